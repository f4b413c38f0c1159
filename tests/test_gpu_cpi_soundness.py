"""Soundness of the compact path index (Section III.B step 1c: refinement
removes dead-end candidates only). For every pattern node u, the refined
candidate list C(u) the GPU builds must contain h(u) for every match h the
oracle finds (the projection of the matches onto u), and C(u) must lie inside
the candidate filter's list (refinement only removes). The oracle's matches are
those of the twin X = {} -> false, whose violations are all the matches."""
import numpy as np
import pytest

from synth import configs
from synth.gfds import GFD

from cases import random_case
from gpu_util import gpu_graph

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")


def _twin(q):
    return GFD(q.node_label, q.edges, [], [], True, q.name + "_twin")


def _check(g, qs, oracle_mod, what, flags=0, induced=True, threads=1):
    dg = gpu_graph(g)
    keep = G.FLAG_KEEP_CANDIDATES | flags
    refined = dg.validate_batch(qs, flags=keep)
    filtered = dg.validate_batch(qs, flags=keep | G.FLAG_NO_REFINE)
    n_proj = 0
    for i, q in enumerate(qs):
        nm, matches = oracle_mod.validate(g, _twin(q), threads=threads, induced=induced)
        assert refined[i].n_matches == nm, f"{what} gfd {i}"
        for u in range(q.k):
            c = refined[i].candidates(u)
            f = filtered[i].candidates(u)
            assert np.all(np.diff(c) > 0) and np.all(np.diff(f) > 0), "lists are sorted and unique"
            assert np.isin(c, f).all(), f"{what} gfd {i} node {u}: refinement added a vertex"
            proj = np.unique(matches[:, u])
            missing = proj[~np.isin(proj, c)]
            assert missing.size == 0, f"{what} gfd {i} node {u}: match images {missing[:8]} pruned"
            n_proj += proj.size
    return n_proj


def test_brute_force_cases(oracle_mod):
    G.load_library()
    total = 0
    for seed in range(80):
        g, q = random_case(seed)
        total += _check(g, [q], oracle_mod, f"seed {seed}")
    assert total > 100


def test_brute_force_cases_non_induced(oracle_mod):
    G.load_library()
    total = 0
    for seed in range(40):
        g, q = random_case(seed)
        total += _check(g, [q], oracle_mod, f"seed {seed}", flags=G.FLAG_NON_INDUCED, induced=False)
    assert total > 100


def test_batched_workload_scaled(oracle_mod):
    G.load_library()
    g, _ = configs.batched(scale=400, n_gfds=1)
    qs = configs.batched_gfds(g, 48)
    assert _check(g, qs, oracle_mod, "batched/400", threads=8) > 1000
