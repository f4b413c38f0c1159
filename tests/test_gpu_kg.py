"""The knowledge-graph-shaped workload: 6-node GFDs x-[e]->y, x-[e']->y',
y->z1, y'->z1, y->z2, y'->z2, x->w with X -> false dependencies, on graphs with
hub out-degrees up to ~1e6 at full size. The plain oracle cannot enumerate
those graphs, so (1) the pattern family is checked exactly against the oracle
on random graphs it can finish, and (2) the full workload is checked through
properties that hold at any size: both enumeration drivers, all kernel
variants, and batched vs one-at-a-time validation give identical results."""
import numpy as np
import pytest

from synth import configs
from synth.gfds import GFD, Literal
from synth.graphs import random_small_graph

from full_size import compare, gpu_rows_for_roots, reorder, rows_at, sample_roots, swap_perm, twin
from gpu_util import assert_same, gpu_graph

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")


@pytest.fixture(scope="module")
def lib_loaded():
    return G.load_library()


def _kg_shaped(rng, k_labels):
    nl = [int(rng.choice(k_labels)) for _ in range(5)] + [-1]
    e1, e2 = (int(rng.choice([-1, 0, 1])) for _ in range(2))
    edges = [(0, 1, e1), (0, 2, e2), (1, 3, -1), (2, 3, -1), (1, 4, -1), (2, 4, -1), (0, 5, -1)]
    if rng.random() < 0.5:
        return GFD(nl, edges, [Literal.const(1, 0, int(rng.integers(0, 3))),
                               Literal.const(2, 0, int(rng.integers(0, 3)))], [], True)
    return GFD(nl, edges, [], [Literal.var(1, 0, 2, 0)], False)


@pytest.mark.parametrize("seed", range(4))
def test_kg_pattern_family_exact(lib_loaded, oracle_mod, seed):
    rng = np.random.default_rng([31, seed])
    g = random_small_graph(500 + seed, 250, n_vlabels=2, n_elabels=2, p_edge=0.06, p_self=0.0,
                           n_attrs=1, n_attr_values=3, p_absent=0.05)
    dg = gpu_graph(g)
    total = 0
    qs = [_kg_shaped(rng, [0, 1, -1]) for _ in range(6)]
    res = dg.validate_batch(qs)
    for i, q in enumerate(qs):
        want = oracle_mod.validate(g, q, threads=8)
        assert_same((res[i].n_matches, res[i].violations()), want, f"seed {seed} gfd {i}")
        total += want[0]
    assert total > 0


def _properties(g, qs):
    dg = gpu_graph(g)
    ref = [(r.n_matches, r.violations()) for r in dg.validate_batch(qs)]
    for flags, variant in ((G.FLAG_HOST_LOOP, 0), (0, 5), (0, 4), (G.FLAG_NO_REFINE, 0)):
        res = dg.validate_batch(qs, flags=flags, kernel_variant=variant)
        for i, r in enumerate(res):
            assert_same((r.n_matches, r.violations()), ref[i], f"{qs[i].name} flags {flags} variant {variant}")
    for i in (0, 1, len(qs) - 1):
        r = dg.validate(qs[i])
        assert_same((r.n_matches, r.violations()), ref[i], f"{qs[i].name} alone")
    return sum(x[0] for x in ref)


def test_kg_scaled_properties(lib_loaded):
    g, qs = configs.kg(scale=20)
    _properties(g, qs)


@pytest.fixture(scope="module")
def kg_full():
    return configs.kg()


@pytest.mark.slow
def test_kg_full_size_properties(lib_loaded, kg_full):
    g, qs = kg_full
    assert np.diff(g.out_off).max() > 500_000          # hub out-degrees near 1e6
    _properties(g, qs)


@pytest.mark.slow
def test_kg_full_size_sampled_roots(lib_loaded, kg_full, oracle_mod):
    """The full KG workload (20M vertices, 200M edges, 32 GFDs) in one batched
    launch, root by root against the oracle. The roots are images of z1 (node
    3, in-degree 2 in the pattern): the matches of a KG pattern concentrate on
    x hubs with out-degrees up to ~1e6, which the oracle cannot search from x
    in seconds, while from z1 each root's work stays small. The oracle runs
    each GFD relabelled so that z1 is node 0 (results are invariant under
    relabelling, a pinned invariant) and the GPU's tuples are compared in that
    column order. About 2,000 (GFD, root) pairs: uniform over label-compatible
    vertices of in-degree >= 2, hubs of in-degree >= 1000 (the top one of every
    pool among them) and z1 images of GPU matches. Matches (through the twin
    X = {} -> false) and violations must be identical."""
    g, qs = kg_full
    dg = gpu_graph(g)
    res = dg.validate_batch(qs)
    total = sum(r.n_matches for r in res)
    tres = dg.validate_batch([twin(q) for q in qs], max_violations_hint=total + 1)
    for i, (r, t) in enumerate(zip(res, tres)):
        assert r.n_matches == t.n_matches == t.n_violations, f"gfd {i}: twin counts differ"
    in_deg = np.bincount(g.out_dst, minlength=g.n_vertices)
    perms = [swap_perm(q.k, 3) for q in qs]
    rel = [q.relabel_nodes(p) for q, p in zip(qs, perms)]
    rng = np.random.default_rng(20261204)
    samples, gpu_m = [], {}
    for i, q in enumerate(rel):
        t = reorder(tres[i].violations(), perms[i])
        samples.append(sample_roots(g, q, in_deg, t, rng, n_uniform=60, n_from_matches=10, n_hubs=4,
                                    min_degree=2))
        gpu_m.update({(i, r): rows_at(t, r).copy() for r, _ in samples[i]})
    gpu_v = gpu_rows_for_roots(res, samples, perms)
    og = oracle_mod.OracleGraph(g)
    st = compare(og, oracle_mod, rel, samples, gpu_m, gpu_v, in_deg, deadline=2.0, hub_deadline=4.0,
                 wall_cap=120.0)
    print("kg full-size sampled roots:", st)
    assert st["roots_done"] >= 2000, st
    assert st["hub_roots_done"] >= 50, st
    # KG matches concentrate on few roots (x hubs and their neighbourhoods):
    # a handful of sampled roots carry hundreds of thousands of matches
    assert st["roots_with_matches"] >= 5 and st["matches_compared"] >= 100_000, st
