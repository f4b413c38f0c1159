"""Parity of the non-induced matching mode (GFD_FLAG_NON_INDUCED) with the
oracle's non-induced mode: identical match counts and sorted violation lists,
under every driver, for single GFDs, batches and serving sessions."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from synth import configs
from synth.gfds import GFD
from synth.graphs import random_small_graph

from cases import complete_bidirected, directed_cycle, edges_graph, out_star, random_case, star_q, undirected_q
from gpu_util import assert_same, gpu_graph, gpu_run

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")

NI = G.FLAG_NON_INDUCED
DRIVERS = {
    "persistent": NI,
    "no_refine": NI | G.FLAG_NO_REFINE,
    "host_loop_graph": NI | G.FLAG_HOST_LOOP,
}


@pytest.fixture(scope="module")
def lib():
    return G.load_library()


@pytest.mark.parametrize("driver", list(DRIVERS), ids=list(DRIVERS))
def test_random_small_vs_oracle(lib, oracle_mod, driver):
    differ = 0
    for seed in range(80):
        g, q = random_case(seed)
        want = oracle_mod.validate(g, q, induced=False)
        got = gpu_run(gpu_graph(g), q, flags=DRIVERS[driver])
        assert_same(got, want, f"seed {seed}")
        differ += want[0] != oracle_mod.validate(g, q)[0]
    assert differ >= 10   # the mode matters on these cases


def test_closed_forms(lib):
    for n in (3, 5, 8):
        dg = gpu_graph(complete_bidirected(n))
        assert gpu_run(dg, undirected_q(3, [(0, 1), (1, 2)]), flags=NI)[0] == n * (n - 1) * (n - 2)
        assert gpu_run(dg, GFD([0, 0, 0], [(0, 1, 0), (1, 2, 0)]), flags=NI)[0] == n * (n - 1) * (n - 2)
    for n, k in [(5, 4), (6, 5)]:
        pairs = [(i, (i + 1) % k) for i in range(k)]
        assert gpu_run(gpu_graph(complete_bidirected(n)), undirected_q(k, pairs), flags=NI)[0] == math.perm(n, k)
    extra = [(2, 5, 0), (3, 4, 0), (1, 6, 0)]
    assert gpu_run(gpu_graph(out_star(6, extra=extra)), star_q(2), flags=NI)[0] == 30
    assert gpu_run(gpu_graph(directed_cycle(3)), GFD([0, 0, 0], [(0, 1, 0), (1, 2, 0)]), flags=NI)[0] == 3
    g = edges_graph(3, [(0, 0, 1), (0, 1, 0), (2, 2, 0), (2, 1, 0)])
    assert gpu_run(gpu_graph(g), GFD([0, 0], [(0, 1, 0)]), flags=NI)[0] == 2
    assert gpu_run(gpu_graph(g), GFD([0, 0], [(0, 0, 1), (0, 1, 0)]), flags=NI)[0] == 1


def test_random_graphs_ragged_chunks(lib, oracle_mod):
    """300-vertex graphs with self-loops and small chunks (ragged tails)."""
    for seed in range(4):
        g = random_small_graph(2000 + seed, 300, n_vlabels=2, n_elabels=2, p_edge=0.03, p_self=0.02,
                               n_attrs=2, n_attr_values=3, p_absent=0.05)
        dg = gpu_graph(g)
        for t, q in enumerate([undirected_q(3, [(0, 1), (1, 2)]), GFD([0, -1, 1], [(0, 1, -1), (2, 1, 0)]),
                               undirected_q(4, [(0, 1), (1, 2), (2, 3), (3, 0)])]):
            want = oracle_mod.validate(g, q, induced=False)
            for chunk in (1024, 0):
                assert_same(gpu_run(dg, q, chunk_rows=chunk, flags=NI), want, f"seed {seed} gfd {t} chunk {chunk}")


def test_batched_workload_scaled(lib, oracle_mod):
    """16 GFDs of the batched recipe on the 1/400 graph, as one batch."""
    g, qs = configs.batched(scale=400, n_gfds=16)
    dg = gpu_graph(g)
    res = dg.validate_batch(qs, flags=NI)
    og = oracle_mod.OracleGraph(g)
    more = 0
    for i, q in enumerate(qs):
        want = oracle_mod.validate(og, q, threads=os.cpu_count() or 8, induced=False)
        assert_same((res[i].n_matches, res[i].violations()), want, f"batch gfd {i} {q.name}")
        more += want[0] > dg.validate(q).n_matches   # the induced count
    assert more > 0


def test_session(lib, oracle_mod):
    g, _ = configs.batched(scale=400, n_gfds=4)
    reqs = configs.serving_requests(g, 12)
    dg = gpu_graph(g)
    s = G.Session(dg, max_slots=4, frontier_budget_bytes=256 << 20, max_violations_hint=1 << 16, flags=NI)
    ids = {s.submit(q): i for i, q in enumerate(reqs)}
    got = {}
    while len(got) < len(reqs):
        s.step()
        for rid, res in s.results():
            got[ids[rid]] = (res.n_matches, res.violations())
    og = oracle_mod.OracleGraph(g)
    for i, q in enumerate(reqs):
        assert_same(got[i], oracle_mod.validate(og, q, threads=os.cpu_count() or 8, induced=False), f"request {i}")
