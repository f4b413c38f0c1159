"""Parity of validation with X pushed into the search (GFD_FLAG_PUSH_X) with
the oracle: the match count equals the oracle's count of matches satisfying X,
and the sorted violation list is the same as without the flag."""
from __future__ import annotations

import os

import numpy as np
import pytest

from synth import configs
from synth.gfds import GFD, Literal

from cases import edges_graph, random_case
from gpu_util import assert_same, gpu_graph, gpu_run

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")

PX = G.FLAG_PUSH_X
DRIVERS = {
    "persistent": PX,
    "non_induced": PX | G.FLAG_NON_INDUCED,
    "host_loop_no_refine": PX | G.FLAG_HOST_LOOP | G.FLAG_NO_REFINE,
}


@pytest.fixture(scope="module")
def lib():
    return G.load_library()


@pytest.mark.parametrize("driver", list(DRIVERS), ids=list(DRIVERS))
def test_random_small_vs_oracle(lib, oracle_mod, driver):
    induced = not (DRIVERS[driver] & G.FLAG_NON_INDUCED)
    fewer = 0
    for seed in range(80):
        g, q = random_case(seed)
        want = oracle_mod.validate(g, q, induced=induced, count="x")
        assert_same(gpu_run(gpu_graph(g), q, flags=DRIVERS[driver]), want, f"seed {seed}")
        fewer += want[0] < oracle_mod.validate(g, q, induced=induced)[0]
    assert fewer >= 20


@pytest.mark.parametrize("induced", [True, False], ids=["induced", "non_induced"])
def test_literals_on_every_node(lib, oracle_mod, induced):
    """Each random case again with extra X literals on one node at a time
    (a variable literal within the node and a constant), the root included."""
    flags = PX | (0 if induced else G.FLAG_NON_INDUCED)
    for seed in range(40):
        g, q = random_case(seed)
        dg = gpu_graph(g)
        for j in range(q.k):
            for extra in ([Literal.var(j, 0, j, 1)], [Literal.const(j, 1, 1)],
                          [Literal.var(j, 0, j, 1), Literal.const(j, 0, 0), Literal.const(j, 1, 0),
                           Literal.const(j, 0, 0)]):
                q2 = GFD(q.node_label, q.edges, list(q.X) + extra, q.Y, q.y_false)
                want = oracle_mod.validate(g, q2, induced=induced, count="x")
                assert_same(gpu_run(dg, q2, flags=flags), want, f"seed {seed} node {j} {extra}")


def _star_with_parity(d):
    attrs = np.array([[5] + [i % 2 for i in range(1, d + 1)], [7] * (d + 1)], np.int64)
    return edges_graph(d + 1, [(0, i, 0) for i in range(1, d + 1)], attrs=attrs)


def test_closed_forms_on_a_star(lib):
    """Out-star with 3 odd and 3 even leaves; constants go to the filter (two
    per node at most, the rest are checked during the search)."""
    dg = gpu_graph(_star_with_parity(6))
    base = GFD([0, 0, 0], [(0, 1, 0), (0, 2, 0)])
    cases = [
        ([], 30),
        ([Literal.const(1, 0, 1)], 15),
        ([Literal.const(1, 0, 1), Literal.const(2, 0, 1)], 6),
        ([Literal.var(1, 0, 2, 0)], 12),
        ([Literal.const(0, 0, 5), Literal.var(1, 0, 2, 0)], 12),
        ([Literal.const(0, 0, 4)], 0),
        ([Literal.const(1, 0, 1), Literal.const(1, 1, 7), Literal.const(1, 0, 1)], 15),   # 3 on one node
        ([Literal.const(1, 1, 7), Literal.const(1, 0, 0), Literal.const(1, 1, 6)], 0),
        ([Literal.var(0, 0, 0, 1)], 0),        # the centre: A0 = 5, A1 = 7
        ([Literal.var(0, 1, 0, 1)], 30),
        ([Literal.var(0, 1, 0, 1), Literal.var(2, 0, 2, 0)], 30),
    ]
    for X, want in cases:
        q = GFD(base.node_label, base.edges, X, [Literal.const(1, 0, 9)], False)
        nx, v = gpu_run(dg, q, flags=PX)
        assert nx == want, X
        assert v.shape[0] == want, X
        nm_all, v_all = gpu_run(dg, q)
        assert nm_all == 30
        np.testing.assert_array_equal(v, v_all)


def test_batched_workload_scaled(lib, oracle_mod):
    """16 GFDs of the batched recipe on the 1/400 graph, as one batch: the
    violations equal the unpushed run's and the counts the oracle's X-count."""
    g, qs = configs.batched(scale=400, n_gfds=16)
    dg = gpu_graph(g)
    res = dg.validate_batch(qs, flags=PX)
    ref = dg.validate_batch(qs)
    og = oracle_mod.OracleGraph(g)
    fewer = 0
    for i, q in enumerate(qs):
        want = oracle_mod.validate(og, q, threads=os.cpu_count() or 8, count="x")
        assert_same((res[i].n_matches, res[i].violations()), want, f"batch gfd {i} {q.name}")
        np.testing.assert_array_equal(res[i].violations(), ref[i].violations())
        fewer += res[i].n_matches < ref[i].n_matches
    assert fewer > 0


def test_session(lib, oracle_mod):
    g, _ = configs.batched(scale=400, n_gfds=4)
    reqs = configs.serving_requests(g, 12)
    dg = gpu_graph(g)
    s = G.Session(dg, max_slots=4, frontier_budget_bytes=256 << 20, max_violations_hint=1 << 16, flags=PX)
    ids = {s.submit(q): i for i, q in enumerate(reqs)}
    got = {}
    while len(got) < len(reqs):
        s.step()
        for rid, res in s.results():
            got[ids[rid]] = (res.n_matches, res.violations())
    og = oracle_mod.OracleGraph(g)
    for i, q in enumerate(reqs):
        assert_same(got[i], oracle_mod.validate(og, q, threads=os.cpu_count() or 8, count="x"), f"request {i}")
