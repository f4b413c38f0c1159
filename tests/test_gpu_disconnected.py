"""Parity of disconnected patterns (matched component after component) with the
oracle: random tiny cases in both matching modes and with X pushed down, closed
forms, a component that starts at level 1 and one that starts deeper, ragged
chunks, and batches mixing connected and disconnected GFDs."""
from __future__ import annotations

import numpy as np
import pytest

from synth.gfds import GFD, Literal
from synth.graphs import random_small_graph

from cases import complete_bidirected, edges_graph, out_star, random_case, random_disconnected_case
from gpu_util import assert_same, gpu_graph, gpu_run

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")

MODES = {
    "induced": (0, True, "all"),
    "non_induced": (G.FLAG_NON_INDUCED, False, "all"),
    "push_x": (G.FLAG_PUSH_X, True, "x"),
    "host_loop": (G.FLAG_HOST_LOOP, True, "all"),
}


@pytest.fixture(scope="module")
def lib():
    return G.load_library()


@pytest.mark.parametrize("mode", list(MODES), ids=list(MODES))
def test_random_small_vs_oracle(lib, oracle_mod, mode):
    flags, induced, count = MODES[mode]
    nonzero = 0
    for seed in range(60):
        g, q = random_disconnected_case(seed)
        want = oracle_mod.validate(g, q, induced=induced, count=count)
        assert_same(gpu_run(gpu_graph(g), q, flags=flags), want, f"seed {seed}")
        nonzero += want[0] > 0
    assert nonzero >= 15


TWO = GFD([0, 0], [])
EDGE_AND_ONE = GFD([0, 0, 0], [(0, 1, 0)])


def test_closed_forms(lib):
    for n in (2, 5, 9):
        assert gpu_run(gpu_graph(edges_graph(n, [])), TWO)[0] == n * (n - 1)
        dg = gpu_graph(complete_bidirected(n))
        assert gpu_run(dg, TWO)[0] == 0
        assert gpu_run(dg, TWO, flags=G.FLAG_NON_INDUCED)[0] == n * (n - 1)
    for d in (2, 4, 7):
        dg = gpu_graph(out_star(d))
        assert gpu_run(dg, TWO)[0] == d * (d - 1)
        assert gpu_run(dg, TWO, flags=G.FLAG_NON_INDUCED)[0] == (d + 1) * d
        assert gpu_run(dg, EDGE_AND_ONE)[0] == 0
        assert gpu_run(dg, EDGE_AND_ONE, flags=G.FLAG_NON_INDUCED)[0] == d * (d - 1)


def test_medium_graphs_and_chunks(lib, oracle_mod):
    """300-vertex graphs: a triangle plus an edge (the second component starts
    deep in the order), two paths, an edge plus an isolated node; small chunks
    give ragged tails and several steps per level."""
    pats = [
        GFD([0, 0, 0, 1, 1], [(0, 1, -1), (1, 2, -1), (2, 0, -1), (3, 4, 0)],
            [Literal.var(0, 0, 3, 0)], [Literal.var(1, 1, 4, 1)]),
        GFD([0, -1, 1, 0], [(0, 1, -1), (2, 3, 1)], [], [Literal.const(1, 0, 1)]),
        GFD([-1, 1, 0], [(0, 1, 0)], [], [Literal.var(0, 0, 2, 0)]),
    ]
    for seed in range(3):
        g = random_small_graph(3000 + seed, 300, n_vlabels=2, n_elabels=2, p_edge=0.02, p_self=0.02,
                               n_attrs=2, n_attr_values=3, p_absent=0.05)
        dg = gpu_graph(g)
        for t, q in enumerate(pats):
            for flags, induced in ((0, True), (G.FLAG_NON_INDUCED, False)):
                want = oracle_mod.validate(g, q, induced=induced)
                for chunk in (0, 1024):
                    assert_same(gpu_run(dg, q, chunk_rows=chunk, flags=flags), want,
                                f"seed {seed} gfd {t} flags {flags} chunk {chunk}")


def test_batch_mixing_connected_and_disconnected(lib, oracle_mod):
    qs = [random_disconnected_case(s)[1] for s in range(12)] + [random_case(s)[1] for s in range(12)]
    g = random_small_graph(4242, 8, n_vlabels=2, n_elabels=2, p_edge=0.3, p_self=0.1,
                           n_attrs=2, n_attr_values=3, p_absent=0.15)
    dg = gpu_graph(g)
    res = dg.validate_batch(qs)
    for i, q in enumerate(qs):
        assert_same((res[i].n_matches, res[i].violations()), oracle_mod.validate(g, q), f"gfd {i}")


def test_session_mixing_connected_and_disconnected(lib, oracle_mod):
    """A serving session (always the general expansion) with connected and
    disconnected requests interleaved, in both matching modes."""
    g = random_small_graph(4343, 9, n_vlabels=2, n_elabels=2, p_edge=0.3, p_self=0.1,
                           n_attrs=2, n_attr_values=3, p_absent=0.15)
    reqs = []
    for s in range(10):
        reqs.append(random_disconnected_case(s)[1])
        reqs.append(random_case(s)[1])
    dg = gpu_graph(g)
    for flags, induced in ((0, True), (G.FLAG_NON_INDUCED, False)):
        sess = G.Session(dg, max_slots=3, frontier_budget_bytes=64 << 20, max_violations_hint=1 << 12, flags=flags)
        ids = {sess.submit(q): i for i, q in enumerate(reqs)}
        got = {}
        while len(got) < len(reqs):
            sess.step()
            for rid, res in sess.results():
                got[ids[rid]] = (res.n_matches, res.violations())
        for i, q in enumerate(reqs):
            assert_same(got[i], oracle_mod.validate(g, q, induced=induced), f"request {i} flags {flags}")
