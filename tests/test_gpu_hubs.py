"""Hubs: adjacency lists longer than the warp kernels keep (over 1024 entries) (they are queued and
scanned by whole blocks in refinement and index construction). Closed forms on
stars of 20,000 leaves, and graphs with planted out- and in-hubs of degree 6,000
compared with the oracle in both matching modes and with X pushed down."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from synth.gfds import GFD, Literal
from synth.graphs import graph_from_edges

from cases import edges_graph, out_star, star_q
from gpu_util import assert_same, gpu_graph, gpu_run

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")


@pytest.fixture(scope="module")
def lib():
    return G.load_library()


def test_big_stars(lib):
    d = 20000
    dg = gpu_graph(out_star(d))
    assert gpu_run(dg, star_q(2))[0] == math.perm(d, 2)
    assert gpu_run(dg, star_q(1))[0] == d
    in_star = edges_graph(d + 1, [(i, 0, 0) for i in range(1, d + 1)])
    q = GFD([0, 0, 0], [(1, 0, 0), (2, 0, 0)])
    assert gpu_run(gpu_graph(in_star), q)[0] == math.perm(d, 2)
    # leaves with a label that only every 7th leaf carries
    vl = np.array([0] + [1 if i % 7 == 0 else 0 for i in range(1, d + 1)], np.int32)
    g = edges_graph(d + 1, [(0, i, 0) for i in range(1, d + 1)], vlabel=vl)
    assert gpu_run(gpu_graph(g), GFD([0, 1, 1], [(0, 1, 0), (0, 2, 0)]))[0] == math.perm(d // 7, 2)


def hub_graph(seed, n=12000, out_hubs=3, in_hubs=2, deg=6000, p_edge=2.5):
    rng = np.random.default_rng([4096, seed])
    E = {}
    hubs = rng.choice(n, size=out_hubs + in_hubs, replace=False)
    for t, h in enumerate(hubs):
        others = rng.choice(n, size=deg, replace=False)
        for o in others:
            if o == h:
                continue
            a, b = (int(h), int(o)) if t < out_hubs else (int(o), int(h))
            E[(a, b)] = int(rng.integers(0, 3))
    m = int(p_edge * n)
    src = rng.integers(0, n, size=m)
    dst = rng.integers(0, n, size=m)
    for a, b in zip(src, dst):
        if a != b:
            E.setdefault((int(a), int(b)), int(rng.integers(0, 3)))
    e = np.array([(a, b, l) for (a, b), l in sorted(E.items())], np.int64)
    vl = rng.integers(0, 6, size=n).astype(np.int32)
    vl[hubs] = 5
    attrs = rng.integers(0, 4, size=(2, n)).astype(np.int64)
    return graph_from_edges(n, e[:, 0], e[:, 1], e[:, 2], vl, attrs)


PATTERNS = [
    GFD([5, 0], [(0, 1, -1)], [], [Literal.const(1, 0, 1)]),
    GFD([5, 1, 2], [(0, 1, -1), (1, 2, -1)], [Literal.const(2, 1, 2)], [Literal.var(1, 0, 2, 0)]),
    GFD([5, -1, -1], [(0, 1, -1), (1, 2, -1), (0, 2, -1)], [], [Literal.var(0, 0, 2, 1)]),
    GFD([0, 5, 1], [(0, 1, 0), (2, 1, -1)], [Literal.const(0, 0, 3)], [Literal.const(2, 1, 0)]),
    GFD([5, 3, 4, 4], [(0, 1, 1), (0, 2, -1), (2, 3, -1)], [], [Literal.var(1, 0, 3, 0)]),
]


@pytest.mark.parametrize("seed", range(2))
@pytest.mark.parametrize("mode", ["induced", "non_induced", "push_x", "no_refine"])
def test_hub_graphs_vs_oracle(lib, oracle_mod, seed, mode):
    g = hub_graph(seed)
    og = oracle_mod.OracleGraph(g)
    dg = gpu_graph(g)
    flags = {"induced": 0, "non_induced": G.FLAG_NON_INDUCED, "push_x": G.FLAG_PUSH_X,
             "no_refine": G.FLAG_NO_REFINE}[mode]
    threads = os.cpu_count() or 8
    wants = [oracle_mod.validate(og, q, threads=threads, induced=mode != "non_induced",
                                 count="x" if mode == "push_x" else "all") for q in PATTERNS]
    for t, q in enumerate(PATTERNS):
        assert_same(gpu_run(dg, q, flags=flags), wants[t], f"seed {seed} pattern {t} {mode}")
    res = dg.validate_batch(PATTERNS, flags=flags)
    for t, q in enumerate(PATTERNS):
        assert_same((res[t].n_matches, res[t].violations()), wants[t], f"batch seed {seed} pattern {t} {mode}")
    assert sum(w[0] for w in wants) > 1000
