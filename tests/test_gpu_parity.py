"""Parity of the CUDA path (through the C-ABI) with the CPU oracle: identical
match counts and identical sorted violation lists (integer work: bit-exact)."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from oracle.bruteforce import brute_force
from synth import configs
from synth.gfds import GFD, Literal
from synth.graphs import graph_from_edges, random_small_graph

from cases import (complete_bidirected, directed_cycle, edges_graph, golden_cases, out_star,
                   random_case, star_q, undirected_q)
from gpu_util import assert_same, gpu_graph, gpu_run, reverse_csr

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")

FLAG_SETS = {
    "persistent": 0,
    "no_refine": G.FLAG_NO_REFINE,
    "host_loop_graph": G.FLAG_HOST_LOOP,
    "host_loop_plain": G.FLAG_HOST_LOOP | G.FLAG_NO_GRAPH,
}


@pytest.fixture(scope="module")
def lib():
    return G.load_library()


@pytest.mark.parametrize("flags", list(FLAG_SETS), ids=list(FLAG_SETS))
def test_random_small_vs_brute_force(lib, oracle_mod, flags):
    for seed in range(80):
        g, q = random_case(seed)
        want = oracle_mod.validate(g, q)
        dg = gpu_graph(g)
        assert_same(gpu_run(dg, q, flags=FLAG_SETS[flags]), want, f"seed {seed}")


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c[0])
def test_golden_toys(lib, case):
    name, g, q, n_matches, viol = case
    got = gpu_run(gpu_graph(g), q)
    assert_same(got, (n_matches, viol), name)


def test_closed_forms(lib):
    for n in (3, 5, 8):
        dg = gpu_graph(complete_bidirected(n))
        assert gpu_run(dg, undirected_q(3, [(0, 1), (1, 2), (0, 2)]))[0] == n * (n - 1) * (n - 2)
        assert gpu_run(dg, undirected_q(3, [(0, 1), (1, 2)]))[0] == 0
    for d, s in [(5, 2), (7, 3), (3, 4)]:
        assert gpu_run(gpu_graph(out_star(d)), star_q(s))[0] == (math.perm(d, s) if s <= d else 0)
    assert gpu_run(gpu_graph(out_star(6, extra=[(2, 5, 0)])), star_q(2))[0] == 28
    q = GFD([0, 0, 0], [(0, 1, 0), (1, 2, 0)])
    for n in (3, 4, 9):
        assert gpu_run(gpu_graph(directed_cycle(n)), q)[0] == (n if n >= 4 else 0)


def test_hub_star_many_tiles(lib, oracle_mod):
    """A hub of out-degree 3000 and the 2-leaf star pattern: 3000*2999 matches
    spread over many tiles and supersteps (chunking), checked by closed form."""
    d = 3000
    g = out_star(d)
    want = d * (d - 1)
    for chunk in (0, 1024, 5000):
        nm, v = gpu_run(gpu_graph(g), star_q(2), chunk_rows=chunk)
        assert nm == want and v.shape == (0, 3)


def test_max_pattern_size(lib, oracle_mod):
    """k = 16 (the largest pattern): a directed path in a directed path graph."""
    n = 40
    g = edges_graph(n, [(i, i + 1, 0) for i in range(n - 1)])
    q = GFD([0] * 16, [(i, i + 1, 0) for i in range(15)], [], [], True)
    want = oracle_mod.validate(g, q)
    assert want[0] == n - 15
    assert_same(gpu_run(gpu_graph(g), q), want, "k=16")
    with pytest.raises(G.GfdError) as e:
        gpu_run(gpu_graph(g), GFD([0] * 17, [(i, i + 1, 0) for i in range(16)]))
    assert e.value.code == G.GFD_ERR_UNSUPPORTED


def test_empty_and_degenerate_graphs(lib, oracle_mod):
    # a graph without edges: single-node patterns match every vertex
    g = edges_graph(5, [], vlabel=np.array([0, 1, 0, 1, 1], np.int32))
    q1 = GFD([1], [], [], [Literal.const(0, 0, 7)])
    assert_same(gpu_run(gpu_graph(g), q1), oracle_mod.validate(g, q1), "no edges")
    assert gpu_run(gpu_graph(g), GFD([0, 0], [(0, 1, 0)]))[0] == 0
    # a single vertex with a self-loop
    g1 = edges_graph(1, [(0, 0, 3)])
    assert gpu_run(gpu_graph(g1), GFD([0], [(0, 0, 3)]))[0] == 1
    assert gpu_run(gpu_graph(g1), GFD([0], []))[0] == 0
    # zero vertices
    g0 = graph_from_edges(0, [], [], [], np.zeros(0, np.int32), np.zeros((1, 0), np.int32))
    assert gpu_run(gpu_graph(g0), GFD([0], []))[0] == 0


@pytest.mark.parametrize("seed", range(6))
def test_random_medium_vs_oracle(lib, oracle_mod, seed):
    """Graphs of a few hundred vertices: many tiles, ragged tails, all shapes."""
    rng = np.random.default_rng([99, seed])
    g = random_small_graph(1000 + seed, 300, n_vlabels=2, n_elabels=2, p_edge=0.03, p_self=0.02,
                           n_attrs=2, n_attr_values=3, p_absent=0.05)
    from synth.gfds import random_pattern_gfd
    dg = gpu_graph(g)
    for t in range(8):
        shape = ["tree", "cycle", "tri_tails", "clique4"][t % 4]
        k = int(rng.integers(4 if shape == "clique4" else 3, 6))
        q = random_pattern_gfd(rng, shape, k, [0, 1, -1], [0, 1, -1], 2, (0, 2), 1,
                               lambda: int(rng.integers(0, 3)), p_both_dirs=0.2)
        want = oracle_mod.validate(g, q)
        for chunk in (0, 1024):
            assert_same(gpu_run(dg, q, chunk_rows=chunk), want, f"seed {seed} gfd {t} chunk {chunk}")


def test_tiny_workload(lib, oracle_mod):
    g, qs = configs.tiny()
    want = oracle_mod.validate(g, qs[0])
    assert want[1].shape[0] == configs.TINY_PLANTED
    dg = gpu_graph(g)
    for flags in FLAG_SETS.values():
        assert_same(gpu_run(dg, qs[0], flags=flags), want, f"tiny flags={flags}")


def test_mid_workload(lib, oracle_mod):
    """The mid workload at full size (1M vertices, 8M edges), exact."""
    g, qs = configs.mid()
    want = oracle_mod.validate(g, qs[0], threads=os.cpu_count() or 8)
    assert want[0] > 10000 and want[1].shape[0] > 0
    dg = gpu_graph(g)
    assert_same(gpu_run(dg, qs[0]), want, "mid")
    assert_same(gpu_run(dg, qs[0], flags=G.FLAG_HOST_LOOP, chunk_rows=4096), want, "mid small chunks")


def _batched_vs_oracle(oracle_mod, scale, n):
    g, qs = configs.batched(scale=scale, n_gfds=n)
    dg = gpu_graph(g)
    res = dg.validate_batch(qs)
    og = oracle_mod.OracleGraph(g)
    total = nonzero = 0
    for i, q in enumerate(qs):
        want = oracle_mod.validate(og, q, threads=os.cpu_count() or 8)
        assert_same((res[i].n_matches, res[i].violations()), want, f"batch gfd {i} {q.name}")
        total += want[0]
        nonzero += want[0] > 0
        if i % 8 == 0:
            assert_same(gpu_run(dg, q), want, f"single gfd {i}")
    assert total > 100000 and nonzero > n // 3


def test_batched_workload_scaled(lib, oracle_mod):
    """The first 64 GFDs of the batched recipe on a 1/400 graph (10K vertices,
    100K edges): the batch equals the oracle and one-at-a-time validation."""
    _batched_vs_oracle(oracle_mod, 400, 64)


@pytest.mark.slow
def test_batched_workload_scaled_all(lib, oracle_mod):
    """All 256 GFDs of the batched recipe on the 1/400 graph."""
    _batched_vs_oracle(oracle_mod, 400, 256)


def test_violation_capacity_regrows(lib, oracle_mod):
    g, qs = configs.tiny()
    want = oracle_mod.validate(g, qs[0])
    assert_same(gpu_run(gpu_graph(g), qs[0], max_violations_hint=1), want, "regrow")


def test_reverse_csr_given(lib, oracle_mod):
    g, q = random_case(3, n_vertices=7)
    assert_same(gpu_run(gpu_graph(g, reverse=reverse_csr(g)), q), oracle_mod.validate(g, q), "reverse given")


def test_rejects_invalid_inputs(lib):
    g = out_star(4)
    dg = gpu_graph(g)
    with pytest.raises(G.GfdError) as e:
        dg.validate(GFD([0] * 17, [(i, i + 1, 0) for i in range(16)]))
    assert e.value.code == G.GFD_ERR_UNSUPPORTED                      # k > 16
    with pytest.raises(G.GfdError) as e:
        dg.validate(GFD([0, 0], [(0, 1, 0)], [Literal.const(0, 5, 1)]))
    assert e.value.code == G.GFD_ERR_INVALID_ARG                      # no attribute 5
    with pytest.raises(G.GfdError) as e:
        dg.validate(GFD([0, 0], [(0, 1, 0), (0, 1, 1)]))
    assert e.value.code == G.GFD_ERR_INVALID_ARG                      # repeated pattern edge
    bad = edges_graph(3, [(0, 1, 0), (0, 2, 0)])
    bad.out_dst = bad.out_dst[::-1].copy()                              # unsorted row
    with pytest.raises(G.GfdError) as e:
        gpu_graph(bad)
    assert e.value.code == G.GFD_ERR_INVALID_ARG
    bad2 = edges_graph(3, [(0, 1, 0), (0, 2, 0)])
    bad2.out_dst = np.array([1, 1], np.int32)                          # repeated edge
    with pytest.raises(G.GfdError):
        gpu_graph(bad2)
    bad3 = edges_graph(3, [(0, 1, 0), (0, 2, 0)])
    bad3.out_dst = np.array([1, 7], np.int32)                          # out of range
    with pytest.raises(G.GfdError):
        gpu_graph(bad3)


def test_kernel_variants_and_autotune(lib, oracle_mod):
    """Every enumeration-kernel variant gives the oracle's answer; the autotuner
    picks one of them and later default calls still agree."""
    g, qs = configs.batched(scale=400, n_gfds=16)
    dg = gpu_graph(g)
    og = oracle_mod.OracleGraph(g)
    want = [oracle_mod.validate(og, q) for q in qs]
    for v in range(1, 7):
        for flags in (0, G.FLAG_HOST_LOOP):
            res = dg.validate_batch(qs, kernel_variant=v, flags=flags, tile_iters=1 + 31 * (v % 2))
            for i, r in enumerate(res):
                assert_same((r.n_matches, r.violations()), want[i], f"variant {v} flags {flags} gfd {i}")
    best = dg.autotune(qs)
    assert 1 <= best["kernel_variant"] <= 6 and best["frontier_budget_bytes"] > 0
    res = dg.validate_batch(qs)
    for i, r in enumerate(res):
        assert_same((r.n_matches, r.violations()), want[i], f"tuned gfd {i}")


def test_batched_violation_fetch(lib, oracle_mod):
    """gfd_results_copy_tuples: one sort and one copy for many results gives
    each result's own sorted list, also across two calls and with empty lists."""
    g, qs = configs.batched(scale=400, n_gfds=24)
    dg = gpu_graph(g)
    res = dg.validate_batch(qs[:16])
    more = [dg.validate(q) for q in qs[16:]]
    allr = res + more
    got = G.violations_all(allr)
    assert len(got) == len(allr)
    empty = 0
    for i, r in enumerate(allr):
        assert_same((r.n_matches, got[i]), (r.n_matches, r.violations()), f"result {i}")
        empty += r.n_violations == 0
    for i in (0, 3, 17):
        assert_same((allr[i].n_matches, got[i]), oracle_mod.validate(g, qs[i], threads=os.cpu_count() or 8),
                    f"oracle {i}")
    assert G.violations_all([]) == []
