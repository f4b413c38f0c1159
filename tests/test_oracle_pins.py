"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(brute force over all maps, closed-form counts, hand-counted toys from the
paper's examples, invariants). CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle.bruteforce import brute_force
from synth import configs
from synth.gfds import GFD, Literal

from cases import (complete_bidirected, directed_cycle, edges_graph, golden_cases, out_star,
                   random_case, star_q, undirected_q)


def _v(oracle_mod, g, q, **kw):
    return oracle_mod.validate(g, q, **kw)


# ------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(80))
def test_oracle_equals_brute_force(oracle_mod, seed):
    g, q = random_case(seed)
    nm, v = _v(oracle_mod, g, q)
    bnm, bv = brute_force(g, q)
    assert nm == bnm
    np.testing.assert_array_equal(v, bv)


def test_brute_force_cases_are_not_trivial(oracle_mod):
    """The random cases must exercise matches and violations, not only zeros."""
    tot_m = tot_v = 0
    for seed in range(80):
        g, q = random_case(seed)
        nm, v = _v(oracle_mod, g, q)
        tot_m += nm > 0
        tot_v += v.shape[0] > 0
    assert tot_m >= 30 and tot_v >= 15


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [3, 4, 6, 9])
def test_complete_graph_triangle(oracle_mod, n):
    """Bidirected K_n, undirected triangle: every ordered triple, n(n-1)(n-2)."""
    nm, _ = _v(oracle_mod, complete_bidirected(n), undirected_q(3, [(0, 1), (1, 2), (0, 2)]))
    assert nm == n * (n - 1) * (n - 2)


@pytest.mark.parametrize("n", [3, 5, 8])
def test_complete_graph_induced_path_is_empty(oracle_mod, n):
    """Induced 3-path in K_n: the end points are always adjacent, so 0 matches."""
    nm, _ = _v(oracle_mod, complete_bidirected(n), undirected_q(3, [(0, 1), (1, 2)]))
    assert nm == 0


@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_complete_graph_clique(oracle_mod, n):
    """Undirected 4-clique in K_n: n!/(n-4)! ordered 4-tuples."""
    pairs = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    nm, _ = _v(oracle_mod, complete_bidirected(n), undirected_q(4, pairs))
    assert nm == math.perm(n, 4)


@pytest.mark.parametrize("d,s", [(2, 2), (5, 2), (6, 3), (7, 4), (4, 4), (3, 4)])
def test_out_star(oracle_mod, d, s):
    """Out-star of degree d, star pattern with s leaves: d!/(d-s)!."""
    nm, _ = _v(oracle_mod, out_star(d), star_q(s))
    assert nm == (math.perm(d, s) if s <= d else 0)


def test_out_star_extra_edge_removes_two(oracle_mod):
    """An edge y_i -> y_j between two leaves removes exactly the 2 tuples that
    map {y, z} onto {y_i, y_j} (additional edges are not allowed)."""
    nm0, _ = _v(oracle_mod, out_star(6), star_q(2))
    nm1, _ = _v(oracle_mod, out_star(6, extra=[(2, 5, 0)]), star_q(2))
    assert nm0 == 30 and nm1 == 28


def test_in_star_direction_matters(oracle_mod):
    """Reversed G edges: the out-star pattern has no match in an in-star."""
    g = edges_graph(5, [(i, 0, 0) for i in range(1, 5)])
    assert _v(oracle_mod, g, star_q(2))[0] == 0
    q = GFD([0, 0, 0], [(1, 0, 0), (2, 0, 0)])
    assert _v(oracle_mod, g, q)[0] == 12


@pytest.mark.parametrize("n", [3, 4, 5, 8])
def test_directed_cycle_path(oracle_mod, n):
    """Directed C_n, pattern x->y->z: n matches for n >= 4, none for n = 3 (z->x)."""
    q = GFD([0, 0, 0], [(0, 1, 0), (1, 2, 0)])
    assert _v(oracle_mod, directed_cycle(n), q)[0] == (n if n >= 4 else 0)


def test_directed_triangle_rotations(oracle_mod):
    """Directed 3-cycle pattern in a directed 3-cycle: its 3 rotations."""
    q = GFD([0, 0, 0], [(0, 1, 0), (1, 2, 0), (2, 0, 0)])
    assert _v(oracle_mod, directed_cycle(3), q)[0] == 3
    assert _v(oracle_mod, complete_bidirected(3), q)[0] == 0


def test_edge_labels_and_wildcards(oracle_mod):
    g = edges_graph(3, [(0, 1, 1), (0, 2, 2)], vlabel=np.array([5, 6, 7], np.int32))
    q1 = GFD([5, 6], [(0, 1, 1)])
    q2 = GFD([5, 6], [(0, 1, 2)])
    q3 = GFD([5, -1], [(0, 1, -1)])
    q4 = GFD([-1, -1], [(0, 1, 2)])
    assert _v(oracle_mod, g, q1)[0] == 1
    assert _v(oracle_mod, g, q2)[0] == 0
    assert _v(oracle_mod, g, q3)[0] == 2
    assert _v(oracle_mod, g, q4)[0] == 1


def test_self_loops(oracle_mod):
    """(a,a) ∈ E_Q ⇔ (h(a),h(a)) ∈ E, labels equal."""
    g = edges_graph(3, [(0, 0, 1), (0, 1, 0), (2, 2, 0), (2, 1, 0)])
    plain = GFD([0, 0], [(0, 1, 0)])
    loop1 = GFD([0, 0], [(0, 0, 1), (0, 1, 0)])
    loopw = GFD([0, 0], [(0, 0, -1), (0, 1, 0)])
    assert _v(oracle_mod, g, plain)[0] == 0          # both sources carry a loop
    assert _v(oracle_mod, g, loop1)[0] == 1          # only vertex 0's loop has label 1
    assert _v(oracle_mod, g, loopw)[0] == 2


# ------------------------------------------------------------- paper toys
@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c[0])
def test_golden_toys(oracle_mod, case):
    name, g, q, n_matches, viol = case
    nm, v = _v(oracle_mod, g, q)
    assert nm == n_matches
    np.testing.assert_array_equal(v, viol)
    bnm, bv = brute_force(g, q)
    assert bnm == n_matches
    np.testing.assert_array_equal(bv, viol)


# ------------------------------------------------------------- invariants
def _tiny_small():
    g, q = configs.tiny(2000, 10000, 20)
    return g, q[0]


def test_tiny_planted_violations(oracle_mod):
    """The planting recipe gives exactly the planted number of violations."""
    g, q = configs.tiny()
    nm, v = _v(oracle_mod, g, q[0])
    assert v.shape == (configs.TINY_PLANTED, 3)
    assert nm >= configs.TINY_PLANTED


def test_relabel_vertices(oracle_mod):
    g, q = _tiny_small()
    perm = np.random.default_rng(5).permutation(g.n_vertices)
    nm, v = _v(oracle_mod, g, q)
    nm2, v2 = _v(oracle_mod, g.permuted(perm), q)
    assert nm == nm2 and nm > 0
    mapped = perm[v]
    mapped = mapped[np.lexsort(mapped.T[::-1])]
    np.testing.assert_array_equal(mapped, v2)


def test_relabel_pattern_nodes(oracle_mod):
    g, q = _tiny_small()
    perm = [2, 0, 1]
    nm, v = _v(oracle_mod, g, q)
    nm2, v2 = _v(oracle_mod, g, q.relabel_nodes(perm))
    assert nm == nm2
    cols = np.empty_like(v)
    cols[:, perm] = v
    np.testing.assert_array_equal(cols[np.lexsort(cols.T[::-1])], v2)


def test_literal_algebra(oracle_mod):
    g, q = _tiny_small()
    base = GFD(q.node_label, q.edges)
    nm, v = _v(oracle_mod, g, base)
    assert v.shape[0] == 0                                   # Y = ∅: G ⊨ φ
    nmf, vf = _v(oracle_mod, g, GFD(q.node_label, q.edges, [], [], True))
    assert nmf == nm and vf.shape[0] == nm                   # X = ∅ → false
    y1, y2 = Literal.var(1, 0, 2, 0), Literal.const(1, 1, 3)
    _, v1 = _v(oracle_mod, g, GFD(q.node_label, q.edges, [], [y1]))
    _, v2 = _v(oracle_mod, g, GFD(q.node_label, q.edges, [], [y2]))
    _, v12 = _v(oracle_mod, g, GFD(q.node_label, q.edges, [], [y1, y2]))
    union = {tuple(r) for r in v1} | {tuple(r) for r in v2}
    assert {tuple(r) for r in v12} == union                   # Vio(Y1 ∪ Y2)
    _, vx = _v(oracle_mod, g, GFD(q.node_label, q.edges, [Literal.const(0, 1, 3)], [y1, y2]))
    assert {tuple(r) for r in vx} <= union                   # more X never adds


def test_root_sample_partition(oracle_mod):
    """Matches split by the image of node 0: sampling roots partitions the output."""
    g, q = _tiny_small()
    nm, v = _v(oracle_mod, g, q)
    roots = np.arange(g.n_vertices, dtype=np.int32)
    a, b = roots[::2], roots[1::2]
    nma, va = _v(oracle_mod, g, q, roots=a)
    nmb, vb = _v(oracle_mod, g, q, roots=b)
    assert nma + nmb == nm
    both = np.concatenate([va, vb])
    np.testing.assert_array_equal(both[np.lexsort(both.T[::-1])], v)
    nm4, v4 = _v(oracle_mod, g, q, threads=4)
    assert nm4 == nm
    np.testing.assert_array_equal(v4, v)


def test_rejects_bad_inputs(oracle_mod):
    g = out_star(3)
    with pytest.raises(ValueError):
        _v(oracle_mod, g, GFD([0, 0], [(0, 1, 0)], [Literal.const(0, 9, 1)]))  # bad attribute
    with pytest.raises(ValueError):
        edges_graph(2, [(0, 1, 0), (0, 1, 1)])               # repeated pair


def test_validate_within_is_a_root_prefix(oracle_mod):
    """The deadline-bounded oracle returns exactly the result of the roots it
    finished: with room for all roots it equals the unbounded run, and what it
    returns under a short deadline equals the unbounded run on roots[:done]."""
    for seed in range(20):
        g, q = random_case(seed)
        og = oracle_mod.OracleGraph(g)
        roots = np.arange(g.n_vertices, dtype=np.int32)
        nm, v, done = oracle_mod.validate_within(og, q, roots, 60.0)
        assert done == g.n_vertices
        assert (nm, v.tolist()) == (lambda r: (r[0], r[1].tolist()))(oracle_mod.validate(og, q))
        nm2, v2, done2 = oracle_mod.validate_within(og, q, roots, 1e-9)
        want = oracle_mod.validate(og, q, roots=roots[:done2]) if done2 else (0, np.zeros((0, q.k), np.int32))
        assert nm2 == want[0]
        np.testing.assert_array_equal(v2, want[1])


# ------------------------------------------------ literal check on given matches
@pytest.mark.parametrize("seed", range(40))
def test_violating_on_match_list_equals_brute_force(oracle_mod, seed):
    """The twin X = {} -> false of a GFD has every match as a violation
    (Section II: nothing satisfies false); the literal check applied to that
    list must give exactly the brute-force violations of the GFD itself."""
    g, q = random_case(seed)
    twin = GFD(q.node_label, q.edges, [], [], True)
    nm, matches = oracle_mod.validate(g, twin)
    bnm, bv = brute_force(g, q)
    assert nm == bnm == matches.shape[0]
    got = oracle_mod.sort_tuples(oracle_mod.violating(oracle_mod.OracleGraph(g), q, matches))
    np.testing.assert_array_equal(got, bv)
