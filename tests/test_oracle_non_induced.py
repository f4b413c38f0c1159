"""Pins of the oracle's non-induced mode (only the pairs in E_Q constrain a
match: the matching of Bi et al. that Section III contrasts with the paper's,
and the reading of the evaluation's path query in Section V, whose end points
"may or may not" be connected). Brute force over all maps, closed forms and
invariants. CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle.bruteforce import brute_force
from synth.gfds import GFD

from cases import complete_bidirected, directed_cycle, edges_graph, out_star, random_case, star_q, undirected_q


def _v(oracle_mod, g, q):
    return oracle_mod.validate(g, q, induced=False)


@pytest.mark.parametrize("seed", range(80))
def test_non_induced_equals_brute_force(oracle_mod, seed):
    g, q = random_case(seed)
    nm, v = _v(oracle_mod, g, q)
    bnm, bv = brute_force(g, q, induced=False)
    assert nm == bnm
    np.testing.assert_array_equal(v, bv)


def test_non_induced_cases_differ_from_induced(oracle_mod):
    """The random cases exercise the difference: some have extra edges among
    matched vertices, and non-induced matches are a superset of induced ones."""
    differ = 0
    for seed in range(80):
        g, q = random_case(seed)
        nm, v = _v(oracle_mod, g, q)
        inm, iv = oracle_mod.validate(g, q)
        assert nm >= inm
        rows = {tuple(r) for r in v}
        assert all(tuple(r) in rows for r in iv)  # same map, same literals
        differ += nm != inm
    assert differ >= 10


@pytest.mark.parametrize("n", [3, 5, 8])
def test_complete_graph_path(oracle_mod, n):
    """Bidirected K_n, undirected 3-path: every ordered triple, n(n-1)(n-2)
    (induced: 0, because the end points are always adjacent)."""
    nm, _ = _v(oracle_mod, complete_bidirected(n), undirected_q(3, [(0, 1), (1, 2)]))
    assert nm == n * (n - 1) * (n - 2)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_complete_graph_directed_path(oracle_mod, n):
    """Directed path x->y->z in bidirected K_n: every ordered triple."""
    q = GFD([0, 0, 0], [(0, 1, 0), (1, 2, 0)])
    assert _v(oracle_mod, complete_bidirected(n), q)[0] == n * (n - 1) * (n - 2)


@pytest.mark.parametrize("n,k", [(5, 4), (6, 5), (7, 3)])
def test_complete_graph_any_connected_pattern(oracle_mod, n, k):
    """In bidirected K_n every connected pattern without self-loops has all
    n!/(n-k)! injective maps as non-induced matches (here: a k-cycle)."""
    pairs = [(i, (i + 1) % k) for i in range(k)]
    assert _v(oracle_mod, complete_bidirected(n), undirected_q(k, pairs))[0] == math.perm(n, k)


def test_out_star_extra_edges_do_not_matter(oracle_mod):
    """Edges between the leaves of an out-star do not remove non-induced
    matches (induced: each such edge removes 2)."""
    for extra in ([], [(2, 5, 0)], [(2, 5, 0), (3, 4, 0), (1, 6, 0)]):
        assert _v(oracle_mod, out_star(6, extra=extra), star_q(2))[0] == math.perm(6, 2)


def test_directed_cycle_path(oracle_mod):
    """Directed C_3, pattern x->y->z: the closing edge z->x is allowed, so the
    3 rotations match (induced: none)."""
    q = GFD([0, 0, 0], [(0, 1, 0), (1, 2, 0)])
    assert _v(oracle_mod, directed_cycle(3), q)[0] == 3
    assert oracle_mod.validate(directed_cycle(3), q)[0] == 0


def test_required_edges_and_labels_still_apply(oracle_mod):
    """Required pattern edges, their labels and directions are still checked."""
    g = edges_graph(3, [(0, 1, 1), (0, 2, 2), (2, 1, 0)], vlabel=np.array([5, 6, 7], np.int32))
    assert _v(oracle_mod, g, GFD([5, 6], [(0, 1, 1)]))[0] == 1
    assert _v(oracle_mod, g, GFD([5, 6], [(0, 1, 2)]))[0] == 0
    assert _v(oracle_mod, g, GFD([6, 5], [(0, 1, 1)]))[0] == 0     # reversed direction
    assert _v(oracle_mod, g, GFD([-1, -1], [(0, 1, -1)]))[0] == 3


def test_self_loops_unconstrained_unless_required(oracle_mod):
    """A data self-loop does not block a pattern node without one; a pattern
    self-loop still needs one with an agreeing label."""
    g = edges_graph(3, [(0, 0, 1), (0, 1, 0), (2, 2, 0), (2, 1, 0)])
    assert _v(oracle_mod, g, GFD([0, 0], [(0, 1, 0)]))[0] == 2    # induced: 0
    assert _v(oracle_mod, g, GFD([0, 0], [(0, 0, 1), (0, 1, 0)]))[0] == 1
    assert _v(oracle_mod, g, GFD([0, 0], [(0, 0, -1), (0, 1, 0)]))[0] == 2
