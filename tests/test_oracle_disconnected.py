"""Pins of the oracle on disconnected patterns (Section II's match definition
applied unchanged: every pair of pattern nodes, across components too, obeys
the match conditions). Brute force over all maps in both matching modes, closed
forms on empty, complete and star graphs. CPU only."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.bruteforce import brute_force
from synth.gfds import GFD

from cases import complete_bidirected, edges_graph, out_star, random_disconnected_case


@pytest.mark.parametrize("induced", [True, False], ids=["induced", "non_induced"])
@pytest.mark.parametrize("seed", range(60))
def test_disconnected_equals_brute_force(oracle_mod, seed, induced):
    g, q = random_disconnected_case(seed)
    for count in ("all", "x"):
        nm, v = oracle_mod.validate(g, q, induced=induced, count=count)
        bnm, bv = brute_force(g, q, induced=induced, count=count)
        assert nm == bnm
        np.testing.assert_array_equal(v, bv)


def test_disconnected_cases_are_not_trivial(oracle_mod):
    nonzero = sum(oracle_mod.validate(*random_disconnected_case(s))[0] > 0 for s in range(60))
    assert nonzero >= 20


TWO = GFD([0, 0], [])                       # two isolated nodes
EDGE_AND_ONE = GFD([0, 0, 0], [(0, 1, 0)])  # an edge and an isolated node


@pytest.mark.parametrize("n", [2, 5, 9])
def test_two_isolated_nodes(oracle_mod, n):
    empty = edges_graph(n, [])
    assert oracle_mod.validate(empty, TWO)[0] == n * (n - 1)
    assert oracle_mod.validate(empty, TWO, induced=False)[0] == n * (n - 1)
    assert oracle_mod.validate(complete_bidirected(n), TWO)[0] == 0
    assert oracle_mod.validate(complete_bidirected(n), TWO, induced=False)[0] == n * (n - 1)


@pytest.mark.parametrize("d", [2, 4, 7])
def test_on_an_out_star(oracle_mod, d):
    """Out-star with d leaves: non-adjacent ordered pairs are leaf pairs,
    d(d-1); every third vertex of an edge's match is adjacent to the centre."""
    g = out_star(d)
    assert oracle_mod.validate(g, TWO)[0] == d * (d - 1)
    assert oracle_mod.validate(g, TWO, induced=False)[0] == (d + 1) * d
    assert oracle_mod.validate(g, EDGE_AND_ONE)[0] == 0
    assert oracle_mod.validate(g, EDGE_AND_ONE, induced=False)[0] == d * (d - 1)
