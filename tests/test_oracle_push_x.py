"""Pins of the oracle's count of X-satisfying matches (what validation with X
pushed into the search enumerates; Section II: only matches with h ⊨ X can be
violations, so Vio is the same). Brute force, closed forms, invariants. CPU only."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.bruteforce import brute_force
from synth.gfds import GFD, Literal

from cases import edges_graph, random_case


@pytest.mark.parametrize("induced", [True, False], ids=["induced", "non_induced"])
@pytest.mark.parametrize("seed", range(80))
def test_x_count_equals_brute_force(oracle_mod, seed, induced):
    g, q = random_case(seed)
    nx, v = oracle_mod.validate(g, q, induced=induced, count="x")
    bnx, bv = brute_force(g, q, induced=induced, count="x")
    assert nx == bnx
    np.testing.assert_array_equal(v, bv)
    nm, v_all = oracle_mod.validate(g, q, induced=induced)
    assert nx <= nm
    np.testing.assert_array_equal(v, v_all)      # the violations do not change
    if not q.X:
        assert nx == nm


def test_x_count_is_not_trivial(oracle_mod):
    fewer = 0
    for seed in range(80):
        g, q = random_case(seed)
        fewer += oracle_mod.validate(g, q, count="x")[0] < oracle_mod.validate(g, q)[0]
    assert fewer >= 20


def _star_with_parity(d):
    """Out-star 0 -> 1..d whose leaf i has A0 = i mod 2 (the centre has A0 = 5)."""
    attrs = np.array([[5] + [i % 2 for i in range(1, d + 1)]], np.int64)
    return edges_graph(d + 1, [(0, i, 0) for i in range(1, d + 1)], attrs=attrs)


def test_closed_forms_on_a_star(oracle_mod):
    """Out-star with 3 odd and 3 even leaves, pattern x -> y, x -> z (30 matches)."""
    g = _star_with_parity(6)
    base = GFD([0, 0, 0], [(0, 1, 0), (0, 2, 0)])
    cases = [
        ([], 30),                                          # X = ∅: every match
        ([Literal.const(1, 0, 1)], 15),                    # y odd: 3 · 5
        ([Literal.const(1, 0, 1), Literal.const(2, 0, 1)], 6),   # both odd: 3 · 2
        ([Literal.var(1, 0, 2, 0)], 12),                   # same parity: 3·2 + 3·2
        ([Literal.const(0, 0, 5), Literal.var(1, 0, 2, 0)], 12),
        ([Literal.const(0, 0, 4)], 0),
    ]
    for X, want in cases:
        q = GFD(base.node_label, base.edges, X, [Literal.const(1, 0, 7)], False)
        nx, v = oracle_mod.validate(g, q, count="x")
        assert nx == want, X
        assert v.shape[0] == want                          # Y fails on every X-match here


def test_more_x_never_adds(oracle_mod):
    for seed in range(40):
        g, q = random_case(seed)
        nx = oracle_mod.validate(g, q, count="x")[0]
        extra = GFD(q.node_label, q.edges, list(q.X) + [Literal.const(0, 0, 1)], q.Y, q.y_false)
        assert oracle_mod.validate(g, extra, count="x")[0] <= nx
