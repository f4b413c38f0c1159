"""Brute-force GFD validation over ALL injective maps — TEST INFRASTRUCTURE ONLY.

The most literal reading of Section II of the paper, used on graphs of a handful
of vertices to pin the C oracle: try every injective h : V_Q → V (P(V, k) maps),
keep those that preserve vertex labels and have (a, b) ∈ E_Q ⇔ (h(a), h(b)) ∈ E
for every ordered pair of pattern nodes (self-pairs included) with equal edge
labels, then apply the literal semantics. No ordering, no pruning.
With induced=False only the pairs in E_Q are required (non-induced mode: pairs
outside E_Q, self-pairs included, are unconstrained).
"""
from __future__ import annotations

import itertools

import numpy as np

ABSENT = np.iinfo(np.int32).min
WILDCARD = -1


def _edge_map(graph):
    src, dst, lab = graph.edge_arrays()
    return {(int(a), int(b)): int(l) for a, b, l in zip(src, dst, lab)}


def _holds(lit, h, attrs):
    va = int(attrs[lit.a][h[lit.x]])
    if va == ABSENT:
        return False
    if lit.kind == 0:
        return va == lit.c
    vb = int(attrs[lit.b][h[lit.y]])
    return vb != ABSENT and va == vb


def brute_force(graph, gfd, induced: bool = True, count: str = "all"):
    """(n_matches, sorted violations [n, k]); count="x" counts only the matches
    whose X literals all hold."""
    E = _edge_map(graph)
    k = gfd.k
    qe = {(a, b): l for (a, b, l) in gfd.edges}
    vl = graph.vlabel
    attrs = graph.attrs
    n_matches = 0
    viol = []
    for h in itertools.permutations(range(graph.n_vertices), k):
        ok = all(gfd.node_label[a] in (WILDCARD, int(vl[h[a]])) for a in range(k))
        if not ok:
            continue
        for a in range(k):
            for b in range(k):
                ql = qe.get((a, b))
                gl = E.get((h[a], h[b]))
                if ql is None and not induced:
                    continue
                if (ql is None) != (gl is None):
                    ok = False
                elif ql is not None and ql != WILDCARD and ql != gl:
                    ok = False
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        x_ok = all(_holds(l, h, attrs) for l in gfd.X)
        n_matches += 1 if (count == "all" or x_ok) else 0
        if not x_ok:
            continue
        if gfd.y_false or not all(_holds(l, h, attrs) for l in gfd.Y):
            viol.append(h)
    v = np.array(sorted(viol), dtype=np.int32).reshape(-1, k)
    return n_matches, v
