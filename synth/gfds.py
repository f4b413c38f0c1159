"""GFDs φ = (Q[x̄], X → Y) and (Q[x̄], X → false) (Section II of the paper), and
seeded random patterns.

Pattern node i is variable x_i. A label of -1 is the wildcard "_". A literal is
either the constant constraint x.A = c (kind 0) or the variable constraint
x.A = y.B (kind 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WILDCARD = -1
CONST = 0
VAR = 1


@dataclass(frozen=True)
class Literal:
    kind: int          # CONST or VAR
    x: int
    a: int
    y: int = 0
    b: int = 0
    c: int = 0

    @staticmethod
    def const(x: int, a: int, c: int) -> "Literal":
        return Literal(CONST, x, a, 0, 0, c)

    @staticmethod
    def var(x: int, a: int, y: int, b: int) -> "Literal":
        return Literal(VAR, x, a, y, b, 0)


@dataclass
class GFD:
    node_label: list                      # [k]
    edges: list                           # [(src, dst, label)], directed
    X: list = field(default_factory=list)
    Y: list = field(default_factory=list)
    y_false: bool = False
    name: str = ""

    @property
    def k(self) -> int:
        return len(self.node_label)

    def relabel_nodes(self, perm) -> "GFD":
        """The same GFD with pattern node i renamed perm[i]."""
        k = self.k
        nl = [0] * k
        for i in range(k):
            nl[perm[i]] = self.node_label[i]
        edges = [(perm[s], perm[d], l) for (s, d, l) in self.edges]

        def mv(lit):
            return Literal(lit.kind, perm[lit.x], lit.a,
                           perm[lit.y] if lit.kind == VAR else 0, lit.b, lit.c)
        return GFD(nl, edges, [mv(l) for l in self.X], [mv(l) for l in self.Y],
                   self.y_false, self.name)


SHAPES = ("tree", "cycle", "clique4", "tri_tails")


def _attach_tails(rng, skel, start, k):
    for i in range(start, k):
        skel.append((int(rng.integers(0, i)), i))


def random_skeleton(rng: np.random.Generator, shape: str, k: int):
    """Undirected connected skeleton of the given shape on k nodes."""
    skel = []
    if shape == "tree":
        _attach_tails(rng, skel, 1, k)
    elif shape == "cycle":
        skel = [(i, (i + 1) % k) for i in range(k)]
    elif shape == "clique4":
        assert k >= 4
        skel = [(a, b) for a in range(4) for b in range(a + 1, 4)]
        _attach_tails(rng, skel, 4, k)
    elif shape == "tri_tails":
        assert k >= 3
        skel = [(0, 1), (1, 2), (0, 2)]
        _attach_tails(rng, skel, 3, k)
    else:
        raise ValueError(shape)
    return skel


def random_literal(rng, k, n_attrs, draw_const):
    if rng.random() < 0.5:
        return Literal.const(int(rng.integers(0, k)), int(rng.integers(0, n_attrs)),
                             int(draw_const()))
    return Literal.var(int(rng.integers(0, k)), int(rng.integers(0, n_attrs)),
                       int(rng.integers(0, k)), int(rng.integers(0, n_attrs)))


def random_pattern_gfd(rng: np.random.Generator, shape: str, k: int, vlabels, elabels,
                       n_attrs: int, n_x, n_y: int, draw_const, p_both_dirs: float = 0.0,
                       y_false: bool = False, permute: bool = True, name: str = "") -> GFD:
    """A GFD whose pattern has the given skeleton shape; each skeleton pair gets one
    randomly oriented edge (or, with probability p_both_dirs, both directions),
    node labels are drawn from `vlabels` and edge labels from `elabels`."""
    skel = random_skeleton(rng, shape, k)
    edges = []
    for (a, b) in skel:
        if rng.random() < p_both_dirs:
            edges.append((a, b, int(rng.choice(elabels))))
            edges.append((b, a, int(rng.choice(elabels))))
        elif rng.random() < 0.5:
            edges.append((a, b, int(rng.choice(elabels))))
        else:
            edges.append((b, a, int(rng.choice(elabels))))
    node_label = [int(rng.choice(vlabels)) for _ in range(k)]
    nx = int(rng.integers(n_x[0], n_x[1] + 1)) if isinstance(n_x, tuple) else int(n_x)
    X = [random_literal(rng, k, n_attrs, draw_const) for _ in range(nx)]
    Y = [] if y_false else [random_literal(rng, k, n_attrs, draw_const) for _ in range(n_y)]
    g = GFD(node_label, edges, X, Y, y_false, name or f"{shape}{k}")
    if permute:
        g = g.relabel_nodes([int(p) for p in rng.permutation(k)])
    return g
