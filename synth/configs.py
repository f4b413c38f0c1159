"""The five seeded workloads: tiny, mid, batched, knowledge-graph shaped, serving.

The paper measures on the Twitch Gamers graph (first 20K nodes, 92,798 edges),
which is not available here; these synthetic power-law labelled graphs stand in
for it. Every draw uses numpy's PCG64 seeded with 20261202 + workload index.
The "sizes" argument scales a workload down (V and E divided by `scale`) for
tests that need the same structure at a size the oracle finishes quickly.
"""
from __future__ import annotations

import numpy as np

from .graphs import Graph, chung_lu_edges, graph_from_edges, zipf_values
from .gfds import GFD, Literal, SHAPES, random_pattern_gfd

SEED_BASE = 20261202


def _rng(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + index, salt])


# --------------------------------------------------------------------------- tiny
TINY_V, TINY_E, TINY_PLANTED = 20_000, 100_000, 50


def tiny_gfd() -> GFD:
    """x(L0) -[e0]-> y(L1), x -[e1]-> z(L2) with ∅ → y.A0 = z.A0."""
    return GFD([0, 1, 2], [(0, 1, 0), (0, 2, 1)], [], [Literal.var(1, 0, 2, 0)],
               False, "tiny")


def tiny(n_vertices: int = TINY_V, n_edges: int = TINY_E,
         n_planted: int = TINY_PLANTED) -> tuple[Graph, list[GFD]]:
    """Directed Chung-Lu (exponent 2.5, independent in/out permutations), 8 vertex
    labels and 4 edge labels uniform, 2 attributes uniform in [0,16).

    Planting is by construction: A0 := 0 on every L1 and L2 vertex, then
    `n_planted` gadgets are added, each a fresh x (L0) and a fresh z (L2) with
    the two edges x -[e0]-> y (y an existing L1 vertex) and x -[e1]-> z and
    nothing else, and z.A0 = 1 + (i mod 15). Each gadget is then the only match
    containing its z, and it violates y.A0 = z.A0; no other match does. The
    gadgets use 2 vertices and 2 edges each out of the V and E budget, and a
    final random renaming of the vertices hides them among the rest.
    """
    rng = _rng(0)
    vc = n_vertices - 2 * n_planted
    ec = n_edges - 2 * n_planted
    src, dst = chung_lu_edges(vc, ec, rng, 2.5, 2.5)
    elab = rng.integers(0, 4, size=ec)
    vlabel = rng.integers(0, 8, size=n_vertices)
    attrs = rng.integers(0, 16, size=(2, n_vertices)).astype(np.int64)
    xs = vc + 2 * np.arange(n_planted)
    zs = xs + 1
    vlabel[xs] = 0
    vlabel[zs] = 2
    l1 = np.flatnonzero(vlabel[:vc] == 1)
    ys = rng.choice(l1, size=n_planted, replace=False)
    attrs[0, (vlabel == 1) | (vlabel == 2)] = 0
    attrs[0, zs] = 1 + (np.arange(n_planted) % 15)
    src = np.concatenate([src, xs, xs])
    dst = np.concatenate([dst, ys, zs])
    elab = np.concatenate([elab, np.zeros(n_planted, np.int64), np.ones(n_planted, np.int64)])
    g = graph_from_edges(n_vertices, src, dst, elab, vlabel, attrs)
    g = g.permuted(rng.permutation(n_vertices))
    g.meta = {"workload": "tiny", "planted": n_planted}
    return g, [tiny_gfd()]


# ----------------------------------------------------------------- shared graph
def powerlaw_graph(index: int, n_vertices: int, n_edges: int, n_vlabels: int,
                   vlabel_s: float, n_elabels: int, n_attrs: int, attr_values: int,
                   attr_s: float, gamma_out: float = 2.5, gamma_in: float = 2.5,
                   out_cap_frac: float | None = None, name: str = "") -> Graph:
    """Directed Chung-Lu graph; Zipf vertex labels, uniform edge labels and Zipf
    attribute values (value = rank - 1)."""
    rng = _rng(index)
    src, dst = chung_lu_edges(n_vertices, n_edges, rng, gamma_out, gamma_in, out_cap_frac)
    elab = rng.integers(0, n_elabels, size=n_edges)
    vlabel = zipf_values(n_vertices, n_vlabels, vlabel_s, rng)
    attrs = np.stack([zipf_values(n_vertices, attr_values, attr_s, rng)
                      for _ in range(n_attrs)])
    g = graph_from_edges(n_vertices, src, dst, elab, vlabel, attrs)
    g.meta = {"workload": name}
    return g


# ---------------------------------------------------------------------------- mid
MID_V, MID_E = 1_000_000, 8_000_000


def mid_gfd() -> GFD:
    """Triangle x->y, y->z, x->z plus the pendant chain z->d->e (core {x,y,z},
    forest d, leaf e), with x.A1 = 7 → y.A2 = z.A2. Every node carries the most
    frequent vertex label and the edges match any edge label: with 16 edge
    labels, fixed edge labels leave almost no labelled triangles in this graph."""
    return GFD([0, 0, 0, 0, 0],
               [(0, 1, -1), (1, 2, -1), (0, 2, -1), (2, 3, -1), (3, 4, -1)],
               [Literal.const(0, 1, 7)], [Literal.var(1, 2, 2, 2)], False, "mid")


def mid(scale: int = 1) -> tuple[Graph, list[GFD]]:
    g = powerlaw_graph(1, MID_V // scale, MID_E // scale, 64, 1.2, 16, 4, 1024, 1.1,
                       name="mid")
    return g, [mid_gfd()]


# ------------------------------------------------------------------------ batched
BATCH_V, BATCH_E, BATCH_N = 4_000_000, 40_000_000, 256


BATCH_CAP = 1e8         # redraw a pattern whose expected match count exceeds this
BATCH_TOP_LABELS = 8    # node labels among the most frequent ones
BATCH_P_WILD_NODE = 0.25
BATCH_P_WILD_EDGE = 0.75


def batched_gfds(graph: Graph, n: int = BATCH_N, n_attrs: int = 4, n_elabels: int = 32,
                 seed_index: int = 2) -> list[GFD]:
    """GFDs with k uniform in 3..8 (4..8 for the 4-clique), shape uniform over
    tree / cycle / 4-clique / triangle-with-tails, one randomly oriented edge per
    skeleton pair. A node label is the wildcard with probability 1/4, else one
    of the 8 most frequent vertex labels drawn in proportion to its frequency;
    an edge label is the wildcard with probability 3/4, else uniform. X has 0-3
    literals and Y one; each is constant or variable with equal odds, constants
    drawn from the attribute distribution. A pattern whose expected match count
    under the configuration model of the graph's degrees exceeds 1e8 is redrawn
    (the paper's queries were chosen to have many embeddings, but bounded)."""
    from .estimate import DegreeMoments
    rng = _rng(seed_index, 1)
    dm = DegreeMoments(graph, n_elabels)
    freq = np.bincount(graph.vlabel, minlength=BATCH_TOP_LABELS).astype(np.float64)
    top = np.argsort(-freq, kind="stable")[:BATCH_TOP_LABELS]
    p_top = freq[top] / max(1.0, freq[top].sum())

    def draw_const():
        return zipf_values(1, 1024, 1.1, rng)[0]

    out = []
    for i in range(n):
        while True:
            shape = SHAPES[int(rng.integers(0, 4))]
            k = int(rng.integers(4 if shape == "clique4" else 3, 9))
            q = random_pattern_gfd(rng, shape, k, [0], [0], n_attrs, (0, 3), 1, draw_const,
                                   name=f"b{i}_{shape}{k}")
            q.node_label = [-1 if rng.random() < BATCH_P_WILD_NODE else int(rng.choice(top, p=p_top))
                            for _ in range(k)]
            q.edges = [(a, b, -1 if rng.random() < BATCH_P_WILD_EDGE else int(rng.integers(0, n_elabels)))
                       for (a, b, _) in q.edges]
            if dm.expected_count(q) <= BATCH_CAP:
                break
        out.append(q)
    return out


def batched(scale: int = 1, n_gfds: int = BATCH_N) -> tuple[Graph, list[GFD]]:
    g = powerlaw_graph(2, BATCH_V // scale, BATCH_E // scale, 128, 1.2, 32, 4, 1024, 1.1,
                       name="batched")
    return g, batched_gfds(g, n_gfds)


# ------------------------------------------------------------- knowledge-graph
KG_V, KG_E, KG_N = 20_000_000, 200_000_000, 32


KG_CAP = 1e8


def kg_gfds(graph: Graph, n: int = KG_N, n_elabels: int = 64, cap: float = KG_CAP) -> list[GFD]:
    """x-[e]->y, x-[e']->y', y->z1, y'->z1, y->z2, y'->z2, x->w (core
    {x,y,y',z1,z2}, leaf w). y and y' carry one of the 8 most frequent vertex
    labels (drawn by frequency), x, z1, z2 such a label or the wildcard with
    equal odds, w the wildcard; e and e' are a uniform edge label or the
    wildcard with equal odds, the shared-neighbour edges and x->w the wildcard.
    Half the GFDs are y.A0 = c1 ∧ y'.A0 = c2 → false (constants drawn from the
    attribute distribution), the others ∅ → y.A0 = y'.A0. A draw whose expected
    match count under the configuration model exceeds `cap` (1e8) is redrawn."""
    from .estimate import DegreeMoments
    rng = _rng(3, 1)
    dm = DegreeMoments(graph, n_elabels)
    freq = np.bincount(graph.vlabel, minlength=8).astype(np.float64)
    top = np.argsort(-freq, kind="stable")[:8]
    p_top = freq[top] / max(1.0, freq[top].sum())

    def lab(p_wild):
        return -1 if rng.random() < p_wild else int(rng.choice(top, p=p_top))

    out = []
    for i in range(n):
        while True:
            nl = [lab(0.5), lab(0.0), lab(0.0), lab(0.5), lab(0.5), -1]
            e1 = -1 if rng.random() < 0.5 else int(rng.integers(0, n_elabels))
            e2 = -1 if rng.random() < 0.5 else int(rng.integers(0, n_elabels))
            edges = [(0, 1, e1), (0, 2, e2), (1, 3, -1), (2, 3, -1), (1, 4, -1), (2, 4, -1), (0, 5, -1)]
            if i % 2 == 0:
                c1, c2 = (int(v) for v in zipf_values(2, 1024, 1.1, rng))
                g = GFD(nl, edges, [Literal.const(1, 0, c1), Literal.const(2, 0, c2)], [], True,
                        f"kg{i}_false")
            else:
                g = GFD(nl, edges, [], [Literal.var(1, 0, 2, 0)], False, f"kg{i}_var")
            if dm.expected_count(g) <= cap:
                break
        out.append(g)
    return out


def kg(scale: int = 1) -> tuple[Graph, list[GFD]]:
    n = KG_V // scale
    # out-weights capped so that no expected out-degree exceeds 10^6
    g = powerlaw_graph(3, n, KG_E // scale, 500, 1.3, 64, 2, 1024, 1.1,
                       gamma_out=2.28, gamma_in=2.5,
                       out_cap_frac=min(1.0, 1e6 / (KG_E // scale)), name="kg")
    return g, kg_gfds(g)


# ------------------------------------------------------------------------ serving
SERVE_RATES = (50, 200, 500, 1000, 2000)


def serving_requests(graph: Graph, n: int, seed_index: int = 4) -> list[GFD]:
    """Single-GFD requests drawn like the batched GFDs (3-8 nodes, 1-4 literals)
    with their own seed."""
    return batched_gfds(graph, n, seed_index=seed_index)


def poisson_arrivals(rate: float, n: int, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds from 0) of n requests of a Poisson process."""
    rng = _rng(4, 1000 + seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
