"""Test inputs shared by the oracle pins and the GPU parity tests: golden toy
fixtures, closed-form graphs and random small cases. Inputs only — no matching."""
from __future__ import annotations

import json
import os

import numpy as np

from synth.graphs import Graph, graph_from_edges, random_small_graph
from synth.gfds import GFD, Literal, random_pattern_gfd

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def lit(t):
    return Literal(int(t[0]), int(t[1]), int(t[2]), int(t[3]), int(t[4]), int(t[5]))


def gfd_from_json(d) -> GFD:
    return GFD([int(x) for x in d["node_label"]], [tuple(int(v) for v in e) for e in d["edges"]],
               [lit(t) for t in d["X"]], [lit(t) for t in d["Y"]], bool(d["y_false"]))


def graph_from_json(d) -> Graph:
    e = np.array(d["edges"], dtype=np.int64).reshape(-1, 3)
    return graph_from_edges(d["n"], e[:, 0], e[:, 1], e[:, 2], d["vlabel"],
                            np.array(d["attrs"], dtype=np.int64))


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def golden_cases():
    """[(name, graph, gfd, n_matches, violations)] from tests/golden/*.json."""
    out = []
    for fn in sorted(os.listdir(GOLDEN)):
        if not fn.endswith(".json"):
            continue
        d = load_golden(fn)
        if "graph" not in d:
            continue
        g = graph_from_json(d["graph"])
        cases = d.get("cases") or [{"gfd": d["gfd"], "expected": d["expected"]}]
        for i, c in enumerate(cases):
            exp = c["expected"]
            v = np.array(exp["violations"], dtype=np.int32).reshape(-1, len(c["gfd"]["node_label"]))
            out.append((f"{fn[:-5]}#{i}", g, gfd_from_json(c["gfd"]), exp["n_matches"], v))
    return out


def edges_graph(n, edges, vlabel=None, attrs=None):
    e = np.array(edges, dtype=np.int64).reshape(-1, 3)
    vlabel = np.zeros(n, np.int32) if vlabel is None else vlabel
    attrs = np.zeros((1, n), np.int64) if attrs is None else attrs
    return graph_from_edges(n, e[:, 0], e[:, 1], e[:, 2], vlabel, attrs)


def complete_bidirected(n):
    return edges_graph(n, [(a, b, 0) for a in range(n) for b in range(n) if a != b])


def out_star(d, extra=()):
    """Centre 0 with edges 0 -> 1..d, plus `extra` edges."""
    return edges_graph(d + 1, [(0, i, 0) for i in range(1, d + 1)] + list(extra))


def directed_cycle(n):
    return edges_graph(n, [(i, (i + 1) % n, 0) for i in range(n)])


def undirected_q(k, pairs, label=0):
    """Pattern with both directions on every skeleton pair (undirected queries)."""
    edges = []
    for a, b in pairs:
        edges += [(a, b, label), (b, a, label)]
    return GFD([0] * k, edges, [], [], False)


def star_q(s):
    return GFD([0] * (s + 1), [(0, i, 0) for i in range(1, s + 1)], [], [], False)


def _induced_pattern(rng, g, k):
    """Pattern copied from the subgraph of G induced by k random vertices (so it
    has at least one match), some labels generalised to the wildcard."""
    src, dst, lab = g.edge_arrays()
    E = {(int(a), int(b)): int(l) for a, b, l in zip(src, dst, lab)}
    for _ in range(50):
        vs = [int(v) for v in rng.choice(g.n_vertices, size=k, replace=False)]
        edges = []
        for i, a in enumerate(vs):
            for j, b in enumerate(vs):
                if (a, b) in E:
                    l = E[(a, b)] if rng.random() > 0.3 else -1
                    edges.append((i, j, l))
        # connected?
        seen, stack = {0}, [0]
        while stack:
            x = stack.pop()
            for (i, j, _) in edges:
                for (p, q) in ((i, j), (j, i)):
                    if p == x and q not in seen:
                        seen.add(q)
                        stack.append(q)
        if len(seen) == k:
            nl = [int(g.vlabel[v]) if rng.random() > 0.3 else -1 for v in vs]
            return nl, edges
    return None


def random_case(seed, max_k=4, n_vertices=None):
    """A random tiny graph (self-loops, reverse edges, absent attributes) and a
    random connected GFD on it (wildcards, both directions, self-loops); most
    patterns are copied from an induced subgraph of G so that matches exist."""
    rng = np.random.default_rng([777, seed])
    n = int(n_vertices or rng.integers(5, 8))
    g = random_small_graph(seed, n, n_vlabels=int(rng.integers(1, 3)),
                           n_elabels=int(rng.integers(1, 3)), p_edge=float(rng.uniform(0.2, 0.5)),
                           p_self=0.1, n_attrs=2, n_attr_values=3, p_absent=0.15)
    k = int(rng.integers(1, max_k + 1))
    planted = _induced_pattern(rng, g, k) if rng.random() < 0.7 else None
    if planted is not None:
        nl, edges = planted
        gfd = GFD(nl, edges, [], [], False)
        tmp = random_pattern_gfd(rng, "tree", k, [0], [0], 2, (0, 2), 1,
                                 lambda: int(rng.integers(0, 3)), permute=False)
        gfd.X, gfd.Y = tmp.X, tmp.Y
        gfd.y_false = bool(rng.random() < 0.2)
        if gfd.y_false:
            gfd.Y = []
        return g, gfd
    shape = ["tree", "cycle", "tri_tails", "clique4"][int(rng.integers(0, 4))]
    k = int(rng.integers(4 if shape == "clique4" else (3 if shape != "tree" else 1), max_k + 1))
    gfd = random_pattern_gfd(rng, shape, k, [0, 1, -1], [0, 1, -1], 2, (0, 2), 1,
                             lambda: int(rng.integers(0, 3)), p_both_dirs=0.3,
                             y_false=bool(rng.random() < 0.2))
    # occasionally a pattern self-loop
    if rng.random() < 0.25:
        a = int(rng.integers(0, k))
        gfd.edges.append((a, a, int(rng.choice([0, 1, -1]))))
    return g, gfd


def random_disconnected_case(seed, max_k=4):
    """A random tiny graph and a GFD whose pattern has at least two connected
    components: the subgraph of G induced by k random vertices (kept only when
    it is disconnected), labels partly generalised, random literals."""
    rng = np.random.default_rng([779, seed])
    while True:
        n = int(rng.integers(5, 8))
        g = random_small_graph(10000 + seed, n, n_vlabels=int(rng.integers(1, 3)),
                               n_elabels=int(rng.integers(1, 3)), p_edge=float(rng.uniform(0.1, 0.35)),
                               p_self=0.1, n_attrs=2, n_attr_values=3, p_absent=0.15)
        src, dst, lab = g.edge_arrays()
        E = {(int(a), int(b)): int(l) for a, b, l in zip(src, dst, lab)}
        for _ in range(50):
            k = int(rng.integers(2, max_k + 1))
            vs = [int(v) for v in rng.choice(g.n_vertices, size=k, replace=False)]
            edges = [(i, j, E[(a, b)] if rng.random() > 0.3 else -1)
                     for i, a in enumerate(vs) for j, b in enumerate(vs) if (a, b) in E]
            seen, stack = {0}, [0]
            while stack:
                x = stack.pop()
                for (i, j, _) in edges:
                    for (p, q) in ((i, j), (j, i)):
                        if p == x and q not in seen:
                            seen.add(q)
                            stack.append(q)
            if len(seen) < k:
                nl = [int(g.vlabel[v]) if rng.random() > 0.3 else -1 for v in vs]
                gfd = GFD(nl, edges, [], [], False)
                tmp = random_pattern_gfd(rng, "tree", k, [0], [0], 2, (0, 2), 1,
                                         lambda: int(rng.integers(0, 3)), permute=False)
                gfd.X, gfd.Y = tmp.X, tmp.Y
                gfd.y_false = bool(rng.random() < 0.2)
                if gfd.y_false:
                    gfd.Y = []
                return g, gfd
        seed += 1000
