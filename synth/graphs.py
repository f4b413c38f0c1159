"""Seeded synthetic graphs G = (V, E, L, F_A) (Section II of the paper).

A graph is a directed edge set E ⊆ V×V with one label per vertex and per edge
and an int32 attribute tuple per vertex. Here it is stored as an out-CSR sorted
by (source, destination), which is both what the C-ABI accepts and what the
oracle reads into its own structures. The attribute value INT32_MIN stands for
"attribute absent".
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ABSENT = np.iinfo(np.int32).min


@dataclass
class Graph:
    n_vertices: int
    out_off: np.ndarray        # int64 [V+1]
    out_dst: np.ndarray        # int32 [E], sorted within each row
    out_elabel: np.ndarray     # int32 [E]
    vlabel: np.ndarray         # int32 [V]
    attrs: np.ndarray          # int32 [n_attrs][V]
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.out_dst.shape[0])

    @property
    def n_attrs(self) -> int:
        return int(self.attrs.shape[0])

    def edge_arrays(self):
        """(src, dst, label) int arrays in CSR order."""
        deg = np.diff(self.out_off)
        src = np.repeat(np.arange(self.n_vertices, dtype=np.int64), deg)
        return src, self.out_dst.astype(np.int64), self.out_elabel

    def permuted(self, perm: np.ndarray) -> "Graph":
        """The same graph with vertex v renamed perm[v]."""
        perm = np.asarray(perm, dtype=np.int64)
        src, dst, lab = self.edge_arrays()
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.shape[0])
        vlabel = self.vlabel[inv]
        attrs = self.attrs[:, inv]
        return graph_from_edges(self.n_vertices, perm[src], perm[dst], lab,
                                vlabel, attrs, dict(self.meta))


def graph_from_edges(n_vertices, src, dst, elabel, vlabel, attrs, meta=None) -> Graph:
    """Build the sorted out-CSR from an edge list with unique (src, dst) pairs."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    elabel = np.asarray(elabel, dtype=np.int32)
    key = src * np.int64(n_vertices) + dst
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.shape[0] > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate (src, dst) pair")
    s = src[order]
    counts = np.bincount(s, minlength=n_vertices).astype(np.int64)
    off = np.zeros(n_vertices + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    attrs = np.asarray(attrs, dtype=np.int32)
    if attrs.ndim != 2:
        attrs = attrs.reshape(-1, n_vertices) if n_vertices else attrs.reshape(0, 0)
    attrs = np.ascontiguousarray(attrs)
    return Graph(n_vertices, off, dst[order].astype(np.int32), elabel[order],
                 np.ascontiguousarray(np.asarray(vlabel, dtype=np.int32)), attrs,
                 meta or {})


def powerlaw_weights(n: int, gamma: float, rng: np.random.Generator,
                     cap_frac: float | None = None) -> np.ndarray:
    """Chung-Lu weights w ∝ (i+1)^(-1/(gamma-1)), placed on a random permutation of
    the vertices. With cap_frac, no weight exceeds cap_frac of the total."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
    if cap_frac is not None:
        # iterate: capping lowers the total, so re-cap until stable
        for _ in range(50):
            cap = cap_frac * w.sum()
            if w.max() <= cap * (1 + 1e-12):
                break
            w = np.minimum(w, cap)
    out = np.empty(n, dtype=np.float64)
    out[rng.permutation(n)] = w
    return out


def _sample(cdf: np.ndarray, m: int, rng: np.random.Generator) -> np.ndarray:
    """m independent draws of index i with probability ∝ cdf[i] - cdf[i-1]."""
    u = rng.random(m) * cdf[-1]
    idx = np.searchsorted(cdf, u, side="right")
    np.minimum(idx, cdf.shape[0] - 1, out=idx)
    return idx


def _sample_sorted(cdf: np.ndarray, m: int, rng: np.random.Generator) -> np.ndarray:
    """The same distribution as _sample, returned in increasing order (sorted
    uniforms make the inverse-CDF search cache friendly)."""
    u = rng.random(m)
    u.sort()
    u *= cdf[-1]
    # draws that fall in [cdf[i-1], cdf[i]) map to i
    below = np.searchsorted(u, cdf, side="left")
    counts = np.diff(below, prepend=0)
    counts[-1] += m - below[-1]
    return np.repeat(np.arange(cdf.shape[0], dtype=np.int64), counts)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    a.sort()
    if a.shape[0] == 0:
        return a
    keep = np.empty(a.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def chung_lu_edges(n: int, m: int, rng: np.random.Generator, gamma_out: float = 2.5,
                   gamma_in: float = 2.5, out_cap_frac: float | None = None):
    """Directed Chung-Lu: each candidate edge draws its source ∝ out-weight and
    its destination ∝ in-weight independently; self-loops and repeated pairs are
    dropped, more candidates are drawn until at least m distinct pairs exist,
    and a seeded uniform random subset of exactly m of them is kept."""
    if m > n * (n - 1):
        raise ValueError("too many edges")
    w_out = powerlaw_weights(n, gamma_out, rng, out_cap_frac)
    w_in = powerlaw_weights(n, gamma_in, rng)
    cdf_out = np.cumsum(w_out)
    cdf_in = np.cumsum(w_in)
    keys = np.empty(0, dtype=np.int64)
    need = m
    while True:
        batch = int(need * 1.15) + 1024
        s = _sample_sorted(cdf_out, batch, rng)[rng.permutation(batch)]   # random pairing
        d = _sample_sorted(cdf_in, batch, rng)
        k = s.astype(np.int64) * n + d
        keys = _sorted_unique(np.concatenate([keys, k[s != d]]))
        if keys.shape[0] >= m:
            break
        need = m - keys.shape[0]
    if keys.shape[0] > m:
        drop = rng.choice(keys.shape[0], keys.shape[0] - m, replace=False)
        mask = np.ones(keys.shape[0], dtype=bool)
        mask[drop] = False
        keys = keys[mask]
    return keys // n, keys % n


def zipf_values(n: int, n_values: int, s: float, rng: np.random.Generator) -> np.ndarray:
    """Values in [0, n_values) with P(value = r-1) ∝ r^(-s)."""
    p = np.arange(1, n_values + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(p)
    return _sample(cdf, n, rng).astype(np.int32)


def random_small_graph(seed: int, n_vertices: int, n_vlabels: int = 2, n_elabels: int = 2,
                       p_edge: float = 0.3, p_self: float = 0.15, n_attrs: int = 2,
                       n_attr_values: int = 3, p_absent: float = 0.1) -> Graph:
    """Tiny Erdos-Renyi style directed graph with self-loops, reverse edges, few
    labels and absent attributes: the brute-force and edge-case workload."""
    rng = np.random.default_rng(seed)
    src, dst = [], []
    for a in range(n_vertices):
        for b in range(n_vertices):
            p = p_self if a == b else p_edge
            if rng.random() < p:
                src.append(a)
                dst.append(b)
    lab = rng.integers(0, n_elabels, size=len(src))
    vlabel = rng.integers(0, n_vlabels, size=n_vertices)
    attrs = rng.integers(0, n_attr_values, size=(n_attrs, n_vertices)).astype(np.int64)
    attrs[rng.random((n_attrs, n_vertices)) < p_absent] = ABSENT
    return graph_from_edges(n_vertices, np.array(src, dtype=np.int64),
                            np.array(dst, dtype=np.int64), lab, vlabel, attrs,
                            {"kind": "small", "seed": seed})
