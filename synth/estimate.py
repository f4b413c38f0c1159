"""Expected homomorphism count of a pattern under the configuration model of a
graph's realized degrees — used only to redraw patterns whose count would
explode. Not a matcher: it never looks at which edges exist.

With P(a -> b) ≈ d_out(a) d_in(b) / E, the expected number of label-preserving
maps of Q factorizes over pattern nodes:
    E^(-|E_Q|) · Π_edges P(label) · Π_u Σ_{v: L(v) ~ L(u)} d_out(v)^{dout(u)} d_in(v)^{din(u)}.
"""
from __future__ import annotations

import numpy as np


class DegreeMoments:
    def __init__(self, graph, n_elabels: int):
        self.E = max(1, graph.n_edges)
        self.dout = np.diff(graph.out_off).astype(np.float64)
        self.din = np.bincount(graph.out_dst, minlength=graph.n_vertices).astype(np.float64)
        self.vlabel = graph.vlabel
        self.p_elabel = 1.0 / n_elabels
        self._by_label = {}
        self._cache = {}

    def _sel(self, label):
        if label not in self._by_label:
            idx = np.flatnonzero(self.vlabel == label) if label >= 0 else None
            self._by_label[label] = (self.dout if idx is None else self.dout[idx],
                                     self.din if idx is None else self.din[idx])
        return self._by_label[label]

    def moment(self, label: int, a: int, b: int) -> float:
        key = (label, a, b)
        if key not in self._cache:
            do, di = self._sel(label)
            self._cache[key] = float(np.sum(do ** a * di ** b))
        return self._cache[key]

    def expected_count(self, gfd) -> float:
        k = gfd.k
        dout = [0] * k
        din = [0] * k
        est = 1.0
        for (s, d, l) in gfd.edges:
            dout[s] += 1
            din[d] += 1
            est /= self.E
            if l >= 0:
                est *= self.p_elabel
        for u in range(k):
            est *= self.moment(gfd.node_label[u], dout[u], din[u])
        return est
