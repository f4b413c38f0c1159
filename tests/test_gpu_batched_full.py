"""The batched workload at full size (4M vertices, 40M edges, 256 GFDs) in the
launch configuration the benchmark times (autotuned, one gfd_validate_batch of
all 256 GFDs), checked root by root against the oracle: for about 2,300
sampled (GFD, root) pairs, uniform over the label-compatible vertices, hubs of
degree >= 1000 (the top hub of every GFD's pool among them) and node-0 images of
GPU matches, the GPU's matches at the root (from the twin X = {} -> false,
validated in the same way) and its violations at the root are identical to the
oracle's; the match count of every GFD equals its twin's."""
from __future__ import annotations

import numpy as np
import pytest

from synth import configs

from full_size import compare, gpu_rows_for_roots, rows_at, sample_roots, twin

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

G = pytest.importorskip("paper_2608_02321_gb300")


def test_full_size_sampled_roots(oracle_mod):
    G.load_library()
    g, qs = configs.batched(scale=1)
    dg = G.Graph(g)
    dg.autotune(qs)
    res = dg.validate_batch(qs)
    total = sum(r.n_matches for r in res)
    tres = dg.validate_batch([twin(q) for q in qs], max_violations_hint=total + 1)
    for i, (r, t) in enumerate(zip(res, tres)):
        assert r.n_matches == t.n_matches == t.n_violations, f"gfd {i}: twin counts differ"
    degree = np.diff(g.out_off) + np.bincount(g.out_dst, minlength=g.n_vertices)
    rng = np.random.default_rng(20261203)
    samples, gpu_m = [], {}
    for i, q in enumerate(qs):          # one GFD's sorted matches on the host at a time
        t = tres[i].violations()
        samples.append(sample_roots(g, q, degree, t, rng, n_uniform=5, n_from_matches=2, n_hubs=2))
        gpu_m.update({(i, r): rows_at(t, r).copy() for r, _ in samples[i]})
        del t
    gpu_v = gpu_rows_for_roots(res, samples)
    og = oracle_mod.OracleGraph(g)
    st = compare(og, oracle_mod, qs, samples, gpu_m, gpu_v, degree, deadline=2.0, hub_deadline=4.0,
                 wall_cap=150.0)
    print("batched full-size sampled roots:", st)
    assert st["roots_done"] >= 2000, st
    assert st["hub_roots_done"] >= 50, st
    assert st["matches_compared"] >= 1000 and st["violations_compared"] >= 100, st
