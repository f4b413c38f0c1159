"""Serving with continuous batching: every request's result is the same when it
runs alone (gfd_validate) and when it runs in the mix of a session, under a
memory budget small enough that requests queue and are admitted as slots free
up, with several running at once."""
import numpy as np
import pytest

from synth import configs

from gpu_util import assert_same

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")


@pytest.fixture(scope="module")
def setup():
    G.load_library()
    g, _ = configs.batched(scale=400, n_gfds=8)
    reqs = configs.serving_requests(g, 40)
    dg = G.Graph(g)
    alone = [dg.validate(q) for q in reqs]
    return g, dg, reqs, [(r.n_matches, r.violations()) for r in alone]


def test_session_results_equal_alone(setup):
    g, dg, reqs, alone = setup
    s = G.Session(dg, max_slots=6, frontier_budget_bytes=256 << 20, max_violations_hint=1 << 16)
    ids = {}
    got = {}
    peak = 0
    # submit in three bursts while the session runs
    for burst in (reqs[:10], reqs[10:25], reqs[25:]):
        for q in burst:
            ids[s.submit(q)] = len(ids)
        for _ in range(3):
            advanced, running, queued = s.step()
            peak = max(peak, advanced)
            for rid, res in s.results():
                got[ids[rid]] = (res.n_matches, res.violations())
    while len(got) < len(reqs):
        advanced, running, queued = s.step()
        peak = max(peak, advanced)
        for rid, res in s.results():
            got[ids[rid]] = (res.n_matches, res.violations())
    assert peak > 1, "requests never overlapped"
    for i in range(len(reqs)):
        assert_same(got[i], alone[i], f"request {i} {reqs[i].name}")


def test_serving_loop_and_serial(setup):
    from paper_2608_02321_gb300 import serving
    g, dg, reqs, alone = setup
    arrivals = configs.poisson_arrivals(500.0, len(reqs))
    summ, results = serving.serve(dg, reqs, arrivals, max_slots=8, budget_bytes=512 << 20,
                                  violation_hint=1 << 16, keep_results=True)
    assert summ["requests"] == len(reqs) and summ["p99_ms"] >= summ["p50_ms"] > 0
    for i, r in enumerate(results):
        assert_same((r.n_matches, r.violations()), alone[i], f"served request {i}")
    ser = serving.serve_serial(dg, reqs, arrivals)
    assert ser["matches"] == summ["matches"] == sum(a[0] for a in alone)


def test_violation_overflow_rerun_in_session(setup):
    g, dg, reqs, alone = setup
    s = G.Session(dg, max_slots=4, max_violations_hint=1)
    ids = {s.submit(q): i for i, q in enumerate(reqs[:12])}
    got = {}
    while len(got) < 12:
        s.step()
        for rid, res in s.results():
            got[ids[rid]] = (res.n_matches, res.violations())
    for i in range(12):
        assert_same(got[i], alone[i], f"overflow request {i}")
