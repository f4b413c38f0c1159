"""Failure detection without a GPU fault: a device-side time limit that runs
out, a frontier budget and an allocation that do not fit, and cancelled serving
requests. Each case must end with a clean error code (or, for a cancellation,
no result) and leave the context usable: the next call on the same graph gives
the oracle's answer. Nothing here faults, traps or hangs the GPU; the time
limit is the enumeration's own bounded exit (the control step stops every slot
and the grid barrier releases every block)."""
import os

import numpy as np
import pytest

from synth import configs

from gpu_util import assert_same, gpu_graph

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")


@pytest.fixture(scope="module")
def workload(oracle_mod):
    G.load_library()
    g, _ = configs.batched(scale=400, n_gfds=1)
    qs = [q for q in configs.batched_gfds(g, 24) if q.k >= 4][:12]
    want = [oracle_mod.validate(g, q, threads=8) for q in qs]
    return g, qs, want


def _check_all(res, want, what):
    for i, r in enumerate(res):
        assert_same((r.n_matches, r.violations()), want[i], f"{what} gfd {i}")


class _env:
    def __init__(self, name, value):
        self.name, self.value = name, value

    def __enter__(self):
        self.old = os.environ.get(self.name)
        os.environ[self.name] = self.value

    def __exit__(self, *exc):
        if self.old is None:
            del os.environ[self.name]
        else:
            os.environ[self.name] = self.old


@pytest.mark.parametrize("flags", [0, "host_loop"])
def test_run_limit_runs_out_then_next_call_is_exact(workload, flags):
    g, qs, want = workload
    flags = G.FLAG_HOST_LOOP if flags == "host_loop" else 0
    dg = gpu_graph(g)
    ref = dg.validate_batch(qs, chunk_rows=1024, flags=flags)
    assert ref[0].stat(G.STAT_STEPS) > 2, "the batch must need several enumeration steps"
    with _env("GFD_RUN_LIMIT_MS", "0"):
        with pytest.raises(G.GfdError) as e:
            dg.validate_batch(qs, chunk_rows=1024, flags=flags)
    assert e.value.code == G.GFD_ERR_TIMEOUT
    _check_all(dg.validate_batch(qs, chunk_rows=1024, flags=flags), want, "after timeout")


def test_frontier_budget_too_small(workload):
    g, qs, want = workload
    dg = gpu_graph(g)
    for budget in (1, 64 << 10):
        with pytest.raises(G.GfdError) as e:
            dg.validate_batch(qs, frontier_budget_bytes=budget)
        assert e.value.code == G.GFD_ERR_OUT_OF_MEMORY
        assert "frontier budget" in str(e.value)
    _check_all(dg.validate_batch(qs), want, "after a refused budget")
    # a budget that holds the minimum is accepted and exact
    _check_all(dg.validate_batch(qs, frontier_budget_bytes=len(qs) << 20), want, "small budget")


def test_allocation_failure_is_reported(workload):
    g, qs, want = workload
    dg = gpu_graph(g)
    with pytest.raises(G.GfdError) as e:
        dg.validate_batch(qs, max_violations_hint=1 << 42)   # an arena of ~150 TB
    assert e.value.code == G.GFD_ERR_OUT_OF_MEMORY
    _check_all(dg.validate_batch(qs), want, "after an allocation failure")


def test_batch_over_the_slot_limit_is_refused(workload):
    """A call over GFD_MAX_SLOTS GFDs is refused before any device work (its
    steps would number their tiles past 32 bits); the graph stays usable."""
    g, qs, want = workload
    dg = gpu_graph(g)
    with pytest.raises(G.GfdError) as e:
        dg.validate_batch([qs[0]] * (G.MAX_SLOTS + 1))
    assert e.value.code == G.GFD_ERR_UNSUPPORTED
    with pytest.raises(G.GfdError) as e:
        G.Session(dg, max_slots=G.MAX_SLOTS + 1)
    assert e.value.code == G.GFD_ERR_INVALID_ARG
    _check_all(dg.validate_batch(qs), want, "after a refused batch")


def _drain(s, limit=100000):
    out = {}
    for _ in range(limit):
        _, running, queued = s.step()
        for rid, r in s.results():
            out[rid] = (r.n_matches, r.violations())
        if running == 0 and queued == 0:
            return out
    raise AssertionError("session did not finish")


def test_session_cancel(workload):
    g, qs, want = workload
    dg = gpu_graph(g)
    s = G.Session(dg, max_slots=2, max_violations_hint=1 << 16)
    ids = [s.submit(q) for q in qs[:6]]
    advanced, running, queued = s.step()
    assert advanced == 2 and queued == 4
    cancelled = {ids[0], ids[4]}      # one admitted first, one still queued
    for rid in cancelled:
        s.cancel(rid)
    with pytest.raises(G.GfdError) as e:
        s.cancel(12345)
    assert e.value.code == G.GFD_ERR_INVALID_ARG
    got = _drain(s)
    assert set(got) == set(ids) - cancelled
    for rid in got:
        assert_same(got[rid], want[ids.index(rid)], f"request {rid}")
    with pytest.raises(G.GfdError):
        s.cancel(ids[1])               # already collected
    # the session keeps working after cancellations
    rid = s.submit(qs[0])
    got = _drain(s)
    assert_same(got[rid], want[0], "resubmitted")


def test_session_budget_too_small_runs_one_at_a_time(workload):
    """A budget below one request's memory: requests are admitted one at a
    time into the idle device (never two at once) and stay exact."""
    g, qs, want = workload
    dg = gpu_graph(g)
    s = G.Session(dg, max_slots=4, frontier_budget_bytes=1 << 20, max_violations_hint=1 << 16)
    ids = [s.submit(q) for q in qs[:5]]
    got = {}
    for _ in range(100000):
        advanced, running, queued = s.step()
        assert advanced <= 1
        for rid, r in s.results():
            got[rid] = (r.n_matches, r.violations())
        if running == 0 and queued == 0:
            break
    assert set(got) == set(ids)
    for rid in ids:
        assert_same(got[rid], want[ids.index(rid)], f"request {rid}")
