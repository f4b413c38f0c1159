"""Serving loop: requests arrive over time and are validated by one native
continuous-batching session (gfd_session_*) against the resident graph.

Requests that arrive while others are running are admitted as slots and
memory free up, and advance together with them on the device. The loop
records each request's latency (completion minus arrival) and the
throughput in matches validated per second. `serve_serial` is the
comparison: the same stream validated one request at a time with
gfd_validate, in arrival order.
"""
from __future__ import annotations

import time

import numpy as np

from . import Graph, Session


def _summary(arrivals, finish, matches, t_end):
    lat = np.asarray(finish) - np.asarray(arrivals)
    return {
        "requests": int(len(arrivals)),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "makespan_s": float(t_end),
        "matches": int(matches),
        "matches_per_s": float(matches / t_end) if t_end > 0 else 0.0,
        "requests_per_s": float(len(arrivals) / t_end) if t_end > 0 else 0.0,
    }


def serve(g: Graph, gfds, arrivals, max_slots: int = 64, budget_bytes: int = 40 << 30,
          violation_hint: int = 1 << 20, stream=None, keep_results: bool = False):
    """Run the stream through a session. Returns (summary, results) where
    results[i] is the Result of gfds[i] when keep_results is set."""
    s = Session(g, max_slots=max_slots, frontier_budget_bytes=budget_bytes,
                max_violations_hint=violation_hint, stream=stream)
    n = len(gfds)
    finish = [0.0] * n
    results = [None] * n
    owner = {}
    matches = 0
    i = 0
    peak_running = 0
    t0 = time.perf_counter()
    running = queued = 0
    while True:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            owner[s.submit(gfds[i])] = i
            i += 1
        outstanding = len(owner) - sum(1 for j in owner.values() if finish[j])
        if outstanding:
            advanced, running, queued = s.step()
            peak_running = max(peak_running, advanced)
        else:
            running = queued = 0
        done_now = s.results()
        t = time.perf_counter() - t0
        for rid, res in done_now:
            j = owner[rid]
            finish[j] = t
            matches += res.n_matches
            if keep_results:
                results[j] = res
        if all(finish) and i == n:
            break
        if running == 0 and queued == 0 and i < n and not done_now:
            wait = arrivals[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    t_end = time.perf_counter() - t0
    summary = _summary(arrivals, finish, matches, t_end)
    summary["peak_running"] = peak_running
    summary["session"] = s.stats()
    return summary, results


def serve_serial(g: Graph, gfds, arrivals, violation_hint: int = 1 << 20, stream=None):
    """The same stream, one gfd_validate call per request in arrival order."""
    n = len(gfds)
    finish = [0.0] * n
    matches = 0
    t0 = time.perf_counter()
    for j in range(n):
        wait = arrivals[j] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        r = g.validate(gfds[j], stream=stream, max_violations_hint=violation_hint)
        matches += r.n_matches
        finish[j] = time.perf_counter() - t0
    return _summary(arrivals, finish, matches, time.perf_counter() - t0)
