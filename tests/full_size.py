"""Sampled-root parity at full size: the GPU's complete outputs of one launch
against the oracle run root by root.

For a GFD phi its twin X = {} -> false has every match as a violation
(Section II: nothing satisfies false), so validating the twin lists all matches
h as tuples. For a sampled root vertex r (an image of pattern node 0) the
oracle, restricted to r, enumerates exactly the matches with h(x_0) = r; the GPU
rows with first column r must be the same tuples, and the violations of phi
among them (the oracle's literal check on those matches) must be the GPU's
violations of phi with first column r. Roots are drawn per GFD from three
strata: uniformly from the label-compatible vertices (no degree cap), from the
high-degree vertices (hubs), and from the node-0 images of the GPU's own
matches (roots with work to compare). A root the oracle does not finish within
its deadline is skipped and counted."""
from __future__ import annotations

import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from synth.gfds import GFD


def twin(q) -> GFD:
    return GFD(list(q.node_label), list(q.edges), [], [], True, q.name + "_matches")


def swap_perm(k: int, root_node: int) -> list:
    """The involution exchanging pattern nodes 0 and root_node: the oracle,
    which starts every search at node 0, then starts at root_node (its result
    is invariant under relabelling the pattern; a pinned invariant)."""
    p = list(range(k))
    p[0], p[root_node] = root_node, 0
    return p


def reorder(t: np.ndarray, perm) -> np.ndarray:
    """Tuples of the relabelled pattern (column j = old node perm[j]), sorted."""
    if t.shape[0] == 0:
        return t[:, perm]
    u = t[:, perm]
    return u[np.lexsort(u.T[::-1])]


def rows_at(t: np.ndarray, root: int) -> np.ndarray:
    """Rows of a lexicographically sorted tuple array whose first column is root."""
    if t.shape[0] == 0:
        return t
    lo = np.searchsorted(t[:, 0], root, "left")
    hi = np.searchsorted(t[:, 0], root, "right")
    return t[lo:hi]


def sample_roots(g, q, degree, gpu_matches, rng, n_uniform, n_from_matches, n_hubs,
                 hub_min=1000, min_degree=0):
    """[(root, kind)] for one GFD: uniform, match-image and hub roots (images
    of pattern node 0; degree is the array that defines hubs and min_degree)."""
    L = q.node_label[0]
    pool = np.arange(g.n_vertices, dtype=np.int64) if L < 0 else np.flatnonzero(g.vlabel == L)
    if min_degree:
        pool = pool[degree[pool] >= min_degree]
    out = []
    if pool.size:
        for r in rng.choice(pool, size=min(n_uniform, pool.size), replace=False):
            out.append((int(r), "uniform"))
    if gpu_matches.shape[0]:
        imgs = np.unique(gpu_matches[:, 0])
        for r in rng.choice(imgs, size=min(n_from_matches, imgs.size), replace=False):
            out.append((int(r), "match"))
    hubs = pool[degree[pool] >= hub_min]
    if hubs.size and n_hubs:
        order = hubs[np.argsort(-degree[hubs], kind="stable")]
        pick = [order[0]]                                  # the top hub of the pool
        rest = order[1:]
        if rest.size:
            pick += list(rng.choice(rest, size=min(n_hubs - 1, rest.size), replace=False))
        for r in pick:
            out.append((int(r), "hub"))
    seen, uniq = set(), []
    for r, kind in out:
        if r not in seen:
            seen.add(r)
            uniq.append((r, kind))
    return uniq


def gpu_rows_for_roots(results, samples, perm=None):
    """{(gfd, root): sorted rows} for the sampled roots, fetching one GFD's
    sorted tuples at a time (keeps host memory to the largest GFD); with perm,
    in the column order of the relabelled pattern."""
    out = {}
    for i, r in enumerate(results):
        t = r.violations()
        if perm is not None:
            t = reorder(t, perm[i])
        for root, _ in samples[i]:
            out[(i, root)] = rows_at(t, root).copy()
        del t
    return out


def compare(og, oracle_mod, qs, samples, gpu_matches, gpu_viol, degree, deadline=2.0,
            hub_deadline=4.0, wall_cap=120.0, threads=None):
    """Run the oracle root by root (the twin, then the literal check of the GFD
    on its matches) and compare with the GPU's rows. Returns statistics."""
    tasks = [(i, r, kind) for i in range(len(qs)) for (r, kind) in samples[i]]
    tasks.sort(key=lambda t: t[2] == "hub")          # hubs last: the cap drops them first
    end = time.monotonic() + wall_cap
    twins = [twin(q) for q in qs]
    failures = []

    def run(task):
        i, r, kind = task
        left = end - time.monotonic()
        if left <= 0:
            return None
        nm, m_or, done = oracle_mod.validate_within(og, twins[i], np.array([r], np.int32),
                                                    min(hub_deadline if kind == "hub" else deadline, left))
        if done != 1:
            return None
        m_gpu = gpu_matches[(i, r)]
        v_or = oracle_mod.sort_tuples(oracle_mod.violating(og, qs[i], m_or))
        v_gpu = gpu_viol[(i, r)]
        if nm != m_gpu.shape[0] or not np.array_equal(m_or, m_gpu) or not np.array_equal(v_or, v_gpu):
            failures.append((i, qs[i].name, r, kind, nm, m_gpu.shape[0], v_or.shape[0], v_gpu.shape[0]))
        return (i, r, kind, nm, v_or.shape[0])

    with ThreadPoolExecutor(threads or os.cpu_count() or 8) as ex:
        res = [x for x in ex.map(run, tasks) if x is not None]
    assert not failures, f"GPU and oracle differ at {len(failures)} roots, e.g. {failures[:5]}"
    hub_done = sum(1 for (i, r, kind, _, _) in res if kind == "hub" and degree[r] >= 1000)
    return {"tasks": len(tasks), "roots_done": len(res), "hub_roots_done": hub_done,
            "matches_compared": sum(x[3] for x in res), "violations_compared": sum(x[4] for x in res),
            "roots_with_matches": sum(1 for x in res if x[3] > 0)}
