#!/usr/bin/env python
"""Benchmark: matches validated per second, batched vs per-GFD, on one GB300.

A step validates the whole GFD batch of the workload against the resident
graph through the C-ABI (gfd_validate_batch): candidate filter, refinement,
index build, core-first enumeration and literal check, all in the library's
CUDA kernels. `value` is whole-job matches/s with the graph already resident;
`e2e` adds, every step, the host-side GFD descriptions going in and the sorted
violation tuples coming back to host memory. `plain` times the same GFDs as
one gfd_validate call each. `--impl reference` times the CPU oracle instead,
on a bounded root sample of the same workload.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one process per GPU, each validating its own replica of
the workload (no data-path collective; the batch does not need one).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matches validated/s, batched vs per-GFD; p50/p99 request latency (1 GB300)"
UNIT = "matches/s"
SRC_ENUM = os.path.join(ROOT, "paper_2608_02321_gb300", "csrc", "enumerate.cu")
PROFILE_NOTE = os.path.join(ROOT, "profiles", "enumerate_batched.md")


# ------------------------------------------------------------------ workloads
def make_workload(name: str, scale: int):
    from synth import configs
    if name == "batched":
        g, qs = configs.batched(scale=scale)
        desc = (f"batched: {g.n_vertices} vertices, {g.n_edges} edges, 128 vertex labels Zipf(1.2), "
                f"32 edge labels, 4 attributes Zipf(1.1); {len(qs)} GFDs of 3-8 nodes "
                f"(tree/cycle/4-clique/triangle-with-tails), 0-3 X literals, 1 Y literal")
    elif name == "mid":
        g, qs = configs.mid(scale=scale)
        desc = f"mid: {g.n_vertices} vertices, {g.n_edges} edges, one 5-node GFD"
    elif name == "tiny":
        g, qs = configs.tiny()
        desc = f"tiny: {g.n_vertices} vertices, {g.n_edges} edges, one 3-node GFD, 50 planted violations"
    elif name == "kg":
        g, qs = configs.kg(scale=scale)
        desc = f"kg: {g.n_vertices} vertices, {g.n_edges} edges, {len(qs)} 6-node GFDs"
    else:
        raise SystemExit(f"unknown workload {name}")
    return g, qs, desc


def literal_attrs(q) -> int:
    s = set()
    for l in list(q.X) + list(q.Y):
        s.add((l.x, l.a))
        if l.kind == 1:
            s.add((l.y, l.b))
    return len(s)


def gfd_bytes(q) -> int:
    return 4 * q.k + 12 * len(q.edges) + 24 * (len(q.X) + len(q.Y)) + 64


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
ROOT_SAMPLE_SEED = 20261205
ROOTS_PER_GFD = 384
ROOTS_PER_TASK = 64
TASK_DEADLINE_S = 2.0


def fixed_root_tasks(g, qs, per_gfd: int = ROOTS_PER_GFD, seed: int = ROOT_SAMPLE_SEED):
    """The seeded root sample both CPU legs time: per GFD, `per_gfd` vertices
    drawn uniformly (images of pattern node 0), in tasks of ROOTS_PER_TASK."""
    rng = np.random.default_rng(seed)
    tasks = []
    for i in range(len(qs)):
        roots = rng.integers(0, g.n_vertices, size=per_gfd).astype(np.int32)
        tasks += [(i, roots[a:a + ROOTS_PER_TASK]) for a in range(0, per_gfd, ROOTS_PER_TASK)]
    return tasks


def oracle_sample(g, qs, threads: int, og=None, tasks=None):
    """The oracle, as it stands, over the fixed root sample on `threads` host
    threads; each task (ROOTS_PER_TASK roots of one GFD) has TASK_DEADLINE_S, and
    the roots after the one in progress at its deadline are dropped with their
    matches (the time is still counted). Returns (matches, wall seconds, roots
    searched to the end, roots dropped)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle
    og = og or oracle.OracleGraph(g)
    tasks = tasks if tasks is not None else fixed_root_tasks(g, qs)

    def run(task):
        i, rs = task
        return oracle.count_within(og, qs[i], rs, TASK_DEADLINE_S)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(run, tasks))
    wall = time.perf_counter() - t0
    done = sum(r[1] for r in res)
    return sum(r[0] for r in res), wall, done, sum(len(t[1]) for t in tasks) - done


def workload_config(desc: str, n_gpus: int) -> dict:
    """The `config` of a bench line (the same for the GPU and the reference arm)."""
    return {"workload": desc, "l2": "inputs larger than L2 and a 512 MB L2 flush before every timed step",
            "parallelism": "replicas" if n_gpus > 1 else "single GPU"}


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, g, qs, desc):
    """The oracle, as it stands, on the host cores: every step times the same
    fixed root sample (the one the GPU arm's cpu_baseline times)."""
    from oracle import oracle
    threads = cpu_threads()
    og = oracle.OracleGraph(g)
    tasks = fixed_root_tasks(g, qs)
    for w in range(args.warmup):
        oracle_sample(g, qs, threads, og, tasks[: max(1, len(tasks) // 8)])
    vals, tot_m, tot_t, done, dropped = [], 0, 0.0, 0, 0
    for s in range(args.steps):
        m, t, d, x = oracle_sample(g, qs, threads, og, tasks)
        vals.append(m / t if t > 0 else 0.0)
        tot_m, tot_t, done, dropped = tot_m + m, tot_t + t, d, x
    value = tot_m / tot_t if tot_t > 0 else 0.0
    sample = (f"fixed seeded sample: {ROOTS_PER_GFD} uniform root vertices (images of pattern node 0) per GFD, "
              f"{len(qs)} GFDs, {done} roots searched to the end and {dropped} dropped at their "
              f"task deadlines ({ROOTS_PER_TASK} roots, {TASK_DEADLINE_S:.0f} s each); "
              f"{tot_m // max(1, args.steps)} matches per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": workload_config(desc, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample, "spread": [min(vals), max(vals)] if vals else None},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ranks
def aggregate(step_ms: float, matches: int, dist=None, device: str = "cpu"):
    """Whole-job figures over the ranks of a replicated run: the step time is
    the slowest rank's, the throughput all ranks' matches over that time."""
    import torch
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    m = torch.tensor([float(matches)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(m, op=dist.ReduceOp.SUM)
    step_max = float(t.item())
    return step_max, float(m.item()) / (step_max / 1000.0)


# ------------------------------------------------------------------ GPU arm
def kernel_traffic(work_items: int):
    """DRAM bytes of one enumeration launch: the traffic per work item of the
    committed small-case ncu capture (one kernel, one launch, a few GB on the
    device) times this launch's work items, if the capture was taken on the
    current source of that kernel; else None."""
    try:
        text = open(PROFILE_NOTE).read()
    except OSError:
        return None
    sha = hashlib.sha256(open(SRC_ENUM, "rb").read()).hexdigest()[:16]
    t = None
    s = None
    for ln in text.splitlines():
        if ln.startswith("traffic_bytes_per_work_item:"):
            t = float(ln.split(":", 1)[1].split()[0])
        if ln.startswith("source_sha256_16:"):
            s = ln.split(":", 1)[1].strip()
    return t * work_items if (t is not None and s == sha) else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfd", choices=["gfd", "reference"])
    ap.add_argument("--workload", default="batched", choices=["batched", "mid", "tiny", "kg"])
    ap.add_argument("--scale", type=int, default=1, help="divide V and E (tests only)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-non-induced", action="store_true",
                    help="skip the non-induced, X-pushdown and disconnected-pattern legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flags", type=int, default=0)
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="frontier budget in GiB (0: the library default)")
    ap.add_argument("--hint", type=int, default=1 << 26,
                    help="violation records stored per call before a re-run")
    ap.add_argument("--serve-rates", default="50,200,500,1000,2000",
                    help="Poisson arrival rates (req/s) of the serving leg; empty: skip")
    ap.add_argument("--serve-requests", type=int, default=3000,
                    help="requests per arrival rate (at most --serve-seconds of arrivals)")
    ap.add_argument("--serve-seconds", type=float, default=12.0)
    ap.add_argument("--n-gfds", type=int, default=0, help="validate only the first N GFDs (profiling)")
    ap.add_argument("--no-autotune", action="store_true", help="skip gfd_autotune before the warm-up")
    ap.add_argument("--kernel-variant", type=int, default=0, help="fixed enumeration kernel variant (1-6)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        g, qs, desc = make_workload(args.workload, args.scale)
        run_reference(args, g, qs, desc)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_2608_02321_gb300 as G
    G.load_library(build_if_missing=False)
    g, qs, desc = make_workload(args.workload, args.scale)
    if args.n_gfds:
        qs = qs[:args.n_gfds]
        desc += f" (first {len(qs)} GFDs only)"
    stream = torch.cuda.current_stream()
    dg = G.Graph(g, stream=stream)
    flags = G.FLAG_PROFILE | args.flags
    hint = args.hint   # violation records stored per call (all GFDs together)
    l2_flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    budget = int(args.budget_gb * (1 << 30))

    def step():
        return dg.validate_batch(qs, stream=stream, flags=flags, max_violations_hint=hint,
                                 frontier_budget_bytes=budget, kernel_variant=args.kernel_variant)

    tuned = None
    if not args.no_autotune and not args.kernel_variant:
        # untimed: pick the enumeration-kernel variant and frontier budget
        tuned = dg.autotune(qs, stream=stream, max_violations_hint=hint,
                            frontier_budget_bytes=budget)
    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    times, enum_ms, enum_launches, launches, phase_ms = [], [], 0, 0, []
    stats = None
    for _ in range(args.steps):
        l2_flush.zero_()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        ms, nl = res[0].profile(G.PROF_ENUM)
        enum_ms.append(ms)
        enum_launches += 1
        launches += sum(res[0].profile(w)[1] for w in range(4))
        phase_ms.append([res[0].profile(w)[0] for w in range(4)])
        stats = res
    clk = clocks.stop()
    matches = sum(r.n_matches for r in stats)
    viols = sum(r.n_violations for r in stats)
    work = sum(r.stat(G.STAT_WORK) for r in stats)
    rows = sum(r.stat(G.STAT_ROWS) for r in stats)
    probes = stats[0].stat(G.STAT_PROBES)
    enum_steps = stats[0].stat(G.STAT_STEPS)
    step_ms = float(np.mean(times))
    step_ms_max, value = aggregate(step_ms, matches, dist, "cuda")

    # counting pass (untimed): what the run's kernels read, for the byte model
    cres = dg.validate_batch(qs, stream=stream, flags=flags | G.FLAG_COUNT, max_violations_hint=hint,
                             frontier_budget_bytes=budget, kernel_variant=args.kernel_variant)
    cnt = cres[0].counters()
    nnz = sum(r.stat(G.STAT_INDEX) for r in cres)
    V = g.n_vertices
    out_bytes = sum(4 * r.k * r.n_violations for r in stats)
    # The algorithmic-byte model of the hot path (filter, refinement, index,
    # enumeration, literal check, output), with the counted quantities:
    model = {
        "filter": 10 * V * cnt["filter_keys"],                         # label + two offsets per vertex and key
        "bitmaps": V // 8 * cnt["bitmaps"],                            # one candidate bitmap per compaction
        "refine_index_scans": 8 * cnt["scan_cands"] + 5 * cnt["scan_entries"],  # offsets + (id, label) per entry
        "index_lists": 8 * nnz,                                        # 2 x 4 B per index entry
        "enum_index_reads": 4 * cnt["items"],                          # 4 B per entry of N_u
        "enum_back_scans": 5 * cnt["back_deg"],                        # backward non-tree adjacency, 5 B per entry
        "enum_negative_probes": 32 * cnt["neg_logd"],                  # one sector per binary-search step
        "literal_reads": 32 * cnt["attr_reads"],                       # one sector per attribute read
        "output": out_bytes,                                           # 4k B per violation
    }
    b_enum = (model["enum_index_reads"] + model["enum_back_scans"] + model["enum_negative_probes"]
              + model["literal_reads"] + model["output"])
    b_step = sum(model.values())
    # what the kernel itself loads: 8 B per index entry (position, id), 16 B
    # per signature, one sector per search step actually taken and per
    # attribute, the partial matches written, the output
    b_kernel = (8 * cnt["items"] + 16 * cnt["sig_loads"] + 32 * cnt["search_loads"] + 32 * cnt["attr_reads"]
                + 8 * cnt["rows"] + out_bytes)
    t_enum = float(np.mean(enum_ms)) / 1000.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = b_enum / t_enum / 1e9 if t_enum > 0 else 0.0
    traffic = kernel_traffic(work)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if peak else None, "traffic": traffic,
                "traffic_source": "ncu DRAM bytes per work item of a small capture x this launch's work items",
                "kernel": "k_persistent (enumeration)", "launch_ms": t_enum * 1000,
                "model": "algorithmic bytes (index reads 4 B per N_u entry, "
                         "backward non-tree adjacency 5 B per entry, 32 B per binary-search step of an absent-edge "
                         "probe, 32 B per literal attribute read, 4k B per violation), counted by an untimed "
                         "counting pass of the same launch",
                "alg_bytes_per_launch": b_enum,
                "dram_frac": (traffic / t_enum / 1e9 / peak) if (traffic and t_enum > 0 and peak) else None,
                "kernel_loads_model": {"bytes": b_kernel, "frac": b_kernel / t_enum / 1e9 / peak if t_enum > 0 else None},
                "step_model": {"bytes": b_step, "frac": b_step / (step_ms / 1000.0) / 1e9 / peak,
                               "terms": model},
                "counters": cnt,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    # e2e: host GFDs in, sorted violation tuples back on the host (one untimed
    # warm-up call first)
    G.violations_all(step())
    e2e_times = []
    d2h = 0
    for _ in range(max(1, min(3, args.steps))):
        l2_flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = step()
        d2h = 0
        for v in G.violations_all(res):   # one sort and one copy for the whole batch
            d2h += v.nbytes + 16
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_times))
    e2e = {"value": matches / e2e_s, "unit": UNIT, "h2d_bytes_per_step": sum(gfd_bytes(q) for q in qs),
           "d2h_bytes_per_step": d2h, "ms_per_step": 1000 * e2e_s,
           "includes": "validate_batch from host GFDs + one device sort and copy of all violation tuples"}

    plain = None
    if not args.no_plain and len(qs) > 1:
        ptimes = []
        for _ in range(max(1, min(2, args.steps))):
            l2_flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pm = 0
            for q in qs:
                r = dg.validate(q, stream=stream, max_violations_hint=hint)
                pm += r.n_matches
            e1.record(stream)
            torch.cuda.synchronize()
            ptimes.append(e0.elapsed_time(e1))
        pms = float(np.mean(ptimes))
        plain = {"value": pm / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms,
                 "launch": f"{len(qs)} gfd_validate calls per step"}

    # the non-induced matching mode (GFD_FLAG_NON_INDUCED) on the same batch:
    # a different result (supersets of the matches and violations), reported
    # beside the headline, never in place of it
    non_induced = None
    push_x = None
    for leg, extra_flag in (("non_induced", G.FLAG_NON_INDUCED), ("push_x", G.FLAG_PUSH_X)):
        if args.no_non_induced:
            break
        nflags = flags | extra_flag
        res = dg.validate_batch(qs, stream=stream, flags=nflags, max_violations_hint=hint,
                                frontier_budget_bytes=budget, kernel_variant=args.kernel_variant)
        ntimes, nenum = [], []
        for _ in range(max(1, min(2, args.steps))):
            l2_flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = dg.validate_batch(qs, stream=stream, flags=nflags, max_violations_hint=hint,
                                    frontier_budget_bytes=budget, kernel_variant=args.kernel_variant)
            e1.record(stream)
            torch.cuda.synchronize()
            ntimes.append(e0.elapsed_time(e1))
            nenum.append(res[0].profile(G.PROF_ENUM)[0])
        nm = sum(r.n_matches for r in res)
        nms = float(np.mean(ntimes))
        line = {"value": nm / (nms / 1000.0), "unit": UNIT, "ms_per_step": nms,
                "enum_ms": float(np.mean(nenum)), "matches_per_step": nm,
                "violations_per_step": sum(r.n_violations for r in res),
                "work_items_per_step": sum(r.stat(G.STAT_WORK) for r in res)}
        if leg == "non_induced":
            non_induced = line
        else:
            # matches counted are those satisfying X; the violations are the
            # headline's, so violations/s compares the two directly
            line["counts"] = "matches satisfying X"
            line["violations_per_s"] = line["violations_per_step"] / (nms / 1000.0)
            line["same_violation_count_as_headline"] = line["violations_per_step"] == viols
            push_x = line

    # disconnected patterns: unions of two batched GFDs with few matches each
    # (the product of the two match counts bounds the union's), one batch
    disconnected = None
    if not args.no_non_induced and len(qs) > 1:
        from synth.gfds import GFD as _GFD
        counts = [r.n_matches for r in stats]
        order = [i for i in sorted(range(len(qs)), key=lambda i: counts[i]) if 1000 <= counts[i] <= 200000]
        unions, used = [], set()
        for a in order:
            if len(unions) == 16:
                break
            if a in used:
                continue
            for b in order:
                if b != a and b not in used and counts[a] * counts[b] <= 3e7:
                    qa, qb = qs[a], qs[b]
                    ka = qa.k
                    unions.append(_GFD(list(qa.node_label) + list(qb.node_label),
                                       list(qa.edges) + [(x + ka, y + ka, l) for (x, y, l) in qb.edges],
                                       qa.X, qa.Y, qa.y_false, name=f"{qa.name}+{qb.name}"))
                    used.update((a, b))
                    break
        if unions:
            res = dg.validate_batch(unions, stream=stream, flags=flags, max_violations_hint=hint)
            dtimes = []
            for _ in range(max(1, min(2, args.steps))):
                l2_flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = dg.validate_batch(unions, stream=stream, flags=flags, max_violations_hint=hint)
                e1.record(stream)
                torch.cuda.synchronize()
                dtimes.append(e0.elapsed_time(e1))
            dm = sum(r.n_matches for r in res)
            dms = float(np.mean(dtimes))
            disconnected = {"value": dm / (dms / 1000.0), "unit": UNIT, "ms_per_step": dms,
                            "gfds": len(unions), "matches_per_step": dm,
                            "violations_per_step": sum(r.n_violations for r in res),
                            "recipe": "pairs of batched GFDs with 1e3-2e5 matches each and a product <= 3e7, "
                                      "joined as two components (X and Y of the first)"}

    # serving: a Poisson stream of single-GFD requests against the resident
    # graph, continuous batching vs one gfd_validate per request
    serving = None
    rates = [float(x) for x in args.serve_rates.split(",") if x.strip()]
    if rates and args.workload == "batched":
        from synth import configs
        from paper_2608_02321_gb300 import serving as srv
        all_reqs = configs.serving_requests(g, args.serve_requests)
        serving = {"max_slots": 64, "budget_gb": 40,
                   "requests_per_rate": f"min({args.serve_requests}, rate x {args.serve_seconds:.0f} s)"}
        for lam in rates:
            reqs = all_reqs[: max(1, min(len(all_reqs), int(lam * args.serve_seconds)))]
            arr = configs.poisson_arrivals(lam, len(reqs), seed=int(lam))
            torch.cuda.synchronize()
            cont, _ = srv.serve(dg, reqs, arr, max_slots=64, budget_bytes=40 << 30, stream=stream)
            torch.cuda.synchronize()
            ser = srv.serve_serial(dg, reqs, arr, stream=stream)
            serving[f"rate_{int(lam)}"] = {
                "requests": len(reqs),
                "continuous": {k: cont[k] for k in ("p50_ms", "p99_ms", "matches_per_s", "requests_per_s",
                                                    "makespan_s", "peak_running", "session")},
                "serial_plain": {k: ser[k] for k in ("p50_ms", "p99_ms", "matches_per_s", "requests_per_s",
                                                     "makespan_s")}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        threads = cpu_threads()
        og = oracle.OracleGraph(g)
        tasks = fixed_root_tasks(g, qs)
        runs = [oracle_sample(g, qs, threads, og, tasks) for _ in range(2)]
        vals = [m / t if t > 0 else 0.0 for (m, t, _, _) in runs]
        m, t, d, x = runs[-1]
        cpu = {"value": float(np.mean(vals)), "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"fixed seeded sample (the reference arm's): {ROOTS_PER_GFD} uniform root vertices "
                         f"(images of pattern node 0) per GFD, {len(qs)} GFDs, {d} roots searched to the end, "
                         f"{x} dropped at task deadlines ({ROOTS_PER_TASK} roots, {TASK_DEADLINE_S:.0f} s each), "
                         f"{m} matches, {t:.1f} s wall",
               "spread": [min(vals), max(vals)]}
        # one thread, on the first eighth of the same sample
        m1, t1, d1, _ = oracle_sample(g, qs, 1, og, tasks[: max(1, len(tasks) // 8)])
        cpu["one_thread"] = {"value": m1 / t1 if t1 > 0 else 0.0, "unit": UNIT, "cores": 1,
                             "sample": f"the first {len(tasks[: max(1, len(tasks) // 8)])} GFDs' roots of the "
                                       f"same sample, {d1} roots, {t1:.1f} s wall"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": workload_config(desc, world),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "plain": plain, "non_induced": non_induced, "push_x": push_x, "disconnected": disconnected, "serving": serving, "autotuned": tuned,
                "batched_over_plain": (value / world) / plain["value"] if plain else None,
                "matches_per_step": matches, "violations_per_step": viols,
                "work_items_per_step": work, "edge_probes_per_step": probes,
                "enumeration_steps": enum_steps,
                "phase_ms": dict(zip(("filter", "refine", "index", "enumerate"),
                                     np.mean(np.array(phase_ms), axis=0).round(2).tolist())),
                "gfds_rerun_for_violation_capacity": sum(r.stat(G.STAT_RERUN) for r in stats),
                "step_ms_all": times, "enum_ms_all": enum_ms}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
