"""Python binding of libgfd.so (include/gfd.h): GFD validation on the GPU.

Argument marshalling only: every step of validation runs in the library's CUDA
kernels. The names follow the C-ABI (graph_load, validate, validate_batch).
If the compiled library is missing and cannot be built, importing the binding
raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgfd.so")

GFD_OK = 0
GFD_ERR_INVALID_ARG = 1
GFD_ERR_UNSUPPORTED = 2
GFD_ERR_OUT_OF_MEMORY = 3
GFD_ERR_OVERFLOW = 4
GFD_ERR_TIMEOUT = 5
GFD_ERR_CUDA = 6
WILDCARD = -1
ATTR_ABSENT = np.iinfo(np.int32).min
MAX_K = 16
MAX_SLOTS = 4095  # GFDs per batch call, running requests per session

FLAG_NO_REFINE = 0x1
FLAG_HOST_LOOP = 0x2
FLAG_PROFILE = 0x4
FLAG_NO_GRAPH = 0x8
FLAG_NON_INDUCED = 0x10
FLAG_PUSH_X = 0x20
FLAG_KEEP_CANDIDATES = 0x40
FLAG_COUNT = 0x80

PROF_FILTER, PROF_REFINE, PROF_INDEX, PROF_ENUM, PROF_SORT = range(5)
STAT_STEPS, STAT_WORK, STAT_ROWS, STAT_PROBES, STAT_CANDIDATES, STAT_INDEX, STAT_RERUN = range(7)
# counters of a GFD_FLAG_COUNT run (gfd_result_stat 7..28)
COUNTERS = ("items", "items_last", "partials", "back_deg", "checks", "sig_settled", "searches",
            "search_loads", "neg_checks", "neg_logd", "sig_loads", "attr_reads", "rows",
            "scan_cands", "scan_entries", "iters", "iter_max_loads", "cyc_tile", "cyc_mid", "cyc_last",
            "iters_mid", "keys_and_bitmaps")


class GfdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gfd error {code}: {msg}")
        self.code = code


class gfd_graph_desc(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_edges", C.c_int64), ("n_attrs", C.c_int32),
                ("out_off", C.c_void_p), ("out_dst", C.c_void_p), ("out_elabel", C.c_void_p),
                ("in_off", C.c_void_p), ("in_src", C.c_void_p), ("in_elabel", C.c_void_p),
                ("vlabel", C.c_void_p), ("attrs", C.c_void_p)]


class gfd_literal(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x", C.c_int32), ("a", C.c_int32),
                ("y", C.c_int32), ("b", C.c_int32), ("c", C.c_int32)]


class gfd_gfd(C.Structure):
    _fields_ = [("k", C.c_int32), ("node_label", C.c_void_p),
                ("m", C.c_int32), ("esrc", C.c_void_p), ("edst", C.c_void_p), ("elabel", C.c_void_p),
                ("nx", C.c_int32), ("X", C.c_void_p), ("ny", C.c_int32), ("Y", C.c_void_p),
                ("y_false", C.c_int32)]


class gfd_opts(C.Structure):
    _fields_ = [("frontier_budget_bytes", C.c_int64), ("chunk_rows", C.c_int32),
                ("kernel_variant", C.c_int32), ("max_violations_hint", C.c_int64),
                ("cuda_stream", C.c_void_p), ("flags", C.c_int32), ("tile_iters", C.c_int32)]


# exported functions: name -> (restype, argtypes)
_SIGS = {
    "gfd_graph_load": (C.c_int, [C.POINTER(gfd_graph_desc), C.POINTER(gfd_opts), C.POINTER(C.c_void_p)]),
    "gfd_graph_free": (None, [C.c_void_p]),
    "gfd_graph_vertices": (C.c_int32, [C.c_void_p]),
    "gfd_graph_edges": (C.c_int64, [C.c_void_p]),
    "gfd_graph_device_bytes": (C.c_int64, [C.c_void_p]),
    "gfd_validate": (C.c_int, [C.c_void_p, C.POINTER(gfd_gfd), C.POINTER(gfd_opts), C.POINTER(C.c_void_p)]),
    "gfd_validate_batch": (C.c_int, [C.c_void_p, C.POINTER(C.POINTER(gfd_gfd)), C.c_int32,
                                     C.POINTER(gfd_opts), C.POINTER(C.c_void_p)]),
    "gfd_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.POINTER(gfd_gfd)), C.c_int32, C.POINTER(gfd_opts),
                              C.POINTER(gfd_opts)]),
    "gfd_result_matches": (C.c_uint64, [C.c_void_p]),
    "gfd_result_violations": (C.c_uint64, [C.c_void_p]),
    "gfd_result_arity": (C.c_int32, [C.c_void_p]),
    "gfd_result_tuples": (C.c_void_p, [C.c_void_p]),
    "gfd_result_copy_tuples": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64]),
    "gfd_results_copy_tuples": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_uint64]),
    "gfd_result_profile": (C.c_double, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "gfd_result_stat": (C.c_uint64, [C.c_void_p, C.c_int32]),
    "gfd_result_candidates": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
    "gfd_result_free": (None, [C.c_void_p]),
    "gfd_session_create": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(gfd_opts), C.POINTER(C.c_void_p)]),
    "gfd_session_submit": (C.c_int, [C.c_void_p, C.POINTER(gfd_gfd), C.POINTER(C.c_int64)]),
    "gfd_session_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "gfd_session_next_result": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_void_p)]),
    "gfd_session_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
    "gfd_session_stat": (C.c_double, [C.c_void_p, C.c_int32]),
    "gfd_session_free": (None, [C.c_void_p]),
    "gfd_node_candidates_noalloc": (C.c_int, [C.c_void_p, C.POINTER(gfd_gfd), C.c_int32, C.c_void_p,
                                              C.c_int64, C.POINTER(C.c_int64), C.c_void_p]),
    "gfd_last_error": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library(build_if_missing: bool = True):
    """Load libgfd.so (building it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            if not build_if_missing:
                raise ImportError(f"{_LIB_PATH} is missing; build it with __graft_entry__.build()")
            from . import build as _b
            _b.build()
        lib = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc != GFD_OK:
        raise GfdError(rc, _lib.gfd_last_error().decode())


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))   # torch.cuda.Stream


def make_opts(frontier_budget_bytes=0, chunk_rows=0, kernel_variant=0, max_violations_hint=0,
              stream=None, flags=0, tile_iters=0) -> gfd_opts:
    o = gfd_opts()
    o.frontier_budget_bytes = int(frontier_budget_bytes)
    o.chunk_rows = int(chunk_rows)
    o.kernel_variant = int(kernel_variant)
    o.max_violations_hint = int(max_violations_hint)
    o.cuda_stream = _stream_handle(stream)
    o.flags = int(flags)
    o.tile_iters = int(tile_iters)
    return o


class _GfdBuf:
    """ctypes image of one GFD (keeps its arrays alive)."""

    def __init__(self, gfd):
        k = len(gfd.node_label)
        self.nl = _i32(gfd.node_label)
        e = np.asarray(gfd.edges, dtype=np.int32).reshape(-1, 3)
        self.es, self.ed, self.el = _i32(e[:, 0]), _i32(e[:, 1]), _i32(e[:, 2])

        def lits(ls):
            arr = (gfd_literal * max(1, len(ls)))()
            for i, l in enumerate(ls):
                arr[i] = gfd_literal(l.kind, l.x, l.a, l.y, l.b, l.c)
            return arr
        self.X = lits(gfd.X)
        self.Y = lits(gfd.Y)
        s = gfd_gfd()
        s.k = k
        s.node_label = _ptr(self.nl)
        s.m = e.shape[0]
        s.esrc, s.edst, s.elabel = _ptr(self.es), _ptr(self.ed), _ptr(self.el)
        s.nx, s.X = len(gfd.X), C.cast(self.X, C.c_void_p)
        s.ny, s.Y = len(gfd.Y), C.cast(self.Y, C.c_void_p)
        s.y_false = 1 if gfd.y_false else 0
        self.s = s


class Result:
    """Matches and violations of one GFD."""

    def __init__(self, handle, graph=None):
        self._h = handle
        # the tuples are sorted on the graph's stream when first read: the
        # graph stays loaded while its results are reachable
        self._g = graph

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.gfd_result_free(self._h)
            self._h = None

    @property
    def n_matches(self) -> int:
        return int(_lib.gfd_result_matches(self._h))

    @property
    def n_violations(self) -> int:
        return int(_lib.gfd_result_violations(self._h))

    @property
    def k(self) -> int:
        return int(_lib.gfd_result_arity(self._h))

    def violations(self) -> np.ndarray:
        """[n_violations, k] int32, lexicographically sorted (sorted on the device)."""
        n, k = self.n_violations, self.k
        if not n:
            return np.empty((0, k), dtype=np.int32)
        out = np.empty((n, k), dtype=np.int32)
        _check(_lib.gfd_result_copy_tuples(self._h, out.ctypes.data_as(C.c_void_p), C.c_uint64(n * k)))
        return out

    def profile(self, which: int):
        """(device milliseconds, launches) of a kernel class (needs FLAG_PROFILE)."""
        n = C.c_int64(0)
        ms = _lib.gfd_result_profile(self._h, int(which), C.byref(n))
        return float(ms), int(n.value)

    def stat(self, which: int) -> int:
        return int(_lib.gfd_result_stat(self._h, int(which)))

    def counters(self) -> dict:
        """The counters of a FLAG_COUNT run (whole call), by name."""
        out = {name: self.stat(7 + i) for i, name in enumerate(COUNTERS)}
        kb = out.pop("keys_and_bitmaps")
        out["filter_keys"], out["bitmaps"] = kb >> 32, kb & 0xffffffff
        return out

    def candidates(self, node: int) -> np.ndarray:
        """The refined candidate list of pattern node `node` (needs
        FLAG_KEEP_CANDIDATES on the batch call), increasing vertex ids."""
        p = C.c_void_p(None)
        n = C.c_int64(0)
        _check(_lib.gfd_result_candidates(self._h, int(node), C.byref(p), C.byref(n)))
        if n.value == 0:
            return np.zeros(0, dtype=np.int32)
        buf = (C.c_int32 * n.value).from_address(p.value)
        return np.frombuffer(buf, dtype=np.int32).copy()


class Graph:
    """A graph resident on the GPU (gfd_graph_load)."""

    def __init__(self, graph, stream=None, reverse=None):
        """graph: CSR arrays (out_off, out_dst, out_elabel, vlabel, attrs).
        reverse: None (the library builds the reverse CSR) or the caller's
        (in_off, in_src, in_elabel), which must describe the same edge set."""
        lib = load_library()
        n = int(graph.n_vertices)
        self.n = n
        off = _i64(graph.out_off)
        dst = _i32(graph.out_dst)
        lab = _i32(graph.out_elabel)
        vl = _i32(graph.vlabel)
        at = _i32(graph.attrs).reshape(-1)
        d = gfd_graph_desc()
        d.n_vertices = n
        d.n_edges = int(dst.shape[0])
        d.n_attrs = int(np.asarray(graph.attrs).shape[0])
        d.out_off, d.out_dst, d.out_elabel = _ptr(off), _ptr(dst), _ptr(lab)
        keep = [off, dst, lab, vl, at]
        if reverse is not None:
            ioff, isrc, ilab = _i64(reverse[0]), _i32(reverse[1]), _i32(reverse[2])
            keep += [ioff, isrc, ilab]
            d.in_off, d.in_src, d.in_elabel = _ptr(ioff), _ptr(isrc), _ptr(ilab)
        d.vlabel, d.attrs = _ptr(vl), _ptr(at)
        o = make_opts(stream=stream)
        h = C.c_void_p(None)
        _check(lib.gfd_graph_load(C.byref(d), C.byref(o), C.byref(h)))
        del keep
        self._h = h
        # The graph's handle and those of its open sessions, shared with the
        # sessions by strong reference. A session runs on the graph's stream
        # and memory pool, so it must be freed first; when a graph and its
        # sessions are garbage in one reference cycle, Python runs their
        # finalisers in any order (and clears weak references before any of
        # them), so whichever finaliser runs first frees the open sessions.
        self._live = {"graph": h, "sessions": set()}

    def __del__(self):
        live = getattr(self, "_live", None)
        if live is None or _lib is None:
            return
        for sh in list(live["sessions"]):
            _lib.gfd_session_free(C.c_void_p(sh))
        live["sessions"].clear()
        if live["graph"] is not None:
            _lib.gfd_graph_free(live["graph"])
            live["graph"] = None
        self._h = None

    @property
    def device_bytes(self) -> int:
        return int(_lib.gfd_graph_device_bytes(self._h))

    def validate(self, gfd, **opts) -> Result:
        o = make_opts(**opts)
        b = _GfdBuf(gfd)
        h = C.c_void_p(None)
        _check(_lib.gfd_validate(self._h, C.byref(b.s), C.byref(o), C.byref(h)))
        return Result(h, self)

    def autotune(self, gfds, **opts) -> dict:
        """Time the enumeration-kernel variants and frontier budgets on this
        batch (gfd_autotune) and keep the fastest for later calls."""
        o = make_opts(**opts)
        bufs = [_GfdBuf(g) for g in gfds]
        arr = (C.POINTER(gfd_gfd) * max(1, len(bufs)))(*[C.pointer(b.s) for b in bufs])
        best = gfd_opts()
        _check(_lib.gfd_autotune(self._h, arr, len(bufs), C.byref(o), C.byref(best)))
        return {"kernel_variant": int(best.kernel_variant), "tile_iters": int(best.tile_iters),
                "frontier_budget_bytes": int(best.frontier_budget_bytes)}

    def validate_batch(self, gfds, **opts) -> list:
        o = make_opts(**opts)
        bufs = [_GfdBuf(g) for g in gfds]
        arr = (C.POINTER(gfd_gfd) * max(1, len(bufs)))(*[C.pointer(b.s) for b in bufs])
        outs = (C.c_void_p * max(1, len(bufs)))()
        _check(_lib.gfd_validate_batch(self._h, arr, len(bufs), C.byref(o), outs))
        return [Result(C.c_void_p(outs[i]), self) for i in range(len(bufs))]


class Session:
    """A serving session with continuous batching (gfd_session_*): submit GFDs
    at any time; each step admits queued requests into free slots within the
    memory budget and advances every running request together."""

    def __init__(self, g: Graph, max_slots: int = 64, **opts):
        self._g = g  # keeps the graph alive
        self._live = g._live
        o = make_opts(**opts)
        h = C.c_void_p(None)
        _check(_lib.gfd_session_create(g._h, int(max_slots), C.byref(o), C.byref(h)))
        self._h = h
        self._live["sessions"].add(h.value)

    def close(self):
        """Release the session (gfd_session_free); later calls are errors.
        A no-op once its graph has been finalised (which freed it)."""
        h, live = getattr(self, "_h", None), getattr(self, "_live", None)
        if h and live is not None and _lib is not None and h.value in live["sessions"]:
            live["sessions"].discard(h.value)
            _lib.gfd_session_free(h)
        self._h = None

    def __del__(self):
        self.close()

    def submit(self, gfd) -> int:
        b = _GfdBuf(gfd)
        rid = C.c_int64(-1)
        _check(_lib.gfd_session_submit(self._h, C.byref(b.s), C.byref(rid)))
        return int(rid.value)

    def step(self):
        """One admission + enumeration round: (requests that advanced together
        in it, requests still running, requests still queued)."""
        a = C.c_int32(0)
        r = C.c_int32(0)
        q = C.c_int32(0)
        _check(_lib.gfd_session_step(self._h, C.byref(a), C.byref(r), C.byref(q)))
        return int(a.value), int(r.value), int(q.value)

    def cancel(self, request_id: int):
        """Drop a queued request, stop a running one or discard an uncollected
        result (gfd_session_cancel)."""
        _check(_lib.gfd_session_cancel(self._h, int(request_id)))

    def stats(self) -> dict:
        """Host time in admissions and in enumeration rounds, rounds run,
        requests admitted, admissions (gfd_session_stat)."""
        names = ("admit_ms", "round_ms", "rounds", "admitted", "admissions")
        return {n: float(_lib.gfd_session_stat(self._h, i)) for i, n in enumerate(names)}

    def results(self):
        """All finished requests since the last call: [(request_id, Result)]."""
        out = []
        while True:
            rid = C.c_int64(-1)
            h = C.c_void_p(None)
            _check(_lib.gfd_session_next_result(self._h, C.byref(rid), C.byref(h)))
            if rid.value < 0:
                return out
            out.append((int(rid.value), Result(h, self._g)))


def node_candidates_noalloc(g: Graph, gfd, node: int, out_ptr: int, out_cap: int, stream=None) -> int:
    """Candidate vertices of pattern node `node` written to the caller's device
    buffer at out_ptr (int32, out_cap elements) without any device allocation by
    the library; returns their number. See include/gfd.h for the limits."""
    b = _GfdBuf(gfd)
    n = C.c_int64(0)
    _check(_lib.gfd_node_candidates_noalloc(g._h, C.byref(b.s), int(node), out_ptr, int(out_cap),
                                            C.byref(n), _stream_handle(stream)))
    return int(n.value)


def graph_load(graph, stream=None, reverse=None) -> Graph:
    return Graph(graph, stream, reverse)


def violations_all(results) -> list:
    """The sorted violation lists of several results ([n_i, k_i] int32 each),
    fetched with one device sort and one copy (gfd_results_copy_tuples)."""
    results = list(results)
    sizes = [r.n_violations * r.k for r in results]
    buf = np.empty(max(1, sum(sizes)), dtype=np.int32)
    hs = (C.c_void_p * max(1, len(results)))(*[r._h for r in results])
    _check(_lib.gfd_results_copy_tuples(hs, len(results), buf.ctypes.data_as(C.c_void_p),
                                        C.c_uint64(sum(sizes))))
    out, at = [], 0
    for r, sz in zip(results, sizes):
        out.append(buf[at:at + sz].reshape(r.n_violations, r.k))
        at += sz
    return out


def validate(g: Graph, gfd, **opts) -> Result:
    return g.validate(gfd, **opts)


def validate_batch(g: Graph, gfds, **opts) -> list:
    return g.validate_batch(gfds, **opts)
