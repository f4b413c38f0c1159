"""ctypes front end of the C oracle (oracle.c) — TEST INFRASTRUCTURE ONLY.

`validate(graph, gfd)` returns (n_matches, violations) where violations is an
int32 array [n_viol, k] sorted lexicographically (Vio of Section II). Root
vertices (the images of pattern node 0) can be restricted to a sample, and split
over host threads; each thread runs the unchanged sequential matcher on its own
slice of roots and the results are concatenated and sorted.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAXK = 16

_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C11, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Lit(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x", C.c_int32), ("a", C.c_int32),
                ("y", C.c_int32), ("b", C.c_int32), ("c", C.c_int32)]


class _Gfd(C.Structure):
    _fields_ = [("k", C.c_int32), ("node_label", C.c_int32 * MAXK), ("m", C.c_int32),
                ("esrc", C.POINTER(C.c_int32)), ("edst", C.POINTER(C.c_int32)),
                ("elab", C.POINTER(C.c_int32)),
                ("nx", C.c_int32), ("X", C.POINTER(_Lit)),
                ("ny", C.c_int32), ("Y", C.POINTER(_Lit)),
                ("y_false", C.c_int32)]


def bind_library(path: str):
    """Load a compiled oracle (liboracle.so or a test-built variant of it)."""
    lib = C.CDLL(path)
    lib.og_graph_new.restype = C.c_void_p
    lib.og_graph_new.argtypes = [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    lib.og_graph_free.argtypes = [C.c_void_p]
    lib.og_validate.restype = C.c_int
    lib.og_validate.argtypes = [C.c_void_p, C.POINTER(_Gfd), C.c_void_p, C.c_int64,
                                C.POINTER(C.c_uint64), C.POINTER(C.c_void_p),
                                C.POINTER(C.c_int64)]
    lib.og_validate_budget.restype = C.c_int
    lib.og_validate_budget.argtypes = [C.c_void_p, C.POINTER(_Gfd), C.c_void_p, C.c_int64, C.c_double,
                                       C.POINTER(C.c_uint64), C.POINTER(C.c_void_p),
                                       C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.og_validate_mode.restype = C.c_int
    lib.og_validate_mode.argtypes = [C.c_void_p, C.POINTER(_Gfd), C.c_int, C.c_void_p, C.c_int64, C.c_double,
                                     C.POINTER(C.c_uint64), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]
    lib.og_violating.restype = C.c_int
    lib.og_violating.argtypes = [C.c_void_p, C.POINTER(_Gfd), C.c_void_p, C.c_int64, C.c_void_p]
    lib.og_free.argtypes = [C.c_void_p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind_library(build_oracle())
    return _lib


def oracle_available() -> bool:
    try:
        _load()
        return True
    except Exception:
        return False


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleGraph:
    """The oracle's own copy of G (sorted out- and in-adjacency)."""

    def __init__(self, graph, lib=None):
        lib = lib or _load()
        self._lib = lib
        src, dst, lab = graph.edge_arrays()
        src = np.ascontiguousarray(src, dtype=np.int64)
        dst = np.ascontiguousarray(dst, dtype=np.int64)
        lab = np.ascontiguousarray(lab, dtype=np.int32)
        vl = np.ascontiguousarray(graph.vlabel, dtype=np.int32)
        at = np.ascontiguousarray(graph.attrs, dtype=np.int32)
        self.n = int(graph.n_vertices)
        self._h = lib.og_graph_new(self.n, int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(lab),
                                   _ptr(vl), int(at.shape[0]), _ptr(at))
        if not self._h:
            raise ValueError("oracle rejected the graph (id out of range or repeated edge)")

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.og_graph_free(self._h)
            self._h = None


def _gfd_struct(gfd):
    k = gfd.k
    if k > MAXK:
        raise ValueError("pattern too large")
    keep = []

    def arr(v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_int32))

    s = _Gfd()
    s.k = k
    for i in range(k):
        s.node_label[i] = gfd.node_label[i]
    s.m = len(gfd.edges)
    s.esrc = arr([e[0] for e in gfd.edges] or [0])
    s.edst = arr([e[1] for e in gfd.edges] or [0])
    s.elab = arr([e[2] for e in gfd.edges] or [0])
    X = (_Lit * max(1, len(gfd.X)))(*[_Lit(l.kind, l.x, l.a, l.y, l.b, l.c) for l in gfd.X])
    Y = (_Lit * max(1, len(gfd.Y)))(*[_Lit(l.kind, l.x, l.a, l.y, l.b, l.c) for l in gfd.Y])
    keep += [X, Y]
    s.nx, s.X = len(gfd.X), C.cast(X, C.POINTER(_Lit))
    s.ny, s.Y = len(gfd.Y), C.cast(Y, C.POINTER(_Lit))
    s.y_false = 1 if gfd.y_false else 0
    return s, keep


def _run(og: OracleGraph, gfd, roots, induced: bool = True, count: str = "all"):
    lib = og._lib
    s, keep = _gfd_struct(gfd)
    nm = C.c_uint64(0)
    nx = C.c_uint64(0)
    vp = C.c_void_p(None)
    nv = C.c_int64(0)
    if roots is None and induced and count == "all":
        rc = lib.og_validate(og._h, C.byref(s), None, 0, C.byref(nm), C.byref(vp), C.byref(nv))
    elif roots is None:
        rc = lib.og_validate_mode(og._h, C.byref(s), 1 if induced else 0, None, 0, 0.0, C.byref(nm),
                                  C.byref(vp), C.byref(nv), None, C.byref(nx))
    else:
        r = np.ascontiguousarray(roots, dtype=np.int32)
        if induced and count == "all":
            rc = lib.og_validate(og._h, C.byref(s), _ptr(r), int(r.shape[0]), C.byref(nm),
                                 C.byref(vp), C.byref(nv))
        else:
            rc = lib.og_validate_mode(og._h, C.byref(s), 1 if induced else 0, _ptr(r), int(r.shape[0]), 0.0,
                                      C.byref(nm), C.byref(vp), C.byref(nv), None, C.byref(nx))
    if count == "x":
        nm = nx
    if rc != 0:
        raise ValueError("oracle rejected the GFD (malformed pattern)")
    k = gfd.k
    n = int(nv.value)
    if n:
        buf = (C.c_int32 * (n * k)).from_address(vp.value)
        out = np.frombuffer(buf, dtype=np.int32).reshape(n, k).copy()
    else:
        out = np.zeros((0, k), dtype=np.int32)
    if vp.value:
        lib.og_free(vp)
    del keep
    return int(nm.value), out


def count_within(og: OracleGraph, gfd, roots, seconds: float, induced: bool = True):
    """(matches, roots searched to the end) for the given roots, stopping after
    about `seconds`; the root in progress at the deadline is not counted."""
    lib = og._lib
    s, keep = _gfd_struct(gfd)
    nm = C.c_uint64(0)
    vp = C.c_void_p(None)
    nv = C.c_int64(0)
    done = C.c_int64(0)
    r = np.ascontiguousarray(roots, dtype=np.int32)
    rc = lib.og_validate_mode(og._h, C.byref(s), 1 if induced else 0, _ptr(r), int(r.shape[0]),
                              float(seconds), C.byref(nm), C.byref(vp), C.byref(nv), C.byref(done), None)
    if vp.value:
        lib.og_free(vp)
    del keep
    if rc != 0:
        raise ValueError("oracle rejected the GFD (malformed pattern)")
    return int(nm.value), int(done.value)


def validate_within(og: OracleGraph, gfd, roots, seconds: float, induced: bool = True):
    """(matches, sorted violations, roots searched to the end) for the given
    roots, stopping after about `seconds`: the matches and violations are those
    of roots[:done] exactly (the root in progress at the deadline is dropped)."""
    lib = og._lib
    s, keep = _gfd_struct(gfd)
    nm = C.c_uint64(0)
    vp = C.c_void_p(None)
    nv = C.c_int64(0)
    done = C.c_int64(0)
    r = np.ascontiguousarray(roots, dtype=np.int32)
    rc = lib.og_validate_mode(og._h, C.byref(s), 1 if induced else 0, _ptr(r), int(r.shape[0]),
                              float(seconds), C.byref(nm), C.byref(vp), C.byref(nv), C.byref(done), None)
    if rc != 0:
        if vp.value:
            lib.og_free(vp)
        raise ValueError("oracle rejected the GFD (malformed pattern)")
    k = gfd.k
    n = int(nv.value)
    out = np.zeros((0, k), dtype=np.int32)
    if n:
        buf = (C.c_int32 * (n * k)).from_address(vp.value)
        out = np.frombuffer(buf, dtype=np.int32).reshape(n, k).copy()
    if vp.value:
        lib.og_free(vp)
    del keep
    return int(nm.value), sort_tuples(out), int(done.value)


def violating(og: OracleGraph, gfd, matches: np.ndarray) -> np.ndarray:
    """The rows of `matches` ([n, k] tuples taken as matches of gfd's pattern)
    that are violations of gfd (X holds, and Y is false or fails): the
    literal check of Section II on its own, in the input order."""
    lib = og._lib
    s, keep = _gfd_struct(gfd)
    t = np.ascontiguousarray(matches, dtype=np.int32).reshape(-1, gfd.k)
    flags = np.zeros(t.shape[0], dtype=np.uint8)
    rc = lib.og_violating(og._h, C.byref(s), _ptr(t), int(t.shape[0]), _ptr(flags))
    del keep
    if rc != 0:
        raise ValueError("oracle rejected the GFD or a tuple")
    return t[flags.astype(bool)]


def sort_tuples(t: np.ndarray) -> np.ndarray:
    """Lexicographic row order (library sort as a step)."""
    if t.shape[0] <= 1:
        return t
    return t[np.lexsort(t.T[::-1])]


def validate(graph_or_og, gfd, roots=None, threads: int = 1, lib=None, induced: bool = True,
             count: str = "all"):
    """(n_matches, sorted violations [n, k]) of one GFD; see module docstring.
    induced=False selects the non-induced mode (only Q's edges constrain h);
    count="x" counts only the matches that satisfy X (the violations are the
    same either way)."""
    og = graph_or_og if isinstance(graph_or_og, OracleGraph) else OracleGraph(graph_or_og, lib)
    if threads <= 1:
        nm, v = _run(og, gfd, roots, induced, count)
        return nm, sort_tuples(v)
    if roots is None:
        roots = np.arange(og.n, dtype=np.int32)
    roots = np.asarray(roots, dtype=np.int32)
    # interleaved slices spread hubs over the threads
    parts = [roots[i::threads * 8] for i in range(threads * 8)]
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(lambda r: _run(og, gfd, r, induced, count), parts))
    nm = sum(r[0] for r in res)
    v = np.concatenate([r[1] for r in res]) if res else np.zeros((0, gfd.k), np.int32)
    return nm, sort_tuples(v)
