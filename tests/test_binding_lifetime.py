"""Lifetime of the Python handles (no GPU): a session runs on its graph's
stream and memory pool, so the library must free every session before its
graph, exactly once, whichever of the two Python finalises first. A fake
library records the calls; the C-ABI itself is not called."""
import ctypes as C
import gc

import numpy as np
import pytest

G = pytest.importorskip("paper_2608_02321_gb300")


class FakeLib:
    def __init__(self):
        self.calls = []
        self.next = 0x1000

    def _new(self, out):
        self.next += 0x10
        C.cast(out, C.POINTER(C.c_void_p))[0] = self.next
        return self.next

    def gfd_graph_load(self, desc, opts, out):
        self.calls.append(("graph_load", self._new(out)))
        return G.GFD_OK

    def gfd_session_create(self, g, max_slots, opts, out):
        self.calls.append(("session_create", self._new(out)))
        return G.GFD_OK

    def gfd_session_free(self, h):
        self.calls.append(("session_free", h.value if isinstance(h, C.c_void_p) else h))

    def gfd_graph_free(self, h):
        self.calls.append(("graph_free", h.value if isinstance(h, C.c_void_p) else h))


class _TinyGraph:
    n_vertices = 2
    out_off = np.array([0, 1, 1])
    out_dst = np.array([1])
    out_elabel = np.array([0])
    vlabel = np.array([0, 0])
    attrs = np.zeros((1, 2), np.int32)


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(G, "_lib", lib)
    monkeypatch.setattr(G, "load_library", lambda *a, **k: lib)
    return lib


def _frees(lib):
    return [c for c in lib.calls if c[0] in ("session_free", "graph_free")]


def _check_order(lib, g_h, s_hs):
    frees = _frees(lib)
    assert sorted(h for k, h in frees if k == "session_free") == sorted(s_hs), "each session freed once"
    assert [h for k, h in frees if k == "graph_free"] == [g_h], "graph freed once"
    assert frees[-1] == ("graph_free", g_h), "sessions freed before the graph"


def test_session_closed_then_graph(fake):
    g = G.Graph(_TinyGraph())
    s = G.Session(g)
    g_h, s_h = g._h.value, s._h.value
    s.close()
    s.close()  # idempotent
    del s, g
    gc.collect()
    _check_order(fake, g_h, [s_h])


@pytest.mark.parametrize("graph_first", [True, False])
def test_finaliser_order(fake, graph_first):
    """Both finalisers run, in either order (as in a collected cycle)."""
    g = G.Graph(_TinyGraph())
    ss = [G.Session(g), G.Session(g)]
    g_h, s_hs = g._h.value, [s._h.value for s in ss]
    if graph_first:
        g.__del__()
        for s in ss:
            s.__del__()
    else:
        for s in ss:
            s.__del__()
        g.__del__()
    _check_order(fake, g_h, s_hs)


def test_reference_cycle_collected(fake):
    """A graph and its sessions held only by a reference cycle (as a traceback
    frame holds them) are freed in a valid order by the cyclic collector."""
    g_hs, s_hs = [], []
    for _ in range(20):
        g = G.Graph(_TinyGraph())
        ss = [G.Session(g) for _ in range(3)]
        box = {"g": g, "ss": ss}
        box["self"] = box
        g._cycle = box
        g_hs.append(g._h.value)
        s_hs += [s._h.value for s in ss]
        del g, ss, box
    gc.collect()
    frees = _frees(fake)
    assert sorted(h for k, h in frees if k == "graph_free") == sorted(g_hs)
    assert sorted(h for k, h in frees if k == "session_free") == sorted(s_hs)
    # every session is freed before the graph it was created on
    owner = {}
    cur = None
    for k, h in fake.calls:
        if k == "graph_load":
            cur = h
        elif k == "session_create":
            owner[h] = cur
    freed_graphs = set()
    for k, h in frees:
        if k == "graph_free":
            freed_graphs.add(h)
        else:
            assert owner[h] not in freed_graphs, "a session was freed after its graph"


def test_results_keep_their_graph(fake, monkeypatch):
    """A result's tuples are sorted on its graph's stream when first read, so
    the graph is released only after its last result."""
    from synth.gfds import GFD

    def validate(g, phi, opts, out):
        fake.calls.append(("validate", fake._new(out)))
        return G.GFD_OK

    def result_free(h):
        fake.calls.append(("result_free", h.value if isinstance(h, C.c_void_p) else h))

    monkeypatch.setattr(fake, "gfd_validate", validate, raising=False)
    monkeypatch.setattr(fake, "gfd_result_free", result_free, raising=False)
    g = G.Graph(_TinyGraph())
    g_h = g._h.value
    r = g.validate(GFD([0, 0], [(0, 1, -1)], [], [], True, "edge"))
    r_h = r._h.value
    del g
    gc.collect()
    assert not any(k == "graph_free" for k, _ in fake.calls), "graph freed while a result is alive"
    del r
    gc.collect()
    frees = [c for c in fake.calls if c[0] in ("result_free", "graph_free")]
    assert frees == [("result_free", r_h), ("graph_free", g_h)]
