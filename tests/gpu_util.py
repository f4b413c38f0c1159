"""Helpers for the GPU parity tests: run the CUDA path through the C-ABI and
the oracle on the same inputs."""
import numpy as np


def reverse_csr(graph):
    """The transpose of the graph's CSR (rows by destination, sources
    increasing), to hand the library a caller-built reverse CSR."""
    n = int(graph.n_vertices)
    off = np.asarray(graph.out_off, dtype=np.int64)
    dst = np.asarray(graph.out_dst, dtype=np.int64)
    lab = np.asarray(graph.out_elabel, dtype=np.int32)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    order = np.lexsort((src, dst))
    ioff = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(dst, minlength=n), out=ioff[1:])
    return ioff, src[order].astype(np.int32), lab[order]


def gpu_graph(graph, **kw):
    import paper_2608_02321_gb300 as G
    return G.Graph(graph, **kw)


def gpu_run(dg, gfd, **opts):
    r = dg.validate(gfd, **opts)
    return r.n_matches, r.violations()


def assert_same(got, want, what=""):
    gm, gv = got
    wm, wv = want
    assert gm == wm, f"{what}: matches {gm} != oracle {wm}"
    assert gv.shape == wv.shape, f"{what}: violations {gv.shape} != oracle {wv.shape}"
    np.testing.assert_array_equal(gv, wv, err_msg=what)
