"""Helpers for the GPU parity tests: run the CUDA path through the C-ABI and
the oracle on the same inputs."""
import numpy as np


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
