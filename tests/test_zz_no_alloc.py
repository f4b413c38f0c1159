"""The allocation-free entry point (gfd_node_candidates_noalloc) against the
existing one (gfd_validate). Some callers may not allocate device memory: a
server whose device memory comes from its own allocator or a budget reserved up
front, or a latency-bound thread that cannot wait for cudaFree's device-wide
synchronisation. For them the library offers the candidate filter of one
pattern node with all scratch in a fixed array of its own. A single-node GFD
with X empty and Y = false has exactly those candidates as its violations, so
gfd_validate gives the expected list; for larger patterns the per-node counts
add up to the candidate total that gfd_validate reports without refinement.
Each check runs twice in a row, because every call reuses the same scratch
array."""
import numpy as np
import pytest

from synth import configs
from synth.gfds import GFD
from synth.graphs import random_small_graph

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")
torch = pytest.importorskip("torch")


def _noalloc(dg, q, node, out):
    n = G.node_candidates_noalloc(dg, q, node, out.data_ptr(), out.numel(),
                                  stream=torch.cuda.current_stream())
    return out[:n].cpu().numpy()


def test_single_node_candidates_equal_validate():
    G.load_library()
    g, qs = configs.tiny()
    dg = G.Graph(g)
    out = torch.empty(g.n_vertices + 16, dtype=torch.int32, device="cuda")
    # wildcard first (large result), then a label (smaller): the second call must
    # not see anything left over from the first
    for label in (-1, 3, 0, -1):
        q = GFD([label], [], [], [], True)
        want = dg.validate(q).violations()[:, 0]
        for _ in range(2):
            got = _noalloc(dg, q, 0, out)
            np.testing.assert_array_equal(got, want)


def test_self_loop_and_degree_filters():
    g = random_small_graph(11, 3000, n_vlabels=3, n_elabels=2, p_edge=0.002, p_self=0.2)
    dg = G.Graph(g)
    out = torch.empty(g.n_vertices, dtype=torch.int32, device="cuda")
    for q in (GFD([1], [(0, 0, 1)], [], [], True),       # self-loop with label 1
              GFD([-1], [(0, 0, -1)], [], [], True),     # any self-loop
              GFD([2], [], [], [], True)):               # no self-loop
        want = dg.validate(q).violations()[:, 0]
        for _ in range(2):
            np.testing.assert_array_equal(_noalloc(dg, q, 0, out), want)


def test_multi_node_counts_equal_candidate_total():
    g, _ = configs.batched(scale=100, n_gfds=8)
    qs = configs.batched_gfds(g, 8)
    dg = G.Graph(g)
    out = torch.empty(g.n_vertices, dtype=torch.int32, device="cuda")
    for q in qs:
        total = sum(len(_noalloc(dg, q, u, out)) for u in range(q.k))
        again = sum(len(_noalloc(dg, q, u, out)) for u in range(q.k))
        r = dg.validate(q, flags=G.FLAG_NO_REFINE)
        assert total == again == r.stat(G.STAT_CANDIDATES)


def test_capacity_and_limits_are_reported():
    g, _ = configs.tiny()
    dg = G.Graph(g)
    small = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(G.GfdError) as e:
        G.node_candidates_noalloc(dg, GFD([-1], [], [], [], True), 0, small.data_ptr(), 4)
    assert e.value.code == G.GFD_ERR_OVERFLOW
    with pytest.raises(G.GfdError) as e:
        G.node_candidates_noalloc(dg, GFD([0], []), 5, small.data_ptr(), 4)
    assert e.value.code == G.GFD_ERR_INVALID_ARG
