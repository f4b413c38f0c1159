"""The knowledge-graph-shaped workload: 6-node GFDs x-[e]->y, x-[e']->y',
y->z1, y'->z1, y->z2, y'->z2, x->w with X -> false dependencies, on graphs with
hub out-degrees up to ~1e6 at full size. The plain oracle cannot enumerate
those graphs, so (1) the pattern family is checked exactly against the oracle
on random graphs it can finish, and (2) the full workload is checked through
properties that hold at any size: both enumeration drivers, all kernel
variants, and batched vs one-at-a-time validation give identical results."""
import numpy as np
import pytest

from synth import configs
from synth.gfds import GFD, Literal
from synth.graphs import random_small_graph

from gpu_util import assert_same, gpu_graph

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2608_02321_gb300")


@pytest.fixture(scope="module")
def lib_loaded():
    return G.load_library()


def _kg_shaped(rng, k_labels):
    nl = [int(rng.choice(k_labels)) for _ in range(5)] + [-1]
    e1, e2 = (int(rng.choice([-1, 0, 1])) for _ in range(2))
    edges = [(0, 1, e1), (0, 2, e2), (1, 3, -1), (2, 3, -1), (1, 4, -1), (2, 4, -1), (0, 5, -1)]
    if rng.random() < 0.5:
        return GFD(nl, edges, [Literal.const(1, 0, int(rng.integers(0, 3))),
                               Literal.const(2, 0, int(rng.integers(0, 3)))], [], True)
    return GFD(nl, edges, [], [Literal.var(1, 0, 2, 0)], False)


@pytest.mark.parametrize("seed", range(4))
def test_kg_pattern_family_exact(lib_loaded, oracle_mod, seed):
    rng = np.random.default_rng([31, seed])
    g = random_small_graph(500 + seed, 250, n_vlabels=2, n_elabels=2, p_edge=0.06, p_self=0.0,
                           n_attrs=1, n_attr_values=3, p_absent=0.05)
    dg = gpu_graph(g)
    total = 0
    qs = [_kg_shaped(rng, [0, 1, -1]) for _ in range(6)]
    res = dg.validate_batch(qs)
    for i, q in enumerate(qs):
        want = oracle_mod.validate(g, q, threads=8)
        assert_same((res[i].n_matches, res[i].violations()), want, f"seed {seed} gfd {i}")
        total += want[0]
    assert total > 0


def _properties(g, qs):
    dg = gpu_graph(g)
    ref = [(r.n_matches, r.violations()) for r in dg.validate_batch(qs)]
    for flags, variant in ((G.FLAG_HOST_LOOP, 0), (0, 5), (0, 4), (G.FLAG_NO_REFINE, 0)):
        res = dg.validate_batch(qs, flags=flags, kernel_variant=variant)
        for i, r in enumerate(res):
            assert_same((r.n_matches, r.violations()), ref[i], f"{qs[i].name} flags {flags} variant {variant}")
    for i in (0, 1, len(qs) - 1):
        r = dg.validate(qs[i])
        assert_same((r.n_matches, r.violations()), ref[i], f"{qs[i].name} alone")
    return sum(x[0] for x in ref)


def test_kg_scaled_properties(lib_loaded):
    g, qs = configs.kg(scale=20)
    _properties(g, qs)


@pytest.mark.slow
def test_kg_full_size_properties(lib_loaded):
    g, qs = configs.kg()
    assert np.diff(g.out_off).max() > 500_000          # hub out-degrees near 1e6
    _properties(g, qs)
