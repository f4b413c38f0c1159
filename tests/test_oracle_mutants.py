"""The oracle pins must catch plausible mistakes: each mutant below is the oracle
with one planted error (compiled on the CPU into a temporary library), and at
least one pin (brute force, closed form or hand-counted toy) must reject it."""
from __future__ import annotations

import math
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from oracle.bruteforce import brute_force

from synth.gfds import GFD

from cases import (complete_bidirected, edges_graph, golden_cases, out_star, random_case,
                   random_disconnected_case, star_q, undirected_q)

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

MUTANTS = {
    "no_injectivity": ("if (hw == v) return 0;", ""),
    "no_reverse_edge_check":
        ("if (!og_pair_ok(s->qedge[w][u], og_edge(g, hw, v))) return 0;", ""),
    "non_induced": ("if (ql == OG_NOEDGE) return gl == OG_NOEDGE;",
                    "if (ql == OG_NOEDGE) return 1;"),
    "no_self_loop_check": ("if (!og_pair_ok(s->qedge[u][u], og_edge(g, v, v))) return 0;", ""),
    "absent_is_a_value": [("if (va == OG_ABSENT) return 0;", ""),
                          ("if (vb == OG_ABSENT) return 0;", "")],
    "ignores_false": ("if (q->y_false) return 1;", ""),
    "ignores_edge_labels": ("return og_label_ok(ql, gl);", "return 1;"),
    "transposed_edge": ("og_pair_ok(s->qedge[u][w], og_edge(g, v, hw))",
                        "og_pair_ok(s->qedge[u][w], og_edge(g, hw, v))"),
    "search_off_by_one": ("if (g->out_nbr[mid] < b) lo = mid + 1;",
                          "if (g->out_nbr[mid] <= b) lo = mid + 1;"),
    "var_literal_wrong_attr": ("vb = og_attr(s->g, l->b, s->h[l->y]);",
                               "vb = og_attr(s->g, l->a, s->h[l->y]);"),
    "vertex_label_ignored": ("if (!og_label_ok(s->q->node_label[u], g->vlabel[v])) return 0;", ""),
    # non-induced mode
    "non_induced_mode_still_induced": ("if (!og_induced && ql == OG_NOEDGE) return 1;", ""),
    "non_induced_mode_drops_required_edges": ("if (!og_induced && ql == OG_NOEDGE) return 1;",
                                              "if (!og_induced) return 1;"),
    # count of X-satisfying matches
    "x_count_ignores_x": ("s->n_x_matches += (uint64_t)og_x_holds(s);", "s->n_x_matches += 1;"),
    # the literal check on given matches
    "violating_row_stride": ("s.h[i] = tuples[t * q->k + i];", "s.h[i] = tuples[t + i];"),
    "violating_ignores_y": ("flags[t] = (uint8_t)og_is_violation(&s);", "flags[t] = (uint8_t)og_x_holds(&s);"),
    # disconnected patterns
    "component_start_skips_last_vertex": ("if (s->pnode[i] < 0) { a = 0; b = g->n; hp = -1; }",
                                          "if (s->pnode[i] < 0) { a = 0; b = g->n - 1; hp = -1; }"),
    "component_start_uses_root_neighbours": ("        s.pnode[i] = -1;                                          /* starts a component */",
                                             "        s.pnode[i] = 0; s.pout[i] = 1;"),
}


def _pins_pass(lib) -> bool:
    def run(g, q):
        return O.validate(g, q, lib=lib)

    for seed in range(80):
        g, q = random_case(seed)
        nm, v = run(g, q)
        bnm, bv = brute_force(g, q)
        if nm != bnm or not np.array_equal(v, bv):
            return False
    for n in (4, 6):
        if run(complete_bidirected(n), undirected_q(3, [(0, 1), (1, 2), (0, 2)]))[0] != n * (n - 1) * (n - 2):
            return False
        if run(complete_bidirected(n), undirected_q(3, [(0, 1), (1, 2)]))[0] != 0:
            return False
    if run(out_star(6), star_q(3))[0] != math.perm(6, 3):
        return False
    for name, g, q, n_matches, viol in golden_cases():
        nm, v = run(g, q)
        if nm != n_matches or not np.array_equal(v, viol):
            return False
    # the non-induced mode's pins
    for seed in range(80):
        g, q = random_case(seed)
        nm, v = O.validate(g, q, lib=lib, induced=False)
        bnm, bv = brute_force(g, q, induced=False)
        if nm != bnm or not np.array_equal(v, bv):
            return False
    if O.validate(complete_bidirected(5), undirected_q(3, [(0, 1), (1, 2)]), lib=lib, induced=False)[0] != 60:
        return False
    # disconnected patterns
    for seed in range(30):
        g, q = random_disconnected_case(seed)
        for induced in (True, False):
            nm, v = O.validate(g, q, lib=lib, induced=induced)
            bnm, bv = brute_force(g, q, induced=induced)
            if nm != bnm or not np.array_equal(v, bv):
                return False
    if O.validate(edges_graph(5, []), GFD([0, 0], []), lib=lib)[0] != 20:
        return False
    # the count of X-satisfying matches
    for seed in range(80):
        g, q = random_case(seed)
        nx, v = O.validate(g, q, lib=lib, count="x")
        bnx, bv = brute_force(g, q, count="x")
        if nx != bnx or not np.array_equal(v, bv):
            return False
    # the literal check on given matches: the twin X = {} -> false lists every
    # match; its violating rows are the GFD's violations
    og_lib = lib
    for seed in range(40):
        g, q = random_case(seed)
        twin = GFD(q.node_label, q.edges, [], [], True)
        _, matches = O.validate(g, twin, lib=og_lib)
        _, v = O.validate(g, q, lib=og_lib)
        got = O.sort_tuples(O.violating(O.OracleGraph(g, og_lib), q, matches))
        if not np.array_equal(got, v):
            return False
    return True


def test_unmutated_oracle_passes(oracle_mod):
    assert _pins_pass(O.bind_library(O.build_oracle()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    edits = MUTANTS[name]
    edits = edits if isinstance(edits, list) else [edits]
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
        src = src.replace(old, new)
    mpath = tmp_path / f"{name}.c"
    mpath.write_text(src)
    lib_path = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(lib_path), str(mpath)],
                   check=True)
    assert not _pins_pass(O.bind_library(str(lib_path))), f"pins did not catch {name}"
