// Host-side planning of one GFD (Section III.B): core-first decomposition of
// the pattern, root and spanning tree of the compact path index, matching
// order, per-level checks of the remaining pattern pairs, filter keys,
// refinement constraints and literal slots.
#pragma once

#include <vector>

#include "common.cuh"

namespace gfd {

// A refinement constraint on level `lvl`: every candidate x of that level needs
// a neighbour in C(q), through an out-edge x -> y (dir 1) or an in-edge
// y -> x (dir 0), with label `lab` (or any label for GFD_WILDCARD).
struct Con {
    int8_t q;
    int8_t dir;
    int32_t lab;
};

struct HostPlan {
    int k = 0;
    int order[MAXK];      // node at level
    int level_of[MAXK];   // level of node
    int core_size = 0;    // levels [0, core_size) are the core (2-core, or the root)
    int forest_end = 0;   // levels [core_size, forest_end) are forest nodes, the rest leaves
                          // (of the first component)
    int n_components = 1; // skeleton components, matched one after another
    LevelPlan lv[MAXK];
    FilterKey key[MAXK];  // candidate filter key per level
    std::vector<Con> td[MAXK];  // constraints from earlier levels
    std::vector<Con> bu[MAXK];  // constraints from later levels
    std::vector<DevLit> lits;   // X then Y
    int nx = 0, ny = 0, y_false = 0;
    bool push_x = false;
};

// Graph statistics used to order the pattern: per vertex label L the moments
// M_L(a, b) = sum over vertices v with label L of d_out(v)^a * d_in(v)^b for
// a, b in 0..3 (moments[16 * L + 4 * a + b]; moments_all over all vertices) and
// the fraction of edges carrying each edge label.
struct PlanStats {
    int64_t n_vertices = 0;
    int64_t n_edges = 0;
    const double* moments = nullptr;      // [65536][16]
    const double* moments_all = nullptr;  // [16]
    const double* elabel_frac = nullptr;  // [256]
};

// Returns GFD_OK or an error code (message set). induced = false plans the
// non-induced matching: no absent-edge checks and no self-loop requirement on
// pattern nodes without one.
// push_x = true places each X literal at the level where both its ends are
// matched and moves constant ones into the candidate filter (up to KEY_ATTRS
// per pattern node).
int make_plan(const gfd_gfd* phi, int32_t n_attrs, const PlanStats& stats, HostPlan* out, bool induced = true,
              bool push_x = false);

}  // namespace gfd
