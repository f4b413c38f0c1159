// Host-side planning of one GFD; see plan.h.
//
// Core-first decomposition (Section III.B, step 2a; the idea of postponing
// Cartesian products, Section III): the core is the 2-core of the undirected
// skeleton of Q (the vertices left after repeatedly removing vertices of
// degree <= 1). Non-core vertices of skeleton degree > 1 form the forest, the
// rest are leaves. The matching order is the core in breadth-first order from
// the root, then the forest, then the leaves. The order inside each of the
// three groups is cost-based, the way CFL-Match orders its paths: starting
// from the root (the vertex v_q from which the compact path index is built,
// Section III.B step 1a), the next vertex is the neighbour of the placed set
// whose addition gives the smallest expected number of partial matches, where
// the expectation is taken under the configuration model of the graph's degree
// distribution per label (an edge a -> b with probability d_out(a) d_in(b) / |E|);
// every core vertex is tried as the root and the order with the smallest sum of
// expected partial matches over all prefixes wins. The spanning
// tree of the index (step 1d) links every later vertex to its earliest-ordered
// skeleton neighbour; all other pattern pairs are checked after a tree match is
// found, including pairs WITHOUT a pattern edge, since a match may not contain
// additional edges (Section II, match definition; Section III on CFL-Match).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace gfd {

namespace {

int32_t exp_of(int32_t qlab) { return qlab == NOEDGE ? EXP_NONE : qlab; }

}  // namespace

int make_plan(const gfd_gfd* phi, int32_t n_attrs, const PlanStats& stats, HostPlan* P, bool induced,
              bool push_x) {
    if (!phi) {
        set_error(GFD_ERR_INVALID_ARG, "NULL GFD");
        return GFD_ERR_INVALID_ARG;
    }
    const int k = phi->k;
    if (k < 1 || !phi->node_label) {
        set_error(GFD_ERR_INVALID_ARG, "pattern needs k >= 1 nodes and node labels");
        return GFD_ERR_INVALID_ARG;
    }
    if (k > MAXK) {
        set_error(GFD_ERR_UNSUPPORTED, "pattern has %d nodes, limit is %d", k, MAXK);
        return GFD_ERR_UNSUPPORTED;
    }
    if (phi->m < 0 || (phi->m > 0 && (!phi->esrc || !phi->edst || !phi->elabel))) {
        set_error(GFD_ERR_INVALID_ARG, "pattern edge arrays missing");
        return GFD_ERR_INVALID_ARG;
    }
    int32_t q[MAXK][MAXK];
    for (int a = 0; a < MAXK; a++)
        for (int b = 0; b < MAXK; b++) q[a][b] = NOEDGE;
    for (int i = 0; i < k; i++) {
        int32_t L = phi->node_label[i];
        if (L < GFD_WILDCARD || L > 65534) {
            set_error(GFD_ERR_INVALID_ARG, "node %d label %d out of range", i, L);
            return GFD_ERR_INVALID_ARG;
        }
    }
    for (int e = 0; e < phi->m; e++) {
        int a = phi->esrc[e], b = phi->edst[e], l = phi->elabel[e];
        if (a < 0 || a >= k || b < 0 || b >= k || l < GFD_WILDCARD || l > 255) {
            set_error(GFD_ERR_INVALID_ARG, "pattern edge %d (%d -> %d, label %d) out of range", e, a, b, l);
            return GFD_ERR_INVALID_ARG;
        }
        if (q[a][b] != NOEDGE) {
            set_error(GFD_ERR_INVALID_ARG, "pattern edge %d -> %d given twice", a, b);
            return GFD_ERR_INVALID_ARG;
        }
        q[a][b] = l;
    }
    const int nlit = phi->nx + (phi->y_false ? 0 : phi->ny);
    if (phi->nx < 0 || phi->ny < 0 || (phi->nx > 0 && !phi->X) || (!phi->y_false && phi->ny > 0 && !phi->Y)) {
        set_error(GFD_ERR_INVALID_ARG, "literal arrays missing");
        return GFD_ERR_INVALID_ARG;
    }
    if (nlit > MAXLIT) {
        set_error(GFD_ERR_UNSUPPORTED, "%d literals, limit is %d", nlit, MAXLIT);
        return GFD_ERR_UNSUPPORTED;
    }
    // undirected skeleton (self-loops excluded)
    bool adj[MAXK][MAXK];
    int deg[MAXK];
    for (int a = 0; a < k; a++) {
        deg[a] = 0;
        for (int b = 0; b < k; b++) {
            adj[a][b] = a != b && (q[a][b] != NOEDGE || q[b][a] != NOEDGE);
            deg[a] += adj[a][b];
        }
    }
    // connected components of the skeleton (a disconnected pattern is matched
    // component after component; its levels that start a component have no
    // tree parent and take their candidates from the candidate list)
    int comp[MAXK], ncomp = 0, comp_size[MAXK];
    for (int a = 0; a < k; a++) comp[a] = -1;
    for (int a0 = 0; a0 < k; a0++) {
        if (comp[a0] >= 0) continue;
        int stack[MAXK], sp = 0;
        comp[a0] = ncomp;
        comp_size[ncomp] = 1;
        stack[sp++] = a0;
        while (sp) {
            const int a = stack[--sp];
            for (int b = 0; b < k; b++)
                if (adj[a][b] && comp[b] < 0) {
                    comp[b] = ncomp;
                    comp_size[ncomp]++;
                    stack[sp++] = b;
                }
        }
        ncomp++;
    }
    // 2-core by repeated removal of vertices of degree <= 1
    bool core[MAXK];
    {
        int d[MAXK];
        for (int a = 0; a < k; a++) {
            core[a] = true;
            d[a] = deg[a];
        }
        bool changed = true;
        while (changed) {
            changed = false;
            for (int a = 0; a < k; a++)
                if (core[a] && d[a] <= 1) {
                    core[a] = false;
                    changed = true;
                    for (int b = 0; b < k; b++)
                        if (adj[a][b] && core[b]) d[b]--;
                }
        }
    }
    bool any_core[MAXK] = {false};  // per component
    for (int a = 0; a < k; a++) any_core[comp[a]] |= core[a];
    // ---- cost model: log of the expected number of maps of the subpattern on
    // a node set (degrees counted inside the set only)
    const double NEG = -std::numeric_limits<double>::infinity();
    auto log_moment = [&](int32_t L, int a, int b) -> double {
        a = std::min(a, 3);
        b = std::min(b, 3);
        double m = stats.moments ? (L == GFD_WILDCARD ? stats.moments_all[4 * a + b]
                                                      : stats.moments[16 * (size_t)L + 4 * a + b])
                                 : 1.0;
        return m > 0 ? std::log(m) : NEG;
    };
    const double logE = std::log((double)std::max<int64_t>(1, stats.n_edges));
    auto log_est = [&](const bool* in) -> double {
        double sum = 0;
        for (int a = 0; a < k; a++) {
            if (!in[a]) continue;
            int dout = 0, din = 0;
            for (int b = 0; b < k; b++) {
                if (b == a || !in[b]) continue;
                if (q[a][b] != NOEDGE) {
                    dout++;
                    double p = q[a][b] == GFD_WILDCARD || !stats.elabel_frac ? 1.0 : stats.elabel_frac[q[a][b]];
                    sum += (p > 0 ? std::log(p) : NEG) - logE;
                }
                if (q[b][a] != NOEDGE) din++;
            }
            sum += log_moment(phi->node_label[a], dout, din);
        }
        return sum;
    };
    // greedy order from `root`: core, then forest, then leaves; returns the
    // sum of expected partial matches over the prefixes
    auto greedy = [&](int root, int* ord, int* core_end, int* forest_end) -> double {
        bool in[MAXK] = {false};
        in[root] = true;
        ord[0] = root;
        int nord = 1;
        double cost = 0;
        for (int phase = 0; phase < 3; phase++) {
            for (;;) {
                int best = -1;
                double best_le = 0;
                for (int u = 0; u < k; u++) {
                    if (in[u]) continue;
                    const bool grp = phase == 0 ? core[u] : phase == 1 ? (!core[u] && deg[u] > 1) : true;
                    if (!grp) continue;
                    bool touches = false;
                    for (int h = 0; h < nord; h++) touches |= adj[ord[h]][u];
                    if (!touches) continue;
                    in[u] = true;
                    const double le = log_est(in);
                    in[u] = false;
                    if (best < 0 || le < best_le) {
                        best = u;
                        best_le = le;
                    }
                }
                if (best < 0) break;
                in[best] = true;
                ord[nord++] = best;
                cost += std::exp(std::min(best_le, 700.0));
            }
            if (phase == 0) *core_end = nord;
            if (phase == 1) *forest_end = nord;
        }
        return nord == comp_size[comp[root]] ? cost : std::numeric_limits<double>::infinity();
    };
    // per component the root of least cost and its greedy order
    int best_root[MAXK];
    double best_cost[MAXK];
    for (int c = 0; c < ncomp; c++) {
        best_root[c] = -1;
        best_cost[c] = 0;
        for (int r = 0; r < k; r++) {
            if (comp[r] != c || (any_core[c] && !core[r])) continue;
            int ord[MAXK], ce = 0, fe = 0;
            const double cost = greedy(r, ord, &ce, &fe);
            if (best_root[c] < 0 || cost < best_cost[c]) {
                best_root[c] = r;
                best_cost[c] = cost;
            }
        }
    }
    // components with fewer expected matches first (their matches are the
    // rows the later components multiply)
    double comp_est[MAXK];
    for (int c = 0; c < ncomp; c++) {
        bool in[MAXK] = {false};
        for (int a = 0; a < k; a++) in[a] = comp[a] == c;
        comp_est[c] = log_est(in);
    }
    int corder[MAXK];
    for (int c = 0; c < ncomp; c++) corder[c] = c;
    std::stable_sort(corder, corder + ncomp, [&](int a, int b) { return comp_est[a] < comp_est[b]; });
    {
        int at = 0;
        for (int t = 0; t < ncomp; t++) {
            const int c = corder[t];
            int ce = 0, fe = 0;
            if (greedy(best_root[c], P->order + at, &ce, &fe) == std::numeric_limits<double>::infinity()) {
                set_error(GFD_ERR_INVALID_ARG, "internal: order incomplete");
                return GFD_ERR_INVALID_ARG;
            }
            if (t == 0) {
                P->core_size = ce;
                P->forest_end = fe;
            }
            at += comp_size[c];
        }
    }
    P->n_components = ncomp;
    P->k = k;
    for (int i = 0; i < k; i++) P->level_of[P->order[i]] = i;

    for (int i = 0; i < k; i++) {
        const int u = P->order[i];
        LevelPlan& L = P->lv[i];
        memset(&L, 0, sizeof(L));
        L.u = (int8_t)u;
        L.par = -1;
        if (i > 0) {
            for (int h = 0; h < i; h++)
                if (adj[P->order[h]][u]) {
                    L.par = (int8_t)h;
                    break;
                }
            if (L.par >= 0) {
                const int p = P->order[L.par];
                if (q[p][u] != NOEDGE) {
                    L.tdir = 1;
                    L.tlab = q[p][u];
                } else {
                    L.tdir = 0;
                    L.tlab = q[u][p];
                }
            }  // else: u starts a component
        }
        // pair checks against every earlier level
        int n = 0;
        for (int h = 0; h < i; h++) {
            const int w = P->order[h];
            const int32_t lu = phi->node_label[u], lw = phi->node_label[w];
            if (lu == GFD_WILDCARD || lw == GFD_WILDCARD || lu == lw) L.inj |= 1u << h;
            const bool skip_out = h == L.par && L.tdir == 0;  // u -> parent is the tree edge
            const bool skip_in = h == L.par && L.tdir == 1;   // parent -> u is the tree edge
            // non-induced matching checks only the pairs that are edges of Q
            if (!skip_out && (induced || q[u][w] != NOEDGE)) {
                L.chk_q[n] = (int8_t)h;
                L.chk_dir[n] = 1;
                L.chk_exp[n] = (int16_t)exp_of(q[u][w]);
                n++;
            }
            if (!skip_in && (induced || q[w][u] != NOEDGE)) {
                L.chk_q[n] = (int8_t)h;
                L.chk_dir[n] = 0;
                L.chk_exp[n] = (int16_t)exp_of(q[w][u]);
                n++;
            }
        }
        // Required edges first: a candidate usually fails there, after one
        // probe, before the absent-edge checks that almost always pass.
        {
            int8_t q2[2 * MAXK], d2[2 * MAXK];
            int16_t e2[2 * MAXK];
            int m2 = 0;
            for (int pass = 0; pass < 2; pass++)
                for (int c = 0; c < n; c++) {
                    const bool required = L.chk_exp[c] != EXP_NONE;
                    if (required == (pass == 0)) {
                        q2[m2] = L.chk_q[c];
                        d2[m2] = L.chk_dir[c];
                        e2[m2] = L.chk_exp[c];
                        m2++;
                    }
                }
            for (int c = 0; c < n; c++) {
                L.chk_q[c] = q2[c];
                L.chk_dir[c] = d2[c];
                L.chk_exp[c] = e2[c];
            }
        }
        L.nchk = (int8_t)n;
        L.nreq = 0;
        while (L.nreq < n && L.chk_exp[L.nreq] != EXP_NONE) L.nreq++;
        for (int c = 0; c < n; c++)
            L.chk_w[c] = (uint32_t)L.chk_q[c] | ((uint32_t)L.chk_dir[c] << 4) |
                         ((uint32_t)(uint16_t)L.chk_exp[c] << 16);
        // alternative generators: required edges to earlier levels other than the
        // spanning-tree parent (the adjacency of their image bounds the candidates)
        L.ngen = 0;
        for (int c = 0; c < n && L.ngen < 3; c++)
            if (L.chk_exp[c] != EXP_NONE && L.chk_q[c] != L.par) L.gen[L.ngen++] = (int8_t)c;
        // candidate filter key (degrees without self-loops)
        FilterKey& K = P->key[i];
        K.label = phi->node_label[u];
        K.dout_min = 0;
        K.din_min = 0;
        for (int w = 0; w < k; w++) {
            if (w == u) continue;
            K.dout_min += q[u][w] != NOEDGE;
            K.din_min += q[w][u] != NOEDGE;
        }
        K.self_exp = !induced && q[u][u] == NOEDGE ? EXP_SKIP : exp_of(q[u][u]);
        K.n_attr = 0;
        for (int t = 0; t < KEY_ATTRS; t++) K.attr_a[t] = K.attr_c[t] = 0;
        // refinement constraints
        P->td[i].clear();
        P->bu[i].clear();
        for (int w = 0; w < k; w++) {
            if (w == u) continue;
            const int h = P->level_of[w];
            if (q[u][w] != NOEDGE) (h < i ? P->td[i] : P->bu[i]).push_back(Con{(int8_t)h, 1, q[u][w]});
            if (q[w][u] != NOEDGE) (h < i ? P->td[i] : P->bu[i]).push_back(Con{(int8_t)h, 0, q[w][u]});
        }
    }
    // literals: checked at the last level, or with X pushed down at the level
    // where both ends are matched (constants in that node's filter key)
    P->lits.clear();
    P->push_x = push_x;
    auto add_lit = [&](const gfd_literal& l, bool is_x) -> int {
        if ((l.kind != 0 && l.kind != 1) || l.x < 0 || l.x >= k || l.a < 0 || l.a >= n_attrs ||
            (l.kind == 1 && (l.y < 0 || l.y >= k || l.b < 0 || l.b >= n_attrs))) {
            set_error(GFD_ERR_INVALID_ARG, "literal refers to a missing node or attribute");
            return GFD_ERR_INVALID_ARG;
        }
        DevLit d;
        d.kind = l.kind;
        d.xl = P->level_of[l.x];
        d.a = l.a;
        d.yl = l.kind == 1 ? P->level_of[l.y] : 0;
        d.b = l.kind == 1 ? l.b : 0;
        d.c = l.c;
        d.lvl = k - 1;
        if (is_x && push_x) {
            FilterKey& K = P->key[d.xl];
            if (l.kind == 0 && K.n_attr < KEY_ATTRS) {
                K.attr_a[K.n_attr] = l.a;
                K.attr_c[K.n_attr] = l.c;
                K.n_attr++;
                d.lvl = -1;
            } else {
                d.lvl = l.kind == 1 ? std::max(d.xl, d.yl) : d.xl;
                // level 0 is never expanded (its candidates are the roots): a
                // literal on the root alone is checked with level 1
                if (k > 1 && d.lvl == 0) d.lvl = 1;
            }
        }
        P->lits.push_back(d);
        return GFD_OK;
    };
    for (int i = 0; i < phi->nx; i++)
        if (int rc = add_lit(phi->X[i], true)) return rc;
    P->nx = phi->nx;
    P->y_false = phi->y_false ? 1 : 0;
    P->ny = 0;
    if (!P->y_false) {
        for (int i = 0; i < phi->ny; i++)
            if (int rc = add_lit(phi->Y[i], false)) return rc;
        P->ny = phi->ny;
    }
    // a canonical order of the filter conditions, so equal keys are shared
    for (int i = 0; i < k; i++) {
        FilterKey& K = P->key[i];
        if (K.n_attr == 2 && (K.attr_a[1] < K.attr_a[0] || (K.attr_a[1] == K.attr_a[0] && K.attr_c[1] < K.attr_c[0]))) {
            std::swap(K.attr_a[0], K.attr_a[1]);
            std::swap(K.attr_c[0], K.attr_c[1]);
        }
    }
    return GFD_OK;
}

}  // namespace gfd
