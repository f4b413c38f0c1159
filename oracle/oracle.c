/*
 * CPU oracle for GFD validation — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
 * file. It shares no code, header or constant with the CUDA library: it is an
 * independent, deliberately plain restatement of the definitions in Section II
 * of the paper (graph model, pattern, match, literals, violations), so that the
 * CUDA path can be compared with it element by element.
 *
 * What it computes (Section II, "match", "satisfies", "violation", Vio):
 *   A match of Q[x̄] in G is a map h : V_Q → V that is injective, keeps vertex
 *   labels (the wildcard "_" = -1 matches any label), and for every ordered pair
 *   (a, b) of pattern nodes — including a == b — has (a, b) ∈ E_Q exactly when
 *   (h(a), h(b)) ∈ E, with equal edge labels when both exist (a match may not
 *   contain additional edges). Matches are maps, so automorphic images count
 *   separately.
 *   x.A = c holds when h(x) has attribute A (value != INT32_MIN) equal to c;
 *   x.A = y.B holds when both attributes exist and are equal; false never holds.
 *   h is a violation when every X literal holds and (Y is `false` or some Y
 *   literal fails). The output is the number of matches and the violating
 *   tuples (h(x_0), ..., h(x_{k-1})) sorted lexicographically.
 *
 *   Non-induced mode (og_validate_mode with induced = 0): the matching of Bi et
 *   al. that Section III contrasts with the paper's definition, and the reading
 *   of the evaluation's path query (Section V: accounts 0 and 2 "may or may not"
 *   be connected). Only the pairs in E_Q constrain h: (a, b) ∈ E_Q implies
 *   (h(a), h(b)) ∈ E with an agreeing label; pairs outside E_Q (self-pairs
 *   included) are unconstrained. Injectivity and vertex labels stay.
 *
 * Algorithm: Ullmann-style backtracking (Section III's description of the
 * generic scheme). Node 0 first, then breadth-first over the undirected
 * skeleton of Q visiting neighbours by increasing node id; a disconnected
 * pattern continues with the lowest unplaced node of the next component. Level
 * 0 tries every vertex of G (or a caller-given subset of them); level i tries
 * the out- or in-neighbours of the image of the first already-placed skeleton
 * neighbour, or every vertex of G when it starts a new component (the match
 * conditions are the same for pairs across components: injective, and in the
 * induced mode no G edge where Q has none).
 * Every candidate is checked against ALL conditions above versus ALL nodes
 * placed before it. Edge lookup is a binary search in the oracle's own sorted
 * copy of the adjacency.
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define OG_ABSENT INT32_MIN
#define OG_NOEDGE (-2)
#define OG_WILDCARD (-1)
#define OG_MAXK 16

typedef struct {
    int32_t n;
    int64_t m;
    int32_t n_attrs;
    int64_t *out_off; int32_t *out_nbr; int32_t *out_lab; /* sorted by neighbour */
    int64_t *in_off;  int32_t *in_nbr;  int32_t *in_lab;  /* sorted by neighbour */
    int32_t *vlabel;
    int32_t *attrs;   /* [n_attrs][n] */
} og_graph;

typedef struct { int32_t kind, x, a, y, b, c; } og_lit;   /* kind 0: x.A=c, 1: x.A=y.B */

typedef struct {
    int32_t k;
    int32_t node_label[OG_MAXK];
    int32_t m;
    const int32_t *esrc, *edst, *elab;
    int32_t nx; const og_lit *X;
    int32_t ny; const og_lit *Y;
    int32_t y_false;
} og_gfd;

/* ------------------------------------------------------------------ graph */

static int og_cmp_pair(const void *pa, const void *pb) {
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    return (a[0] > b[0]) - (a[0] < b[0]);
}

/* Build one adjacency direction: for every edge (key[e] -> nbr[e], lab[e]) put
 * (nbr, lab) in row key, rows sorted by nbr. Returns 0, or 1 on a repeated pair. */
static int og_build_dir(int32_t n, int64_t m, const int64_t *key, const int64_t *nbr,
                        const int32_t *lab, int64_t **off_o, int32_t **nbr_o,
                        int32_t **lab_o) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(m > 0 ? m : 1));
    int32_t *onbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *olab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t e, v;
    int dup = 0;
    for (e = 0; e < m; e++) off[key[e] + 1]++;
    for (v = 0; v < n; v++) off[v + 1] += off[v];
    for (e = 0; e < m; e++) {
        int64_t p = off[key[e]] + fill[key[e]]++;
        pairs[2 * p] = (int32_t)nbr[e];
        pairs[2 * p + 1] = lab[e];
    }
    for (v = 0; v < n; v++) {
        int64_t a = off[v], b = off[v + 1];
        qsort(pairs + 2 * a, (size_t)(b - a), 2 * sizeof(int32_t), og_cmp_pair);
        for (e = a; e < b; e++) {
            onbr[e] = pairs[2 * e];
            olab[e] = pairs[2 * e + 1];
            if (e > a && onbr[e] == onbr[e - 1]) dup = 1;
        }
    }
    free(fill);
    free(pairs);
    *off_o = off; *nbr_o = onbr; *lab_o = olab;
    return dup;
}

void og_graph_free(og_graph *g) {
    if (!g) return;
    free(g->out_off); free(g->out_nbr); free(g->out_lab);
    free(g->in_off); free(g->in_nbr); free(g->in_lab);
    free(g->vlabel); free(g->attrs);
    free(g);
}

/* Copies the edge list (src[e] -> dst[e] with label lab[e]), vertex labels and
 * attributes. Returns NULL on an out-of-range id or a repeated (src, dst). */
og_graph *og_graph_new(int32_t n, int64_t m, const int64_t *src, const int64_t *dst,
                       const int32_t *lab, const int32_t *vlabel, int32_t n_attrs,
                       const int32_t *attrs) {
    og_graph *g;
    int64_t e;
    for (e = 0; e < m; e++)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return NULL;
    g = (og_graph *)calloc(1, sizeof(og_graph));
    g->n = n; g->m = m; g->n_attrs = n_attrs;
    if (og_build_dir(n, m, src, dst, lab, &g->out_off, &g->out_nbr, &g->out_lab) ||
        og_build_dir(n, m, dst, src, lab, &g->in_off, &g->in_nbr, &g->in_lab)) {
        og_graph_free(g);
        return NULL;
    }
    g->vlabel = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    memcpy(g->vlabel, vlabel, sizeof(int32_t) * (size_t)n);
    g->attrs = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)(n_attrs > 0 ? n_attrs : 1));
    memcpy(g->attrs, attrs, sizeof(int32_t) * (size_t)n * (size_t)n_attrs);
    return g;
}

/* Label of the edge a -> b, or OG_NOEDGE. */
static int32_t og_edge(const og_graph *g, int32_t a, int32_t b) {
    int64_t lo = g->out_off[a], hi = g->out_off[a + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->out_nbr[mid] < b) lo = mid + 1;
        else hi = mid;
    }
    if (lo < g->out_off[a + 1] && g->out_nbr[lo] == b) return g->out_lab[lo];
    return OG_NOEDGE;
}

/* --------------------------------------------------------------- matching */

typedef struct {
    const og_graph *g;
    const og_gfd *q;
    int32_t qedge[OG_MAXK][OG_MAXK];   /* label of pattern edge a -> b, or OG_NOEDGE */
    int32_t order[OG_MAXK];            /* order[i] = pattern node placed at level i */
    int32_t pnode[OG_MAXK];            /* first earlier-placed skeleton neighbour */
    int32_t pout[OG_MAXK];             /* 1: iterate out-nbrs of h(pnode), 0: in-nbrs */
    int32_t h[OG_MAXK];                /* h[node] = vertex */
    uint64_t n_matches;
    uint64_t n_x_matches;              /* matches with h ⊨ X */
    int32_t *viol; int64_t n_viol, cap_viol;
    double deadline;                   /* monotonic seconds; 0 = none */
    uint64_t calls;
    int aborted;
} og_state;

static double og_now(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static int og_label_ok(int32_t want, int32_t have) {
    return want == OG_WILDCARD || want == have;
}

/* Matching mode of the call running on this thread: 1 induced, 0 non-induced. */
static _Thread_local int og_induced = 1;

/* Do pattern edge label `ql` (or OG_NOEDGE) and graph edge label `gl` (or
 * OG_NOEDGE) agree? Both absent, or both present with equal label / wildcard;
 * in non-induced mode an absent pattern pair accepts anything. */
static int og_pair_ok(int32_t ql, int32_t gl) {
    if (!og_induced && ql == OG_NOEDGE) return 1;
    if (ql == OG_NOEDGE) return gl == OG_NOEDGE;
    if (gl == OG_NOEDGE) return 0;
    return og_label_ok(ql, gl);
}

static int32_t og_attr(const og_graph *g, int32_t a, int32_t v) {
    return g->attrs[(int64_t)a * g->n + v];
}

static int og_lit_holds(const og_state *s, const og_lit *l) {
    int32_t va = og_attr(s->g, l->a, s->h[l->x]);
    int32_t vb;
    if (va == OG_ABSENT) return 0;
    if (l->kind == 0) return va == l->c;
    vb = og_attr(s->g, l->b, s->h[l->y]);
    if (vb == OG_ABSENT) return 0;
    return va == vb;
}

/* Does the match in s->h satisfy X (every X literal holds)? */
static int og_x_holds(const og_state *s) {
    const og_gfd *q = s->q;
    int i, x_ok = 1;
    for (i = 0; i < q->nx; i++) x_ok = x_ok && og_lit_holds(s, &q->X[i]);
    return x_ok;
}

/* Is the match in s->h a violation: h satisfies X, and Y is false or some Y
 * literal fails? */
static int og_is_violation(const og_state *s) {
    const og_gfd *q = s->q;
    int i, y_ok = 1;
    if (!og_x_holds(s)) return 0;
    if (q->y_false) return 1;
    for (i = 0; i < q->ny; i++) y_ok = y_ok && og_lit_holds(s, &q->Y[i]);
    return !y_ok;
}

static void og_record(og_state *s) {
    const og_gfd *q = s->q;
    s->n_matches++;
    s->n_x_matches += (uint64_t)og_x_holds(s);
    if (!og_is_violation(s)) return;
    if (s->n_viol == s->cap_viol) {
        s->cap_viol = s->cap_viol ? 2 * s->cap_viol : 1024;
        s->viol = (int32_t *)realloc(s->viol, sizeof(int32_t) * (size_t)s->cap_viol * (size_t)q->k);
    }
    memcpy(s->viol + s->n_viol * q->k, s->h, sizeof(int32_t) * (size_t)q->k);
    s->n_viol++;
}

/* May vertex v be the image of pattern node order[i], given levels 0..i-1? */
static int og_candidate_ok(const og_state *s, int i, int32_t v) {
    const og_graph *g = s->g;
    int32_t u = s->order[i];
    int j;
    if (!og_label_ok(s->q->node_label[u], g->vlabel[v])) return 0;
    if (!og_pair_ok(s->qedge[u][u], og_edge(g, v, v))) return 0;
    for (j = 0; j < i; j++) {
        int32_t w = s->order[j];
        int32_t hw = s->h[w];
        if (hw == v) return 0;                                        /* injective */
        if (!og_pair_ok(s->qedge[u][w], og_edge(g, v, hw))) return 0; /* u -> w */
        if (!og_pair_ok(s->qedge[w][u], og_edge(g, hw, v))) return 0; /* w -> u */
    }
    return 1;
}

static void og_extend(og_state *s, int i) {
    const og_graph *g = s->g;
    int32_t u, hp;
    int64_t e, a, b;
    if (i == s->q->k) { og_record(s); return; }
    u = s->order[i];
    if (s->pnode[i] < 0) { a = 0; b = g->n; hp = -1; }           /* every vertex */
    else {
        hp = s->h[s->pnode[i]];
        if (s->pout[i]) { a = g->out_off[hp]; b = g->out_off[hp + 1]; }
        else            { a = g->in_off[hp];  b = g->in_off[hp + 1]; }
    }
    for (e = a; e < b; e++) {
        int32_t v = hp < 0 ? (int32_t)e : s->pout[i] ? g->out_nbr[e] : g->in_nbr[e];
        if (s->aborted) return;
        if (s->deadline > 0 && (++s->calls & 0xfff) == 0 && og_now() > s->deadline) {
            s->aborted = 1;
            return;
        }
        if (!og_candidate_ok(s, i, v)) continue;
        s->h[u] = v;
        og_extend(s, i + 1);
    }
}

/* Validate one GFD; induced = 1 is the paper's matching, 0 the non-induced
 * mode described at the top. *n_x_matches (if not NULL) receives the number of
 * matches that satisfy X (Section II: only they can be violations). roots: the vertices tried for pattern node 0 (NULL: all of V).
 * seconds > 0 bounds the run: the root being searched when time runs out is
 * dropped together with its matches, and *roots_done tells how many roots were
 * searched to the end (all of them when there is no bound).
 * Returns 0 on success, 1 for a malformed pattern. On success the
 * caller owns *viol_out (free with og_free). */
int og_validate_mode(const og_graph *g, const og_gfd *q, int induced, const int32_t *roots, int64_t n_roots,
                     double seconds, uint64_t *n_matches, int32_t **viol_out, int64_t *n_viol,
                     int64_t *roots_done, uint64_t *n_x_matches) {
    og_state s;
    int32_t placed[OG_MAXK];
    int i, j, head, tail;
    int64_t r;
    memset(&s, 0, sizeof(s));
    s.g = g; s.q = q;
    og_induced = induced ? 1 : 0;
    if (q->k < 1 || q->k > OG_MAXK) return 1;
    for (i = 0; i < OG_MAXK; i++)
        for (j = 0; j < OG_MAXK; j++) s.qedge[i][j] = OG_NOEDGE;
    for (i = 0; i < q->m; i++) {
        if (q->esrc[i] < 0 || q->esrc[i] >= q->k || q->edst[i] < 0 || q->edst[i] >= q->k)
            return 1;
        if (s.qedge[q->esrc[i]][q->edst[i]] != OG_NOEDGE) return 1; /* repeated edge */
        s.qedge[q->esrc[i]][q->edst[i]] = q->elab[i];
    }
    for (i = 0; i < q->nx + q->ny; i++) {
        const og_lit *l = i < q->nx ? &q->X[i] : &q->Y[i - q->nx];
        if (l->x < 0 || l->x >= q->k || l->a < 0 || l->a >= g->n_attrs) return 1;
        if (l->kind == 1 && (l->y < 0 || l->y >= q->k || l->b < 0 || l->b >= g->n_attrs))
            return 1;
        if (l->kind != 0 && l->kind != 1) return 1;
    }
    /* order: node 0, then BFS over the undirected skeleton by increasing id;
     * each further component from its lowest node */
    for (i = 0; i < q->k; i++) placed[i] = -1;
    tail = 0;
    for (i = 0; i < q->k; i++) {
        if (placed[i] >= 0) continue;
        head = tail;
        placed[i] = tail;
        s.order[tail++] = i;
        while (head < tail) {
            int32_t a = s.order[head++];
            for (j = 0; j < q->k; j++) {
                if (j == a || placed[j] >= 0) continue;
                if (s.qedge[a][j] == OG_NOEDGE && s.qedge[j][a] == OG_NOEDGE) continue;
                placed[j] = tail;
                s.order[tail++] = j;
            }
        }
    }
    for (i = 1; i < q->k; i++) {
        int32_t u = s.order[i];
        s.pnode[i] = -1;                                          /* starts a component */
        for (j = 0; j < i; j++) {
            int32_t w = s.order[j];
            if (s.qedge[w][u] != OG_NOEDGE) { s.pnode[i] = w; s.pout[i] = 1; break; }
            if (s.qedge[u][w] != OG_NOEDGE) { s.pnode[i] = w; s.pout[i] = 0; break; }
        }
    }
    s.deadline = seconds > 0 ? og_now() + seconds : 0;
    for (r = 0; r < (roots ? n_roots : (int64_t)g->n); r++) {
        int32_t v = roots ? roots[r] : (int32_t)r;
        uint64_t m0 = s.n_matches, x0 = s.n_x_matches;
        int64_t v0 = s.n_viol;
        if (v < 0 || v >= g->n) continue;
        if (!og_candidate_ok(&s, 0, v)) continue;
        s.h[0] = v;
        og_extend(&s, 1);
        if (s.aborted) {          /* drop the unfinished root */
            s.n_matches = m0;
            s.n_x_matches = x0;
            s.n_viol = v0;
            break;
        }
    }
    if (roots_done) *roots_done = r;
    *n_matches = s.n_matches;
    if (n_x_matches) *n_x_matches = s.n_x_matches;
    *viol_out = s.viol;
    *n_viol = s.n_viol;
    return 0;
}

/* The paper's (induced) matching, bounded in time as og_validate_mode. */
int og_validate_budget(const og_graph *g, const og_gfd *q, const int32_t *roots, int64_t n_roots,
                       double seconds, uint64_t *n_matches, int32_t **viol_out, int64_t *n_viol,
                       int64_t *roots_done) {
    return og_validate_mode(g, q, 1, roots, n_roots, seconds, n_matches, viol_out, n_viol, roots_done, NULL);
}

int og_validate(const og_graph *g, const og_gfd *q, const int32_t *roots, int64_t n_roots,
                uint64_t *n_matches, int32_t **viol_out, int64_t *n_viol) {
    return og_validate_mode(g, q, 1, roots, n_roots, 0.0, n_matches, viol_out, n_viol, NULL, NULL);
}

/* The literal check alone on given matches: flags[i] = 1 when the k-tuple
 * tuples[i] = (h(x_0), ..., h(x_{k-1})), taken as a match of q's pattern (not
 * checked as one), is a violation of q, else 0. Returns 0, or 1 for a
 * malformed GFD or an out-of-range vertex. */
int og_violating(const og_graph *g, const og_gfd *q, const int32_t *tuples, int64_t n, uint8_t *flags) {
    og_state s;
    int64_t t;
    int i;
    memset(&s, 0, sizeof(s));
    s.g = g; s.q = q;
    if (q->k < 1 || q->k > OG_MAXK) return 1;
    for (i = 0; i < q->nx + q->ny; i++) {
        const og_lit *l = i < q->nx ? &q->X[i] : &q->Y[i - q->nx];
        if (l->x < 0 || l->x >= q->k || l->a < 0 || l->a >= g->n_attrs) return 1;
        if (l->kind == 1 && (l->y < 0 || l->y >= q->k || l->b < 0 || l->b >= g->n_attrs))
            return 1;
        if (l->kind != 0 && l->kind != 1) return 1;
    }
    for (t = 0; t < n; t++) {
        for (i = 0; i < q->k; i++) {
            s.h[i] = tuples[t * q->k + i];
            if (s.h[i] < 0 || s.h[i] >= g->n) return 1;
        }
        flags[t] = (uint8_t)og_is_violation(&s);
    }
    return 0;
}

/* --------------------------------------------------------------- sorting */

static _Thread_local int og_sort_k;

static int og_cmp_tuple(const void *pa, const void *pb) {
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    int i;
    for (i = 0; i < og_sort_k; i++)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

/* Sort n k-tuples lexicographically in place (Vio is a set; this fixes an order). */
void og_sort_tuples(int32_t *t, int64_t n, int32_t k) {
    if (n <= 1 || k <= 0) return;
    og_sort_k = k;
    qsort(t, (size_t)n, sizeof(int32_t) * (size_t)k, og_cmp_tuple);
}

void og_free(void *p) { free(p); }
