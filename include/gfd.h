/*
 * gfd.h — C-ABI of the GB300 GFD validation library (libgfd.so).
 *
 * The calls follow the paper's statement of the validation problem (Section II,
 * "the validation problem"): given a graph G and a set Σ of GFDs, find
 * Vio(Σ, G), the matches h(x̄) of each φ = (Q[x̄], X → Y) that satisfy X and
 * not Y (or satisfy X when Y is `false`). The matching itself follows
 * Section III.B (FastGFDs): a compact path index (candidate filtering by label
 * and degree, breadth-first refinement that removes dead ends, index edges
 * along a spanning tree of Q, remaining edges checked afterwards) and a
 * core-first matching order.
 *
 * Conventions for every call:
 *   - Return value: GFD_OK (0) or one of the GFD_ERR_* codes. On an error,
 *     gfd_last_error() returns a message for the calling thread and no output
 *     pointer is written.
 *   - Inputs are read during the call only (copied where kept); the caller keeps
 *     ownership of everything it passes in. All input pointers are HOST pointers.
 *   - Handles returned by the library (gfd_graph, gfd_result) are owned by the
 *     caller and released with the matching *_free call; *_free(NULL) is a no-op.
 *   - All GPU work is issued on opts->cuda_stream (a cudaStream_t) when given,
 *     else on a stream owned by the graph handle. Calls are blocking: when they
 *     return, the results they report are final.
 *   - Every wait the library performs on the device is bounded; a wait that runs
 *     out returns GFD_ERR_TIMEOUT instead of hanging.
 */
#ifndef GFD_H
#define GFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfd_graph gfd_graph;    /* opaque, device-resident, library-owned */
typedef struct gfd_result gfd_result;  /* opaque, library-owned */
typedef struct gfd_session gfd_session; /* opaque serving session */

enum {
    GFD_OK = 0,
    GFD_ERR_INVALID_ARG = 1,   /* malformed graph, pattern or literal */
    GFD_ERR_UNSUPPORTED = 2,   /* valid but outside what the library handles */
    GFD_ERR_OUT_OF_MEMORY = 3, /* device or host allocation failed */
    GFD_ERR_OVERFLOW = 4,      /* a bounded buffer could not hold the result */
    GFD_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    GFD_ERR_CUDA = 6           /* a CUDA runtime call failed */
};

/* Label value "_" that matches any label (Section II, wildcard). */
#define GFD_WILDCARD (-1)
/* Attribute value meaning "vertex has no such attribute" (Section II: a literal
 * is satisfied only when the attribute exists). */
#define GFD_ATTR_ABSENT INT32_MIN
/* Largest pattern handled: |V_Q| <= GFD_MAX_K. */
#define GFD_MAX_K 16
/* Most GFDs one gfd_validate_batch (or gfd_autotune) call takes, and most slots
 * of a session: every step of the enumeration numbers its work tiles in 32
 * bits, and a slot's step holds up to 2^20 tiles. Split larger batches. */
#define GFD_MAX_SLOTS 4095

/*
 * Graph G = (V, E, L, F_A) (Section II, "directed labeled graphs with
 * attributes"): V = {0 .. n_vertices-1}, E ⊆ V×V a set (at most one edge per
 * ordered pair, self-loops allowed), a label per vertex and per edge, and an
 * int32 attribute tuple per vertex. Layout:
 *   out_off    [n_vertices+1]  CSR row offsets, out_off[0] = 0, non-decreasing,
 *                              out_off[n_vertices] = n_edges
 *   out_dst    [n_edges]       destinations, strictly increasing within a row
 *   out_elabel [n_edges]       edge labels, 0 <= label <= 255
 *   in_off/in_src/in_elabel    the reverse CSR (rows by destination, sources
 *                              strictly increasing); all three NULL = built by
 *                              the library. If given, must describe the same E.
 *   vlabel     [n_vertices]    vertex labels, 0 <= label <= 65534
 *   attrs      [n_attrs][n_vertices]  structure of arrays; GFD_ATTR_ABSENT = none
 * Limits: n_edges < 2^32, and n_vertices <= 2^(32 - b) where b is the number of
 * bits of the largest edge label (at least 1); beyond them GFD_ERR_UNSUPPORTED.
 */
typedef struct {
    int32_t n_vertices;
    int64_t n_edges;
    int32_t n_attrs;
    const int64_t *out_off;
    const int32_t *out_dst;
    const int32_t *out_elabel;
    const int64_t *in_off;
    const int32_t *in_src;
    const int32_t *in_elabel;
    const int32_t *vlabel;
    const int32_t *attrs;
} gfd_graph_desc;

/* Attribute constraint (Section II): kind 0 is the constant constraint
 * x.A = c (fields x, a, c); kind 1 is the variable constraint x.A = y.B
 * (fields x, a, y, b). x and y are pattern node ids, a and b attribute ids. */
typedef struct {
    int32_t kind;
    int32_t x, a;
    int32_t y, b;
    int32_t c;
} gfd_literal;

/*
 * GFD φ = (Q[x̄], X → Y) or (Q[x̄], X → false) (Section II). Pattern node i is
 * the variable x_i (μ is the identity). node_label[k]: label or GFD_WILDCARD.
 * Directed pattern edges esrc[i] -> edst[i] with label elabel[i] (or
 * GFD_WILDCARD), at most one per ordered pair. X has nx literals, Y has ny;
 * y_false != 0 means the right-hand side is `false` (Y is then ignored).
 * Limits: 1 <= k <= GFD_MAX_K, else GFD_ERR_UNSUPPORTED. A disconnected Q is
 * matched component after component (Section II's conditions hold across
 * components too: injective, and with induced matching no G edge between the
 * images of nodes in different components); the work grows with the product of
 * the components' match counts, and a step whose fan-out sum exceeds 2^40
 * returns GFD_ERR_OVERFLOW.
 */
typedef struct {
    int32_t k;
    const int32_t *node_label;
    int32_t m;
    const int32_t *esrc;
    const int32_t *edst;
    const int32_t *elabel;
    int32_t nx;
    const gfd_literal *X;
    int32_t ny;
    const gfd_literal *Y;
    int32_t y_false;
} gfd_gfd;

/* gfd_opts.flags */
#define GFD_FLAG_NO_REFINE     0x1  /* candidate filter only: skip the top-down and
                                       bottom-up refinement (results unchanged) */
#define GFD_FLAG_HOST_LOOP     0x2  /* drive the enumeration from a host loop of
                                       per-step launches instead of one persistent
                                       cooperative launch (results unchanged) */
#define GFD_FLAG_PROFILE       0x4  /* time each kernel class with CUDA events;
                                       read back with gfd_result_profile() */
#define GFD_FLAG_NO_GRAPH      0x8  /* host loop without CUDA-graph capture */
#define GFD_FLAG_NON_INDUCED   0x10 /* non-induced matching: only the pairs in E_Q
                                       constrain a match ((a,b) in E_Q implies
                                       (h(a),h(b)) in E with an agreeing label);
                                       pairs outside E_Q, self-pairs included, are
                                       free. The matching of Bi et al. that
                                       Section III contrasts with the paper's
                                       (induced) definition, and the reading of
                                       the path query of Section V. Changes the
                                       result: matches and Vio are supersets. */
#define GFD_FLAG_PUSH_X        0x20 /* apply X during the search: constant X
                                       literals in the candidate filter (two per
                                       pattern node), the others as soon as both
                                       ends are matched. Only matches satisfying
                                       X can be violations (Section II), so Vio is
                                       unchanged; gfd_result_matches then counts
                                       the matches that satisfy X. */

#define GFD_FLAG_KEEP_CANDIDATES 0x40 /* keep a host copy of every pattern node's
                                       refined candidate list C(u) (Section III.B
                                       step 1c) in the result, read with
                                       gfd_result_candidates (batch calls only;
                                       for inspection and tests) */

#define GFD_FLAG_COUNT         0x80 /* counting pass: run the enumeration with an
                                       instrumented kernel that counts what the
                                       run reads (gfd_result_stat 7..28); the
                                       results are unchanged, the run is slower */

/* Tuning options; a NULL gfd_opts* or zero fields select the defaults. */
typedef struct {
    int64_t frontier_budget_bytes; /* device bytes for partial-match buffers
                                      (0: the tuned choice, else min(128 GiB,
                                      half the free device memory)). A budget
                                      that cannot hold 1024 partial matches per
                                      level of every GFD of a call gives
                                      GFD_ERR_OUT_OF_MEMORY (calls with
                                      chunk_rows set, and sessions, use at
                                      least 1024 instead) */
    int32_t chunk_rows;            /* partial matches expanded per step and GFD */
    int32_t kernel_variant;        /* enumeration kernel: 0 = the graph's tuned
                                      choice (gfd_autotune) or the default;
                                      1..6 = a fixed variant (threads per block
                                      and minimum resident blocks per SM:
                                      256/4, 256/6, 256/8, 128/12, 256/5, 512/3) */
    int64_t max_violations_hint;   /* violations the run stores before it must
                                      run again with exactly enough room (all
                                      GFDs of a call together) */
    void *cuda_stream;             /* cudaStream_t to issue work on */
    int32_t flags;                 /* GFD_FLAG_* */
    int32_t tile_iters;            /* work items per block visit, in units of the
                                      block size (0: tuned choice or 8) */
} gfd_opts;

/* Copy a graph to the device, validate it (row order, ranges, label limits,
 * reverse CSR consistency) and keep it resident. *out is set on GFD_OK. */
int gfd_graph_load(const gfd_graph_desc *desc, const gfd_opts *opts, gfd_graph **out);

/* Release a graph handle and its device memory (the graph G of Section II
 * loaded by gfd_graph_load). Waits for work still running on the graph's
 * stream; NULL is a no-op. Free the graph's sessions first. Its results stay
 * valid for their counts, for tuples already read to the host and for
 * gfd_result_free, but tuples not yet read are sorted on the graph's stream
 * (unless the call named another): read them before freeing the graph. */
void gfd_graph_free(gfd_graph *g);

/* Autotuner: validate the batch phis[0..n) once per enumeration-kernel variant,
 * tile size (8 or 32 block-sized iterations) and frontier budget (the budget of
 * opts, or the default, and a quarter of it), time the device work of each run
 * with CUDA events, and keep the fastest choice in the graph handle, where later
 * calls with kernel_variant 0, tile_iters 0 and no frontier budget of their own
 * use it. *best (may be NULL) receives opts with the chosen kernel_variant,
 * tile_iters and frontier_budget_bytes. The trial runs' results are discarded. */
int gfd_autotune(gfd_graph *g, const gfd_gfd *const *phis, int32_t n, const gfd_opts *opts,
                 gfd_opts *best);

/* |V|, |E| (Section II, G = (V, E, L, F_A)) and the resident device bytes of
 * a loaded graph; 0 for NULL. */
int32_t gfd_graph_vertices(const gfd_graph *g);
int64_t gfd_graph_edges(const gfd_graph *g);
int64_t gfd_graph_device_bytes(const gfd_graph *g);

/* Validate one GFD: every match of Q is enumerated and checked (Section II,
 * Vio({φ}, G); Section III.B, the CPI and core-first matching). *out receives
 * the result handle on GFD_OK. */
int gfd_validate(const gfd_graph *g, const gfd_gfd *phi, const gfd_opts *opts,
                 gfd_result **out);

/* Validate n GFDs against the same resident graph in one batched run: the
 * candidate filters are shared between GFDs and all GFDs' matches are expanded
 * together by one persistent launch (Section II, Vio(Σ, G) as the per-GFD
 * lists). out[i] receives the result of phis[i]; on an error no entry is set.
 * n above GFD_MAX_SLOTS gives GFD_ERR_UNSUPPORTED. */
int gfd_validate_batch(const gfd_graph *g, const gfd_gfd *const *phis, int32_t n,
                       const gfd_opts *opts, gfd_result **out);

/* Number of matches h of Q in G (Section II, "match": all of them, whether or
 * not h satisfies X; with GFD_FLAG_PUSH_X only those that satisfy X). 0 for
 * NULL. */
uint64_t gfd_result_matches(const gfd_result *r);
/* Number of violations |Vio({φ}, G)| (Section II: matches that satisfy X and
 * not Y, or satisfy X when Y is false). 0 for NULL. */
uint64_t gfd_result_violations(const gfd_result *r);
/* k = |x̄|, the length of each violation tuple h(x̄) (Section II). 0 for NULL. */
int32_t gfd_result_arity(const gfd_result *r);
/* The violations as [n_violations][k] int32 tuples (h(x_0), ..., h(x_{k-1})),
 * sorted lexicographically; host memory owned by the result. The sort and the
 * copy to the host happen on the first call. NULL on error (see
 * gfd_last_error) or when there are no violations. */
const int32_t *gfd_result_tuples(gfd_result *r);
/* The same tuples written straight into caller-owned host memory `out` of
 * `capacity` int32 (at least n_violations * k), without a copy owned by the
 * result: the device sorts them and copies them to `out` on every call that
 * comes before a gfd_result_tuples call (after one, they are copied from the
 * result's buffer). Returns GFD_OK, GFD_ERR_INVALID_ARG (NULL or too small a
 * buffer), GFD_ERR_OUT_OF_MEMORY or a CUDA error code. */
int gfd_result_copy_tuples(gfd_result *r, int32_t *out, uint64_t capacity);
/* The sorted tuples of n results (say, one gfd_validate_batch) written back to
 * back into caller-owned host memory `out` of `capacity` int32: result 0's
 * n_violations * k ints, then result 1's, and so on. One device sort over all of
 * them (keyed by result, then tuple) and one copy, instead of one per result.
 * The results may come from calls on different streams: the sort runs on the
 * stream of the first result with violations and waits for the others' streams.
 * Returns GFD_OK, GFD_ERR_INVALID_ARG (NULL arguments or too small a buffer),
 * GFD_ERR_OUT_OF_MEMORY or a CUDA error code. */
int gfd_results_copy_tuples(gfd_result *const *rs, int32_t n, int32_t *out, uint64_t capacity);
/* Device time in milliseconds spent in kernel class `which` (0 candidate
 * filter, 1 refinement, 2 index build, 3 enumeration, 4 result sort) and the
 * number of launches, when GFD_FLAG_PROFILE was set; else 0. */
double gfd_result_profile(const gfd_result *r, int32_t which, int64_t *launches);
/* Statistics of the run: 0 supersteps, 1 work items expanded, 2 partial
 * matches written, 3 edge-lookup probes (whole run), 4 candidate-list entries
 * (sum over pattern nodes), 5 index entries, 6 number of extra runs made
 * because the violations of the call outgrew max_violations_hint. With
 * GFD_FLAG_COUNT, 7..28 are the whole call's counters of what its kernels read:
 * 7 work items (entries of the index lists N_u, Section III.B, or of another
 * candidate list), 8 of them at the last level, 9 partial matches expanded,
 * 10 sum over expanded partial matches of the adjacency lengths of their
 * backward non-tree neighbours' images, 11 pair checks, 12 of them settled by
 * the neighbourhood signature, 13 adjacency binary searches, 14 adjacency
 * entries those searches read, 15 absent-edge checks, 16 sum over absent-edge
 * checks of ceil(log2(d + 1)) (d the shorter adjacency list), 17 signature
 * loads, 18 attribute loads of literal checks, 19 partial matches written,
 * 20 candidates whose adjacency the refinement and index build scanned, 21
 * adjacency entries they read, 22 warp iterations of the expansion, 23 sum over
 * them of the largest number of search loads one lane made, 24..26 SM cycles
 * warps spent setting up tiles, in iterations at intermediate levels and at the
 * last level, 27 warp iterations at intermediate levels, 28 the number of
 * distinct filter keys (high 32 bits) and of candidate bitmaps compacted (low
 * 32 bits). */
uint64_t gfd_result_stat(const gfd_result *r, int32_t which);
/* The refined candidate list C(u) of pattern node `node` (Section III.B step
 * 1c: label and degree filter, then top-down and bottom-up refinement), kept by
 * a batch call made with GFD_FLAG_KEEP_CANDIDATES: *list receives increasing
 * vertex ids in host memory owned by the result, *n their number. Every match
 * h has h(node) in this list (refinement removes only dead ends). Returns
 * GFD_OK, or GFD_ERR_INVALID_ARG (NULL argument, node out of range, or the
 * result kept no lists). */
int gfd_result_candidates(const gfd_result *r, int32_t node, const int32_t **list, int64_t *n);
/* Release a result and its device and host buffers; NULL is a no-op. */
void gfd_result_free(gfd_result *r);

/*
 * Serving session with continuous batching (Section II's validation problem
 * answered per request). Requests are single GFDs, queued by
 * gfd_session_submit. Each gfd_session_step admits queued requests, in arrival
 * order, into free slots while their device memory (index, partial-match
 * buffers and a violation buffer of opts->max_violations_hint tuples, default
 * 2^20) fits opts->frontier_budget_bytes; builds their indexes together; then
 * runs one round of enumeration steps over ALL running requests at once, so
 * requests admitted later overlap on the device with those already running.
 * Requests that finish in that round are moved to the result queue, read with
 * gfd_session_next_result in completion order. The graph stays resident and
 * the session's slot tables are reused across requests. opts->flags apply to
 * every request of the session (GFD_FLAG_NON_INDUCED, GFD_FLAG_PUSH_X);
 * disconnected patterns are admitted like any other.
 */
/* max_slots: requests running at once, 1..GFD_MAX_SLOTS (else
 * GFD_ERR_INVALID_ARG). */
int gfd_session_create(const gfd_graph *g, int32_t max_slots, const gfd_opts *opts,
                       gfd_session **out);
/* Queue one GFD (copied); *request_id identifies its result. The GFD is
 * checked here: an invalid one is rejected with the usual error codes. */
int gfd_session_submit(gfd_session *s, const gfd_gfd *phi, int64_t *request_id);
/* Admit, run one round of enumeration steps, collect finished requests.
 * *n_advanced: requests that ran together in this round; *n_running and
 * *n_queued: requests still running and still waiting afterwards (any of the
 * three may be NULL). */
int gfd_session_step(gfd_session *s, int32_t *n_advanced, int32_t *n_running, int32_t *n_queued);
/* Pop one finished request: *request_id = -1 and *out = NULL when none is
 * ready. The caller owns *out (gfd_result_free). */
int gfd_session_next_result(gfd_session *s, int64_t *request_id, gfd_result **out);
/* Cancel a request of the session: a queued one is dropped, a running one is
 * stopped and its device memory released, a finished but uncollected one has
 * its result freed; no result for it is delivered afterwards. Call it between
 * gfd_session_step calls. Returns GFD_OK, or GFD_ERR_INVALID_ARG when the
 * session holds no request with that id (unknown, or already collected). */
int gfd_session_cancel(gfd_session *s, int64_t request_id);
/* Session statistics since creation, for monitoring: 0 host milliseconds spent
 * admitting requests (planning, index builds), 1 device milliseconds of
 * enumeration rounds, 2 rounds run, 3 requests admitted, 4 admissions (groups
 * of requests admitted together). 0 for NULL or another `which`. While an
 * admission keeps the host busy, gfd_session_step queues as many rounds as
 * recent admissions took (running averages), so the device keeps working. */
double gfd_session_stat(const gfd_session *s, int32_t which);
/* Wait for the session's work, release it and any uncollected results. Free
 * every session of a graph before the graph: a session issues its work on the
 * graph's stream unless opts->cuda_stream names another. */
void gfd_session_free(gfd_session *s);

/* Candidate filter of pattern node `node` of phi (its label, its out- and
 * in-degree in Q as lower bounds on the data vertex's degrees without
 * self-loops, and its self-loop), written to the caller's DEVICE buffer d_out as
 * increasing vertex ids; *n_out (host) receives how many there are.
 * The paper has no counterpart: this is an extra entry point for callers that
 * may not allocate device memory themselves or through a library. Examples are
 * a server whose device memory is handed out by its own allocator or reserved
 * up front under a fixed budget (an allocation by the library would bypass that
 * accounting, or fail once the reservation holds the free memory), and
 * latency-bound threads that cannot wait for cudaFree, which synchronises the
 * whole device. The same filter runs inside gfd_validate.
 * It allocates nothing: its only scratch is a fixed 64 KiB array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits. Graphs are therefore limited to 2^26 vertices (GFD_ERR_UNSUPPORTED
 * beyond). The first call on each device looks up that array's device address
 * and the multiprocessor count; make that first call before any stream
 * capture. All calls share the array and each call clears it before use:
 * calls that overlap on the GPU race on it, so serialise them (one stream, or
 * wait for the previous call). out_cap is the capacity of d_out in elements;
 * more candidates than that give GFD_ERR_OVERFLOW with *n_out set. The call
 * copies the count to the host and waits for its own work on cuda_stream
 * (NULL: the graph's stream) before returning. */
int gfd_node_candidates_noalloc(const gfd_graph *g, const gfd_gfd *phi, int32_t node,
                                int32_t *d_out, int64_t out_cap, int64_t *n_out,
                                void *cuda_stream);

/* Message for the calling thread's last non-OK return ("" if none); the
 * library owns the string, valid until the thread's next failing call. */
const char *gfd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GFD_H */
