// Internal structures shared by the library's translation units.
//
// Device data layout (all resident in HBM):
//   graph:   out_off/in_off u32 [V+1]; out_adj/in_adj u32 [E] packed as
//            (neighbour << lbits) | edge_label, rows sorted by neighbour;
//            vinfo u32 [V] = vertex label (low 16 bits) | (self-loop label + 1) << 16
//            (0 in the high half = no self-loop); attrs i32 [n_attrs][V];
//            sig u64x2 [V] = (out-, in-neighbourhood signature).
//   index:   per (GFD, level) a candidate bitmap [nwords] u32, its exclusive
//            popcount prefix [nwords] u32 (so rank(v) is O(1)), the sorted
//            candidate list i32, and for every level i >= 1 the index edges of
//            the spanning-tree edge (parent(i), i): off u32 [|C(parent)|+1],
//            idx int2 [nnz] = (position in C(i), vertex id).
//   frontier: per (GFD, level l >= 1) a buffer of partial matches, row-major
//            [chunk][2(l+1)+2] i32 = l+1 vertex ids, l+1 candidate positions, the
//            generator chosen for level l+1 and the start of the parent's index
//            edges for level l+1, plus the exclusive prefix of each row's fan-out
//            u64 [chunk]. Rows with no fan-out are not stored.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gfd.h"

namespace gfd {

constexpr int MAXK = 16;
constexpr int MAXLIT = 32;
// expectation for an ordered vertex pair of the pattern
constexpr int16_t EXP_SKIP = -3;  // already guaranteed by construction
constexpr int16_t EXP_NONE = -2;  // the data graph must have no such edge
constexpr int16_t EXP_ANY = -1;   // an edge with any label
constexpr int32_t NOEDGE = -2;

// packed per-level counter: rows in the high ROW_BITS bits, fan-out sum below
constexpr int ROW_SHIFT = 40;
constexpr uint64_t WORK_MASK = (1ull << ROW_SHIFT) - 1;

struct DevGraph {
    int32_t n;
    int32_t n_attrs;
    int32_t lbits;
    uint32_t lmask;
    int64_t m;
    uint32_t nwords;  // ceil(V / 32)
    const uint32_t* out_off;
    const uint32_t* in_off;
    const uint32_t* out_adj;
    const uint32_t* in_adj;
    const uint32_t* vinfo;
    const int32_t* attrs;
    // neighbourhood signatures: sig[v].x has bit sig_bit(w) set for every
    // out-neighbour w of v, sig[v].y for every in-neighbour; a clear bit proves
    // that the edge is absent
    const ulonglong2* sig;
};

// Signature bit of a vertex id: the top 6 bits of a Fibonacci (multiplicative)
// hash.
__host__ __device__ __forceinline__ uint32_t sig_bit(uint32_t v) { return (v * 0x9E3779B1u) >> 26; }

// Candidate filter key (Section III.B step 1a-1b): label, degree lower bounds
// (self-loops excluded on both sides) and the self-loop expectation.
constexpr int KEY_ATTRS = 2;  // constant X literals a filter key can carry

struct FilterKey {
    int32_t label;     // or GFD_WILDCARD
    uint32_t dout_min;
    uint32_t din_min;
    int32_t self_exp;  // EXP_NONE, EXP_ANY, a label, or EXP_SKIP (no condition)
    int32_t n_attr;    // attribute conditions attr[a] = c (pushed-down constant X literals)
    int32_t attr_a[KEY_ATTRS];
    int32_t attr_c[KEY_ATTRS];
};

// ints of a stored partial match of level l (l+1 ids, l+1 candidate positions,
// generator, index base), padded to a multiple of 16 bytes for vector loads
__host__ __device__ constexpr int row_width(int l) { return (2 * (l + 1) + 2 + 3) & ~3; }

struct LevelPlan {
    int8_t u;          // pattern node matched at this level
    int8_t par;        // level of its spanning-tree parent (-1 at level 0)
    int8_t tdir;       // 1: tree edge parent -> u, 0: u -> parent
    int8_t nchk;       // number of entries in chk_q
    int8_t ngen;       // number of alternative candidate generators in gen
    int8_t gen[3];     // chk entries (required, not the tree parent) whose other
                       // end's adjacency may generate the candidates instead
    int8_t nreq;       // chk entries [0, nreq) are required edges, the rest absent
    int32_t tlab;      // tree edge label or GFD_WILDCARD
    uint32_t inj;      // bit q: v must differ from the vertex at level q
    int8_t chk_q[2 * MAXK];   // earlier level of each pair check
    int8_t chk_dir[2 * MAXK]; // 1: edge u -> node(q), 0: node(q) -> u
    int16_t chk_exp[2 * MAXK];// expectation (EXP_NONE / EXP_ANY / label)
    uint32_t chk_w[2 * MAXK]; // the same packed: q | dir << 4 | (uint16_t)exp << 16
};

struct DevLit {
    int32_t kind;  // 0: x.A = c, 1: x.A = y.B
    int32_t xl;    // level of x
    int32_t a;
    int32_t yl;    // level of y
    int32_t b;
    int32_t c;
    int32_t lvl;   // level whose candidates are checked against it (-1: in the filter)
};

// Everything the device needs about one GFD slot.
struct SlotDesc {
    int32_t k;
    int32_t nx, ny, y_false;
    int32_t push_x;  // X applied during the search: count only matches with h |= X
    int32_t order[MAXK];
    LevelPlan lv[MAXK];
    DevLit lit[MAXLIT];  // X literals then Y literals
    // index
    uint32_t* bm[MAXK];
    uint32_t* rank[MAXK];
    int32_t* cand[MAXK];
    uint32_t cand_cap[MAXK];
    uint32_t* cpi_off[MAXK];  // level i >= 1
    int2* cpi_idx[MAXK];      // (position in C(i), vertex id) per index edge
    uint64_t cpi_cap[MAXK];
    // frontier
    int32_t* rows[MAXK];      // level l >= 1
    uint64_t* wpre[MAXK];     // level l >= 1
    uint64_t chunk;           // max work items per step (= row capacity)
    // violation output of this slot (serving); null: the run's shared arena
    int32_t* viol;
    uint64_t viol_cap;
};

// Mutable per-slot state (device).
struct SlotState {
    int32_t cur;        // level being expanded, -1 when finished
    int32_t err;
    uint32_t ncand[MAXK];     // candidate list sizes
    uint64_t nrows[MAXK];     // rows held at level l
    uint64_t total[MAXK];     // work items at level l
    uint64_t cursor[MAXK];    // work items of level l already expanded
    uint64_t ctr[MAXK];       // packed rows/work counter of level l (filled by l-1)
    uint64_t cb, ce;          // current step's work range at level `cur`
    uint64_t n_matches;
    uint64_t n_viol;
    uint64_t st_work, st_rows, st_probes, st_steps, st_cpi;
    uint32_t tile;            // work items per tile in the current step
};

// Counters of the counting pass (GFD_FLAG_COUNT): what one run's kernels
// read, per kind of access, for the algorithmic-byte model of the roofline.
enum : int {
    CNT_ITEMS = 0,     // work items expanded (entries of N_u or of a generator's list)
    CNT_ITEMS_LAST,    // of them at the last level
    CNT_PARTIALS,      // partial matches expanded (stored rows, and roots, with fan-out)
    CNT_BACK_DEG,      // sum over expanded partial matches of the degrees (in the edge's
                       // direction) of the images of their backward non-tree neighbours
    CNT_CHECKS,        // pair checks made (required and absent edges)
    CNT_SIG_SETTLED,   // of them settled by the neighbourhood signature
    CNT_SEARCHES,      // binary searches of an adjacency list made
    CNT_SEARCH_LOADS,  // adjacency entries those searches loaded
    CNT_NEG_CHECKS,    // absent-edge checks made
    CNT_NEG_LOGD,      // sum over absent-edge checks of ceil(log2(d + 1)), d the shorter list
    CNT_SIG_LOADS,     // neighbourhood-signature loads
    CNT_ATTR_READS,    // attribute loads of the literal checks
    CNT_ROWS,          // partial matches written
    CNT_SCAN_CANDS,    // refinement and index build: candidates whose adjacency was scanned
    CNT_SCAN_ENTRIES,  // refinement and index build: adjacency entries read
    CNT_ITERS,         // warp iterations of the expansion (32 work items each at most)
    CNT_ITER_MAX_LOADS,// sum over warp iterations of the largest number of search
                       // loads one lane made (the warp waits for its slowest lane)
    CNT_CYC_TILE,      // SM cycles warps spent setting up tiles (row range searches)
    CNT_CYC_MID,       // SM cycles of warp iterations at intermediate levels
    CNT_CYC_LAST,      // SM cycles of warp iterations at the last level
    CNT_ITERS_MID,     // warp iterations at intermediate levels
    CNT_HOST,          // filled by the host: distinct filter keys << 32 | bitmaps
    N_CNT = 22
};

// Scheduler state shared by all slots of a run (device).
struct Sched {
    int32_t n_slots;
    int32_t active;
    int32_t err;
    uint32_t total_tiles;
    uint32_t tile;            // work items per tile in the current step
    uint32_t bar_count;       // grid barrier
    uint32_t bar_gen;
    uint32_t pad;
    uint64_t steps;
    uint64_t timeout_ns;      // limit of one grid-barrier wait
    uint64_t probes;
    uint64_t t_start;         // globaltimer at the first step
    uint64_t run_limit_ns;    // limit of the whole enumeration
    // violations of all slots: records [slot, h(x_0), ..., h(x_{k-1})] of
    // vstride ints appended at varena_used; records past varena_cap are counted
    // but not stored
    int32_t* varena;
    uint64_t varena_cap;
    uint64_t varena_used;
    int32_t vstride;
    int32_t pad2;
    uint64_t cnt[N_CNT];      // counting pass only
    // next tile of the current step handed out to a warp that finished its
    // first one (tiles below the warp count go to warps by index); on its own
    // cache line, away from the fields every warp reads
    alignas(128) uint32_t tile_next;
};

// device error codes (Sched::err, SlotState::err)
enum : int32_t {
    DERR_NONE = 0,
    DERR_COUNTER_OVERFLOW = 1,
    DERR_TIMEOUT = 2,
    DERR_CAPACITY = 3,
};

__host__ __device__ inline bool label_ok(int32_t want, int32_t have) {
    return want == GFD_WILDCARD || want == have;
}

// Agreement of a pattern expectation with a data-graph edge label (NOEDGE if
// the edge is absent): Section II, (a,b) ∈ E_Q ⇔ (h(a),h(b)) ∈ E with equal labels.
__host__ __device__ inline bool exp_ok(int32_t e, int32_t gl) {
    if (e == EXP_NONE) return gl == NOEDGE;
    if (gl == NOEDGE) return false;
    return e == EXP_ANY || e == gl;
}

// ---------------------------------------------------------------- host side
struct Status {
    int code = GFD_OK;
    const char* where = "";
};

void set_error(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define GFD_CUDA(call)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::gfd::cuda_fail(_e, #call); \
    } while (0)

}  // namespace gfd
