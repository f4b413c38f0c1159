// Core-first match enumeration over the compact path index (Section III.B,
// step 2) with the literal check and violation output (Section II) fused into
// the last level.
//
// Execution model: a breadth-first / depth-first hybrid over many GFD slots at
// once. Each slot keeps one buffer of partial matches per level. A step takes
// a bounded chunk of "work items" from the deepest unfinished level of every
// active slot: work item w of level l is the pair (partial match r, o-th index
// edge of r's tree parent), found by binary search in the exclusive prefix of
// the rows' fan-outs, so hub vertices are split evenly over threads. Each work
// item yields at most one partial match of level l+1, so a level-l chunk of
// `chunk` items always fits the next buffer; when a level is exhausted the slot
// pops back to the previous level (depth-first), bounding memory.
//
// A candidate v for pattern node u = order[i] extending partial match m passes
// when: v != m[q] for earlier label-compatible levels q (injectivity), and for
// every earlier level q and both directions, the data-graph edge between v and
// m[q] agrees with the pattern (present with an equal label where Q has the
// edge, absent where it has not: a match may not contain additional edges,
// Section II; the CFL-Match index alone would allow them, Section III). The
// spanning-tree edge to the parent is guaranteed by the index and skipped.
//
// Survivors are appended with one atomic per block on a packed 64-bit counter
// (rows << 40 | fan-out sum), which gives each row both its index and the
// exclusive prefix of fan-outs needed by the next step's search, consistently.
//
// The scheduler (k_control) runs in one block between steps. Two drivers: a
// persistent cooperative kernel with a bounded grid barrier between phases, or
// a host loop of (expand, control) launches, optionally captured in CUDA graphs.
#include <cub/cub.cuh>

#include <algorithm>
#include <type_traits>

#include "engine.h"

namespace gfd {

namespace {

constexpr int CTRL_THREADS = 1024;
constexpr uint64_t LAST_LEVEL_CHUNK = 1ull << 25;  // work items per step at the last level
// generator stored in a row for a next level that starts a pattern component:
// its candidates are the level's candidate list (fan-out |C| for every row)
constexpr int GEN_LIST = 4;

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per-thread counters of the counting pass (empty unless COUNT), added into
// Sched::cnt once per warp at the end of the expansion.
template <bool COUNT>
struct Counters {
    __device__ __forceinline__ void add(int, uint64_t) {}
    __device__ __forceinline__ uint32_t* loads() { return nullptr; }
    __device__ __forceinline__ void iteration(bool) {}
    __device__ __forceinline__ void mark() {}
    __device__ __forceinline__ void cycles(int) {}
    __device__ __forceinline__ void flush(Sched*) {}
};
template <>
struct Counters<true> {
    uint64_t c[N_CNT] = {};
    uint32_t search_loads = 0;  // of the current warp iteration
    __device__ __forceinline__ void add(int i, uint64_t v) { c[i] += v; }
    __device__ __forceinline__ uint32_t* loads() { return &search_loads; }
    long long t0 = 0;  // clock at the start of the current phase
    __device__ __forceinline__ void mark() { t0 = clock64(); }
    // SM cycles since mark() into counter i (lane 0 counts for the warp)
    __device__ __forceinline__ void cycles(int i) {
        const long long t = clock64();
        if ((threadIdx.x & 31) == 0) c[i] += (uint64_t)(t - t0);
        t0 = t;
    }
    // end of a warp iteration (all lanes): the slowest lane's search loads
    __device__ __forceinline__ void iteration(bool last) {
        const uint32_t mx = __reduce_max_sync(0xffffffffu, search_loads);
        if ((threadIdx.x & 31) == 0) {
            c[CNT_ITERS] += 1;
            c[CNT_ITER_MAX_LOADS] += mx;
            if (!last) c[CNT_ITERS_MID] += 1;
        }
        c[CNT_SEARCH_LOADS] += search_loads;
        search_loads = 0;
        cycles(last ? CNT_CYC_LAST : CNT_CYC_MID);
    }
    __device__ void flush(Sched* s) {
        for (int i = 0; i < N_CNT; i++) {
            uint64_t v = c[i];
            for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long*)&s->cnt[i], (unsigned long long)v);
        }
    }
};

__device__ __forceinline__ uint32_t ceil_log2_1(uint32_t d) { return 32 - __clz(d); }  // ceil(log2(d + 1))

// Label of the data-graph edge a -> b, or NOEDGE: binary search in the shorter
// of out(a) and in(b) (both sorted by neighbour id). loads (counting pass
// only, else null) accumulates the adjacency entries read.
__device__ __forceinline__ int32_t edge_label(const DevGraph& g, uint32_t a, uint32_t a_out0, uint32_t a_out1,
                                              uint32_t b, uint32_t b_in0, uint32_t b_in1,
                                              uint32_t* loads = nullptr) {
    const uint32_t* arr;
    uint32_t lo, hi, key;
    if (a_out1 - a_out0 <= b_in1 - b_in0) {
        arr = g.out_adj;
        lo = a_out0;
        hi = a_out1;
        key = b;
    } else {
        arr = g.in_adj;
        lo = b_in0;
        hi = b_in1;
        key = a;
    }
    const uint32_t end = hi;
    const uint32_t kk = key << g.lbits;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (loads) ++*loads;
        if (__ldg(arr + mid) < kk) lo = mid + 1;
        else hi = mid;
    }
    if (lo < end) {
        if (loads) ++*loads;
        const uint32_t p = __ldg(arr + lo);
        if ((p >> g.lbits) == key) return (int32_t)(p & g.lmask);
    }
    return NOEDGE;
}

// m: the partial match in shared memory, level q at m[32 q] (one column per lane)
__device__ __forceinline__ bool lit_holds(const DevGraph& g, const DevLit& L, const uint32_t* m,
                                          uint32_t* reads = nullptr) {
    if (reads) ++*reads;
    const int32_t va = __ldg(g.attrs + (uint64_t)L.a * g.n + m[L.xl << 5]);
    if (va == GFD_ATTR_ABSENT) return false;
    if (L.kind == 0) return va == L.c;
    if (reads) ++*reads;
    const int32_t vb = __ldg(g.attrs + (uint64_t)L.b * g.n + m[L.yl << 5]);
    return vb != GFD_ATTR_ABSENT && va == vb;
}

// The same with the vertex of level lv given in a register (v) instead of the
// shared-memory column (used when another lane's column holds the earlier
// levels).
__device__ __forceinline__ uint32_t level_vertex(const uint32_t* m, int q, int lv, uint32_t v) {
    return q == lv ? v : m[q << 5];
}
__device__ __forceinline__ bool lit_holds_at(const DevGraph& g, const DevLit& L, const uint32_t* m, int lv, uint32_t v,
                                             uint32_t* reads = nullptr) {
    if (reads) ++*reads;
    const int32_t va = __ldg(g.attrs + (uint64_t)L.a * g.n + level_vertex(m, L.xl, lv, v));
    if (va == GFD_ATTR_ABSENT) return false;
    if (L.kind == 0) return va == L.c;
    if (reads) ++*reads;
    const int32_t vb = __ldg(g.attrs + (uint64_t)L.b * g.n + level_vertex(m, L.yl, lv, v));
    return vb != GFD_ATTR_ABSENT && va == vb;
}

// Partial matches of the second-to-last level with at most this many
// candidates at the last level are expanded by the warp that makes them,
// without being stored.
constexpr uint32_t FUSE_FANOUT = 64;
// Tiles of a step that fuses the last level are this many times smaller.
constexpr uint64_t FUSED_TILE_DIV = 2;
// Number the last level's tiles after the other intermediate levels' (else
// both are numbered together, in slot order).
constexpr bool LAST_LEVEL_TILES_LAST = true;

// Largest r in [0, n) with S[r] <= w (S non-decreasing, S[0] <= w). The index
// offsets are read-only during enumeration; the frontier prefix is rewritten
// between steps, so it is read through L2 only (ld.global.cg).
__device__ __forceinline__ uint32_t find_row(const uint32_t* S, uint64_t n, uint64_t w) {
    uint64_t lo = 0, hi = n;  // invariant: S[lo] <= w, answer in [lo, hi)
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(S + mid) <= w) lo = mid;
        else hi = mid;
    }
    return (uint32_t)lo;
}
__device__ __forceinline__ uint32_t find_row(const uint64_t* S, uint64_t n, uint64_t w) {
    uint64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (__ldcg((const unsigned long long*)S + mid) <= w) lo = mid;
        else hi = mid;
    }
    return (uint32_t)lo;
}

// Loads of data rewritten between steps (frontier rows and prefixes, the
// per-step tile prefix): plain weak loads, which may be served from L1. In the
// persistent kernel the grid barrier orders them after the previous step's
// writes: every writer's block fences at gpu scope before arriving, each
// block's thread 0 fences at gpu scope after observing the release, and the
// block barrier orders the block's other threads after that fence, so by the
// PTX memory model the loads observe the writes (the pattern of a cooperative
// grid synchronisation). In the host-driven loop the kernel boundary orders them.
__device__ __forceinline__ uint32_t ld_front(const uint32_t* p) { return *p; }
__device__ __forceinline__ uint64_t ld_front(const uint64_t* p) { return *p; }

// r in [lo, hi) with S[r] <= w < S[r+1]: the search limited to the rows of a tile.
__device__ __forceinline__ uint32_t find_row_in(const uint32_t* S, uint32_t lo, uint32_t hi, uint64_t w) {
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(S + mid) <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t find_row_in(const uint64_t* S, uint32_t lo, uint32_t hi, uint64_t w) {
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldcg((const unsigned long long*)S + mid) <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One half of a vertex's neighbourhood signature: 0 its out-neighbours, 1 its
// in-neighbours. An edge a -> b needs both b's bit in a's out-signature and
// a's bit in b's in-signature, so either clear bit proves it absent.
__device__ __forceinline__ uint64_t sig_half(const DevGraph& g, uint32_t x, int half) {
    return __ldg(reinterpret_cast<const unsigned long long*>(g.sig) + 2 * (uint64_t)x + half);
}

// position of v in the sorted candidate list of a level: O(1) from the bitmap
// and its per-word popcount prefix
__device__ __forceinline__ int32_t cand_rank(const uint32_t* bm, const uint32_t* rank, uint32_t v) {
    return (int32_t)(__ldg(rank + (v >> 5)) + __popc(__ldg(bm + (v >> 5)) & ((1u << (v & 31)) - 1u)));
}

// Warp-parallel search: largest r in [lo, hi) with S[r] <= w, given S[lo] <= w.
// Each round probes 32 evenly spaced entries and keeps the last one <= w.
template <typename T>
__device__ __forceinline__ uint32_t warp_find(const T* S, uint64_t lo, uint64_t hi, uint64_t w, int lane) {
    while (hi - lo > 32) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t idx = lo + (uint64_t)lane * step;
        const bool le = idx < hi && (uint64_t)ld_front(S + idx) <= w;
        const uint32_t b = __ballot_sync(0xffffffffu, le);
        const int j = 31 - __clz(b);
        lo = lo + (uint64_t)j * step;
        hi = min(hi, lo + step);
    }
    const uint64_t idx = lo + lane;
    const bool le = idx < hi && (uint64_t)ld_front(S + idx) <= w;
    const uint32_t b = __ballot_sync(0xffffffffu, le);
    return (uint32_t)(lo + 31 - __clz(b));
}

// Exclusive warp scan of 64-bit values; *total receives the warp's sum.
__device__ __forceinline__ uint64_t warp_excl_scan(uint64_t x, int lane, uint64_t* total) {
    uint64_t incl = x;
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    *total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - x;
}

// The expansion step, warp-synchronous: every warp takes its own tiles of
// work items (no block-wide barrier in the loop). A tile belongs to one slot
// and one level; the warp finds them (and the rows the tile covers) with
// lane-parallel searches, then processes 32 work items per iteration.
// GEN = false: the common case (connected patterns, X checked at the last
// level only), compiled without the general paths so that it keeps its
// registers; GEN = true adds component starts and X pushed down.
template <int NT, bool GEN, bool COUNT>
__device__ void expand_warps(const EnumArgs& A) {
    // Per warp in shared memory: the lanes' partial matches (level q of lane t
    // at [32 q + t], so the lanes' dynamically indexed reads hit distinct
    // banks) and the current tile's pair checks, packed.
    __shared__ uint32_t s_m[NT / 32][MAXK * 32];
    __shared__ uint32_t s_chk[NT / 32][2 * MAXK];
    __shared__ uint32_t s_chk2[NT / 32][2 * MAXK];  // the last level's, for fused expansion
    Counters<COUNT> cn;
    uint32_t attr_reads = 0;
    const int lane = threadIdx.x & 31;
    uint32_t* const m = &s_m[threadIdx.x >> 5][lane];
    uint32_t* const cw = s_chk[threadIdx.x >> 5];
    uint32_t* const cw2 = s_chk2[threadIdx.x >> 5];
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const DevGraph& g = A.g;
    const uint32_t total_tiles = *(volatile uint32_t*)&A.sched->total_tiles;
    uint32_t probes = 0;  // a statistic (saturates per warp)
    for (uint64_t t = gwarp; t < total_tiles;) {
        cn.mark();
        // the step's tiles: those of fusing slots first, then those of the other
        // intermediate levels, then the last level's
        const uint32_t* tb = A.tile_base;
        if (t >= __ldcg(A.tile_base + A.n_slots)) tb += A.n_slots + 1;
        if (t >= __ldcg(A.tile_base + 2 * A.n_slots + 1)) tb = A.tile_base + 2 * (A.n_slots + 1);
        const int s = (int)warp_find(tb, 0, (uint64_t)A.n_slots, t, lane);
        const SlotDesc* __restrict__ D = A.slots + s;
        SlotState* S = A.state + s;
        const int k = D->k;
        // scheduler fields are rewritten between steps: read them through L2
        const int l = __ldcg(&S->cur);
        const int i = k == 1 ? 0 : l + 1;  // level being matched
        const bool last = i == k - 1;
        const uint64_t tile = __ldcg(&S->tile);  // work items per tile of this slot in this step
        const uint64_t wb = __ldcg((const unsigned long long*)&S->cb) + (t - __ldcg(tb + s)) * tile;
        const uint64_t we = min(wb + tile, (uint64_t)__ldcg((const unsigned long long*)&S->ce));
        const LevelPlan& LP = D->lv[i];
        const int nchk = LP.nchk;
        __syncwarp();  // the previous tile's checks are no longer read
        if (lane < nchk) cw[lane] = LP.chk_w[lane];
        __syncwarp();
        const uint32_t* S0 = i > 0 ? D->cpi_off[i] : nullptr;
        const uint64_t* Sl = l >= 1 ? D->wpre[l] : nullptr;
        const int32_t* rows_l = l >= 1 ? D->rows[l] : nullptr;
        const uint64_t nrows = k == 1 ? 0 : (l == 0 ? (uint64_t)S->ncand[0]
                                                    : (uint64_t)__ldcg((const unsigned long long*)&S->nrows[l]));
        const int rw = row_width(l);  // ints per row at level l: ids, positions, generator, index base
        // level 1 starts a component: root r's items are [r c1, (r+1) c1)
        const bool list1 = GEN && k > 1 && l == 0 && LP.par < 0;
        const uint64_t c1 = list1 ? (uint64_t)S->ncand[1] : 0;
        uint32_t rlo = 0, rhi1 = 0;
        if (k > 1 && !list1) {
            if (l == 0) {
                rlo = warp_find(S0, 0, nrows, wb, lane);
                rhi1 = warp_find(S0, rlo, nrows, we - 1, lane) + 1;
            } else {
                // stored rows all have fan-out >= 1, so the window search never
                // runs past the tile's last row: the end of the row range need
                // not be searched
                rlo = warp_find(Sl, 0, nrows, wb, lane);
                rhi1 = (uint32_t)nrows;
            }
        }
        // The tile's items, compiled for the last level (literal check,
        // violations) and for the others (fan-out, new partial matches), each
        // for the roots (level 0: candidate list, 32-bit index offsets) and for
        // stored partial matches (rows, 64-bit prefixes), so that no path
        // carries another's registers.
        auto run_tile = [&](auto last_tag, auto root_tag) {
            constexpr bool LAST = decltype(last_tag)::value;
            constexpr bool ROOT = decltype(root_tag)::value;  // expanding the roots (ROOT)
            uint32_t tile_matches = 0;
            uint32_t cur = rlo;  // row of the first work item of the iteration
            // a tile that makes partial matches of the second-to-last level
            // expands the last level of those with small fan-outs at once
            // (fused); the last level's pair checks are staged too
            const bool fuse = !LAST && k >= 3 && i == k - 2;
            if (fuse) {
                __syncwarp();
                if (lane < D->lv[k - 1].nchk) cw2[lane] = D->lv[k - 1].chk_w[lane];
                __syncwarp();
            }
            cn.cycles(CNT_CYC_TILE);
            for (uint64_t w0 = wb; w0 < we; w0 += 32) {
                const uint64_t w = w0 + lane;
                bool ok = w < we;
                uint32_t v = 0;
                int32_t j = 0;
                const int32_t* rowp = nullptr;
                uint32_t r = 0;
                // Rows of this iteration's 32 work items: stored rows have fan-out
                // >= 1, so they lie in the window [cur, cur + 32); one coalesced load
                // of the window's prefixes and a 5-step shuffle search per lane. A
                // lane left at the window's end checks the next prefix and falls
                // back to a binary search (root candidates may have no fan-out).
                uint64_t sr = 0;
                if (list1) {
                    r = ok ? (uint32_t)(w / c1) : 0u;
                    sr = (uint64_t)r * c1;
                } else if (k > 1) {
                    const uint64_t widx = (uint64_t)cur + lane;
                    const uint64_t sv = widx < rhi1 ? (ROOT ? (uint64_t)__ldg(S0 + widx) : ld_front(Sl + widx))
                                                    : ~0ull;
                    int pos = 0;
                    for (int step = 16; step >= 1; step >>= 1) {
                        const uint64_t x = __shfl_sync(0xffffffffu, sv, pos + step);
                        if (x <= w) pos += step;
                    }
                    sr = __shfl_sync(0xffffffffu, sv, pos);
                    r = cur + pos;
                    if (ok && pos == 31 && r + 1 < rhi1) {
                        const uint64_t nxt = ROOT ? (uint64_t)__ldg(S0 + r + 1) : ld_front(Sl + r + 1);
                        if (nxt <= w) {
                            r = ROOT ? find_row_in(S0, r, rhi1, w) : find_row_in(Sl, r, rhi1, w);
                            sr = ROOT ? (uint64_t)__ldg(S0 + r) : ld_front(Sl + r);
                        }
                    }
                    cur = __shfl_sync(0xffffffffu, r, 31);
                }
                if (ok) {
                    cn.add(CNT_ITEMS, 1);
                    if (LAST) cn.add(CNT_ITEMS_LAST, 1);
                    if (k == 1) {
                        j = (int32_t)w;
                        v = (uint32_t)D->cand[0][j];
                    } else {
                        // the item's offset within its row's candidates, and the
                        // position of its index edge (both below 2^32: fan-outs and
                        // index lists are 32-bit)
                        const uint32_t o = (uint32_t)(w - sr);
                        uint32_t ent;
                        int choice = 0;
                        if (ROOT) {
                            // the roots' index edges are level 1's, in work-item order
                            // (or level 1's candidate list when it starts a component)
                            ent = list1 ? o : (uint32_t)w;
                            choice = list1 ? GEN_LIST : 0;
                            m[0] = (uint32_t)D->cand[0][r];
                        } else {
                            // the row's ids in 16-byte loads (rows are padded to 16 B;
                            // m has room for the LAST group), generator and index base
                            // in one 8-byte load
                            rowp = rows_l + (uint64_t)r * rw;
                            const int4* r4 = reinterpret_cast<const int4*>(rowp);
                            for (int q = 0; q <= l; q += 4) {
                                const int4 t4 = r4[q >> 2];
                                m[q << 5] = (uint32_t)t4.x;
                                m[(q + 1) << 5] = (uint32_t)t4.y;
                                m[(q + 2) << 5] = (uint32_t)t4.z;
                                m[(q + 3) << 5] = (uint32_t)t4.w;
                            }
                            const int2 gb = *reinterpret_cast<const int2*>(rowp + 2 * (l + 1));
                            choice = gb.x;
                            ent = (uint32_t)gb.y + o;
                        }
                        int skip = -1;
                        // the first pair check's earlier image is the same for all the
                        // row's candidates: its signature half (the one that holds v
                        // if the edge exists) is loaded while the candidate is fetched
                        uint64_t sx0 = 0;
                        if (nchk > 0) {
                            const uint32_t w0c = cw[0];
                            sx0 = sig_half(g, m[(w0c & 15u) << 5], (w0c >> 4) & 1u);
                        }
                        if (COUNT && o == 0) {
                            // the row's first item: the partial match is expanded once;
                            // a merge-based intersection would scan the adjacency of
                            // each backward non-tree neighbour's image
                            cn.add(CNT_PARTIALS, 1);
                            uint64_t bd = 0;
                            for (int c = 0; c < nchk; c++) {
                                if (LP.chk_exp[c] == EXP_NONE) continue;
                                const uint32_t x = m[LP.chk_q[c] << 5];
                                bd += LP.chk_dir[c] ? g.in_off[x + 1] - g.in_off[x] : g.out_off[x + 1] - g.out_off[x];
                            }
                            cn.add(CNT_BACK_DEG, bd);
                        }
                        if (choice == 0) {
                            // candidates from the index edges of the spanning-tree parent
                            const int2 e = __ldg(D->cpi_idx[i] + ent);
                            j = e.x;
                            v = (uint32_t)e.y;
                        } else if (GEN && choice == GEN_LIST) {
                            // the level starts a component: its candidate list
                            j = (int32_t)ent;
                            v = (uint32_t)__ldg(D->cand[i] + ent);
                        } else {
                            // candidates from the adjacency of the other end of a
                            // required back edge (the shorter list): keep those in
                            // C(u) and probe the spanning-tree edge instead
                            const int cg = LP.gen[choice - 1];
                            skip = cg;
                            const uint32_t x = m[LP.chk_q[cg] << 5];
                            const uint32_t p = LP.chk_dir[cg] ? __ldg(g.in_adj + __ldg(g.in_off + x) + o)
                                                              : __ldg(g.out_adj + __ldg(g.out_off + x) + o);
                            v = p >> g.lbits;
                            ok = exp_ok(LP.chk_exp[cg], (int32_t)(p & g.lmask)) &&
                                 ((__ldg(D->bm[i] + (v >> 5)) >> (v & 31)) & 1u);
                            if (ok) {
                                j = cand_rank(D->bm[i], D->rank[i], v);
                                const uint32_t xp = m[LP.par << 5];
                                // tree edge xp -> v (tdir 1) or v -> xp: the parent's
                                // signature first, then v's
                                bool maybe = (sig_half(g, xp, LP.tdir ? 0 : 1) >> sig_bit(v)) & 1ull;
                                cn.add(CNT_SIG_LOADS, 1);
                                if (maybe) {
                                    maybe = (sig_half(g, v, LP.tdir ? 1 : 0) >> sig_bit(xp)) & 1ull;
                                    cn.add(CNT_SIG_LOADS, 1);
                                }
                                int32_t gl = NOEDGE;
                                cn.add(CNT_CHECKS, 1);
                                if (maybe) {
                                    cn.add(CNT_SEARCHES, 1);
                                    gl = LP.tdir ? edge_label(g, xp, g.out_off[xp], g.out_off[xp + 1], v, g.in_off[v], g.in_off[v + 1], cn.loads())
                                                 : edge_label(g, v, g.out_off[v], g.out_off[v + 1], xp, g.in_off[xp], g.in_off[xp + 1], cn.loads());
                                } else {
                                    cn.add(CNT_SIG_SETTLED, 1);
                                }
                                probes++;
                                ok = exp_ok(LP.tlab, gl);
                            }
                        }
                        // injectivity
                        for (int q = 0; q <= l && ok; q++)
                            if (((LP.inj >> q) & 1u) && m[q << 5] == v) ok = false;
                        // every other pattern pair, both directions (required edges
                        // first): v's neighbourhood signatures settle most pairs (a
                        // clear bit proves the edge absent); the rest search the
                        // shorter adjacency list
                        if (ok && nchk > 0) {
                            const uint32_t bv = sig_bit(v);
                            uint64_t svo = 0, svi = 0;  // v's signature, loaded when needed
                            bool have_sv = false;
                            for (int c = 0; c < nchk && ok; c++) {
                                if (c == skip) continue;
                                const uint32_t wd = cw[c];
                                const uint32_t x = m[(wd & 15u) << 5];
                                const bool out = (wd >> 4) & 1u;  // edge v -> x, else x -> v
                                const int32_t ex = (int32_t)(int16_t)(wd >> 16);
                                int32_t gl = NOEDGE;
                                cn.add(CNT_CHECKS, 1);
                                // v's bit in x's signature (x's in-neighbours for v -> x),
                                // then x's bit in v's: a clear bit proves the edge absent
                                const uint64_t sx = c == 0 ? sx0 : sig_half(g, x, out ? 1 : 0);
                                if (c != 0) cn.add(CNT_SIG_LOADS, 1);
                                bool maybe = (sx >> bv) & 1ull;
                                if (maybe) {
                                    if (!have_sv) {
                                        const ulonglong2 sg = __ldg(g.sig + v);
                                        svo = sg.x;
                                        svi = sg.y;
                                        have_sv = true;
                                        cn.add(CNT_SIG_LOADS, 1);
                                    }
                                    maybe = ((out ? svo : svi) >> sig_bit(x)) & 1ull;
                                }
                                if (COUNT && ex == EXP_NONE) {
                                    const uint32_t dv = out ? g.out_off[v + 1] - g.out_off[v] : g.in_off[v + 1] - g.in_off[v];
                                    const uint32_t dx = out ? g.in_off[x + 1] - g.in_off[x] : g.out_off[x + 1] - g.out_off[x];
                                    cn.add(CNT_NEG_CHECKS, 1);
                                    cn.add(CNT_NEG_LOGD, ceil_log2_1(min(dv, dx)));
                                }
                                if (maybe) {
                                    cn.add(CNT_SEARCHES, 1);
                                    gl = out ? edge_label(g, v, g.out_off[v], g.out_off[v + 1], x, g.in_off[x], g.in_off[x + 1],
                                                          cn.loads())
                                             : edge_label(g, x, g.out_off[x], g.out_off[x + 1], v, g.in_off[v], g.in_off[v + 1],
                                                          cn.loads());
                                } else {
                                    cn.add(CNT_SIG_SETTLED, 1);
                                }
                                probes++;
                                ok = exp_ok(ex, gl);
                            }
                        }
                    }
                    m[i << 5] = v;
                    // X pushed down: the X literals whose ends are matched at this
                    // level (before the LAST one; the LAST level checks its own below)
                    if (GEN && ok && D->push_x && !LAST)
                        for (int q = 0; q < D->nx && ok; q++)
                            if (D->lit[q].lvl == i) ok = lit_holds(g, D->lit[q], m, COUNT ? &attr_reads : nullptr);
                }
                if (LAST) {
                    // complete match: check the X literals of this level, count it
                    // (with X pushed down only if they hold), check Y, emit a violation
                    bool viol = false;
                    if (ok) {
                        bool x_ok = true;
                        for (int q = 0; q < D->nx && x_ok; q++)
                            if (!GEN || D->lit[q].lvl == i) x_ok = lit_holds(g, D->lit[q], m, COUNT ? &attr_reads : nullptr);
                        if (GEN) tile_matches += x_ok || !D->push_x;
                        else tile_matches++;
                        if (x_ok) {
                            bool y_ok = !D->y_false;
                            for (int q = 0; q < D->ny && y_ok; q++)
                                y_ok = lit_holds(g, D->lit[D->nx + q], m, COUNT ? &attr_reads : nullptr);
                            viol = !y_ok;
                        }
                    }
                    const uint32_t vb = __ballot_sync(0xffffffffu, viol);
                    if (vb) {
                        unsigned long long base = 0;
                        if (lane == 0) {
                            const unsigned long long nv = __popc(vb);
                            const unsigned long long old = atomicAdd((unsigned long long*)&S->n_viol, nv);
                            base = D->viol ? old : atomicAdd((unsigned long long*)&A.sched->varena_used, nv);
                        }
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (viol) {
                            const uint64_t idx = base + __popc(vb & ((1u << lane) - 1u));
                            if (D->viol) {
                                // the slot's own buffer: tuples in pattern-node order
                                if (idx < D->viol_cap) {
                                    int32_t* out = D->viol + idx * k;
                                    for (int q = 0; q < k; q++) out[D->order[q]] = (int32_t)m[q << 5];
                                }
                            } else if (idx < A.sched->varena_cap) {
                                // the run's arena: [slot, tuple in pattern-node order]
                                int32_t* rec = A.sched->varena + idx * A.sched->vstride;
                                rec[0] = s;
                                for (int q = 0; q < k; q++) rec[1 + D->order[q]] = (int32_t)m[q << 5];
                            }
                        }
                    }
                } else {
                    // partial match of level i: append it with its fan-out for level
                    // i+1, taken from the shortest candidate generator (dead ends,
                    // with no fan-out, are dropped)
                    uint64_t fo = 0;
                    uint32_t nbase = 0;
                    int gen = 0;
                    if (ok) {
                        const LevelPlan& L2 = D->lv[i + 1];
                        const int pn = L2.par;
                        if (GEN && pn < 0) {
                            // level i+1 starts a component: its whole candidate list
                            gen = GEN_LIST;
                            fo = S->ncand[i + 1];
                        } else {
                            const uint32_t ppn = pn == i ? (uint32_t)j : (ROOT ? r : (uint32_t)rowp[l + 1 + pn]);
                            const uint32_t* co = D->cpi_off[i + 1];
                            nbase = __ldg(co + ppn);
                            fo = __ldg(co + ppn + 1) - nbase;
                        }
                        for (int q = 0; q < L2.ngen; q++) {
                            const int cg = L2.gen[q];
                            const uint32_t x = m[L2.chk_q[cg] << 5];
                            const uint32_t d = L2.chk_dir[cg] ? __ldg(g.in_off + x + 1) - __ldg(g.in_off + x)
                                                              : __ldg(g.out_off + x + 1) - __ldg(g.out_off + x);
                            if (d < fo) {
                                fo = d;
                                gen = q + 1;
                            }
                        }
                    }
                    ok = ok && fo > 0;
                    const bool fuse_me = fuse && ok && fo <= FUSE_FANOUT;  // expanded below, not stored
                    const bool row_me = ok && !fuse_me;
                    const uint64_t packed = row_me ? ((1ull << ROW_SHIFT) | fo) : 0ull;
                    uint64_t total;
                    const uint64_t excl = warp_excl_scan(packed, lane, &total);
                    if (total) {
                        unsigned long long old = 0;
                        if (lane == 0) {
                            old = atomicAdd((unsigned long long*)&S->ctr[i], (unsigned long long)total);
                            if ((old & WORK_MASK) + (total & WORK_MASK) > WORK_MASK ||
                                (old >> ROW_SHIFT) + (total >> ROW_SHIFT) > D->chunk)
                                atomicExch(&S->err, DERR_COUNTER_OVERFLOW);
                        }
                        old = __shfl_sync(0xffffffffu, old, 0);
                        // the warp's new partial matches take rows [row0, row0 + its
                        // count) of the level's buffer, in lane order
                        if (row_me) {
                            const uint64_t row = (old >> ROW_SHIFT) + (excl >> ROW_SHIFT);
                            if (row < D->chunk) {
                                cn.add(CNT_ROWS, 1);
                                // the row (ids, positions, generator, index base,
                                // padding) in 16-byte stores, four ints at a time
                                const int nw = row_width(i);
                                int32_t* dst = D->rows[i] + row * nw;
                                for (int t = 0; t < nw; t += 4) {
                                    int32_t e4[4];
    #pragma unroll
                                    for (int c = 0; c < 4; c++) {
                                        const int idx = t + c;
                                        int32_t val = 0;
                                        if (idx <= i) {
                                            val = (int32_t)m[idx << 5];
                                        } else if (idx <= 2 * i + 1) {
                                            const int q = idx - i - 1;
                                            val = q == i ? j : (ROOT ? (int32_t)r : rowp[l + 1 + q]);
                                        } else if (idx == 2 * i + 2) {
                                            val = gen;
                                        } else if (idx == 2 * i + 3) {
                                            val = (int32_t)nbase;
                                        }
                                        e4[c] = val;
                                    }
                                    *reinterpret_cast<int4*>(dst + t) = make_int4(e4[0], e4[1], e4[2], e4[3]);
                                }
                                D->wpre[i][row] = (old & WORK_MASK) + (excl & WORK_MASK);
                            }
                        }
                    }
                    if (fuse) {
                        // The last level of the lanes' new partial matches with small
                        // fan-outs, by the whole warp, 32 items at a time: item t
                        // belongs to the lane whose [fex, fex + ffo) holds t; that
                        // lane's shared-memory column holds the partial match.
                        const uint32_t ffo = fuse_me ? (uint32_t)fo : 0u;
                        uint32_t fin = ffo;
                        for (int d = 1; d < 32; d <<= 1) {
                            const uint32_t y = __shfl_up_sync(0xffffffffu, fin, d);
                            if (lane >= d) fin += y;
                        }
                        const uint32_t fex = fin - ffo;
                        const uint32_t ftot = __shfl_sync(0xffffffffu, fin, 31);
                        if (lane == 0 && ftot) atomicAdd((unsigned long long*)&S->st_work, (unsigned long long)ftot);
                        __syncwarp();  // the lanes' columns, written above, are read by other lanes
                        const int L = k - 1;
                        const LevelPlan& LQ = D->lv[L];
                        const int nchk2 = LQ.nchk;
                        for (uint32_t fb = 0; fb < ftot; fb += 32) {
                            const uint32_t it = fb + lane;
                            int own = 0;
                            for (int st = 16; st >= 1; st >>= 1) {
                                const uint32_t x = __shfl_sync(0xffffffffu, fex, own + st);
                                if (x <= it) own += st;
                            }
                            const uint32_t fo2 = it - __shfl_sync(0xffffffffu, fex, own);
                            const uint32_t onb = __shfl_sync(0xffffffffu, nbase, own);
                            const int och = __shfl_sync(0xffffffffu, gen, own);
                            const uint32_t* mo = &s_m[threadIdx.x >> 5][own];
                            bool iok = it < ftot;
                            uint32_t fv = 0;
                            int fskip = -1;
                            if (iok) {
                                cn.add(CNT_ITEMS, 1);
                                cn.add(CNT_ITEMS_LAST, 1);
                                if (COUNT && fo2 == 0) {
                                    cn.add(CNT_PARTIALS, 1);
                                    uint64_t bd = 0;
                                    for (int c = 0; c < nchk2; c++) {
                                        if (LQ.chk_exp[c] == EXP_NONE) continue;
                                        const uint32_t x = mo[LQ.chk_q[c] << 5];
                                        bd += LQ.chk_dir[c] ? g.in_off[x + 1] - g.in_off[x] : g.out_off[x + 1] - g.out_off[x];
                                    }
                                    cn.add(CNT_BACK_DEG, bd);
                                }
                                if (och == 0) {
                                    fv = (uint32_t)__ldg(D->cpi_idx[L] + onb + fo2).y;
                                } else if (GEN && och == GEN_LIST) {
                                    fv = (uint32_t)__ldg(D->cand[L] + fo2);
                                } else {
                                    // from the adjacency of the other end of a required back
                                    // edge: keep those in C(u) and probe the tree edge
                                    const int cg = LQ.gen[och - 1];
                                    fskip = cg;
                                    const uint32_t x = mo[LQ.chk_q[cg] << 5];
                                    const uint32_t pe = LQ.chk_dir[cg] ? __ldg(g.in_adj + __ldg(g.in_off + x) + fo2)
                                                                       : __ldg(g.out_adj + __ldg(g.out_off + x) + fo2);
                                    fv = pe >> g.lbits;
                                    iok = exp_ok(LQ.chk_exp[cg], (int32_t)(pe & g.lmask)) &&
                                          ((__ldg(D->bm[L] + (fv >> 5)) >> (fv & 31)) & 1u);
                                    if (iok) {
                                        const uint32_t xp = mo[LQ.par << 5];
                                        bool maybe = (sig_half(g, xp, LQ.tdir ? 0 : 1) >> sig_bit(fv)) & 1ull;
                                        if (maybe) maybe = (sig_half(g, fv, LQ.tdir ? 1 : 0) >> sig_bit(xp)) & 1ull;
                                        int32_t gl = NOEDGE;
                                        cn.add(CNT_CHECKS, 1);
                                        if (maybe) {
                                            cn.add(CNT_SEARCHES, 1);
                                            gl = LQ.tdir ? edge_label(g, xp, g.out_off[xp], g.out_off[xp + 1], fv, g.in_off[fv],
                                                                      g.in_off[fv + 1], cn.loads())
                                                         : edge_label(g, fv, g.out_off[fv], g.out_off[fv + 1], xp, g.in_off[xp],
                                                                      g.in_off[xp + 1], cn.loads());
                                        } else {
                                            cn.add(CNT_SIG_SETTLED, 1);
                                        }
                                        probes++;
                                        iok = exp_ok(LQ.tlab, gl);
                                    }
                                }
                                // injectivity, then the other pattern pairs
                                for (int q = 0; q < L && iok; q++)
                                    if (((LQ.inj >> q) & 1u) && mo[q << 5] == fv) iok = false;
                                if (iok && nchk2 > 0) {
                                    const uint32_t bv = sig_bit(fv);
                                    uint64_t svo = 0, svi = 0;
                                    bool have_sv = false;
                                    for (int c = 0; c < nchk2 && iok; c++) {
                                        if (c == fskip) continue;
                                        const uint32_t wd = cw2[c];
                                        const uint32_t x = mo[(wd & 15u) << 5];
                                        const bool out = (wd >> 4) & 1u;
                                        const int32_t ex = (int32_t)(int16_t)(wd >> 16);
                                        cn.add(CNT_CHECKS, 1);
                                        cn.add(CNT_SIG_LOADS, 1);
                                        bool maybe = (sig_half(g, x, out ? 1 : 0) >> bv) & 1ull;
                                        if (maybe) {
                                            if (!have_sv) {
                                                const ulonglong2 sg = __ldg(g.sig + fv);
                                                svo = sg.x;
                                                svi = sg.y;
                                                have_sv = true;
                                            }
                                            maybe = ((out ? svo : svi) >> sig_bit(x)) & 1ull;
                                        }
                                        int32_t gl = NOEDGE;
                                        if (maybe) {
                                            cn.add(CNT_SEARCHES, 1);
                                            gl = out ? edge_label(g, fv, g.out_off[fv], g.out_off[fv + 1], x, g.in_off[x],
                                                                  g.in_off[x + 1], cn.loads())
                                                     : edge_label(g, x, g.out_off[x], g.out_off[x + 1], fv, g.in_off[fv],
                                                                  g.in_off[fv + 1], cn.loads());
                                        } else {
                                            cn.add(CNT_SIG_SETTLED, 1);
                                        }
                                        probes++;
                                        iok = exp_ok(ex, gl);
                                    }
                                }
                            }
                            // complete match: X, count, Y, emit (as at the last level)
                            bool fviol = false;
                            if (iok) {
                                bool x_ok = true;
                                for (int q = 0; q < D->nx && x_ok; q++)
                                    if (!GEN || D->lit[q].lvl == L)
                                        x_ok = lit_holds_at(g, D->lit[q], mo, L, fv, COUNT ? &attr_reads : nullptr);
                                if (GEN) tile_matches += x_ok || !D->push_x;
                                else tile_matches++;
                                if (x_ok) {
                                    bool y_ok = !D->y_false;
                                    for (int q = 0; q < D->ny && y_ok; q++)
                                        y_ok = lit_holds_at(g, D->lit[D->nx + q], mo, L, fv, COUNT ? &attr_reads : nullptr);
                                    fviol = !y_ok;
                                }
                            }
                            const uint32_t vb = __ballot_sync(0xffffffffu, fviol);
                            if (vb) {
                                unsigned long long base = 0;
                                if (lane == 0) {
                                    const unsigned long long nv = __popc(vb);
                                    const unsigned long long oldv = atomicAdd((unsigned long long*)&S->n_viol, nv);
                                    base = D->viol ? oldv : atomicAdd((unsigned long long*)&A.sched->varena_used, nv);
                                }
                                base = __shfl_sync(0xffffffffu, base, 0);
                                if (fviol) {
                                    const uint64_t idx = base + __popc(vb & ((1u << lane) - 1u));
                                    if (D->viol) {
                                        if (idx < D->viol_cap) {
                                            int32_t* outp = D->viol + idx * k;
                                            for (int q = 0; q < k; q++) outp[D->order[q]] = (int32_t)level_vertex(mo, q, L, fv);
                                        }
                                    } else if (idx < A.sched->varena_cap) {
                                        int32_t* rec = A.sched->varena + idx * A.sched->vstride;
                                        rec[0] = s;
                                        for (int q = 0; q < k; q++) rec[1 + D->order[q]] = (int32_t)level_vertex(mo, q, L, fv);
                                    }
                                }
                            }
                        }
                    }
                }
                cn.iteration(LAST);
            }
            if (LAST || fuse) {
                const unsigned long long tm = __reduce_add_sync(0xffffffffu, tile_matches);
                if (lane == 0 && tm) atomicAdd((unsigned long long*)&S->n_matches, tm);
            }
        };
        if (last) {
            if (l == 0) run_tile(std::true_type{}, std::true_type{});
            else run_tile(std::true_type{}, std::false_type{});
        } else {
            if (l == 0) run_tile(std::false_type{}, std::true_type{});
            else run_tile(std::false_type{}, std::false_type{});
        }
        uint32_t nt = 0;
        if (lane == 0) nt = atomicAdd(&A.sched->tile_next, 1u);
        t = nwarps + __shfl_sync(0xffffffffu, nt, 0);
    }
    // probe statistics: one atomic per warp
    const unsigned long long p = __reduce_add_sync(0xffffffffu, probes);
    if (lane == 0 && p) atomicAdd((unsigned long long*)&A.sched->probes, p);
    if (COUNT) {
        cn.add(CNT_ATTR_READS, attr_reads);
        cn.flush(A.sched);
    }
}

// Start the enumeration of a slot whose index is built: level 0 holds the root
// candidates, whose work items are the index edges to level 1.
__device__ void slot_start(const SlotDesc* D, SlotState* S) {
    S->cur = 0;
    S->cursor[0] = 0;
    S->cb = S->ce = 0;
    S->nrows[0] = S->ncand[0];
    S->total[0] = D->k == 1             ? (uint64_t)S->ncand[0]
                : D->lv[1].par < 0      ? (uint64_t)S->ncand[0] * S->ncand[1]  // level 1 starts a component
                                        : (uint64_t)D->cpi_off[1][S->ncand[0]];
}

// One block: finish the last step of every slot and plan the next one.
template <int CT>
__device__ void control_step(const EnumArgs& A, bool first) {
    using Scan = cub::BlockScan<unsigned long long, CT>;
    using Scan32 = cub::BlockScan<uint32_t, CT>;
    __shared__ typename Scan::TempStorage tmp;
    __shared__ typename Scan32::TempStorage tmp32;
    __shared__ unsigned long long carry_s;
    __shared__ uint32_t carry_last_s;
    __shared__ int32_t active_s;
    __shared__ int32_t expired_s;
    __shared__ unsigned long long work_s;
    if (threadIdx.x == 0) {
        carry_s = 0;
        carry_last_s = 0;
        active_s = 0;
        work_s = 0;
        // bound the whole enumeration in time: past the limit every slot stops
        const uint64_t now = globaltimer_ns();
        if (first || A.sched->t_start == 0) A.sched->t_start = now;
        expired_s = now - A.sched->t_start > A.sched->run_limit_ns;
        if (expired_s) A.sched->err = DERR_TIMEOUT;
    }
    __syncthreads();
    for (int base = 0; base < A.n_slots; base += CT) {
        const int s = base + threadIdx.x;
        if (s < A.n_slots) {
            const SlotDesc* D = A.slots + s;
            SlotState* S = A.state + s;
            const int k = D->k;
            if (first) {
                slot_start(D, S);
            } else if (S->cur >= 0) {
                const int l = S->cur;
                S->cursor[l] = S->ce;
                S->st_steps++;
                if (k > 1 && l + 1 <= k - 2) {
                    const uint64_t c = __ldcg((const unsigned long long*)&S->ctr[l + 1]);
                    const uint64_t rows = c >> ROW_SHIFT;
                    if (rows > 0) {
                        S->nrows[l + 1] = rows;
                        S->total[l + 1] = c & WORK_MASK;
                        S->cursor[l + 1] = 0;
                        S->cur = l + 1;
                        S->st_rows += rows;
                    }
                }
            }
            while (S->cur >= 0 && S->cursor[S->cur] >= S->total[S->cur]) S->cur--;
            if (__ldcg(&S->err) || expired_s) S->cur = -1;
            if (S->cur >= 0) {
                const int l = S->cur;
                S->cb = S->cursor[l];
                // the last level writes no partial matches, so its steps are not
                // bounded by the row buffers
                const bool to_last = k == 1 || l + 1 == k - 1;
                const uint64_t step = to_last ? max(D->chunk, (uint64_t)LAST_LEVEL_CHUNK) : D->chunk;
                S->ce = min(S->cb + step, S->total[l]);
                if (k > 1 && l + 1 <= k - 2) S->ctr[l + 1] = 0;
                S->st_work += S->ce - S->cb;
                atomicAdd(&active_s, 1);
                atomicAdd(&work_s, (unsigned long long)(S->ce - S->cb));
            }
        }
    }
    __syncthreads();
    // Tile size of this step: the largest (up to A.tile) that still gives every
    // warp about four tiles, so that a step with little work (one slot at an
    // intermediate level) is spread over all warps.
    uint64_t tile = (uint64_t)A.tile;
    if (A.n_warps > 0) {
        const uint64_t per = work_s / (4ull * (uint64_t)A.n_warps);
        tile = min(tile, max((uint64_t)32, (uint64_t)((per + 31) & ~(uint64_t)31)));
    }
    // A slot whose step makes the second-to-last level's partial matches also
    // expands most of their last level inside the same tiles (fused, up to
    // FUSE_FANOUT items per partial match): its tiles are cut smaller, so that
    // no single tile holds the step's end. The step's tiles are numbered
    // heaviest first: the fusing slots', those of the other intermediate
    // levels (which store partial matches), the last level's. tile_base holds
    // three prefixes over the slots, each class from the end of the one before:
    // [0, n] fusing (F tiles), [n + 1, 2n + 1] intermediate (M), [2n + 2, 3n + 2]
    // last level. The first two counts are scanned packed in 64 bits (each total
    // is below 2^32).
    const uint64_t tile_fused = max((uint64_t)32, (tile / FUSED_TILE_DIV) & ~(uint64_t)31);
    const int n = A.n_slots;
    for (int base = 0; base < n; base += CT) {
        const int s = base + threadIdx.x;
        unsigned long long fm = 0;  // fusing << 32 | intermediate
        uint32_t nl = 0;             // last level
        if (s < n) {
            SlotState* S = A.state + s;
            if (S->cur >= 0) {
                const int k = A.slots[s].k;
                const bool fused = k >= 3 && S->cur + 1 == k - 2;
                const bool to_last = k == 1 || S->cur + 1 == k - 1;
                const uint64_t ts = fused ? tile_fused : tile;
                S->tile = (uint32_t)ts;
                const uint64_t nt = (S->ce - S->cb + ts - 1) / ts;
                if (fused) fm = nt << 32;
                else if (to_last && LAST_LEVEL_TILES_LAST) nl = (uint32_t)nt;
                else fm = nt;
            }
        }
        unsigned long long excl, total;
        Scan(tmp).ExclusiveSum(fm, excl, total);
        uint32_t lexcl, ltotal;
        Scan32(tmp32).ExclusiveSum(nl, lexcl, ltotal);
        if (s < n) {
            A.tile_base[s] = (uint32_t)((carry_s + excl) >> 32);
            A.tile_base[n + 1 + s] = (uint32_t)(carry_s + excl);  // F added below
            A.tile_base[2 * n + 2 + s] = carry_last_s + lexcl;   // F + M added below
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_s += total;
            carry_last_s += ltotal;
        }
        __syncthreads();
    }
    const uint32_t nfused = (uint32_t)(carry_s >> 32), nmid = (uint32_t)carry_s, nlast = carry_last_s;
    for (int s = threadIdx.x; s < n; s += CT) {
        A.tile_base[n + 1 + s] += nfused;
        A.tile_base[2 * n + 2 + s] += nfused + nmid;
    }
    if (threadIdx.x == 0) {
        A.tile_base[n] = nfused;
        A.tile_base[2 * n + 1] = nfused + nmid;
        A.tile_base[3 * n + 2] = nfused + nmid + nlast;
        A.sched->total_tiles = nfused + nmid + nlast;
        A.sched->tile = (uint32_t)tile;
        A.sched->tile_next = 0;
        A.sched->active = active_s;
        A.sched->steps++;
        __threadfence();
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CTRL_THREADS) k_control(EnumArgs A, int first) {
    control_step<CTRL_THREADS>(A, first != 0);
}

template <int NT, int MINB, bool GEN>
__global__ void __launch_bounds__(NT, MINB) k_expand(EnumArgs A) {
    expand_warps<NT, GEN, false>(A);
}

// Bounded grid barrier (cooperative launch guarantees co-residency): the last
// arriving block bumps the generation; the others wait for it, up to
// sched->timeout_ns, after which they record DERR_TIMEOUT and give up.
__device__ bool grid_barrier(Sched* s) {
    __syncthreads();
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        volatile uint32_t* genp = &s->bar_gen;
        const uint32_t gen = *genp;
        __threadfence();
        const uint32_t arrived = atomicAdd(&s->bar_count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(&s->bar_count, 0u);
            __threadfence();
            atomicAdd(&s->bar_gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (*genp == gen) {
                if (*(volatile int32_t*)&s->err) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > s->timeout_ns) {
                    atomicExch(&s->err, DERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <int NT, int MINB, bool GEN, bool COUNT = false>
__global__ void __launch_bounds__(NT, MINB) k_persistent(EnumArgs A) {
    for (;;) {
        expand_warps<NT, GEN, COUNT>(A);
        if (!grid_barrier(A.sched)) return;
        if (blockIdx.x == 0) control_step<NT>(A, false);
        if (!grid_barrier(A.sched)) return;
        if (*(volatile int32_t*)&A.sched->active == 0) return;
    }
}

template <int NT, int MINB, bool GEN, bool COUNT = false>
int launch_persistent(const EnumArgs& a, cudaStream_t st, int64_t* launches) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<NT, MINB, GEN, COUNT>, NT, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) {
        set_error(GFD_ERR_CUDA, "persistent enumeration kernel cannot be resident");
        return GFD_ERR_CUDA;
    }
    const int grid = sms * per_sm;
    EnumArgs args = a;
    args.n_warps = grid * (NT / 32);
    void* params[] = {&args};
    e = cudaLaunchCooperativeKernel((const void*)k_persistent<NT, MINB, GEN, COUNT>, dim3(grid), dim3(NT), params, 0,
                                    st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel");
    if (launches) *launches += 1;
    return GFD_OK;
}

template <int NT, int MINB, bool GEN>
int expand_grid() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand<NT, MINB, GEN>, NT, 0);
    return sms * std::max(per_sm, 1);
}

template <int NT, int MINB, bool GEN>
int host_loop(const EnumArgs& a0, bool use_graph, cudaStream_t st, int64_t* launches) {
    const int grid = expand_grid<NT, MINB, GEN>();
    EnumArgs a = a0;
    a.n_warps = grid * (NT / 32);
    int32_t* h_active = nullptr;
    cudaError_t e = cudaMallocHost(&h_active, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    const int per_check = 8;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int rc = GFD_OK;
    if (use_graph) {
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int it = 0; it < per_check; it++) {
                k_expand<NT, MINB, GEN><<<grid, NT, 0, st>>>(a);
                k_control<<<1, CTRL_THREADS, 0, st>>>(a, 0);
            }
            e = cudaStreamEndCapture(st, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            cudaFreeHost(h_active);
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e, "CUDA graph capture of the enumeration steps");
        }
    }
    for (int64_t round = 0;; round++) {
        if (use_graph) {
            e = cudaGraphLaunch(exec, st);
            if (launches) *launches += 2 * per_check;
        } else {
            for (int it = 0; it < per_check; it++) {
                k_expand<NT, MINB, GEN><<<grid, NT, 0, st>>>(a);
                k_control<<<1, CTRL_THREADS, 0, st>>>(a, 0);
            }
            e = cudaGetLastError();
            if (launches) *launches += 2 * per_check;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_active, &a.sched->active, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "enumeration step");
            break;
        }
        if (*h_active == 0) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFreeHost(h_active);
    return rc;
}

// one thread per violation record: append it to its GFD's list
__global__ void k_split(const SlotDesc* slots, const int32_t* arena, uint64_t n, int32_t stride,
                        int32_t* const* lists, unsigned long long* cursor) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t* rec = arena + r * stride;
        const int s = rec[0];
        const int k = slots[s].k;
        // one atomic per group of lanes with the same slot (records of one
        // slot arrive in runs, so a warp usually needs one or two)
        const int lane = threadIdx.x & 31;
        const uint32_t peers = __match_any_sync(__activemask(), s);
        const int leader = __ffs(peers) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&cursor[s], (unsigned long long)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        const uint64_t pos = base + __popc(peers & ((1u << lane) - 1u));
        int32_t* dst = lists[s] + pos * k;
        for (int q = 0; q < k; q++) dst[q] = rec[1 + q];
    }
}

__global__ void k_mark_idle(SlotState* state, int n) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) state[s].cur = -1;
}

// Slots admitted between steps: start them (the next control step plans their
// first chunk), finishing at once when level 0 has no work. The slot ids
// travel in the kernel parameters.
struct SlotIds {
    int n;
    int v[64];
};

__global__ void k_init_slots(EnumArgs A, SlotIds ids) {
    const int i = threadIdx.x;
    if (i >= ids.n) return;
    const int s = ids.v[i];
    SlotState* S = A.state + s;
    slot_start(A.slots + s, S);
    if (S->total[0] == 0) S->cur = -1;
}

}  // namespace

int mark_idle(SlotState* state, int n, cudaStream_t st) {
    k_mark_idle<<<std::max(1, (n + 255) / 256), 256, 0, st>>>(state, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GFD_OK : cuda_fail(e, "k_mark_idle");
}

int init_slots(const EnumArgs& a, const int* host_ids, int n, cudaStream_t st) {
    for (int b = 0; b < n; b += 64) {
        SlotIds ids{};
        ids.n = std::min(64, n - b);
        for (int i = 0; i < ids.n; i++) ids.v[i] = host_ids[b + i];
        k_init_slots<<<1, 64, 0, st>>>(a, ids);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GFD_OK : cuda_fail(e, "k_init_slots");
}

int launch_split(const SlotDesc* slots, const int32_t* arena, uint64_t n, int32_t stride, int32_t* const* lists,
                 unsigned long long* cursor, cudaStream_t st) {
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sms() * 16);
    k_split<<<std::max(grid, 1), 256, 0, st>>>(slots, arena, n, stride, lists, cursor);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GFD_OK : cuda_fail(e, "k_split");
}

namespace {

template <int NT, int MINB, bool GEN>
int capture_steps_t(const EnumArgs& a0, int steps, cudaStream_t st, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    const int grid = expand_grid<NT, MINB, GEN>();
    EnumArgs a = a0;
    a.n_warps = grid * (NT / 32);
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int it = 0; it < steps; it++) {
            k_expand<NT, MINB, GEN><<<grid, NT, 0, st>>>(a);
            k_control<<<1, CTRL_THREADS, 0, st>>>(a, 0);
        }
        e = cudaStreamEndCapture(st, graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, *graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "CUDA graph capture of the enumeration steps");
    return GFD_OK;
}

template <int NT, int MINB, bool GEN>
int run_variant(const EnumArgs& a, bool persistent, bool use_graph, cudaStream_t st, int64_t* launches) {
    return persistent ? launch_persistent<NT, MINB, GEN>(a, st, launches) : host_loop<NT, MINB, GEN>(a, use_graph, st, launches);
}

}  // namespace

// Kernel variants: threads per block and the minimum resident blocks per SM the
// compiler must allow (which caps registers per thread).
int variant_threads(int v) {
    switch (v) {
        case 3: return 128;
        case 5: return 512;
        default: return 256;
    }
}

int capture_steps(const EnumArgs& a, int variant, int steps, cudaStream_t st, cudaGraph_t* graph,
                  cudaGraphExec_t* exec) {
    // a session admits any request later: the general expansion
    constexpr bool GEN = true;
    switch (variant) {
        case 1: return capture_steps_t<256, 6, GEN>(a, steps, st, graph, exec);
        case 2: return capture_steps_t<256, 8, GEN>(a, steps, st, graph, exec);
        case 3: return capture_steps_t<128, 12, GEN>(a, steps, st, graph, exec);
        case 4: return capture_steps_t<256, 5, GEN>(a, steps, st, graph, exec);
        case 5: return capture_steps_t<512, 3, GEN>(a, steps, st, graph, exec);
        default: return capture_steps_t<256, 4, GEN>(a, steps, st, graph, exec);
    }
}

namespace {

template <bool GEN>
int run_any_variant(const EnumArgs& a, bool persistent, bool use_graph, int variant, cudaStream_t st,
                    int64_t* launches) {
    switch (variant) {
        case 1: return run_variant<256, 6, GEN>(a, persistent, use_graph, st, launches);
        case 2: return run_variant<256, 8, GEN>(a, persistent, use_graph, st, launches);
        case 3: return run_variant<128, 12, GEN>(a, persistent, use_graph, st, launches);
        case 4: return run_variant<256, 5, GEN>(a, persistent, use_graph, st, launches);
        case 5: return run_variant<512, 3, GEN>(a, persistent, use_graph, st, launches);
        default: return run_variant<256, 4, GEN>(a, persistent, use_graph, st, launches);
    }
}

}  // namespace

int enum_init(const EnumArgs& a, cudaStream_t st) {
    k_control<<<1, CTRL_THREADS, 0, st>>>(a, 1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GFD_OK : cuda_fail(e, "k_control");
}

int enum_run(const EnumArgs& a, bool persistent, bool use_graph, int variant, bool general, cudaStream_t st,
             cudaEvent_t ev0, cudaEvent_t ev1, int64_t* launches, bool count) {
    if (ev0) cudaEventRecord(ev0, st);
    const int rc = count     ? launch_persistent<256, 4, true, true>(a, st, launches)
                 : general ? run_any_variant<true>(a, persistent, use_graph, variant, st, launches)
                           : run_any_variant<false>(a, persistent, use_graph, variant, st, launches);
    if (ev1) cudaEventRecord(ev1, st);
    return rc;
}

}  // namespace gfd
