// Compact path index construction (Section III.B, step 1).
//
//   k_filter   step 1a-1b: candidates by label and degree (and self-loop, and
//              pushed-down constant X literals), one coalesced pass over vertex
//              data for all filter keys;
//   k_scatter  step 1c: mark vertices adjacent (in the direction and with the
//   k_and      label of a pattern edge) to the candidates of another level,
//              then intersect;
//   k_prune    step 1c: remove candidates with no such neighbour among the
//              candidates of another level (early exit at the first one);
//              top-down and bottom-up use whichever of the two is cheaper;
//   k_compact  bitmap -> exclusive popcount prefix (O(1) rank) + sorted list;
//   k_cpi_*    step 1d: for each spanning-tree edge, the index edges from
//              every parent candidate to the positions of its child candidates;
//   *_hub      the same for adjacency lists over HUB_LIST entries, one block
//              per list (queued by the warp kernels).
//
// Every launch processes a table of jobs; blocks (or warps) stride over the
// items of each job with a per-job rotation so that small jobs spread out.
#include <cub/cub.cuh>

#include <map>
#include <mutex>

#include "engine.h"

namespace gfd {

namespace {

constexpr int FILTER_THREADS = 256;
constexpr int COMPACT_THREADS = 256;
constexpr uint32_t COMPACT_WORDS = 1024;  // words (or counts) per chunk
constexpr int WARP_KERNEL_THREADS = 256;

__device__ __forceinline__ uint64_t gwarp_id() {
    return (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ uint64_t nwarps_total() { return ((uint64_t)gridDim.x * blockDim.x) >> 5; }

__device__ __forceinline__ bool bit_of(const uint32_t* bm, uint32_t x) {
    return (bm[x >> 5] >> (x & 31)) & 1u;
}

__global__ void k_filter(DevGraph g, const FilterKey* __restrict__ keys, int nkeys, uint32_t* __restrict__ out) {
    extern __shared__ FilterKey sk[];
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) sk[i] = keys[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (uint64_t w = gwarp_id(); w < g.nwords; w += nwarps_total()) {
        const uint32_t v = (uint32_t)w * 32 + lane;
        const bool valid = v < (uint32_t)g.n;
        uint32_t vi = 0, dout = 0, din = 0;
        if (valid) {
            vi = g.vinfo[v];
            dout = g.out_off[v + 1] - g.out_off[v];
            din = g.in_off[v + 1] - g.in_off[v];
        }
        const int32_t L = (int32_t)(vi & 0xffffu);
        const bool has_self = (vi >> 16) != 0;
        const int32_t self_lab = (int32_t)(vi >> 16) - 1;
        dout -= has_self;
        din -= has_self;
        for (int k = 0; k < nkeys; k++) {
            const FilterKey& key = sk[k];  // fields read from shared memory as needed
            bool self_ok = key.self_exp == EXP_SKIP ? true
                         : key.self_exp == EXP_NONE ? !has_self
                         : key.self_exp == EXP_ANY  ? has_self
                                                    : (has_self && self_lab == key.self_exp);
            bool p = valid && label_ok(key.label, L) && dout >= key.dout_min && din >= key.din_min && self_ok;
            for (int t = 0; t < key.n_attr; t++) {  // pushed-down constant X literals
                const int32_t va = p ? g.attrs[(uint64_t)key.attr_a[t] * g.n + v] : GFD_ATTR_ABSENT;
                p = p && va != GFD_ATTR_ABSENT && va == key.attr_c[t];
            }
            uint32_t b = __ballot_sync(0xffffffffu, p);
            if (lane == 0) out[(uint64_t)k * g.nwords + w] = b;
        }
    }
}

// One block per (job, chunk of AND_WORDS words) item, so that every job's words
// are spread over the GPU and no thread walks the job table.
constexpr uint32_t AND_WORDS = 2048;
constexpr int AND_THREADS = 256;

__global__ void __launch_bounds__(AND_THREADS) k_and(DevGraph g, const AndJob* __restrict__ jobs, int njobs,
                                                      uint32_t nchunks) {
    for (uint64_t it = blockIdx.x; it < (uint64_t)njobs * nchunks; it += gridDim.x) {
        const AndJob& J = jobs[it / nchunks];
        const uint32_t w0 = (uint32_t)(it % nchunks) * AND_WORDS;
        const uint32_t w1 = min(g.nwords, w0 + AND_WORDS);
        const int ntmp = J.ntmp;
        for (uint32_t w = w0 + threadIdx.x; w < w1; w += AND_THREADS) {
            uint32_t x = J.src[w];
            for (int t = 0; t < ntmp; t++) x &= J.tmp[t][w];
            J.bm[w] = x;
        }
    }
}

// Compaction in two passes over (job, chunk) items so that even one job uses
// the whole GPU: k_compact_sums counts set bits per chunk of COMPACT_WORDS
// words; k_compact_write adds the counts of the preceding chunks, scans its own
// chunk and writes rank[w] (set bits before word w) and the candidate list.
__global__ void __launch_bounds__(COMPACT_THREADS) k_compact_sums(DevGraph g, const CompactJob* __restrict__ jobs,
                                                                  int njobs, uint32_t nchunks) {
    using Reduce = cub::BlockReduce<uint32_t, COMPACT_THREADS>;
    __shared__ typename Reduce::TempStorage tmp;
    for (uint64_t it = blockIdx.x; it < (uint64_t)njobs * nchunks; it += gridDim.x) {
        const CompactJob& J = jobs[it / nchunks];
        const uint32_t c = (uint32_t)(it % nchunks);
        uint32_t cnt = 0;
        for (uint32_t w = c * COMPACT_WORDS + threadIdx.x; w < min(g.nwords, (c + 1) * COMPACT_WORDS);
             w += COMPACT_THREADS)
            cnt += __popc(J.bm[w]);
        cnt = Reduce(tmp).Sum(cnt);
        if (threadIdx.x == 0) J.csum[c] = cnt;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(COMPACT_THREADS) k_compact_write(DevGraph g, const CompactJob* __restrict__ jobs,
                                                                   int njobs, uint32_t nchunks) {
    using Scan = cub::BlockScan<uint32_t, COMPACT_THREADS>;
    using Reduce = cub::BlockReduce<uint32_t, COMPACT_THREADS>;
    __shared__ union {
        typename Scan::TempStorage scan;
        typename Reduce::TempStorage reduce;
    } tmp;
    __shared__ uint32_t base_s;
    constexpr int WPT = COMPACT_WORDS / COMPACT_THREADS;  // words per thread
    for (uint64_t it = blockIdx.x; it < (uint64_t)njobs * nchunks; it += gridDim.x) {
        const CompactJob& J = jobs[it / nchunks];
        const uint32_t c = (uint32_t)(it % nchunks);
        uint32_t before = 0;
        for (uint32_t q = threadIdx.x; q < c; q += COMPACT_THREADS) before += J.csum[q];
        before = Reduce(tmp.reduce).Sum(before);
        if (threadIdx.x == 0) base_s = before;
        __syncthreads();
        const uint32_t w0 = c * COMPACT_WORDS + threadIdx.x * WPT;
        uint32_t words[WPT];
        uint32_t cnt = 0;
        for (int q = 0; q < WPT; q++) {
            words[q] = w0 + q < g.nwords ? J.bm[w0 + q] : 0u;
            cnt += __popc(words[q]);
        }
        uint32_t excl, total;
        Scan(tmp.scan).ExclusiveSum(cnt, excl, total);
        uint32_t r = base_s + excl;
        for (int q = 0; q < WPT; q++) {
            if (w0 + q >= g.nwords) break;
            J.rank[w0 + q] = r;
            uint32_t x = words[q];
            while (x) {
                const int bpos = __ffs(x) - 1;
                J.cand[r++] = (int32_t)((w0 + q) * 32 + bpos);
                x &= x - 1;
            }
        }
        if (c == nchunks - 1 && threadIdx.x == 0) *J.count = base_s + total;
        __syncthreads();
    }
}

// The adjacency kernels below give each lane of a warp one candidate and let
// the lane scan a short list alone; lists longer than SHORT_LIST are left to
// the whole warp, one after the other (ballot of the long ones), scanned 32
// entries at a time without idling lanes on short lists; hub lists (over
// HUB_LIST entries) are queued for a block each.
constexpr uint32_t SHORT_LIST = 32;

// A lane scanning a short list alone reads UNROLL entries per round and then
// their UNROLL bitmap words, so that each round costs two dependent loads
// rather than two per entry.
constexpr int UNROLL = 4;

constexpr int HUB_THREADS = 512;

// Queue the lanes whose list is a hub (warp-synchronous: every lane calls it);
// true for the lanes whose item was stored.
__device__ __forceinline__ bool hub_push(const HubQueue& q, bool want, unsigned long long item, int lane) {
    const uint32_t b = __ballot_sync(0xffffffffu, want);
    if (!b) return false;
    const int leader = __ffs(b) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(q.n, (uint32_t)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    const uint32_t pos = base + __popc(b & ((1u << lane) - 1u));
    if (want && pos < q.cap) {
        q.item[pos] = item;
        return true;
    }
    return false;
}

__device__ __forceinline__ uint32_t hub_count(const HubQueue& q) { return min(*q.n, q.cap); }

// The adjacency kernels below take (job, group of 32 candidates) items from one
// flat index: k_job_groups writes the exclusive prefix of the jobs' group
// counts (total at [njobs]), and job_of finds an item's job by binary search,
// so no warp walks the whole job table.
__device__ __forceinline__ uint32_t job_count(const ScatterJob& J) { return *J.qcount; }
__device__ __forceinline__ uint32_t job_count(const PruneJob& J) { return *J.count; }
__device__ __forceinline__ uint32_t job_count(const CpiJob& J) { return *J.pcount; }

constexpr int JOB_SCAN_THREADS = 1024;

template <typename Job>
__global__ void __launch_bounds__(JOB_SCAN_THREADS) k_job_groups(const Job* __restrict__ jobs, int njobs,
                                                                  uint32_t* pre) {
    using Scan = cub::BlockScan<uint32_t, JOB_SCAN_THREADS>;
    __shared__ typename Scan::TempStorage tmp;
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < njobs; b += JOB_SCAN_THREADS) {
        const int j = b + threadIdx.x;
        const uint32_t groups = j < njobs ? (job_count(jobs[j]) + 31) / 32 : 0;
        uint32_t excl, total;
        Scan(tmp).ExclusiveSum(groups, excl, total);
        if (j < njobs) pre[j] = carry + excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) pre[njobs] = carry;
}

// the job whose items [pre[j], pre[j+1]) hold item it (pre[njobs] > it)
__device__ __forceinline__ int job_of(const uint32_t* pre, int njobs, uint32_t it) {
    int lo = 0, hi = njobs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Counting pass: add this thread's scanned candidates and adjacency entries to
// the run's counters (all lanes of the warp call it; one atomic per warp).
template <bool COUNT>
__device__ __forceinline__ void scan_flush(const HubQueue& q, uint64_t cands, uint64_t entries) {
    if (!COUNT || !q.scan) return;
    for (int d = 16; d >= 1; d >>= 1) {
        cands += __shfl_xor_sync(0xffffffffu, cands, d);
        entries += __shfl_xor_sync(0xffffffffu, entries, d);
    }
    if ((threadIdx.x & 31) == 0) {
        if (cands) atomicAdd(&q.scan[0], (unsigned long long)cands);
        if (entries) atomicAdd(&q.scan[1], (unsigned long long)entries);
    }
}

__device__ __forceinline__ void load_group(const uint32_t* adj, uint32_t e, uint32_t e1, uint32_t (&p)[UNROLL]) {
#pragma unroll
    for (int t = 0; t < UNROLL; t++) p[t] = e + t < e1 ? __ldg(adj + e + t) : 0u;
}

template <bool COUNT>
__global__ void k_scatter(DevGraph g, const ScatterJob* __restrict__ jobs, int njobs, HubQueue hq) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    uint64_t sc = 0, se = 0;
    const uint32_t ngroups = hq.jpre[njobs];
    for (uint64_t it = gw; it < ngroups; it += nw) {
        // the warp's group of 32 candidates: job j, group grp of that job
        const int j = job_of(hq.jpre, njobs, (uint32_t)it);
        const uint64_t grp = it - hq.jpre[j];
        const ScatterJob J = jobs[j];
        const uint32_t n = *J.qcount;
        const uint32_t* off = J.scan_out ? g.out_off : g.in_off;
        const uint32_t* adj = J.scan_out ? g.out_adj : g.in_adj;
        {
            const uint64_t a = grp * 32 + lane;
            uint32_t e0 = 0, e1 = 0;
            if (a < n) {
                const uint32_t v = (uint32_t)J.qcand[a];
                e0 = off[v];
                e1 = off[v + 1];
            }
            if (hub_push(hq, e1 - e0 > HUB_LIST, ((unsigned long long)j << 40) | a, lane)) e1 = e0;
            const bool is_long = e1 - e0 > SHORT_LIST;
            sc += a < n && e1 > e0;
            se += e1 - e0;
            if (!is_long)
                for (uint32_t e = e0; e < e1; e += UNROLL) {
                    uint32_t p[UNROLL], f[UNROLL];
                    load_group(adj, e, e1, p);
#pragma unroll
                    for (int t = 0; t < UNROLL; t++)
                        f[t] = e + t < e1 ? __ldg(J.filter + ((p[t] >> g.lbits) >> 5)) : 0u;
#pragma unroll
                    for (int t = 0; t < UNROLL; t++) {
                        const uint32_t x = p[t] >> g.lbits;
                        if (e + t < e1 && label_ok(J.lab, (int32_t)(p[t] & g.lmask)) && ((f[t] >> (x & 31)) & 1u))
                            atomicOr(&J.marks[x >> 5], 1u << (x & 31));
                    }
                }
            for (uint32_t lm = __ballot_sync(0xffffffffu, is_long); lm; lm &= lm - 1) {
                const int src = __ffs(lm) - 1;
                const uint32_t b0 = __shfl_sync(0xffffffffu, e0, src), b1 = __shfl_sync(0xffffffffu, e1, src);
                for (uint32_t e = b0 + lane; e < b1; e += 32) {
                    const uint32_t p = adj[e];
                    const uint32_t x = p >> g.lbits;
                    if (label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.filter, x))
                        atomicOr(&J.marks[x >> 5], 1u << (x & 31));
                }
            }
        }
    }
    scan_flush<COUNT>(hq, sc, se);
}

// Does the list adj[e0, e1) hold a neighbour in bm with an allowed label? One
// lane alone (short lists) or the whole warp (cooperative).
__device__ __forceinline__ bool any_hit_serial(const DevGraph& g, const uint32_t* adj, uint32_t e0, uint32_t e1,
                                               int32_t lab, const uint32_t* bm, uint64_t& read) {
    for (uint32_t e = e0; e < e1; e += UNROLL) {
        read += min((uint32_t)UNROLL, e1 - e);
        uint32_t p[UNROLL], w[UNROLL];
        load_group(adj, e, e1, p);
#pragma unroll
        for (int t = 0; t < UNROLL; t++) w[t] = e + t < e1 ? __ldg(bm + ((p[t] >> g.lbits) >> 5)) : 0u;
        bool hit = false;
#pragma unroll
        for (int t = 0; t < UNROLL; t++)
            hit |= e + t < e1 && label_ok(lab, (int32_t)(p[t] & g.lmask)) && ((w[t] >> ((p[t] >> g.lbits) & 31)) & 1u);
        if (hit) return true;
    }
    return false;
}

__device__ __forceinline__ bool any_hit_warp(const DevGraph& g, const uint32_t* adj, uint32_t e0, uint32_t e1,
                                             int32_t lab, const uint32_t* bm, int lane, uint64_t& read) {
    for (uint32_t b = e0; b < e1; b += 32) {
        if (lane == 0) read += min(32u, e1 - b);
        const uint32_t e = b + lane;
        bool hit = false;
        if (e < e1) {
            const uint32_t p = adj[e];
            hit = label_ok(lab, (int32_t)(p & g.lmask)) && bit_of(bm, p >> g.lbits);
        }
        if (__any_sync(0xffffffffu, hit)) return true;
    }
    return false;
}

template <bool COUNT>
__global__ void k_prune(DevGraph g, const PruneJob* __restrict__ jobs, int njobs, HubQueue hq) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    uint64_t sc = 0, se = 0;
    const uint32_t ngroups = hq.jpre[njobs];
    for (uint64_t it = gw; it < ngroups; it += nw) {
        // the warp's group of 32 candidates: job j, group grp of that job
        const int j = job_of(hq.jpre, njobs, (uint32_t)it);
        const uint64_t grp = it - hq.jpre[j];
        const PruneJob& J = jobs[j];
        const uint32_t n = *J.count;
        const int ncon = J.ncon;
        {
            const uint64_t a = grp * 32 + lane;
            const bool valid = a < n;
            const uint32_t v = valid ? (uint32_t)J.cand[a] : 0u;
            bool keep = valid;
            for (int c = 0; c < ncon; c++) {
                const uint32_t* off = J.con_dir[c] ? g.out_off : g.in_off;
                const uint32_t* adj = J.con_dir[c] ? g.out_adj : g.in_adj;
                uint32_t e0 = 0, e1 = 0;
                if (keep) {
                    e0 = off[v];
                    e1 = off[v + 1];
                }
                // a hub's constraint is decided by a block later (it clears the bit
                // when nothing hits); the other constraints go on here
                const bool queued = hub_push(hq, keep && e1 - e0 > HUB_LIST,
                                             ((unsigned long long)j << 40) | ((unsigned long long)c << 32) | a, lane);
                const bool is_long = keep && !queued && e1 - e0 > SHORT_LIST;
                sc += keep && !queued;
                if (keep && !queued && !is_long) keep = any_hit_serial(g, adj, e0, e1, J.con_lab[c], J.con_bm[c], se);
                for (uint32_t lm = __ballot_sync(0xffffffffu, is_long); lm; lm &= lm - 1) {
                    const int src = __ffs(lm) - 1;
                    const uint32_t b0 = __shfl_sync(0xffffffffu, e0, src), b1 = __shfl_sync(0xffffffffu, e1, src);
                    const bool hit = any_hit_warp(g, adj, b0, b1, J.con_lab[c], J.con_bm[c], lane, se);
                    if (lane == src) keep = hit;
                }
            }
            if (valid && !keep) atomicAnd(&J.bm[v >> 5], ~(1u << (v & 31)));
        }
    }
    scan_flush<COUNT>(hq, sc, se);
}

// off[a] = number of children of parent candidate a
template <bool COUNT>
__global__ void k_cpi_count(DevGraph g, const CpiJob* __restrict__ jobs, int njobs, HubQueue hq) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    uint64_t sc = 0, se = 0;
    const uint32_t ngroups = hq.jpre[njobs];
    for (uint64_t it = gw; it < ngroups; it += nw) {
        // the warp's group of 32 candidates: job j, group grp of that job
        const int j = job_of(hq.jpre, njobs, (uint32_t)it);
        const uint64_t grp = it - hq.jpre[j];
        const CpiJob J = jobs[j];
        const uint32_t n = *J.pcount;
        const uint32_t* off = J.out ? g.out_off : g.in_off;
        const uint32_t* adj = J.out ? g.out_adj : g.in_adj;
        {
            const uint64_t a = grp * 32 + lane;
            uint32_t e0 = 0, e1 = 0;
            if (a < n) {
                const uint32_t v = (uint32_t)J.pcand[a];
                e0 = off[v];
                e1 = off[v + 1];
            }
            const bool queued = hub_push(hq, e1 - e0 > HUB_LIST, ((unsigned long long)j << 40) | a, lane);
            if (queued) e1 = e0;  // counted by a block later
            const bool is_long = e1 - e0 > SHORT_LIST;
            sc += a < n && e1 > e0;
            se += e1 - e0;
            uint32_t cnt = 0;
            if (!is_long)
                for (uint32_t e = e0; e < e1; e += UNROLL) {
                    uint32_t p[UNROLL], w[UNROLL];
                    load_group(adj, e, e1, p);
#pragma unroll
                    for (int t = 0; t < UNROLL; t++) w[t] = e + t < e1 ? __ldg(J.cbm + ((p[t] >> g.lbits) >> 5)) : 0u;
#pragma unroll
                    for (int t = 0; t < UNROLL; t++)
                        cnt += e + t < e1 && label_ok(J.lab, (int32_t)(p[t] & g.lmask)) &&
                               ((w[t] >> ((p[t] >> g.lbits) & 31)) & 1u);
                }
            for (uint32_t lm = __ballot_sync(0xffffffffu, is_long); lm; lm &= lm - 1) {
                const int src = __ffs(lm) - 1;
                const uint32_t b0 = __shfl_sync(0xffffffffu, e0, src), b1 = __shfl_sync(0xffffffffu, e1, src);
                uint32_t c = 0;
                for (uint32_t e = b0 + lane; e < b1; e += 32) {
                    const uint32_t p = adj[e];
                    c += label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.cbm, p >> g.lbits);
                }
                c = __reduce_add_sync(0xffffffffu, c);
                if (lane == src) cnt = c;
            }
            if (a < n && !queued) J.off[a] = cnt;
        }
    }
    scan_flush<COUNT>(hq, sc, se);
}

// Exclusive scan of the per-candidate counts off[0..n) in place, off[n] =
// total, in two passes over (job, chunk) items like the compaction above.
__global__ void __launch_bounds__(COMPACT_THREADS) k_cpi_sums(const CpiJob* __restrict__ jobs, int njobs,
                                                              uint32_t nchunks) {
    using Reduce = cub::BlockReduce<uint64_t, COMPACT_THREADS>;
    __shared__ typename Reduce::TempStorage tmp;
    for (uint64_t it = blockIdx.x; it < (uint64_t)njobs * nchunks; it += gridDim.x) {
        const CpiJob& J = jobs[it / nchunks];
        const uint32_t c = (uint32_t)(it % nchunks);
        const uint32_t n = *J.pcount;
        if ((uint64_t)c * COMPACT_WORDS >= n && c > 0) continue;
        uint64_t cnt = 0;
        for (uint32_t a = c * COMPACT_WORDS + threadIdx.x; a < min(n, (c + 1) * COMPACT_WORDS); a += COMPACT_THREADS)
            cnt += J.off[a];
        cnt = Reduce(tmp).Sum(cnt);
        if (threadIdx.x == 0) J.csum[c] = cnt;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(COMPACT_THREADS) k_cpi_scan(const CpiJob* __restrict__ jobs, int njobs,
                                                              uint32_t nchunks, int32_t* err) {
    using Scan = cub::BlockScan<uint64_t, COMPACT_THREADS>;
    using Reduce = cub::BlockReduce<uint64_t, COMPACT_THREADS>;
    __shared__ union {
        typename Scan::TempStorage scan;
        typename Reduce::TempStorage reduce;
    } tmp;
    __shared__ uint64_t base_s;
    constexpr int EPT = COMPACT_WORDS / COMPACT_THREADS;
    for (uint64_t it = blockIdx.x; it < (uint64_t)njobs * nchunks; it += gridDim.x) {
        const CpiJob& J = jobs[it / nchunks];
        const uint32_t c = (uint32_t)(it % nchunks);
        const uint32_t n = *J.pcount;
        const uint32_t last = n / COMPACT_WORDS;  // chunk holding off[n]
        if (c > last) continue;
        uint64_t before = 0;
        for (uint32_t q = threadIdx.x; q < c; q += COMPACT_THREADS) before += J.csum[q];
        before = Reduce(tmp.reduce).Sum(before);
        if (threadIdx.x == 0) base_s = before;
        __syncthreads();
        const uint32_t a0 = c * COMPACT_WORDS + threadIdx.x * EPT;
        uint32_t vals[EPT];
        uint64_t cnt = 0;
        for (int q = 0; q < EPT; q++) {
            vals[q] = a0 + q < n ? J.off[a0 + q] : 0u;
            cnt += vals[q];
        }
        uint64_t excl, total;
        Scan(tmp.scan).ExclusiveSum(cnt, excl, total);
        uint64_t r = base_s + excl;
        const bool overflow = base_s + total > J.cap || base_s + total > 0xffffffffull;
        for (int q = 0; q < EPT; q++) {
            if (a0 + q >= n) break;
            J.off[a0 + q] = overflow ? 0u : (uint32_t)r;
            r += vals[q];
        }
        if (c == last && threadIdx.x == 0) {
            uint64_t tot = base_s + total;
            if (overflow) {
                atomicExch(err, DERR_CAPACITY);
                tot = 0;  // leave an empty index
            }
            J.off[n] = (uint32_t)tot;
            if (J.nnz_stat) atomicAdd((unsigned long long*)J.nnz_stat, (unsigned long long)tot);
        }
        __syncthreads();
    }
}

template <bool COUNT>
__global__ void k_cpi_fill(DevGraph g, const CpiJob* __restrict__ jobs, int njobs, HubQueue hq) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    uint64_t sc = 0, se = 0;
    const uint32_t ngroups = hq.jpre[njobs];
    for (uint64_t it = gw; it < ngroups; it += nw) {
        // the warp's group of 32 candidates: job j, group grp of that job
        const int j = job_of(hq.jpre, njobs, (uint32_t)it);
        const uint64_t grp = it - hq.jpre[j];
        const CpiJob J = jobs[j];
        const uint32_t n = *J.pcount;
        const uint32_t* off = J.out ? g.out_off : g.in_off;
        const uint32_t* adj = J.out ? g.out_adj : g.in_adj;
        {
            const uint64_t a = grp * 32 + lane;
            uint32_t e0 = 0, e1 = 0, o = 0, oend = 0;
            if (a < n) {
                const uint32_t v = (uint32_t)J.pcand[a];
                o = J.off[a];
                oend = J.off[a + 1];
                if (oend > o) {  // a parent without index edges skips its list
                    e0 = off[v];
                    e1 = off[v + 1];
                }
            }
            if (hub_push(hq, e1 - e0 > HUB_LIST, ((unsigned long long)j << 40) | a, lane)) e1 = e0;
            const bool is_long = e1 - e0 > SHORT_LIST;
            sc += a < n && e1 > e0;
            se += e1 - e0;
            if (!is_long)
                for (uint32_t e = e0; e < e1; e += UNROLL) {
                    uint32_t p[UNROLL], w[UNROLL], rk[UNROLL];
                    load_group(adj, e, e1, p);
#pragma unroll
                    for (int t = 0; t < UNROLL; t++) {
                        const uint32_t x = p[t] >> g.lbits;
                        w[t] = e + t < e1 ? __ldg(J.cbm + (x >> 5)) : 0u;
                        rk[t] = e + t < e1 ? __ldg(J.crank + (x >> 5)) : 0u;
                    }
#pragma unroll
                    for (int t = 0; t < UNROLL; t++) {
                        const uint32_t x = p[t] >> g.lbits;
                        if (e + t < e1 && label_ok(J.lab, (int32_t)(p[t] & g.lmask)) && ((w[t] >> (x & 31)) & 1u)) {
                            if (o < oend && o < J.cap)
                                J.idx[o] = make_int2((int32_t)(rk[t] + __popc(w[t] & ((1u << (x & 31)) - 1))), (int32_t)x);
                            o++;
                        }
                    }
                }
            for (uint32_t lm = __ballot_sync(0xffffffffu, is_long); lm; lm &= lm - 1) {
                const int src = __ffs(lm) - 1;
                const uint32_t b0 = __shfl_sync(0xffffffffu, e0, src), b1 = __shfl_sync(0xffffffffu, e1, src);
                uint32_t w = __shfl_sync(0xffffffffu, o, src);
                const uint32_t wend = __shfl_sync(0xffffffffu, oend, src);
                for (uint32_t bb = b0; bb < b1; bb += 32) {
                    const uint32_t e = bb + lane;
                    bool hit = false;
                    uint32_t x = 0;
                    if (e < b1) {
                        const uint32_t p = adj[e];
                        x = p >> g.lbits;
                        hit = label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.cbm, x);
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                    if (hit) {
                        const uint32_t slot = w + __popc(bal & ((1u << lane) - 1));
                        if (slot < wend && slot < J.cap) {
                            const uint32_t word = J.cbm[x >> 5];
                            J.idx[slot] = make_int2((int32_t)(J.crank[x >> 5] + __popc(word & ((1u << (x & 31)) - 1))),
                                                    (int32_t)x);
                        }
                    }
                    w += __popc(bal);
                }
            }
        }
    }
    scan_flush<COUNT>(hq, sc, se);
}

// ---- hub lists, one block per queued (job, candidate[, constraint]) item

__global__ void __launch_bounds__(HUB_THREADS) k_scatter_hub(DevGraph g, const ScatterJob* __restrict__ jobs,
                                                            HubQueue hq) {
    const uint32_t nq = hub_count(hq);
    for (uint32_t t = blockIdx.x; t < nq; t += gridDim.x) {
        const unsigned long long it = hq.item[t];
        const ScatterJob& J = jobs[it >> 40];
        const uint32_t v = (uint32_t)J.qcand[(uint32_t)it];
        const uint32_t* off = J.scan_out ? g.out_off : g.in_off;
        const uint32_t* adj = J.scan_out ? g.out_adj : g.in_adj;
        const uint32_t e1 = off[v + 1];
        if (hq.scan && threadIdx.x == 0) {
            atomicAdd(&hq.scan[0], 1ull);
            atomicAdd(&hq.scan[1], (unsigned long long)(e1 - off[v]));
        }
        for (uint32_t e = off[v] + threadIdx.x; e < e1; e += HUB_THREADS) {
            const uint32_t p = __ldg(adj + e);
            const uint32_t x = p >> g.lbits;
            if (label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.filter, x))
                atomicOr(&J.marks[x >> 5], 1u << (x & 31));
        }
    }
}

// A queued prune constraint: the candidate stays only if some neighbour hits.
__global__ void __launch_bounds__(HUB_THREADS) k_prune_hub(DevGraph g, const PruneJob* __restrict__ jobs,
                                                          HubQueue hq) {
    const uint32_t nq = hub_count(hq);
    for (uint32_t t = blockIdx.x; t < nq; t += gridDim.x) {
        const unsigned long long it = hq.item[t];
        const PruneJob& J = jobs[it >> 40];
        const int c = (int)((it >> 32) & 0xff);
        const uint32_t v = (uint32_t)J.cand[(uint32_t)it];
        const uint32_t* off = J.con_dir[c] ? g.out_off : g.in_off;
        const uint32_t* adj = J.con_dir[c] ? g.out_adj : g.in_adj;
        const uint32_t e0 = off[v], e1 = off[v + 1];
        bool found = false;
        uint32_t read = 0;
        for (uint32_t b = e0; b < e1; b += HUB_THREADS) {  // block-uniform bounds
            const uint32_t e = b + threadIdx.x;
            bool hit = false;
            read += min((uint32_t)HUB_THREADS, e1 - b);
            if (e < e1) {
                const uint32_t p = __ldg(adj + e);
                hit = label_ok(J.con_lab[c], (int32_t)(p & g.lmask)) && bit_of(J.con_bm[c], p >> g.lbits);
            }
            if (__syncthreads_or(hit)) {
                found = true;
                break;
            }
        }
        if (hq.scan && threadIdx.x == 0) {
            atomicAdd(&hq.scan[0], 1ull);
            atomicAdd(&hq.scan[1], (unsigned long long)read);
        }
        if (!found && threadIdx.x == 0) atomicAnd(&J.bm[v >> 5], ~(1u << (v & 31)));
    }
}

__global__ void __launch_bounds__(HUB_THREADS) k_cpi_count_hub(DevGraph g, const CpiJob* __restrict__ jobs,
                                                              HubQueue hq) {
    using Reduce = cub::BlockReduce<uint32_t, HUB_THREADS>;
    __shared__ typename Reduce::TempStorage tmp;
    const uint32_t nq = hub_count(hq);
    for (uint32_t t = blockIdx.x; t < nq; t += gridDim.x) {
        const unsigned long long it = hq.item[t];
        const CpiJob& J = jobs[it >> 40];
        const uint32_t a = (uint32_t)it;
        const uint32_t v = (uint32_t)J.pcand[a];
        const uint32_t* off = J.out ? g.out_off : g.in_off;
        const uint32_t* adj = J.out ? g.out_adj : g.in_adj;
        const uint32_t e1 = off[v + 1];
        uint32_t cnt = 0;
        if (hq.scan && threadIdx.x == 0) {
            atomicAdd(&hq.scan[0], 1ull);
            atomicAdd(&hq.scan[1], (unsigned long long)(e1 - off[v]));
        }
        for (uint32_t e = off[v] + threadIdx.x; e < e1; e += HUB_THREADS) {
            const uint32_t p = __ldg(adj + e);
            cnt += label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.cbm, p >> g.lbits);
        }
        const uint32_t total = Reduce(tmp).Sum(cnt);
        if (threadIdx.x == 0) J.off[a] = total;
        __syncthreads();  // tmp is reused by the next item
    }
}

// Ordered fill of a hub's index edges: tiles of HUB_THREADS entries, a block
// scan gives each hit its slot after the hits of the earlier tiles.
__global__ void __launch_bounds__(HUB_THREADS) k_cpi_fill_hub(DevGraph g, const CpiJob* __restrict__ jobs,
                                                             HubQueue hq) {
    using Scan = cub::BlockScan<uint32_t, HUB_THREADS>;
    __shared__ typename Scan::TempStorage tmp;
    const uint32_t nq = hub_count(hq);
    for (uint32_t t = blockIdx.x; t < nq; t += gridDim.x) {
        const unsigned long long it = hq.item[t];
        const CpiJob& J = jobs[it >> 40];
        const uint32_t a = (uint32_t)it;
        const uint32_t v = (uint32_t)J.pcand[a];
        const uint32_t* off = J.out ? g.out_off : g.in_off;
        const uint32_t* adj = J.out ? g.out_adj : g.in_adj;
        const uint32_t e0 = off[v], e1 = off[v + 1];
        const uint32_t o = J.off[a], oend = J.off[a + 1];
        uint32_t running = 0;
        if (hq.scan && threadIdx.x == 0) {
            atomicAdd(&hq.scan[0], 1ull);
            atomicAdd(&hq.scan[1], (unsigned long long)(e1 - e0));
        }
        for (uint32_t b = e0; b < e1; b += HUB_THREADS) {  // block-uniform bounds
            const uint32_t e = b + threadIdx.x;
            bool hit = false;
            uint32_t x = 0, word = 0;
            if (e < e1) {
                const uint32_t p = __ldg(adj + e);
                x = p >> g.lbits;
                word = J.cbm[x >> 5];
                hit = label_ok(J.lab, (int32_t)(p & g.lmask)) && ((word >> (x & 31)) & 1u);
            }
            uint32_t excl, total;
            Scan(tmp).ExclusiveSum(hit ? 1u : 0u, excl, total);
            if (hit) {
                const uint64_t slot = (uint64_t)o + running + excl;
                if (slot < oend && slot < J.cap)
                    J.idx[slot] = make_int2((int32_t)(J.crank[x >> 5] + __popc(word & ((1u << (x & 31)) - 1))),
                                            (int32_t)x);
            }
            running += total;
            __syncthreads();  // tmp is reused by the next tile
        }
    }
}

// number of index edges of each job (read back to size the index exactly)
__global__ void k_cpi_totals(const CpiJob* __restrict__ jobs, int njobs, uint32_t* totals) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < njobs) totals[j] = jobs[j].off[*jobs[j].pcount];
}

// Blocks of a grid-stride kernel: as many as the device holds at once. A
// larger grid leaves a partial second wave, whose blocks start only as
// first-wave blocks exit and then run their share at a fraction of the
// occupancy. Cached per (kernel, device).
int resident_grid(const void* fn, int threads) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = device_sms();
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(fn, dev);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();  // the launch itself reports a kernel that cannot run
        per_sm = 1;
    }
    const int grid = sms * per_sm;
    cache.emplace(key, grid);
    return grid;
}

template <typename F>
int grid_of(F* fn, int threads) {
    return resident_grid((const void*)fn, threads);
}

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return GFD_OK;
}

}  // namespace

int launch_filter(const DevGraph& g, const FilterKey* d_keys, int nkeys, uint32_t* d_out, cudaStream_t st) {
    if (nkeys <= 0 || g.nwords == 0) return GFD_OK;
    int blocks = (int)std::min<uint64_t>((g.nwords * 32 + FILTER_THREADS - 1) / FILTER_THREADS, (uint64_t)device_sms() * 8);
    // keys staged in shared memory: at most KEYS_PER_LAUNCH per launch
    constexpr int KEYS_PER_LAUNCH = 4096;
    for (int k0 = 0; k0 < nkeys; k0 += KEYS_PER_LAUNCH) {
        const int cnt = std::min(KEYS_PER_LAUNCH, nkeys - k0);
        const size_t smem = sizeof(FilterKey) * cnt;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_filter)");
        }
        k_filter<<<std::max(blocks, 1), FILTER_THREADS, smem, st>>>(g, d_keys + k0, cnt,
                                                                    d_out + (uint64_t)k0 * g.nwords);
        if (int rc = check_launch("k_filter")) return rc;
    }
    return GFD_OK;
}

int launch_and(const DevGraph& g, const AndJob* d_jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0 || g.nwords == 0) return GFD_OK;
    const uint32_t nch = (g.nwords + AND_WORDS - 1) / AND_WORDS;
    const int grid = (int)std::min<uint64_t>((uint64_t)njobs * nch, (uint64_t)device_sms() * 16);
    k_and<<<grid, AND_THREADS, 0, st>>>(g, d_jobs, njobs, nch);
    return check_launch("k_and");
}

uint32_t compact_chunks(const DevGraph& g) {
    return std::max<uint32_t>(1, (g.nwords + COMPACT_WORDS - 1) / COMPACT_WORDS);
}

int launch_compact(const DevGraph& g, const CompactJob* d_jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    const uint32_t nch = compact_chunks(g);
    const int grid = (int)std::min<uint64_t>((uint64_t)njobs * nch, (uint64_t)device_sms() * 8);
    k_compact_sums<<<grid, COMPACT_THREADS, 0, st>>>(g, d_jobs, njobs, nch);
    k_compact_write<<<grid, COMPACT_THREADS, 0, st>>>(g, d_jobs, njobs, nch);
    return check_launch("k_compact");
}

static int hub_reset(const HubQueue& hq, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hq.n, 0, sizeof(uint32_t), st);
    return e == cudaSuccess ? GFD_OK : cuda_fail(e, "hub queue reset");
}

int launch_scatter(const DevGraph& g, const ScatterJob* d_jobs, int njobs, const HubQueue& hq, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    if (int rc = hub_reset(hq, st)) return rc;
    k_job_groups<ScatterJob><<<1, JOB_SCAN_THREADS, 0, st>>>(d_jobs, njobs, hq.jpre);
    if (hq.scan) k_scatter<true><<<grid_of(k_scatter<true>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    else k_scatter<false><<<grid_of(k_scatter<false>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    k_scatter_hub<<<grid_of(k_scatter_hub, HUB_THREADS), HUB_THREADS, 0, st>>>(g, d_jobs, hq);
    return check_launch("k_scatter");
}

int launch_prune(const DevGraph& g, const PruneJob* d_jobs, int njobs, const HubQueue& hq, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    if (int rc = hub_reset(hq, st)) return rc;
    k_job_groups<PruneJob><<<1, JOB_SCAN_THREADS, 0, st>>>(d_jobs, njobs, hq.jpre);
    if (hq.scan) k_prune<true><<<grid_of(k_prune<true>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    else k_prune<false><<<grid_of(k_prune<false>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    k_prune_hub<<<grid_of(k_prune_hub, HUB_THREADS), HUB_THREADS, 0, st>>>(g, d_jobs, hq);
    return check_launch("k_prune");
}

uint32_t cpi_chunks(uint64_t max_parent_candidates) {
    return (uint32_t)(max_parent_candidates / COMPACT_WORDS + 1);
}

int launch_cpi_count(const DevGraph& g, const CpiJob* d_jobs, int njobs, uint32_t nchunks, int32_t* d_err,
                     uint32_t* d_totals, const HubQueue& hq, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    if (int rc = hub_reset(hq, st)) return rc;
    k_job_groups<CpiJob><<<1, JOB_SCAN_THREADS, 0, st>>>(d_jobs, njobs, hq.jpre);
    if (hq.scan) k_cpi_count<true><<<grid_of(k_cpi_count<true>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    else k_cpi_count<false><<<grid_of(k_cpi_count<false>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    k_cpi_count_hub<<<grid_of(k_cpi_count_hub, HUB_THREADS), HUB_THREADS, 0, st>>>(g, d_jobs, hq);
    const int grid = (int)std::min<uint64_t>((uint64_t)njobs * nchunks, (uint64_t)device_sms() * 8);
    k_cpi_sums<<<grid, COMPACT_THREADS, 0, st>>>(d_jobs, njobs, nchunks);
    k_cpi_scan<<<grid, COMPACT_THREADS, 0, st>>>(d_jobs, njobs, nchunks, d_err);
    k_cpi_totals<<<(njobs + 255) / 256, 256, 0, st>>>(d_jobs, njobs, d_totals);
    return check_launch("k_cpi_count");
}

int launch_cpi_fill(const DevGraph& g, const CpiJob* d_jobs, int njobs, const HubQueue& hq, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    if (int rc = hub_reset(hq, st)) return rc;
    k_job_groups<CpiJob><<<1, JOB_SCAN_THREADS, 0, st>>>(d_jobs, njobs, hq.jpre);
    if (hq.scan) k_cpi_fill<true><<<grid_of(k_cpi_fill<true>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    else k_cpi_fill<false><<<grid_of(k_cpi_fill<false>, WARP_KERNEL_THREADS), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs, hq);
    k_cpi_fill_hub<<<grid_of(k_cpi_fill_hub, HUB_THREADS), HUB_THREADS, 0, st>>>(g, d_jobs, hq);
    return check_launch("k_cpi_fill");
}

}  // namespace gfd
