// Compact path index construction (Section III.B, step 1).
//
//   k_filter   step 1a-1b: candidates by label and degree (and self-loop),
//              one coalesced pass over vertex data for all filter keys;
//   k_scatter  step 1c, top-down: mark vertices adjacent (in the direction and
//   k_and      with the label of a pattern edge) to the candidates of an
//              earlier level, then intersect;
//   k_prune    step 1c, bottom-up: remove dead ends, i.e. candidates with no
//              neighbour among the candidates of a later level;
//   k_compact  bitmap -> exclusive popcount prefix (O(1) rank) + sorted list;
//   k_cpi_*    step 1d: for each spanning-tree edge, the index edges from
//              every parent candidate to the positions of its child candidates.
//
// Every launch processes a table of jobs; blocks (or warps) stride over the
// items of each job with a per-job rotation so that small jobs spread out.
#include <cub/cub.cuh>

#include "engine.h"

namespace gfd {

namespace {

constexpr int FILTER_THREADS = 256;
constexpr int COMPACT_THREADS = 1024;
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
            const FilterKey key = sk[k];
            bool self_ok = key.self_exp == EXP_NONE ? !has_self
                         : key.self_exp == EXP_ANY  ? has_self
                                                    : (has_self && self_lab == key.self_exp);
            bool p = valid && label_ok(key.label, L) && dout >= key.dout_min && din >= key.din_min && self_ok;
            uint32_t b = __ballot_sync(0xffffffffu, p);
            if (lane == 0) out[(uint64_t)k * g.nwords + w] = b;
        }
    }
}

__global__ void k_and(DevGraph g, const AndJob* __restrict__ jobs, int njobs) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (int j = 0; j < njobs; j++) {
        const AndJob J = jobs[j];
        for (uint64_t w = (tid + (uint64_t)j * 7919) % nt; w < g.nwords; w += nt) {
            uint32_t x = J.src[w];
            for (int t = 0; t < J.ntmp; t++) x &= J.tmp[t][w];
            J.bm[w] = x;
        }
    }
}

// One block per job: rank[w] = number of set bits before word w; cand = the
// set bits in increasing order; *count = total.
__global__ void __launch_bounds__(COMPACT_THREADS) k_compact(DevGraph g, const CompactJob* __restrict__ jobs, int njobs) {
    using Scan = cub::BlockScan<uint32_t, COMPACT_THREADS>;
    __shared__ typename Scan::TempStorage tmp;
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
        const CompactJob J = jobs[j];
        uint32_t carry = 0;
        for (uint32_t base = 0; base < g.nwords; base += COMPACT_THREADS) {
            const uint32_t w = base + threadIdx.x;
            const uint32_t word = w < g.nwords ? J.bm[w] : 0u;
            uint32_t excl, total;
            Scan(tmp).ExclusiveSum((uint32_t)__popc(word), excl, total);
            if (w < g.nwords) {
                const uint32_t r = carry + excl;
                J.rank[w] = r;
                uint32_t x = word, o = r;
                while (x) {
                    const int b = __ffs(x) - 1;
                    J.cand[o++] = (int32_t)(w * 32 + b);
                    x &= x - 1;
                }
            }
            carry += total;
            __syncthreads();
        }
        if (threadIdx.x == 0) *J.count = carry;
        __syncthreads();
    }
}

__global__ void k_scatter(DevGraph g, const ScatterJob* __restrict__ jobs, int njobs) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    for (int j = 0; j < njobs; j++) {
        const ScatterJob J = jobs[j];
        const uint32_t n = *J.qcount;
        const uint32_t* off = J.scan_out ? g.out_off : g.in_off;
        const uint32_t* adj = J.scan_out ? g.out_adj : g.in_adj;
        for (uint64_t a = (gw + (uint64_t)j * 7919) % nw; a < n; a += nw) {
            const uint32_t v = (uint32_t)J.qcand[a];
            const uint32_t e1 = off[v + 1];
            for (uint32_t e = off[v] + lane; e < e1; e += 32) {
                const uint32_t p = adj[e];
                const uint32_t x = p >> g.lbits;
                if (label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.filter, x))
                    atomicOr(&J.marks[x >> 5], 1u << (x & 31));
            }
        }
    }
}

__global__ void k_prune(DevGraph g, const PruneJob* __restrict__ jobs, int njobs) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    for (int j = 0; j < njobs; j++) {
        const PruneJob& J = jobs[j];
        const uint32_t n = *J.count;
        const int ncon = J.ncon;
        for (uint64_t a = (gw + (uint64_t)j * 7919) % nw; a < n; a += nw) {
            const uint32_t v = (uint32_t)J.cand[a];
            bool keep = true;
            for (int c = 0; c < ncon && keep; c++) {
                const uint32_t* off = J.con_dir[c] ? g.out_off : g.in_off;
                const uint32_t* adj = J.con_dir[c] ? g.out_adj : g.in_adj;
                const uint32_t* bm = J.con_bm[c];
                const int32_t lab = J.con_lab[c];
                const uint32_t e1 = off[v + 1];
                bool found = false;
                for (uint32_t e0 = off[v]; e0 < e1 && !found; e0 += 32) {
                    const uint32_t e = e0 + lane;
                    bool hit = false;
                    if (e < e1) {
                        const uint32_t p = adj[e];
                        hit = label_ok(lab, (int32_t)(p & g.lmask)) && bit_of(bm, p >> g.lbits);
                    }
                    found = __any_sync(0xffffffffu, hit);
                }
                keep = found;
            }
            if (!keep && lane == 0) atomicAnd(&J.bm[v >> 5], ~(1u << (v & 31)));
        }
    }
}

// off[a] = number of children of parent candidate a
__global__ void k_cpi_count(DevGraph g, const CpiJob* __restrict__ jobs, int njobs) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    for (int j = 0; j < njobs; j++) {
        const CpiJob J = jobs[j];
        const uint32_t n = *J.pcount;
        const uint32_t* off = J.out ? g.out_off : g.in_off;
        const uint32_t* adj = J.out ? g.out_adj : g.in_adj;
        for (uint64_t a = (gw + (uint64_t)j * 7919) % nw; a < n; a += nw) {
            const uint32_t v = (uint32_t)J.pcand[a];
            const uint32_t e1 = off[v + 1];
            uint32_t cnt = 0;
            for (uint32_t e = off[v] + lane; e < e1; e += 32) {
                const uint32_t p = adj[e];
                cnt += label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.cbm, p >> g.lbits);
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0) J.off[a] = cnt;
        }
    }
}

// One block per job: exclusive scan of off[0..n), off[n] = total.
__global__ void __launch_bounds__(COMPACT_THREADS) k_cpi_scan(const CpiJob* __restrict__ jobs, int njobs, int32_t* err) {
    using Scan = cub::BlockScan<uint64_t, COMPACT_THREADS>;
    __shared__ typename Scan::TempStorage tmp;
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
        const CpiJob J = jobs[j];
        const uint32_t n = *J.pcount;
        uint64_t carry = 0;
        for (uint32_t base = 0; base < n; base += COMPACT_THREADS) {
            const uint32_t a = base + threadIdx.x;
            const uint64_t c = a < n ? J.off[a] : 0;
            uint64_t excl, total;
            Scan(tmp).ExclusiveSum(c, excl, total);
            if (a < n) J.off[a] = (uint32_t)(carry + excl);
            carry += total;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (carry > J.cap || carry > 0xffffffffull) {
                atomicExch(err, DERR_CAPACITY);
                carry = 0;  // leave an empty, consistent index
            }
            J.off[n] = (uint32_t)carry;
            if (J.nnz_stat) atomicAdd((unsigned long long*)J.nnz_stat, (unsigned long long)carry);
        }
        __syncthreads();
    }
}

__global__ void k_cpi_fill(DevGraph g, const CpiJob* __restrict__ jobs, int njobs) {
    const int lane = threadIdx.x & 31;
    const uint64_t gw = gwarp_id(), nw = nwarps_total();
    for (int j = 0; j < njobs; j++) {
        const CpiJob J = jobs[j];
        const uint32_t n = *J.pcount;
        const uint32_t* off = J.out ? g.out_off : g.in_off;
        const uint32_t* adj = J.out ? g.out_adj : g.in_adj;
        for (uint64_t a = (gw + (uint64_t)j * 7919) % nw; a < n; a += nw) {
            const uint32_t v = (uint32_t)J.pcand[a];
            const uint32_t e1 = off[v + 1];
            uint32_t o = J.off[a];
            const uint32_t oend = J.off[a + 1];
            for (uint32_t e0 = off[v]; e0 < e1; e0 += 32) {
                const uint32_t e = e0 + lane;
                bool hit = false;
                uint32_t x = 0;
                if (e < e1) {
                    const uint32_t p = adj[e];
                    x = p >> g.lbits;
                    hit = label_ok(J.lab, (int32_t)(p & g.lmask)) && bit_of(J.cbm, x);
                }
                const uint32_t b = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const uint32_t slot = o + __popc(b & ((1u << lane) - 1));
                    if (slot < oend && slot < J.cap) {
                        const uint32_t word = J.cbm[x >> 5];
                        J.idx[slot] = (int32_t)(J.crank[x >> 5] + __popc(word & ((1u << (x & 31)) - 1)));
                    }
                }
                o += __popc(b);
            }
        }
    }
}

int grid_warps(int sms_mult = 8) { return 152 * sms_mult; }

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return GFD_OK;
}

}  // namespace

int launch_filter(const DevGraph& g, const FilterKey* d_keys, int nkeys, uint32_t* d_out, cudaStream_t st) {
    if (nkeys <= 0 || g.nwords == 0) return GFD_OK;
    int blocks = (int)std::min<uint64_t>((g.nwords * 32 + FILTER_THREADS - 1) / FILTER_THREADS, 152 * 8);
    size_t smem = sizeof(FilterKey) * nkeys;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    k_filter<<<std::max(blocks, 1), FILTER_THREADS, smem, st>>>(g, d_keys, nkeys, d_out);
    return check_launch("k_filter");
}

int launch_and(const DevGraph& g, const AndJob* d_jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    k_and<<<grid_warps(4), 256, 0, st>>>(g, d_jobs, njobs);
    return check_launch("k_and");
}

int launch_compact(const DevGraph& g, const CompactJob* d_jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    k_compact<<<std::min(njobs, 152 * 2), COMPACT_THREADS, 0, st>>>(g, d_jobs, njobs);
    return check_launch("k_compact");
}

int launch_scatter(const DevGraph& g, const ScatterJob* d_jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    k_scatter<<<grid_warps(), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs);
    return check_launch("k_scatter");
}

int launch_prune(const DevGraph& g, const PruneJob* d_jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    k_prune<<<grid_warps(), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs);
    return check_launch("k_prune");
}

int launch_cpi(const DevGraph& g, const CpiJob* d_jobs, int njobs, int32_t* d_err, cudaStream_t st) {
    if (njobs <= 0) return GFD_OK;
    k_cpi_count<<<grid_warps(), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs);
    k_cpi_scan<<<std::min(njobs, 152 * 2), COMPACT_THREADS, 0, st>>>(d_jobs, njobs, d_err);
    k_cpi_fill<<<grid_warps(), WARP_KERNEL_THREADS, 0, st>>>(g, d_jobs, njobs);
    return check_launch("k_cpi");
}

}  // namespace gfd
