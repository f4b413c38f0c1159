// gfd_node_candidates_noalloc: the candidate filter of one pattern node
// (label, degree and self-loop test), computed without allocating any device
// memory. It is meant for callers that may not allocate: a server whose device
// memory is handed out by its own allocator or reserved up front under a fixed
// budget (a library cudaMalloc would bypass that accounting, or fail once the
// reservation holds the free memory), and latency-bound threads that cannot
// wait for cudaFree, which synchronises the whole device. The caller passes
// the graph handle (already resident), the GFD, and a device buffer for the
// output; the only temporary storage is the file-scope array below.
//
// The kernel is a single-pass, order-preserving stream compaction: blocks take
// tiles of TILE consecutive vertices in order from an atomic counter, count the
// vertices that pass, and chain the tile totals with a decoupled look-back over
// per-tile descriptors. Those descriptors, the tile counter, an error word and
// the total are the scratch memory: NA_MAX_TILES tiles of 8192 vertices, so at
// most 2^26 vertices (64 KiB of descriptors plus 64 bytes of counters). Every
// GPU that loads the library keeps this array until the process exits.
#include <cub/cub.cuh>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "engine.h"

namespace gfd {

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_TILE = NA_THREADS * 32;          // vertices per tile
constexpr int NA_MAX_TILES = 8192;                // => at most 2^26 vertices
constexpr int NA_HEADER = 8;                      // counter words before the descriptors
constexpr uint64_t NA_FLAG_AGG = 1ull << 62;      // tile total published
constexpr uint64_t NA_FLAG_PREFIX = 1ull << 63;   // inclusive prefix published
constexpr uint64_t NA_VALUE = (1ull << 62) - 1;

// [0] tile counter, [1] error (1 = a look-back wait gave up), [2] total count,
// [NA_HEADER + t] descriptor of tile t. Zeroed by every call before its launch.
static __device__ __align__(256) unsigned long long g_na_scratch[NA_HEADER + NA_MAX_TILES];

std::mutex g_na_mu;
void* g_na_ptr[64] = {};  // device address of g_na_scratch, per device
int g_na_sms[64] = {};    // multiprocessor count, per device

__global__ void __launch_bounds__(NA_THREADS)
k_node_candidates(DevGraph g, FilterKey key, unsigned long long* scratch, int32_t* out, uint64_t cap,
                  uint32_t ntiles) {
    using Scan = cub::BlockScan<uint32_t, NA_THREADS>;
    __shared__ typename Scan::TempStorage tmp;
    __shared__ uint32_t tile_s;
    __shared__ uint64_t base_s;
    volatile unsigned long long* desc = scratch + NA_HEADER;
    for (;;) {
        if (threadIdx.x == 0) tile_s = (uint32_t)atomicAdd(&scratch[0], 1ull);
        __syncthreads();
        const uint32_t t = tile_s;
        if (t >= ntiles) return;
        // 32 consecutive vertices per thread
        const uint32_t v0 = t * NA_TILE + threadIdx.x * 32;
        uint32_t mask = 0;
        for (int b = 0; b < 32; b++) {
            const uint32_t v = v0 + b;
            if (v >= (uint32_t)g.n) break;
            const uint32_t vi = g.vinfo[v];
            const bool has_self = (vi >> 16) != 0;
            const int32_t self_lab = (int32_t)(vi >> 16) - 1;
            const uint32_t dout = g.out_off[v + 1] - g.out_off[v] - has_self;
            const uint32_t din = g.in_off[v + 1] - g.in_off[v] - has_self;
            const bool self_ok = key.self_exp == EXP_NONE ? !has_self
                               : key.self_exp == EXP_ANY  ? has_self
                                                          : (has_self && self_lab == key.self_exp);
            if (label_ok(key.label, (int32_t)(vi & 0xffffu)) && dout >= key.dout_min &&
                din >= key.din_min && self_ok)
                mask |= 1u << b;
        }
        uint32_t excl, total;
        Scan(tmp).ExclusiveSum((uint32_t)__popc(mask), excl, total);
        if (threadIdx.x == 0) {
            uint64_t prefix = 0;
            if (t == 0) {
                desc[0] = NA_FLAG_PREFIX | total;
            } else {
                desc[t] = NA_FLAG_AGG | total;
                __threadfence();
                // look back until a tile with a published inclusive prefix
                int64_t j = (int64_t)t - 1;
                uint64_t spins = 0;
                while (j >= 0) {
                    const uint64_t d = desc[j];
                    if (d & NA_FLAG_PREFIX) {
                        prefix += d & NA_VALUE;
                        break;
                    }
                    if (d & NA_FLAG_AGG) {
                        prefix += d & NA_VALUE;
                        j--;
                        continue;
                    }
                    if (++spins > (1ull << 22)) {  // bounded wait: give up, report
                        atomicExch(&scratch[1], 1ull);
                        break;
                    }
                    __nanosleep(32);
                }
                __threadfence();
                desc[t] = NA_FLAG_PREFIX | (prefix + total);
            }
            if (t == ntiles - 1) scratch[2] = prefix + total;
            base_s = prefix;
        }
        __syncthreads();
        uint64_t o = base_s + excl;
        uint32_t m = mask;
        while (m) {
            const int b = __ffs(m) - 1;
            if (o < cap) out[o] = (int32_t)(v0 + b);
            o++;
            m &= m - 1;
        }
        __syncthreads();
    }
}

// Device address of the scratch array on the current device and the device's
// multiprocessor count, looked up once per device (the host-side symbol is only
// a stand-in for the array and must never be handed to a kernel).
int scratch_ptr(unsigned long long** out, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error(GFD_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
        return GFD_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        int n_sm = 0;
        e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(multiprocessors)");
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_na_sms[dev] = n_sm > 0 ? n_sm : 1;
        g_na_ptr[dev] = p;
    }
    *out = (unsigned long long*)g_na_ptr[dev];
    *sms = g_na_sms[dev];
    return GFD_OK;
}

}  // namespace

int node_candidates_noalloc(const gfd_graph* g, const gfd_gfd* phi, int32_t node, int32_t* d_out,
                            int64_t out_cap, int64_t* n_out, void* cuda_stream) {
    if (!g || !phi || !n_out || out_cap < 0 || (out_cap > 0 && !d_out)) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_node_candidates_noalloc: NULL argument or negative capacity");
        return GFD_ERR_INVALID_ARG;
    }
    if (node < 0 || node >= phi->k) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_node_candidates_noalloc: node %d outside the pattern", node);
        return GFD_ERR_INVALID_ARG;
    }
    const uint64_t ntiles = ((uint64_t)g->n + NA_TILE - 1) / NA_TILE;
    if (ntiles > (uint64_t)NA_MAX_TILES) {
        set_error(GFD_ERR_UNSUPPORTED,
                  "gfd_node_candidates_noalloc: %d vertices exceed the fixed scratch limit of %llu", g->n,
                  (unsigned long long)NA_MAX_TILES * NA_TILE);
        return GFD_ERR_UNSUPPORTED;
    }
    HostPlan plan;  // host memory only
    if (int rc = make_plan(phi, g->n_attrs, g->plan_stats(), &plan)) return rc;
    const FilterKey key = plan.key[plan.level_of[node]];
    unsigned long long* scratch = nullptr;
    int sms = 1;
    if (int rc = scratch_ptr(&scratch, &sms)) return rc;
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : g->stream;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (NA_HEADER + ntiles), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
    if (ntiles > 0) {
        // four resident blocks per multiprocessor take the tiles in order
        const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)sms * 4);
        k_node_candidates<<<grid, NA_THREADS, 0, st>>>(g->dg, key, scratch, d_out, (uint64_t)out_cap,
                                                       (uint32_t)ntiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_node_candidates");
    }
    unsigned long long hdr[3] = {0, 0, 0};
    e = cudaMemcpyAsync(hdr, scratch, sizeof(hdr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "gfd_node_candidates_noalloc readback");
    if (hdr[1]) {
        set_error(GFD_ERR_TIMEOUT, "gfd_node_candidates_noalloc: a look-back wait gave up");
        return GFD_ERR_TIMEOUT;
    }
    *n_out = (int64_t)hdr[2];
    if ((int64_t)hdr[2] > out_cap) {
        set_error(GFD_ERR_OVERFLOW, "gfd_node_candidates_noalloc: %llu candidates, output holds %lld",
                  (unsigned long long)hdr[2], (long long)out_cap);
        return GFD_ERR_OVERFLOW;
    }
    return GFD_OK;
}

}  // namespace gfd

extern "C" int gfd_node_candidates_noalloc(const gfd_graph* g, const gfd_gfd* phi, int32_t node, int32_t* d_out,
                                           int64_t out_cap, int64_t* n_out, void* cuda_stream) {
    return gfd::node_candidates_noalloc(g, phi, node, d_out, out_cap, n_out, cuda_stream);
}
