// gfd_graph_load / gfd_graph_free: make G = (V, E, L, F_A) (Section II)
// resident on the device.
//
// The caller's int64/int32 CSR is copied once, checked on the device (rows
// strictly increasing, ids in range, labels in range, reverse CSR equal to the
// transpose of the forward one) and packed into the layout of common.cuh.
#include <cub/cub.cuh>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace gfd {

namespace {

// error bits written by the validation kernels
enum : uint32_t {
    BAD_OFFSETS = 1u,
    BAD_ORDER = 2u,
    BAD_RANGE = 4u,
    BAD_LABEL = 8u,
    BAD_REVERSE = 16u,
};

__global__ void k_check_offsets(const int64_t* off, int32_t n, int64_t m, uint32_t* bad) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = off[v];
        bool ok = o >= 0 && o <= m;
        if (v == 0) ok = ok && o == 0;
        if (v == n) ok = ok && o == m;
        if (v > 0) ok = ok && off[v - 1] <= o;
        if (!ok) atomicOr(bad, BAD_OFFSETS);
    }
}

// One warp per row: check order / range / label and pack (nbr << lbits) | label.
__global__ void k_pack_rows(const int64_t* off, const int32_t* nbr, const int32_t* lab, int32_t n,
                            int32_t lbits, uint32_t* off32, uint32_t* adj, uint32_t* bad) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int64_t a = off[v], b = off[v + 1];
        if (lane == 0) off32[v] = (uint32_t)a;
        uint32_t err = 0;
        for (int64_t e = a + lane; e < b; e += 32) {
            int32_t x = nbr[e];
            int32_t l = lab[e];
            if (x < 0 || x >= n) err |= BAD_RANGE;
            if (l < 0 || l > 255 || (l >> lbits) != 0) err |= BAD_LABEL;
            if (e > a && nbr[e - 1] >= x) err |= BAD_ORDER;
            adj[e] = ((uint32_t)x << lbits) | (uint32_t)(l & 255);
        }
        err = __reduce_or_sync(0xffffffffu, err);
        if (lane == 0 && err) atomicOr(bad, err);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off32[n] = (uint32_t)off[n];
}

__global__ void k_vinfo(const int32_t* vlabel, const uint32_t* out_off, const uint32_t* out_adj,
                        int32_t n, int32_t lbits, uint32_t lmask, uint32_t* vinfo, uint32_t* bad) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t L = vlabel[v];
        if (L < 0 || L > 65534) atomicOr(bad, BAD_LABEL);
        uint32_t lo = out_off[v], hi = out_off[v + 1];
        const uint32_t key = (uint32_t)v << lbits;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (out_adj[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        uint32_t self = 0;
        if (lo < out_off[v + 1] && (out_adj[lo] >> lbits) == (uint32_t)v) self = (out_adj[lo] & lmask) + 1;
        vinfo[v] = ((uint32_t)L & 0xffffu) | (self << 16);
    }
}

// One warp per vertex: OR of the signature bits of its out-neighbours (half 0)
// or in-neighbours (half 1).
__global__ void k_signature(const uint32_t* off, const uint32_t* adj, int32_t n, int32_t lbits, int half,
                            unsigned long long* sig) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        unsigned long long b = 0;
        for (uint32_t e = off[v] + lane; e < off[v + 1]; e += 32) b |= 1ull << sig_bit(adj[e] >> lbits);
        const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)b);
        const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(b >> 32));
        if (lane == 0) sig[2 * v + half] = ((unsigned long long)hi << 32) | lo;
    }
}

// keys[e] = (dst << 32) | src over the forward CSR, labels alongside.
__global__ void k_transpose_keys(const uint32_t* off, const uint32_t* adj, int32_t n, int32_t lbits,
                                 uint32_t lmask, uint64_t* keys, uint8_t* labs) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        for (uint32_t e = off[v] + lane; e < off[v + 1]; e += 32) {
            uint32_t p = adj[e];
            keys[e] = ((uint64_t)(p >> lbits) << 32) | (uint64_t)v;
            labs[e] = (uint8_t)(p & lmask);
        }
    }
}

__global__ void k_in_degree(const uint64_t* keys, int64_t m, uint32_t* deg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[keys[e] >> 32], 1u);
}

__global__ void k_pack_in(const uint64_t* keys, const uint8_t* labs, int64_t m, int32_t lbits,
                          uint32_t* in_adj) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        in_adj[e] = ((uint32_t)(keys[e] & 0xffffffffu) << lbits) | labs[e];
}

__global__ void k_compare(const uint32_t* a, const uint32_t* b, int64_t n, uint32_t* bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        if (a[e] != b[e]) atomicOr(bad, BAD_REVERSE);
}

// per vertex label: count, out-degree sum, in-degree sum
__global__ void k_label_stats(const uint32_t* vinfo, const uint32_t* out_off, const uint32_t* in_off,
                              int32_t n, unsigned long long* stats /* [65536][3] */) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t L = vinfo[v] & 0xffffu;
        atomicAdd(&stats[3 * L + 0], 1ull);
        atomicAdd(&stats[3 * L + 1], (unsigned long long)(out_off[v + 1] - out_off[v]));
        atomicAdd(&stats[3 * L + 2], (unsigned long long)(in_off[v + 1] - in_off[v]));
    }
}

template <typename T>
int dev_alloc(T** p, size_t count, int64_t* bytes) {
    size_t b = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(GFD_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed: %s", b,
                  cudaGetErrorString(e));
        return GFD_ERR_OUT_OF_MEMORY;
    }
    if (bytes) *bytes += (int64_t)b;
    return GFD_OK;
}

struct TmpFree {
    std::vector<void*> ptrs;
    ~TmpFree() {
        for (void* p : ptrs) cudaFree(p);
    }
};

int grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)device_sms() * 16));
}

std::string bad_text(uint32_t bad) {
    std::string s;
    if (bad & BAD_OFFSETS) s += " offsets not a valid CSR;";
    if (bad & BAD_ORDER) s += " adjacency row not strictly increasing (repeated or unsorted edge);";
    if (bad & BAD_RANGE) s += " vertex id out of range;";
    if (bad & BAD_LABEL) s += " label out of range;";
    if (bad & BAD_REVERSE) s += " reverse CSR differs from the transpose of the forward CSR;";
    return s;
}

}  // namespace

int device_sms() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 1;  // not cached: a later call may succeed
    }
    cache.emplace(dev, sms);
    return sms;
}

int graph_load(const gfd_graph_desc* d, const gfd_opts* o, gfd_graph** out) {
    if (!d || !out) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_graph_load: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    const int32_t n = d->n_vertices;
    const int64_t m = d->n_edges;
    if (n < 0 || m < 0 || d->n_attrs < 0 || !d->out_off || (m > 0 && (!d->out_dst || !d->out_elabel)) ||
        (n > 0 && !d->vlabel) || (d->n_attrs > 0 && n > 0 && !d->attrs)) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_graph_load: negative size or missing array");
        return GFD_ERR_INVALID_ARG;
    }
    const bool have_in = d->in_off || d->in_src || d->in_elabel;
    if (have_in && (!d->in_off || (m > 0 && (!d->in_src || !d->in_elabel)))) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_graph_load: reverse CSR given only in part");
        return GFD_ERR_INVALID_ARG;
    }
    if (m >= (int64_t)UINT32_MAX) {
        set_error(GFD_ERR_UNSUPPORTED, "gfd_graph_load: %lld edges, limit is 2^32-1", (long long)m);
        return GFD_ERR_UNSUPPORTED;
    }
    // edge-label bit width from the largest label (checked again on the device)
    int32_t maxlab = 0;
    for (int64_t e = 0; e < m; e++) maxlab = std::max(maxlab, d->out_elabel[e]);
    if (maxlab > 255) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_graph_load: edge label %d > 255", maxlab);
        return GFD_ERR_INVALID_ARG;
    }
    int32_t lbits = 1;
    while ((1 << lbits) <= maxlab) lbits++;
    if ((int64_t)n > (1ll << (32 - lbits))) {
        set_error(GFD_ERR_UNSUPPORTED, "gfd_graph_load: %d vertices with %d-bit edge labels exceed 2^%d",
                  n, lbits, 32 - lbits);
        return GFD_ERR_UNSUPPORTED;
    }

    cudaStream_t st = o && o->cuda_stream ? (cudaStream_t)o->cuda_stream : nullptr;
    gfd_graph* g = new gfd_graph();
    g->n = n;
    g->m = m;
    g->n_attrs = d->n_attrs;
    g->lbits = lbits;
    auto fail = [&](int code) {
        graph_free(g);
        return code;
    };
    cudaError_t ce = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return fail(cuda_fail(ce, "cudaStreamCreate"));
    if (!st) st = g->stream;

    int rc;
    uint32_t *out_off, *in_off, *out_adj, *in_adj, *vinfo;
    int32_t* attrs;
    if ((rc = dev_alloc(&out_off, (size_t)n + 1, &g->bytes)) ||
        (rc = dev_alloc(&in_off, (size_t)n + 1, &g->bytes)) ||
        (rc = dev_alloc(&out_adj, (size_t)m, &g->bytes)) ||
        (rc = dev_alloc(&in_adj, (size_t)m, &g->bytes)) ||
        (rc = dev_alloc(&vinfo, (size_t)n, &g->bytes)) ||
        (rc = dev_alloc(&attrs, (size_t)n * std::max(1, d->n_attrs), &g->bytes))) {
        return fail(rc);
    }
    unsigned long long* sig;
    if ((rc = dev_alloc(&sig, 2 * (size_t)std::max(1, n), &g->bytes))) return fail(rc);
    g->allocs = {out_off, in_off, out_adj, in_adj, vinfo, attrs, sig};

    TmpFree tmp;
    int64_t* d_off;
    int32_t *d_nbr, *d_lab, *d_vl;
    uint32_t* d_bad;
    if ((rc = dev_alloc(&d_off, (size_t)n + 1, nullptr)) || (rc = dev_alloc(&d_nbr, (size_t)m, nullptr)) ||
        (rc = dev_alloc(&d_lab, (size_t)m, nullptr)) || (rc = dev_alloc(&d_vl, (size_t)n, nullptr)) ||
        (rc = dev_alloc(&d_bad, 1, nullptr)))
        return fail(rc);
    tmp.ptrs = {d_off, d_nbr, d_lab, d_vl, d_bad};
#define CK(call)                                         \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return fail(cuda_fail(_e, #call)); \
    } while (0)
    CK(cudaMemsetAsync(d_bad, 0, sizeof(uint32_t), st));
    CK(cudaMemcpyAsync(d_off, d->out_off, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, st));
    if (m) {
        CK(cudaMemcpyAsync(d_nbr, d->out_dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_lab, d->out_elabel, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    }
    if (n) CK(cudaMemcpyAsync(d_vl, d->vlabel, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    if (n && d->n_attrs)
        CK(cudaMemcpyAsync(attrs, d->attrs, sizeof(int32_t) * (size_t)n * d->n_attrs, cudaMemcpyHostToDevice, st));
    const uint32_t lmask = (1u << lbits) - 1;
    k_check_offsets<<<grid_for(n + 1), 256, 0, st>>>(d_off, n, m, d_bad);
    uint32_t bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_graph_load: forward CSR:%s", bad_text(bad).c_str());
        return fail(GFD_ERR_INVALID_ARG);
    }
    k_pack_rows<<<grid_for((int64_t)n * 32), 256, 0, st>>>(d_off, d_nbr, d_lab, n, lbits, out_off, out_adj, d_bad);
    k_vinfo<<<grid_for(n), 256, 0, st>>>(d_vl, out_off, out_adj, n, lbits, lmask, vinfo, d_bad);
    CK(cudaGetLastError());
    // the kernels below index arrays by neighbour id: stop here on a bad row
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_graph_load: forward CSR:%s", bad_text(bad).c_str());
        return fail(GFD_ERR_INVALID_ARG);
    }

    // reverse CSR: stable radix sort of (dst, src) keys
    {
        uint64_t *k0, *k1;
        uint8_t *l0, *l1;
        uint32_t* deg;
        if ((rc = dev_alloc(&k0, (size_t)m, nullptr)) || (rc = dev_alloc(&k1, (size_t)m, nullptr)) ||
            (rc = dev_alloc(&l0, (size_t)m, nullptr)) || (rc = dev_alloc(&l1, (size_t)m, nullptr)) ||
            (rc = dev_alloc(&deg, (size_t)n + 1, nullptr)))
            return fail(rc);
        tmp.ptrs.insert(tmp.ptrs.end(), {k0, k1, l0, l1, deg});
        k_transpose_keys<<<grid_for((int64_t)n * 32), 256, 0, st>>>(out_off, out_adj, n, lbits, lmask, k0, l0);
        cub::DoubleBuffer<uint64_t> kb(k0, k1);
        cub::DoubleBuffer<uint8_t> lb(l0, l1);
        int endbit = 32;
        while ((1ll << (endbit - 32)) < (int64_t)n + 1 && endbit < 64) endbit++;
        size_t tb = 0;
        CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, kb, lb, (int64_t)m, 0, endbit, st));
        void* tstore;
        if ((rc = dev_alloc((uint8_t**)&tstore, tb, nullptr))) return fail(rc);
        tmp.ptrs.push_back(tstore);
        CK(cub::DeviceRadixSort::SortPairs(tstore, tb, kb, lb, (int64_t)m, 0, endbit, st));
        CK(cudaMemsetAsync(deg, 0, sizeof(uint32_t) * ((size_t)n + 1), st));
        k_in_degree<<<grid_for(m), 256, 0, st>>>(kb.Current(), m, deg);
        size_t sb = 0;
        CK(cub::DeviceScan::ExclusiveSum(nullptr, sb, deg, in_off, n + 1, st));
        void* sstore;
        if ((rc = dev_alloc((uint8_t**)&sstore, sb, nullptr))) return fail(rc);
        tmp.ptrs.push_back(sstore);
        CK(cub::DeviceScan::ExclusiveSum(sstore, sb, deg, in_off, n + 1, st));
        k_pack_in<<<grid_for(m), 256, 0, st>>>(kb.Current(), lb.Current(), m, lbits, in_adj);
        k_signature<<<grid_for((int64_t)n * 32), 256, 0, st>>>(out_off, out_adj, n, lbits, 0, sig);
        k_signature<<<grid_for((int64_t)n * 32), 256, 0, st>>>(in_off, in_adj, n, lbits, 1, sig);
        CK(cudaGetLastError());
        if (have_in) {
            // the caller's reverse CSR must be exactly the transpose
            uint32_t *uoff, *uadj;
            if ((rc = dev_alloc(&uoff, (size_t)n + 1, nullptr)) || (rc = dev_alloc(&uadj, (size_t)m, nullptr)))
                return fail(rc);
            tmp.ptrs.insert(tmp.ptrs.end(), {uoff, uadj});
            CK(cudaMemcpyAsync(d_off, d->in_off, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, st));
            if (m) {
                CK(cudaMemcpyAsync(d_nbr, d->in_src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
                CK(cudaMemcpyAsync(d_lab, d->in_elabel, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
            }
            k_check_offsets<<<grid_for(n + 1), 256, 0, st>>>(d_off, n, m, d_bad);
            k_pack_rows<<<grid_for((int64_t)n * 32), 256, 0, st>>>(d_off, d_nbr, d_lab, n, lbits, uoff, uadj, d_bad);
            k_compare<<<grid_for(n + 1), 256, 0, st>>>(uoff, in_off, n + 1, d_bad);
            k_compare<<<grid_for(m), 256, 0, st>>>(uadj, in_adj, m, d_bad);
            CK(cudaGetLastError());
        }
    }
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    // label statistics for planning and capacity bounds
    {
        unsigned long long* dstats;
        if ((rc = dev_alloc(&dstats, 65536 * 3, nullptr))) return fail(rc);
        tmp.ptrs.push_back(dstats);
        CK(cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * 65536 * 3, st));
        k_label_stats<<<grid_for(n), 256, 0, st>>>(vinfo, out_off, in_off, n, dstats);
        g->label_stats.assign(65536 * 3, 0);
        CK(cudaMemcpyAsync(g->label_stats.data(), dstats, sizeof(unsigned long long) * 65536 * 3,
                           cudaMemcpyDeviceToHost, st));
    }
    std::vector<uint32_t> h_in_off((size_t)n + 1);
    CK(cudaMemcpyAsync(h_in_off.data(), in_off, sizeof(uint32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_graph_load:%s", bad_text(bad).c_str());
        return fail(GFD_ERR_INVALID_ARG);
    }
#undef CK
    // degree moments per vertex label and edge-label frequencies for planning
    g->moments.assign((size_t)65536 * 16, 0.0);
    g->moments_all.assign(16, 0.0);
    for (int32_t v = 0; v < n; v++) {
        const double dout = (double)(d->out_off[v + 1] - d->out_off[v]);
        const double din = (double)(h_in_off[v + 1] - h_in_off[v]);
        double* M = &g->moments[16 * (size_t)(d->vlabel[v] & 0xffff)];
        double pa = 1.0;
        for (int a = 0; a < 4; a++) {
            double pb = pa;
            for (int b = 0; b < 4; b++) {
                M[4 * a + b] += pb;
                pb *= din;
            }
            pa *= dout;
        }
    }
    for (size_t L = 0; L < 65536; L++)
        if (g->label_stats[3 * L])
            for (int c = 0; c < 16; c++) g->moments_all[c] += g->moments[16 * L + c];
    g->elabel_frac.assign(256, 0.0);
    for (int64_t e = 0; e < m; e++) g->elabel_frac[d->out_elabel[e] & 255] += 1.0;
    for (auto& f : g->elabel_frac) f /= (double)std::max<int64_t>(1, m);
    DevGraph& dg = g->dg;
    dg.n = n;
    dg.n_attrs = d->n_attrs;
    dg.lbits = lbits;
    dg.lmask = lmask;
    dg.m = m;
    dg.nwords = (uint32_t)(((int64_t)n + 31) / 32);
    dg.out_off = out_off;
    dg.in_off = in_off;
    dg.out_adj = out_adj;
    dg.in_adj = in_adj;
    dg.vinfo = vinfo;
    dg.attrs = attrs;
    dg.sig = (const ulonglong2*)sig;
    *out = g;
    return GFD_OK;
}

void graph_free(gfd_graph* g) {
    if (!g) return;
    if (g->eng) engine_free(g->eng);
    for (void* p : g->allocs) cudaFree(p);
    if (g->stream) cudaStreamDestroy(g->stream);
    cudaGetLastError();  // a failure here must not surface in a later, unrelated call
    delete g;
}

}  // namespace gfd
