// Orchestration of one validation run over a batch of GFD slots.
//
// Host: plan every GFD (plan.cpp), deduplicate candidate-filter keys across
// GFDs (the shared candidate cache), derive every buffer's capacity from the
// graph's per-label statistics, lay all device buffers out in one stream-
// ordered allocation and upload all descriptors and job tables in one copy.
// Device: one filter pass for all keys, the refinement and index phases (each
// launch covers every GFD), then the enumeration driver. Nothing waits on the
// host between phases; the host reads back the counters once at the end.
#include <cub/cub.cuh>

#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "engine.h"

namespace gfd {

struct Engine {
    cudaMemPool_t pool = nullptr;
};

void engine_free(Engine* e) {
    if (!e) return;
    if (e->pool) cudaMemPoolDestroy(e->pool);
    delete e;
}

namespace {

constexpr int PROF_FILTER = 0, PROF_REFINE = 1, PROF_INDEX = 2, PROF_ENUM = 3;

struct Layout {
    size_t size = 256;  // offset 0 is reserved so that no buffer is at a null offset
    size_t take(size_t bytes) {
        size_t off = size;
        size = (size + bytes + 255) & ~(size_t)255;
        return off;
    }
};

int get_pool(gfd_graph* g, cudaMemPool_t* out) {
    if (!g->eng) g->eng = new Engine();
    if (!g->eng->pool) {
        int dev = 0;
        GFD_CUDA(cudaGetDevice(&dev));
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        GFD_CUDA(cudaMemPoolCreate(&g->eng->pool, &props));
        uint64_t thr = UINT64_MAX;
        GFD_CUDA(cudaMemPoolSetAttribute(g->eng->pool, cudaMemPoolAttrReleaseThreshold, &thr));
    }
    *out = g->eng->pool;
    return GFD_OK;
}

uint64_t env_u64(const char* name, uint64_t dflt) {
    const char* s = getenv(name);
    if (!s || !*s) return dflt;
    return strtoull(s, nullptr, 10);
}

struct ProfEvents {
    bool on = false;
    cudaEvent_t ev[2 * 5] = {};
    ~ProfEvents() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
    int init(bool enable) {
        on = enable;
        if (!on) return GFD_OK;
        for (auto& e : ev) GFD_CUDA(cudaEventCreate(&e));
        return GFD_OK;
    }
    void begin(int w, cudaStream_t st) {
        if (on) cudaEventRecord(ev[2 * w], st);
    }
    void end(int w, cudaStream_t st) {
        if (on) cudaEventRecord(ev[2 * w + 1], st);
    }
    double ms(int w) {
        if (!on) return 0;
        float t = 0;
        if (cudaEventElapsedTime(&t, ev[2 * w], ev[2 * w + 1]) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return t;
    }
};

}  // namespace

int run_batch(gfd_graph* g, const gfd_gfd* const* phis, int32_t n, const gfd_opts* o, gfd_result** out) {
    if (!g || (!phis && n > 0) || !out || n < 0) {
        set_error(GFD_ERR_INVALID_ARG, "validate: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    if (n == 0) return GFD_OK;
    const DevGraph& dg = g->dg;
    const uint32_t nwords = dg.nwords;
    const int32_t flags = o ? o->flags : 0;
    const bool refine = !(flags & GFD_FLAG_NO_REFINE);
    const bool persistent = !(flags & GFD_FLAG_HOST_LOOP);
    const bool use_graph = !(flags & GFD_FLAG_NO_GRAPH);
    const int block_threads = (o && o->block_threads == 512) ? 512 : 256;
    cudaStream_t st = (o && o->cuda_stream) ? (cudaStream_t)o->cuda_stream : g->stream;

    // ---------------------------------------------------------------- plans
    std::vector<HostPlan> plans(n);
    for (int s = 0; s < n; s++) {
        int rc = make_plan(phis[s], g->n_attrs, g->plan_stats(), &plans[s]);
        if (rc) return rc;
    }
    // filter keys (deduplicated across all GFDs and levels)
    std::vector<FilterKey> keys;
    std::map<std::tuple<int32_t, uint32_t, uint32_t, int32_t>, int> key_id;
    std::vector<std::array<int, MAXK>> slot_key(n);
    for (int s = 0; s < n; s++)
        for (int i = 0; i < plans[s].k; i++) {
            const FilterKey& K = plans[s].key[i];
            auto t = std::make_tuple(K.label, K.dout_min, K.din_min, K.self_exp);
            auto it = key_id.find(t);
            if (it == key_id.end()) {
                it = key_id.emplace(t, (int)keys.size()).first;
                keys.push_back(K);
            }
            slot_key[s][i] = it->second;
        }
    const int nkeys = (int)keys.size();

    // ---------------------------------------------------------------- capacities
    auto lab_count = [&](int32_t L) -> uint64_t {
        return L == GFD_WILDCARD ? (uint64_t)g->n : (uint64_t)g->label_stats[3 * (size_t)L];
    };
    auto lab_deg = [&](int32_t L, bool outdir) -> uint64_t {
        return L == GFD_WILDCARD ? (uint64_t)g->m : (uint64_t)g->label_stats[3 * (size_t)L + (outdir ? 1 : 2)];
    };
    int64_t budget = o && o->frontier_budget_bytes > 0 ? o->frontier_budget_bytes : 0;
    if (!budget) {
        size_t fr = 0, tot = 0;
        GFD_CUDA(cudaMemGetInfo(&fr, &tot));
        budget = (int64_t)std::min<size_t>((size_t)64 << 30, fr / 3);
    }
    // violation arena: records shared by all GFDs of the run
    const uint64_t vcap = o && o->max_violations_hint > 0 ? (uint64_t)o->max_violations_hint : (1ull << 22);

    std::vector<SlotDesc> descs(n);
    Layout L;
    struct Off {
        size_t bm[MAXK], rank[MAXK], cand[MAXK], cpi_off[MAXK], cpi_idx[MAXK], rows[MAXK], wpre[MAXK];
    };
    std::vector<Off> offs(n);
    size_t td_need = 0;
    for (int lvl = 0; lvl < MAXK; lvl++) {
        size_t c = 0;
        for (int s = 0; s < n; s++)
            if (lvl < plans[s].k) c += plans[s].td[lvl].size();
        td_need = std::max(td_need, c);
    }
    for (int s = 0; s < n; s++) {
        const HostPlan& P = plans[s];
        SlotDesc& D = descs[s];
        memset(&D, 0, sizeof(D));
        D.k = P.k;
        D.nx = P.nx;
        D.ny = P.ny;
        D.y_false = P.y_false;
        for (int i = 0; i < P.k; i++) {
            D.order[i] = P.order[i];
            D.lv[i] = P.lv[i];
        }
        for (size_t q = 0; q < P.lits.size(); q++) D.lit[q] = P.lits[q];
        uint64_t row_bytes = 0;
        for (int l = 1; l <= P.k - 2; l++) row_bytes += 4ull * (2 * (l + 1) + 1) + 8;
        uint64_t chunk = o && o->chunk_rows > 0 ? (uint64_t)o->chunk_rows
                                                : (row_bytes ? (uint64_t)budget / n / row_bytes : (1ull << 24) - 1);
        chunk = std::max<uint64_t>(1024, std::min<uint64_t>(chunk, (1ull << 24) - 1));
        D.chunk = chunk;
        Off& F = offs[s];
        for (int i = 0; i < P.k; i++) {
            const int32_t lab = phis[s]->node_label[P.order[i]];
            D.cand_cap[i] = (uint32_t)std::min<uint64_t>(lab_count(lab), (uint64_t)g->n);
            F.bm[i] = L.take(4ull * nwords);
            F.rank[i] = L.take(4ull * nwords);
            F.cand[i] = L.take(4ull * std::max<uint32_t>(1, D.cand_cap[i]));
        }
        for (int i = 1; i < P.k; i++) {
            const int par = P.lv[i].par;
            const int32_t plab = phis[s]->node_label[P.order[par]];
            D.cpi_cap[i] = std::min<uint64_t>(lab_deg(plab, P.lv[i].tdir == 1), (uint64_t)g->m);
            F.cpi_off[i] = L.take(4ull * (D.cand_cap[par] + 1ull));
            F.cpi_idx[i] = L.take(4ull * std::max<uint64_t>(1, D.cpi_cap[i]));
        }
        for (int l = 1; l <= P.k - 2; l++) {
            F.rows[l] = L.take(4ull * (2 * (l + 1) + 1) * chunk);
            F.wpre[l] = L.take(8ull * chunk);
        }
    }
    const size_t off_keybm = L.take(4ull * nwords * std::max(1, nkeys));
    const size_t off_keys = L.take(sizeof(FilterKey) * std::max(1, nkeys));
    const size_t off_tmp = L.take(4ull * nwords * std::max<size_t>(1, td_need));
    // the violation arena and its split tables lie before the region that is
    // uploaded from the host image (they need no initial contents)
    int kmax = 1;
    for (auto& P : plans) kmax = std::max(kmax, P.k);
    const int vstride = kmax + 1;
    const size_t off_varena = L.take(4ull * vstride * vcap);
    const size_t off_vptr = L.take(sizeof(int32_t*) * n);
    const size_t off_vcur = L.take(8ull * n);
    const size_t off_desc = L.take(sizeof(SlotDesc) * n);
    const size_t off_state = L.take(sizeof(SlotState) * n);
    const size_t off_sched = L.take(sizeof(Sched));
    const size_t off_tiles = L.take(4ull * (n + 1));
    const size_t off_err = L.take(4);

    // ---------------------------------------------------------------- job tables
    std::vector<AndJob> and_jobs;
    std::vector<CompactJob> compact_jobs;
    std::vector<ScatterJob> scatter_jobs;
    std::vector<PruneJob> prune_jobs;
    std::vector<CpiJob> cpi_jobs;
    struct Phase {
        int kind;  // 0 and, 1 compact, 2 scatter, 3 prune, 4 memset tmp
        size_t first, count;
        int prof;
    };
    std::vector<Phase> phases;
    // pointers are relative to the pool base until the pool exists: build with
    // a null base, then add the base when uploading (see rebase below)
    auto P8 = [](size_t off) { return (uint8_t*)nullptr + off; };
    auto state_ncand = [&](int s, int i) {
        return (uint32_t*)(P8(off_state + sizeof(SlotState) * s + offsetof(SlotState, ncand) + 4 * i));
    };
    auto keybm = [&](int key) { return (uint32_t*)P8(off_keybm + 4ull * nwords * key); };
    int maxk = 0;
    for (auto& P : plans) maxk = std::max(maxk, P.k);
    for (int s = 0; s < n; s++) {
        const HostPlan& P = plans[s];
        SlotDesc& D = descs[s];
        const Off& F = offs[s];
        for (int i = 0; i < P.k; i++) {
            D.bm[i] = (uint32_t*)P8(F.bm[i]);
            D.rank[i] = (uint32_t*)P8(F.rank[i]);
            D.cand[i] = (int32_t*)P8(F.cand[i]);
            if (i >= 1) {
                D.cpi_off[i] = (uint32_t*)P8(F.cpi_off[i]);
                D.cpi_idx[i] = (int32_t*)P8(F.cpi_idx[i]);
            }
        }
        for (int l = 1; l <= P.k - 2; l++) {
            D.rows[l] = (int32_t*)P8(F.rows[l]);
            D.wpre[l] = (uint64_t*)P8(F.wpre[l]);
        }
    }
    auto compact_job = [&](int s, int i) {
        CompactJob J;
        J.bm = descs[s].bm[i];
        J.rank = descs[s].rank[i];
        J.cand = descs[s].cand[i];
        J.count = state_ncand(s, i);
        return J;
    };
    if (!refine) {
        size_t a0 = and_jobs.size(), c0 = compact_jobs.size();
        for (int s = 0; s < n; s++)
            for (int i = 0; i < plans[s].k; i++) {
                AndJob J{};
                J.bm = descs[s].bm[i];
                J.src = keybm(slot_key[s][i]);
                J.ntmp = 0;
                and_jobs.push_back(J);
                compact_jobs.push_back(compact_job(s, i));
            }
        phases.push_back({0, a0, and_jobs.size() - a0, PROF_REFINE});
        phases.push_back({1, c0, compact_jobs.size() - c0, PROF_REFINE});
    } else {
        // top-down, level by level
        for (int lvl = 0; lvl < maxk; lvl++) {
            size_t a0 = and_jobs.size(), c0 = compact_jobs.size(), s0 = scatter_jobs.size();
            size_t tmp_used = 0;
            for (int s = 0; s < n; s++) {
                const HostPlan& P = plans[s];
                if (lvl >= P.k) continue;
                AndJob J{};
                J.bm = descs[s].bm[lvl];
                J.src = keybm(slot_key[s][lvl]);
                J.ntmp = 0;
                for (const Con& c : P.td[lvl]) {
                    uint32_t* marks = (uint32_t*)P8(off_tmp + 4ull * nwords * tmp_used++);
                    ScatterJob S{};
                    S.qcand = descs[s].cand[c.q];
                    S.qcount = state_ncand(s, c.q);
                    S.filter = J.src;
                    S.marks = marks;
                    // x needs an out-neighbour y in C(q) (x -> y): follow in-edges of y
                    S.scan_out = c.dir ? 0 : 1;
                    S.lab = c.lab;
                    scatter_jobs.push_back(S);
                    J.tmp[J.ntmp++] = marks;
                }
                and_jobs.push_back(J);
                compact_jobs.push_back(compact_job(s, lvl));
            }
            if (tmp_used) phases.push_back({4, 0, tmp_used, PROF_REFINE});
            if (scatter_jobs.size() > s0) phases.push_back({2, s0, scatter_jobs.size() - s0, PROF_REFINE});
            phases.push_back({0, a0, and_jobs.size() - a0, PROF_REFINE});
            phases.push_back({1, c0, compact_jobs.size() - c0, PROF_REFINE});
        }
        // bottom-up, reverse level order
        for (int lvl = maxk - 1; lvl >= 0; lvl--) {
            size_t p0 = prune_jobs.size(), c0 = compact_jobs.size();
            for (int s = 0; s < n; s++) {
                const HostPlan& P = plans[s];
                if (lvl >= P.k || P.bu[lvl].empty()) continue;
                PruneJob J{};
                J.cand = descs[s].cand[lvl];
                J.count = state_ncand(s, lvl);
                J.bm = descs[s].bm[lvl];
                for (const Con& c : P.bu[lvl]) {
                    J.con_bm[J.ncon] = descs[s].bm[c.q];
                    J.con_dir[J.ncon] = c.dir;
                    J.con_lab[J.ncon] = c.lab;
                    J.ncon++;
                }
                prune_jobs.push_back(J);
                compact_jobs.push_back(compact_job(s, lvl));
            }
            if (prune_jobs.size() > p0) {
                phases.push_back({3, p0, prune_jobs.size() - p0, PROF_REFINE});
                phases.push_back({1, c0, compact_jobs.size() - c0, PROF_REFINE});
            }
        }
    }
    for (int s = 0; s < n; s++)
        for (int i = 1; i < plans[s].k; i++) {
            const int par = plans[s].lv[i].par;
            CpiJob J{};
            J.pcand = descs[s].cand[par];
            J.pcount = state_ncand(s, par);
            J.cbm = descs[s].bm[i];
            J.crank = descs[s].rank[i];
            J.off = descs[s].cpi_off[i];
            J.idx = descs[s].cpi_idx[i];
            J.cap = descs[s].cpi_cap[i];
            J.out = plans[s].lv[i].tdir;
            J.lab = plans[s].lv[i].tlab;
            J.nnz_stat = (uint64_t*)P8(off_state + sizeof(SlotState) * s + offsetof(SlotState, st_cpi));
            cpi_jobs.push_back(J);
        }
    // per-chunk scratch of the compaction and index scans
    const uint32_t cmp_chunks = compact_chunks(dg);
    const size_t off_cmp_sums = L.take(4ull * cmp_chunks * std::max<size_t>(1, compact_jobs.size()));
    for (size_t j = 0; j < compact_jobs.size(); j++)
        compact_jobs[j].csum = (uint32_t*)P8(off_cmp_sums + 4ull * cmp_chunks * j);
    uint64_t max_pcand = 0;
    for (int s = 0; s < n; s++)
        for (int i = 1; i < plans[s].k; i++) max_pcand = std::max<uint64_t>(max_pcand, descs[s].cand_cap[plans[s].lv[i].par]);
    const uint32_t cpi_nch = cpi_chunks(max_pcand);
    const size_t off_cpi_sums = L.take(8ull * cpi_nch * std::max<size_t>(1, cpi_jobs.size()));
    for (size_t j = 0; j < cpi_jobs.size(); j++) cpi_jobs[j].csum = (uint64_t*)P8(off_cpi_sums + 8ull * cpi_nch * j);
    const size_t off_and = L.take(sizeof(AndJob) * std::max<size_t>(1, and_jobs.size()));
    const size_t off_cmp = L.take(sizeof(CompactJob) * std::max<size_t>(1, compact_jobs.size()));
    const size_t off_sct = L.take(sizeof(ScatterJob) * std::max<size_t>(1, scatter_jobs.size()));
    const size_t off_prn = L.take(sizeof(PruneJob) * std::max<size_t>(1, prune_jobs.size()));
    const size_t off_cpi = L.take(sizeof(CpiJob) * std::max<size_t>(1, cpi_jobs.size()));
    const size_t upload_begin = off_keys;  // keys .. end are uploaded from one host image
    (void)upload_begin;

    // ---------------------------------------------------------------- allocate
    cudaMemPool_t pool;
    if (int rc = get_pool(g, &pool)) return rc;
    uint8_t* base = nullptr;
    cudaError_t ce = cudaMallocFromPoolAsync((void**)&base, L.size, pool, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        set_error(GFD_ERR_OUT_OF_MEMORY, "device workspace of %zu bytes: %s", L.size, cudaGetErrorString(ce));
        return GFD_ERR_OUT_OF_MEMORY;
    }
    struct PoolFree {
        uint8_t* p;
        cudaStream_t st;
        ~PoolFree() {
            if (p) cudaFreeAsync(p, st);
        }
    } pool_free{base, st};
    // rebase every pool-relative pointer
    auto rb = [&](auto* p) -> decltype(p) {
        return p ? (decltype(p))(base + ((uint8_t*)p - (uint8_t*)nullptr)) : p;
    };
    for (auto& D : descs) {
        for (int i = 0; i < MAXK; i++) {
            D.bm[i] = rb(D.bm[i]);
            D.rank[i] = rb(D.rank[i]);
            D.cand[i] = rb(D.cand[i]);
            D.cpi_off[i] = rb(D.cpi_off[i]);
            D.cpi_idx[i] = rb(D.cpi_idx[i]);
            D.rows[i] = rb(D.rows[i]);
            D.wpre[i] = rb(D.wpre[i]);
        }
    }
    for (auto& J : and_jobs) {
        J.bm = rb(J.bm);
        J.src = rb(J.src);
        for (int t = 0; t < J.ntmp; t++) J.tmp[t] = rb(J.tmp[t]);
    }
    for (auto& J : compact_jobs) {
        J.bm = rb(J.bm);
        J.rank = rb(J.rank);
        J.cand = rb(J.cand);
        J.count = rb(J.count);
        J.csum = rb(J.csum);
    }
    for (auto& J : scatter_jobs) {
        J.qcand = rb(J.qcand);
        J.qcount = rb(J.qcount);
        J.filter = rb(J.filter);
        J.marks = rb(J.marks);
    }
    for (auto& J : prune_jobs) {
        J.cand = rb(J.cand);
        J.count = rb(J.count);
        J.bm = rb(J.bm);
        for (int c = 0; c < J.ncon; c++) J.con_bm[c] = rb(J.con_bm[c]);
    }
    for (auto& J : cpi_jobs) {
        J.pcand = rb(J.pcand);
        J.pcount = rb(J.pcount);
        J.cbm = rb(J.cbm);
        J.crank = rb(J.crank);
        J.off = rb(J.off);
        J.idx = rb(J.idx);
        J.nnz_stat = rb(J.nnz_stat);
        J.csum = rb(J.csum);
    }
    // host image of [off_keys, L.size): keys, tmp (untouched), descs, zeroed
    // state/sched/tiles/err, job tables — uploaded in one copy
    const size_t img0 = off_desc;
    std::vector<uint8_t> img(L.size - img0, 0);
    memcpy(img.data() + (off_desc - img0), descs.data(), sizeof(SlotDesc) * n);
    Sched sched{};
    sched.n_slots = n;
    sched.tile = (uint32_t)block_threads * 8;
    sched.timeout_ns = env_u64("GFD_WAIT_LIMIT_MS", 10000) * 1000000ull;
    sched.run_limit_ns = env_u64("GFD_RUN_LIMIT_MS", 600000) * 1000000ull;
    sched.varena = (int32_t*)(base + off_varena);
    sched.varena_cap = vcap;
    sched.vstride = vstride;
    memcpy(img.data() + (off_sched - img0), &sched, sizeof(sched));
    memcpy(img.data() + (off_and - img0), and_jobs.data(), sizeof(AndJob) * and_jobs.size());
    memcpy(img.data() + (off_cmp - img0), compact_jobs.data(), sizeof(CompactJob) * compact_jobs.size());
    memcpy(img.data() + (off_sct - img0), scatter_jobs.data(), sizeof(ScatterJob) * scatter_jobs.size());
    memcpy(img.data() + (off_prn - img0), prune_jobs.data(), sizeof(PruneJob) * prune_jobs.size());
    memcpy(img.data() + (off_cpi - img0), cpi_jobs.data(), sizeof(CpiJob) * cpi_jobs.size());
    ProfEvents prof;
    if (int rc = prof.init((flags & GFD_FLAG_PROFILE) != 0)) return rc;
    int64_t launches[5] = {0, 0, 0, 0, 0};
    GFD_CUDA(cudaMemcpyAsync(base + off_keys, keys.data(), sizeof(FilterKey) * nkeys, cudaMemcpyHostToDevice, st));
    GFD_CUDA(cudaMemcpyAsync(base + img0, img.data(), img.size(), cudaMemcpyHostToDevice, st));

    // ---------------------------------------------------------------- device phases
    prof.begin(PROF_FILTER, st);
    if (int rc = launch_filter(dg, (const FilterKey*)(base + off_keys), nkeys, (uint32_t*)(base + off_keybm), st))
        return rc;
    launches[PROF_FILTER]++;
    prof.end(PROF_FILTER, st);
    prof.begin(PROF_REFINE, st);
    for (const Phase& ph : phases) {
        int rc = GFD_OK;
        switch (ph.kind) {
            case 0: rc = launch_and(dg, (const AndJob*)(base + off_and) + ph.first, (int)ph.count, st); break;
            case 1: rc = launch_compact(dg, (const CompactJob*)(base + off_cmp) + ph.first, (int)ph.count, st); break;
            case 2: rc = launch_scatter(dg, (const ScatterJob*)(base + off_sct) + ph.first, (int)ph.count, st); break;
            case 3: rc = launch_prune(dg, (const PruneJob*)(base + off_prn) + ph.first, (int)ph.count, st); break;
            case 4: {
                cudaError_t e = cudaMemsetAsync(base + off_tmp, 0, 4ull * nwords * ph.count, st);
                rc = e == cudaSuccess ? GFD_OK : cuda_fail(e, "cudaMemsetAsync");
                break;
            }
        }
        if (rc) return rc;
        launches[PROF_REFINE] += ph.kind == 4 ? 0 : (ph.kind == 1 ? 2 : 1);
    }
    prof.end(PROF_REFINE, st);
    prof.begin(PROF_INDEX, st);
    if (int rc = launch_cpi(dg, (const CpiJob*)(base + off_cpi), (int)cpi_jobs.size(), cpi_nch,
                            (int32_t*)(base + off_err), st))
        return rc;
    launches[PROF_INDEX] += cpi_jobs.empty() ? 0 : 4;
    prof.end(PROF_INDEX, st);

    EnumArgs A;
    A.g = dg;
    A.slots = (const SlotDesc*)(base + off_desc);
    A.state = (SlotState*)(base + off_state);
    A.sched = (Sched*)(base + off_sched);
    A.tile_base = (uint32_t*)(base + off_tiles);
    A.n_slots = n;
    A.tile = (int32_t)sched.tile;
    if (int rc = enum_init(A, st)) return rc;
    if (int rc = enum_run(A, persistent, use_graph, block_threads, st, prof.on ? prof.ev[2 * PROF_ENUM] : nullptr,
                          prof.on ? prof.ev[2 * PROF_ENUM + 1] : nullptr, &launches[PROF_ENUM]))
        return rc;
    launches[PROF_ENUM] += 1;

    // ---------------------------------------------------------------- read back
    std::vector<SlotState> states(n);
    Sched hs{};
    int32_t herr = 0;
    GFD_CUDA(cudaMemcpyAsync(states.data(), base + off_state, sizeof(SlotState) * n, cudaMemcpyDeviceToHost, st));
    GFD_CUDA(cudaMemcpyAsync(&hs, base + off_sched, sizeof(Sched), cudaMemcpyDeviceToHost, st));
    GFD_CUDA(cudaMemcpyAsync(&herr, base + off_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GFD_CUDA(cudaStreamSynchronize(st));
    if (hs.err == DERR_TIMEOUT) {
        set_error(GFD_ERR_TIMEOUT, "a device-side limit ran out (grid barrier wait or enumeration time)");
        return GFD_ERR_TIMEOUT;
    }
    if (herr) {
        set_error(GFD_ERR_OVERFLOW, "index capacity exceeded");
        return GFD_ERR_OVERFLOW;
    }
    for (int s = 0; s < n; s++)
        if (states[s].err) {
            set_error(GFD_ERR_OVERFLOW, "GFD %d: partial-match counter overflow (lower chunk_rows)", s);
            return GFD_ERR_OVERFLOW;
        }
    if (hs.varena_used > vcap) {
        // the violations did not fit: run again with room for exactly all of them
        gfd_opts o2 = o ? *o : gfd_opts{};
        o2.max_violations_hint = (int64_t)hs.varena_used;
        o2.cuda_stream = st;
        const int rc = run_batch(g, phis, n, &o2, out);
        if (rc == GFD_OK)
            for (int s = 0; s < n; s++) out[s]->stat[6] += 1;
        return rc;
    }
    // split the arena into one violation list per GFD (order within a list is
    // arbitrary; gfd_result_tuples sorts)
    std::vector<int32_t*> vbuf(n, nullptr);
    struct VFree {
        std::vector<int32_t*>* v;
        cudaStream_t st;
        ~VFree() {
            for (auto p : *v)
                if (p) cudaFreeAsync(p, st);
        }
    } vfree{&vbuf, st};
    for (int s = 0; s < n; s++) {
        if (!states[s].n_viol) continue;
        ce = cudaMallocFromPoolAsync((void**)&vbuf[s], 4ull * states[s].n_viol * plans[s].k, pool, st);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            set_error(GFD_ERR_OUT_OF_MEMORY, "violation list: %s", cudaGetErrorString(ce));
            return GFD_ERR_OUT_OF_MEMORY;
        }
    }
    if (hs.varena_used) {
        GFD_CUDA(cudaMemcpyAsync(base + off_vptr, vbuf.data(), sizeof(int32_t*) * n, cudaMemcpyHostToDevice, st));
        GFD_CUDA(cudaMemsetAsync(base + off_vcur, 0, 8ull * n, st));
        if (int rc = launch_split(A.slots, sched.varena, hs.varena_used, vstride, (int32_t* const*)(base + off_vptr),
                                  (unsigned long long*)(base + off_vcur), st))
            return rc;
    }
    for (int s = 0; s < n; s++) {
        gfd_result* r = new gfd_result();
        r->k = plans[s].k;
        r->n_matches = states[s].n_matches;
        r->n_viol = states[s].n_viol;
        r->d_viol = vbuf[s];
        vbuf[s] = nullptr;
        r->stream = st;
        for (int w = 0; w < 5; w++) {
            r->prof_ms[w] = prof.ms(w);
            r->prof_launch[w] = launches[w];
        }
        r->stat[0] = hs.steps;
        r->stat[1] = states[s].st_work;
        r->stat[2] = states[s].st_rows;
        r->stat[3] = hs.probes;
        uint64_t nc = 0;
        for (int i = 0; i < plans[s].k; i++) nc += states[s].ncand[i];
        r->stat[4] = nc;
        r->stat[5] = states[s].st_cpi;
        out[s] = r;
    }
    return GFD_OK;
}

// ---------------------------------------------------------------- result sort
namespace {

__global__ void k_iota(uint32_t* p, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

// key[i] = (t[perm[i]][c0] << 32) | t[perm[i]][c1]  (c0 < 0: high half zero)
__global__ void k_gather_key(const int32_t* t, int k, const uint32_t* perm, uint64_t n, int c0, int c1, uint64_t* key) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t* row = t + (uint64_t)perm[i] * k;
        const uint64_t hi = c0 >= 0 ? (uint64_t)(uint32_t)row[c0] : 0;
        key[i] = (hi << 32) | (uint64_t)(uint32_t)row[c1];
    }
}

__global__ void k_gather_rows(const int32_t* t, int k, const uint32_t* perm, uint64_t n, int32_t* out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n * k; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = i / k, c = i % k;
        out[i] = t[(uint64_t)perm[r] * k + c];
    }
}

}  // namespace

// Lexicographic order of the violation tuples (Vio is a set; this fixes a
// canonical order): least-significant-first stable radix sorts over pairs of
// columns, carrying a permutation.
int result_fetch(gfd_result* r) {
    if (r->fetched) return GFD_OK;
    const uint64_t n = r->n_viol;
    const int k = r->k;
    r->tuples.assign(n * k, 0);
    if (n == 0) {
        r->fetched = true;
        return GFD_OK;
    }
    cudaStream_t st = r->stream;
    uint32_t *p0, *p1;
    uint64_t *k0, *k1;
    int32_t* sorted;
    GFD_CUDA(cudaMallocAsync((void**)&p0, 4 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&p1, 4 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&k0, 8 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&k1, 8 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&sorted, 4 * n * k, st));
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, 152 * 16);
    k_iota<<<grid, 256, 0, st>>>(p0, n);
    size_t tb = 0;
    cub::DoubleBuffer<uint64_t> kb(k0, k1);
    cub::DoubleBuffer<uint32_t> pb(p0, p1);
    GFD_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, kb, pb, (int64_t)n, 0, 64, st));
    void* tmp;
    GFD_CUDA(cudaMallocAsync(&tmp, tb, st));
    int rc = GFD_OK;
    for (int c1 = k - 1; c1 >= 0; c1 -= 2) {
        const int c0 = c1 - 1;
        k_gather_key<<<grid, 256, 0, st>>>(r->d_viol, k, pb.Current(), n, c0, c1, kb.Current());
        cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tb, kb, pb, (int64_t)n, 0, c0 >= 0 ? 64 : 32, st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cub::DeviceRadixSort::SortPairs");
            break;
        }
    }
    if (rc == GFD_OK) {
        k_gather_rows<<<grid, 256, 0, st>>>(r->d_viol, k, pb.Current(), n, sorted);
        cudaError_t e = cudaMemcpyAsync(r->tuples.data(), sorted, 4 * n * k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "violation copy");
    }
    cudaFreeAsync(tmp, st);
    cudaFreeAsync(p0, st);
    cudaFreeAsync(p1, st);
    cudaFreeAsync(k0, st);
    cudaFreeAsync(k1, st);
    cudaFreeAsync(sorted, st);
    if (rc == GFD_OK) r->fetched = true;
    return rc;
}

}  // namespace gfd
