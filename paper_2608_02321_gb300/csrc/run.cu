// Orchestration of validation runs: batches (gfd_validate, gfd_validate_batch)
// and continuous-batching serving sessions (gfd_session_*).
//
// Device memory is organised in two kinds of blocks:
//   - slot tables (one per run or session): a SlotDesc and a SlotState per GFD
//     slot, the scheduler state, the per-step tile prefix and, for batch runs,
//     the shared violation arena;
//   - one workspace per group of GFDs admitted together: candidate bitmaps,
//     ranks and lists, index edges, partial-match buffers, index-build job
//     tables and scratch.
// For a group the host plans every GFD (plan.cpp), deduplicates candidate-filter
// keys across the group (the shared candidate cache), derives every buffer's
// capacity from the graph's per-label statistics, allocates the workspace from
// the graph's stream-ordered pool, uploads descriptors and job tables, and
// launches one filter pass for all keys plus the refinement and index phases
// (each launch covers every GFD of the group). Nothing waits on the host until
// the counters are read back at the end.
#include <cub/cub.cuh>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
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
    size_t size = 256;  // offset 0 is reserved
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

int pool_alloc(cudaMemPool_t pool, size_t bytes, cudaStream_t st, void** out, const char* what) {
    cudaError_t e = cudaMallocFromPoolAsync(out, std::max<size_t>(bytes, 256), pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        set_error(GFD_ERR_OUT_OF_MEMORY, "%s: %zu device bytes: %s", what, bytes, cudaGetErrorString(e));
        return GFD_ERR_OUT_OF_MEMORY;
    }
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

// ------------------------------------------------------------------ slot tables
struct Tables {
    int max_slots = 0;
    uint8_t* base = nullptr;
    SlotDesc* desc = nullptr;
    SlotState* state = nullptr;
    Sched* sched = nullptr;
    uint32_t* tiles = nullptr;
    int32_t* err = nullptr;
    int32_t** vptr = nullptr;
    unsigned long long* vcur = nullptr;
    int32_t* varena = nullptr;  // batch runs only
    uint64_t vcap = 0;
    int vstride = 0;
    int32_t tile = 2048;
};

namespace {

int tables_alloc(cudaMemPool_t pool, int max_slots, int block_threads, int tile_iters, int kmax_arena,
                 uint64_t vcap, bool bounded_run, cudaStream_t st, Tables* T) {
    Layout L;
    const size_t o_desc = L.take(sizeof(SlotDesc) * max_slots);
    const size_t o_state = L.take(sizeof(SlotState) * max_slots);
    const size_t o_sched = L.take(sizeof(Sched));
    const size_t o_tiles = L.take(4ull * 3 * (max_slots + 1));  // three tile prefixes
    const size_t o_err = L.take(4);
    const size_t zero_end = L.size;
    const size_t o_vptr = L.take(sizeof(int32_t*) * max_slots);
    const size_t o_vcur = L.take(8ull * max_slots);
    const int vstride = kmax_arena + 1;
    const size_t o_arena = kmax_arena > 0 ? L.take(4ull * vstride * vcap) : 0;
    void* base = nullptr;
    if (int rc = pool_alloc(pool, L.size, st, &base, "slot tables")) return rc;
    T->max_slots = max_slots;
    T->base = (uint8_t*)base;
    T->desc = (SlotDesc*)(T->base + o_desc);
    T->state = (SlotState*)(T->base + o_state);
    T->sched = (Sched*)(T->base + o_sched);
    T->tiles = (uint32_t*)(T->base + o_tiles);
    T->err = (int32_t*)(T->base + o_err);
    T->vptr = (int32_t**)(T->base + o_vptr);
    T->vcur = (unsigned long long*)(T->base + o_vcur);
    T->varena = kmax_arena > 0 ? (int32_t*)(T->base + o_arena) : nullptr;
    T->vcap = kmax_arena > 0 ? vcap : 0;
    T->vstride = vstride;
    T->tile = 32 * tile_iters;  // work items per warp visit
    GFD_CUDA(cudaMemsetAsync(T->base + o_desc, 0, zero_end - o_desc, st));
    Sched s{};
    s.n_slots = max_slots;
    s.tile = (uint32_t)T->tile;
    s.timeout_ns = env_u64("GFD_WAIT_LIMIT_MS", 10000) * 1000000ull;
    // a run as a whole is bounded in time; a session's host drives bounded
    // rounds of steps and has no overall limit
    s.run_limit_ns = bounded_run ? env_u64("GFD_RUN_LIMIT_MS", 600000) * 1000000ull : UINT64_MAX;
    s.varena = T->varena;
    s.varena_cap = T->vcap;
    s.vstride = vstride;
    GFD_CUDA(cudaMemcpyAsync(T->sched, &s, sizeof(s), cudaMemcpyHostToDevice, st));
    return GFD_OK;
}

EnumArgs enum_args(const gfd_graph* g, const Tables& T) {
    EnumArgs A;
    A.g = g->dg;
    A.slots = T.desc;
    A.state = T.state;
    A.sched = T.sched;
    A.tile_base = T.tiles;
    A.n_slots = T.max_slots;
    A.tile = T.tile;
    A.n_warps = 0;
    return A;
}

// ------------------------------------------------------------------ groups
struct Phase {
    int kind;  // 0 and, 1 compact, 2 scatter, 3 prune, 4 clear marks
    size_t first, count;
};

}  // namespace

struct Group {
    int n = 0;
    std::vector<int> slot;
    std::vector<HostPlan> plans;
    std::vector<SlotDesc> descs;
    std::vector<std::array<int, MAXK>> slot_key;
    std::vector<FilterKey> keys;
    uint8_t* base = nullptr;
    size_t bytes = 0;
    struct Off {
        size_t bm[MAXK], rank[MAXK], cand[MAXK], cpi_off[MAXK], cpi_idx[MAXK], rows[MAXK], wpre[MAXK];
    };
    std::vector<Off> offs;
    size_t o_keybm = 0, o_keys = 0, o_tmp = 0, o_cmp_sums = 0, o_cpi_sums = 0, o_cpi_tot = 0;
    size_t o_hubq = 0, o_hubn = 0;  // hub queue of the adjacency kernels
    size_t o_jpre = 0;               // per-launch prefix of the jobs' group counts
    uint8_t* cpi_base = nullptr;  // index edges, sized after counting
    size_t cpi_bytes = 0;
    size_t cpi_bound = 0;  // upper bound of cpi_bytes known at planning time
    size_t o_jobs = 0, o_and = 0, o_cmp = 0, o_sct = 0, o_prn = 0, o_cpi = 0, jobs_end = 0;
    uint32_t cmp_chunks = 1, cpi_nch = 1;
    size_t td_need = 0;
    std::vector<AndJob> and_jobs;
    std::vector<CompactJob> compact_jobs;
    std::vector<ScatterJob> scatter_jobs;
    std::vector<PruneJob> prune_jobs;
    std::vector<CpiJob> cpi_jobs;
    std::vector<Phase> phases;
    std::vector<SlotState> state_img;  // host image of the cleared states (kept until copied)
    int live = 0;  // slots of this group still running (sessions)
};

namespace {

// Top-down constraint "x in C(i) needs a neighbour in C(q) through an edge
// leaving x (dir 1) or entering x (dir 0)": scattering from C(q) scans the
// opposite-direction adjacency of the q label class; gathering scans the
// dir-direction adjacency of the i label class but stops at the first hit
// (counted as half of it).
bool td_gather_cheaper(const gfd_graph* g, int32_t label_q, int32_t label_i, int dir) {
    auto degsum = [&](int32_t L, bool out) -> double {
        return L == GFD_WILDCARD ? (double)g->m : (double)g->label_stats[3 * (size_t)L + (out ? 1 : 2)];
    };
    const double scatter = degsum(label_q, dir == 0);
    const double gather = 0.5 * degsum(label_i, dir == 1);
    return gather < scatter;
}

// Plans, capacities and the workspace layout of a group (host only). With
// strict_budget, a frontier_per_slot that cannot hold MIN_CHUNK partial matches
// at every level of some GFD is an error instead of being raised to that.
constexpr uint64_t MIN_CHUNK = 1024;
int group_plan(gfd_graph* g, const gfd_gfd* const* phis, int n, const gfd_opts* o, int64_t frontier_per_slot,
               Group* G, bool strict_budget = false) {
    const uint32_t nwords = g->dg.nwords;
    G->n = n;
    G->plans.resize(n);
    for (int s = 0; s < n; s++)
        if (int rc = make_plan(phis[s], g->n_attrs, g->plan_stats(), &G->plans[s],
                               !(o && (o->flags & GFD_FLAG_NON_INDUCED)), o && (o->flags & GFD_FLAG_PUSH_X)))
            return rc;
    std::map<std::vector<int64_t>, int> key_id;
    G->slot_key.resize(n);
    for (int s = 0; s < n; s++)
        for (int i = 0; i < G->plans[s].k; i++) {
            const FilterKey& K = G->plans[s].key[i];
            std::vector<int64_t> t = {K.label, K.dout_min, K.din_min, K.self_exp, K.n_attr};
            for (int a = 0; a < K.n_attr; a++) {
                t.push_back(K.attr_a[a]);
                t.push_back(K.attr_c[a]);
            }
            auto it = key_id.find(t);
            if (it == key_id.end()) {
                it = key_id.emplace(t, (int)G->keys.size()).first;
                G->keys.push_back(K);
            }
            G->slot_key[s][i] = it->second;
        }
    auto lab_count = [&](int32_t L) -> uint64_t {
        return L == GFD_WILDCARD ? (uint64_t)g->n : (uint64_t)g->label_stats[3 * (size_t)L];
    };
    auto lab_deg = [&](int32_t L, bool outdir) -> uint64_t {
        return L == GFD_WILDCARD ? (uint64_t)g->m : (uint64_t)g->label_stats[3 * (size_t)L + (outdir ? 1 : 2)];
    };
    Layout L;
    G->descs.assign(n, SlotDesc{});
    G->offs.resize(n);
    for (int lvl = 0; lvl < MAXK; lvl++) {
        size_t c = 0, b = 0;
        for (int s = 0; s < n; s++)
            if (lvl < G->plans[s].k) {
                c += G->plans[s].td[lvl].size();
                b += G->plans[s].bu[lvl].size();
            }
        G->td_need = std::max(G->td_need, std::max(c, b));
    }
    for (int s = 0; s < n; s++) {
        const HostPlan& P = G->plans[s];
        SlotDesc& D = G->descs[s];
        memset(&D, 0, sizeof(D));
        D.k = P.k;
        D.nx = P.nx;
        D.ny = P.ny;
        D.y_false = P.y_false;
        D.push_x = P.push_x ? 1 : 0;
        for (int i = 0; i < P.k; i++) {
            D.order[i] = P.order[i];
            D.lv[i] = P.lv[i];
        }
        for (size_t q = 0; q < P.lits.size(); q++) D.lit[q] = P.lits[q];
        uint64_t row_bytes = 0;
        for (int l = 1; l <= P.k - 2; l++) row_bytes += 4ull * row_width(l) + 8;
        uint64_t chunk = o && o->chunk_rows > 0 ? (uint64_t)o->chunk_rows
                                                : (row_bytes ? (uint64_t)frontier_per_slot / row_bytes : (1ull << 24) - 1);
        if (strict_budget && !(o && o->chunk_rows > 0) && chunk < MIN_CHUNK) {
            set_error(GFD_ERR_OUT_OF_MEMORY,
                      "frontier budget of %lld bytes per GFD holds fewer than %llu partial matches per level of GFD "
                      "%d (it needs %llu bytes)",
                      (long long)frontier_per_slot, (unsigned long long)MIN_CHUNK, s,
                      (unsigned long long)(MIN_CHUNK * row_bytes));
            return GFD_ERR_OUT_OF_MEMORY;
        }
        chunk = std::max<uint64_t>(MIN_CHUNK, std::min<uint64_t>(chunk, (1ull << 24) - 1));
        D.chunk = chunk;
        Group::Off& F = G->offs[s];
        for (int i = 0; i < P.k; i++) {
            const int32_t lab = phis[s]->node_label[P.order[i]];
            D.cand_cap[i] = (uint32_t)std::min<uint64_t>(lab_count(lab), (uint64_t)g->n);
            F.bm[i] = L.take(4ull * nwords);
            F.rank[i] = L.take(4ull * nwords);
            F.cand[i] = L.take(4ull * std::max<uint32_t>(1, D.cand_cap[i]));
        }
        for (int i = 1; i < P.k; i++) {
            const int par = P.lv[i].par;
            if (par < 0) continue;  // starts a component: no index edges
            const int32_t plab = phis[s]->node_label[P.order[par]];
            D.cpi_cap[i] = std::min<uint64_t>(lab_deg(plab, P.lv[i].tdir == 1), (uint64_t)g->m);
            F.cpi_off[i] = L.take(4ull * (D.cand_cap[par] + 1ull));
            G->cpi_bound += 8ull * std::max<uint64_t>(1, D.cpi_cap[i]) + 256;
        }
        for (int l = 1; l <= P.k - 2; l++) {
            F.rows[l] = L.take(4ull * row_width(l) * chunk);
            F.wpre[l] = L.take(8ull * chunk);
        }
    }
    const int nkeys = (int)G->keys.size();
    G->o_keybm = L.take(4ull * nwords * std::max(1, nkeys));
    G->o_tmp = L.take(4ull * nwords * std::max<size_t>(1, G->td_need));
    // job counts, known before any pointer is
    const bool refine = !(o && (o->flags & GFD_FLAG_NO_REFINE));
    size_t n_compact = 0, n_cpi = 0, n_and = 0, n_sct = 0, n_prn = 0;
    for (int s = 0; s < n; s++) {
        const HostPlan& P = G->plans[s];
        for (int i = 1; i < P.k; i++) n_cpi += P.lv[i].par >= 0;
        n_and += P.k;
        n_compact += P.k;
        for (int i = 0; i < P.k; i++) {
            n_sct += refine ? P.td[i].size() + P.bu[i].size() : 0;
            const bool pr = refine && !P.bu[i].empty();   // bottom-up: an AND and a gather at most
            const bool tdg = refine && !P.td[i].empty();  // at most one top-down gather per level
            n_prn += pr + tdg;
            n_and += pr;
            n_compact += 2 * pr + tdg;
        }
    }
    G->cmp_chunks = compact_chunks(g->dg);
    uint64_t max_pcand = 0;
    for (int s = 0; s < n; s++)
        for (int i = 1; i < G->plans[s].k; i++)
            if (G->plans[s].lv[i].par >= 0)
                max_pcand = std::max<uint64_t>(max_pcand, G->descs[s].cand_cap[G->plans[s].lv[i].par]);
    G->cpi_nch = cpi_chunks(max_pcand);
    G->o_cmp_sums = L.take(4ull * G->cmp_chunks * std::max<size_t>(1, n_compact));
    G->o_cpi_sums = L.take(8ull * G->cpi_nch * std::max<size_t>(1, n_cpi));
    G->o_cpi_tot = L.take(4ull * std::max<size_t>(1, n_cpi));
    G->o_hubq = L.take(8ull * HUB_CAP);
    G->o_hubn = L.take(4);
    G->o_jpre = L.take(4ull * (std::max(n_sct, std::max(n_prn, n_cpi)) + 1));
    // the region uploaded from the host: keys and job tables
    G->o_jobs = L.size;
    G->o_keys = L.take(sizeof(FilterKey) * std::max(1, nkeys));
    G->o_and = L.take(sizeof(AndJob) * std::max<size_t>(1, n_and));
    G->o_cmp = L.take(sizeof(CompactJob) * std::max<size_t>(1, n_compact));
    G->o_sct = L.take(sizeof(ScatterJob) * std::max<size_t>(1, n_sct));
    G->o_prn = L.take(sizeof(PruneJob) * std::max<size_t>(1, n_prn));
    G->o_cpi = L.take(sizeof(CpiJob) * std::max<size_t>(1, n_cpi));
    G->jobs_end = L.size;
    G->bytes = L.size;
    return GFD_OK;
}

// Absolute pointers, job tables and their upload; the descriptors go to the
// slot tables at the group's slots, whose states are cleared.
int group_build(gfd_graph* g, Group* G, const Tables& T, bool refine, cudaStream_t st) {
    const uint32_t nwords = g->dg.nwords;
    uint8_t* base = G->base;
    const int n = G->n;
    auto state_ncand = [&](int s, int i) { return &T.state[G->slot[s]].ncand[i]; };
    auto keybm = [&](int key) { return (uint32_t*)(base + G->o_keybm + 4ull * nwords * key); };
    int maxk = 0;
    for (auto& P : G->plans) maxk = std::max(maxk, P.k);
    for (int s = 0; s < n; s++) {
        const HostPlan& P = G->plans[s];
        SlotDesc& D = G->descs[s];
        const Group::Off& F = G->offs[s];
        for (int i = 0; i < P.k; i++) {
            D.bm[i] = (uint32_t*)(base + F.bm[i]);
            D.rank[i] = (uint32_t*)(base + F.rank[i]);
            D.cand[i] = (int32_t*)(base + F.cand[i]);
            if (i >= 1) {
                D.cpi_off[i] = P.lv[i].par >= 0 ? (uint32_t*)(base + F.cpi_off[i]) : nullptr;
                D.cpi_idx[i] = nullptr;  // allocated once the index edges are counted
            }
        }
        for (int l = 1; l <= P.k - 2; l++) {
            D.rows[l] = (int32_t*)(base + F.rows[l]);
            D.wpre[l] = (uint64_t*)(base + F.wpre[l]);
        }
    }
    auto compact_job = [&](int s, int i) {
        CompactJob J{};
        J.bm = G->descs[s].bm[i];
        J.rank = G->descs[s].rank[i];
        J.cand = G->descs[s].cand[i];
        J.count = state_ncand(s, i);
        J.csum = (uint32_t*)(base + G->o_cmp_sums + 4ull * G->cmp_chunks * G->compact_jobs.size());
        return J;
    };
    G->phases.clear();
    if (!refine) {
        size_t a0 = G->and_jobs.size(), c0 = G->compact_jobs.size();
        for (int s = 0; s < n; s++)
            for (int i = 0; i < G->plans[s].k; i++) {
                AndJob J{};
                J.bm = G->descs[s].bm[i];
                J.src = keybm(G->slot_key[s][i]);
                G->and_jobs.push_back(J);
                G->compact_jobs.push_back(compact_job(s, i));
            }
        G->phases.push_back({0, a0, G->and_jobs.size() - a0});
        G->phases.push_back({1, c0, G->compact_jobs.size() - c0});
    } else {
        // top-down, level by level. Each constraint from an earlier level is
        // applied in the cheaper direction: scatter marks from the earlier
        // level's candidates (cost ~ their degree sum), or, after compaction,
        // keep the level's own candidates that have a neighbour there
        // (a gather that stops at the first hit).
        for (int lvl = 0; lvl < maxk; lvl++) {
            size_t a0 = G->and_jobs.size(), c0 = G->compact_jobs.size(), s0 = G->scatter_jobs.size();
            size_t p0 = G->prune_jobs.size();
            size_t tmp_used = 0;
            std::vector<int> gathered;
            for (int s = 0; s < n; s++) {
                const HostPlan& P = G->plans[s];
                if (lvl >= P.k) continue;
                AndJob J{};
                J.bm = G->descs[s].bm[lvl];
                J.src = keybm(G->slot_key[s][lvl]);
                PruneJob Pj{};
                Pj.cand = G->descs[s].cand[lvl];
                Pj.count = state_ncand(s, lvl);
                Pj.bm = G->descs[s].bm[lvl];
                for (const Con& c : P.td[lvl]) {
                    const int32_t lq = G->plans[s].key[c.q].label, li = G->plans[s].key[lvl].label;
                    if (td_gather_cheaper(g, lq, li, c.dir)) {
                        Pj.con_bm[Pj.ncon] = G->descs[s].bm[c.q];
                        Pj.con_dir[Pj.ncon] = c.dir;
                        Pj.con_lab[Pj.ncon] = c.lab;
                        Pj.ncon++;
                        continue;
                    }
                    uint32_t* marks = (uint32_t*)(base + G->o_tmp + 4ull * nwords * tmp_used++);
                    ScatterJob S{};
                    S.qcand = G->descs[s].cand[c.q];
                    S.qcount = state_ncand(s, c.q);
                    S.filter = J.src;
                    S.marks = marks;
                    // x needs an out-neighbour y in C(q) (x -> y): follow in-edges of y
                    S.scan_out = c.dir ? 0 : 1;
                    S.lab = c.lab;
                    G->scatter_jobs.push_back(S);
                    J.tmp[J.ntmp++] = marks;
                }
                G->and_jobs.push_back(J);
                G->compact_jobs.push_back(compact_job(s, lvl));
                if (Pj.ncon) {
                    G->prune_jobs.push_back(Pj);
                    gathered.push_back(s);
                }
            }
            if (tmp_used) G->phases.push_back({4, 0, tmp_used});
            if (G->scatter_jobs.size() > s0) G->phases.push_back({2, s0, G->scatter_jobs.size() - s0});
            G->phases.push_back({0, a0, G->and_jobs.size() - a0});
            G->phases.push_back({1, c0, G->compact_jobs.size() - c0});
            if (!gathered.empty()) {
                const size_t c1 = G->compact_jobs.size();
                for (int s : gathered) G->compact_jobs.push_back(compact_job(s, lvl));
                G->phases.push_back({3, p0, G->prune_jobs.size() - p0});
                G->phases.push_back({1, c1, G->compact_jobs.size() - c1});
            }
        }
        // bottom-up, reverse level order; each constraint from a later level
        // is applied in the cheaper direction, as top-down
        for (int lvl = maxk - 1; lvl >= 0; lvl--) {
            size_t a0 = G->and_jobs.size(), c0 = G->compact_jobs.size(), s0 = G->scatter_jobs.size();
            size_t p0 = G->prune_jobs.size();
            size_t tmp_used = 0;
            std::vector<int> gathered;
            for (int s = 0; s < n; s++) {
                const HostPlan& P = G->plans[s];
                if (lvl >= P.k || P.bu[lvl].empty()) continue;
                AndJob A{};
                A.bm = G->descs[s].bm[lvl];
                A.src = G->descs[s].bm[lvl];
                PruneJob J{};
                J.cand = G->descs[s].cand[lvl];
                J.count = state_ncand(s, lvl);
                J.bm = G->descs[s].bm[lvl];
                for (const Con& c : P.bu[lvl]) {
                    const int32_t lq = P.key[c.q].label, li = P.key[lvl].label;
                    if (td_gather_cheaper(g, lq, li, c.dir)) {
                        J.con_bm[J.ncon] = G->descs[s].bm[c.q];
                        J.con_dir[J.ncon] = c.dir;
                        J.con_lab[J.ncon] = c.lab;
                        J.ncon++;
                        continue;
                    }
                    uint32_t* marks = (uint32_t*)(base + G->o_tmp + 4ull * nwords * tmp_used++);
                    ScatterJob S{};
                    S.qcand = G->descs[s].cand[c.q];
                    S.qcount = state_ncand(s, c.q);
                    S.filter = G->descs[s].bm[lvl];
                    S.marks = marks;
                    S.scan_out = c.dir ? 0 : 1;
                    S.lab = c.lab;
                    G->scatter_jobs.push_back(S);
                    A.tmp[A.ntmp++] = marks;
                }
                if (A.ntmp) {
                    G->and_jobs.push_back(A);
                    G->compact_jobs.push_back(compact_job(s, lvl));
                }
                if (J.ncon) {
                    G->prune_jobs.push_back(J);
                    gathered.push_back(s);
                }
            }
            if (tmp_used) G->phases.push_back({4, 0, tmp_used});
            if (G->scatter_jobs.size() > s0) G->phases.push_back({2, s0, G->scatter_jobs.size() - s0});
            if (G->and_jobs.size() > a0) {
                G->phases.push_back({0, a0, G->and_jobs.size() - a0});
                G->phases.push_back({1, c0, G->compact_jobs.size() - c0});
            }
            if (!gathered.empty()) {
                const size_t c1 = G->compact_jobs.size();
                for (int s : gathered) G->compact_jobs.push_back(compact_job(s, lvl));
                G->phases.push_back({3, p0, G->prune_jobs.size() - p0});
                G->phases.push_back({1, c1, G->compact_jobs.size() - c1});
            }
        }
    }
    for (int s = 0; s < n; s++)
        for (int i = 1; i < G->plans[s].k; i++) {
            const int par = G->plans[s].lv[i].par;
            if (par < 0) continue;  // starts a component
            CpiJob J{};
            J.pcand = G->descs[s].cand[par];
            J.pcount = state_ncand(s, par);
            J.cbm = G->descs[s].bm[i];
            J.crank = G->descs[s].rank[i];
            J.off = G->descs[s].cpi_off[i];
            J.idx = G->descs[s].cpi_idx[i];
            J.cap = G->descs[s].cpi_cap[i];
            J.out = G->plans[s].lv[i].tdir;
            J.lab = G->plans[s].lv[i].tlab;
            J.nnz_stat = &T.state[G->slot[s]].st_cpi;
            J.csum = (uint64_t*)(base + G->o_cpi_sums + 8ull * G->cpi_nch * G->cpi_jobs.size());
            G->cpi_jobs.push_back(J);
        }
    // one host image of keys and job tables (each table within its region)
    const size_t need[6] = {sizeof(FilterKey) * G->keys.size(), sizeof(AndJob) * G->and_jobs.size(),
                            sizeof(CompactJob) * G->compact_jobs.size(), sizeof(ScatterJob) * G->scatter_jobs.size(),
                            sizeof(PruneJob) * G->prune_jobs.size(), sizeof(CpiJob) * G->cpi_jobs.size()};
    const size_t at[7] = {G->o_keys, G->o_and, G->o_cmp, G->o_sct, G->o_prn, G->o_cpi, G->jobs_end};
    for (int t = 0; t < 6; t++)
        if (at[t] + need[t] > at[t + 1]) {
            set_error(GFD_ERR_CUDA, "internal: job table %d needs %zu bytes, region holds %zu", t, need[t],
                      at[t + 1] - at[t]);
            return GFD_ERR_CUDA;
        }
    std::vector<uint8_t> img(G->jobs_end - G->o_jobs, 0);
    auto put = [&](size_t off, const void* p, size_t bytes) {
        if (bytes) memcpy(img.data() + (off - G->o_jobs), p, bytes);
    };
    put(G->o_keys, G->keys.data(), sizeof(FilterKey) * G->keys.size());
    put(G->o_and, G->and_jobs.data(), sizeof(AndJob) * G->and_jobs.size());
    put(G->o_cmp, G->compact_jobs.data(), sizeof(CompactJob) * G->compact_jobs.size());
    put(G->o_sct, G->scatter_jobs.data(), sizeof(ScatterJob) * G->scatter_jobs.size());
    put(G->o_prn, G->prune_jobs.data(), sizeof(PruneJob) * G->prune_jobs.size());
    put(G->o_cpi, G->cpi_jobs.data(), sizeof(CpiJob) * G->cpi_jobs.size());
    GFD_CUDA(cudaMemcpyAsync(base + G->o_jobs, img.data(), img.size(), cudaMemcpyHostToDevice, st));
    // descriptors into the slot tables (contiguous runs in one copy) and states
    // cleared, idle (cur = -1): a serving session's running enumeration may
    // read these slots' states while they are built, and must see them idle
    // until they are started
    G->state_img.assign(n, SlotState{});
    for (auto& z : G->state_img) z.cur = -1;
    for (int s = 0; s < n;) {
        int e = s + 1;
        while (e < n && G->slot[e] == G->slot[e - 1] + 1) e++;
        GFD_CUDA(cudaMemcpyAsync(&T.desc[G->slot[s]], &G->descs[s], sizeof(SlotDesc) * (e - s),
                                 cudaMemcpyHostToDevice, st));
        GFD_CUDA(cudaMemcpyAsync(&T.state[G->slot[s]], &G->state_img[s], sizeof(SlotState) * (e - s),
                                 cudaMemcpyHostToDevice, st));
        s = e;
    }
    return GFD_OK;
}

int group_launch(gfd_graph* g, Group* G, const Tables& T, cudaMemPool_t pool, cudaStream_t st, ProfEvents& prof,
                 int64_t* launches, bool count = false) {
    const DevGraph& dg = g->dg;
    uint8_t* base = G->base;
    const HubQueue hq{(unsigned long long*)(base + G->o_hubq), (uint32_t*)(base + G->o_hubn), HUB_CAP,
                      count ? (unsigned long long*)&T.sched->cnt[CNT_SCAN_CANDS] : nullptr,
                      (uint32_t*)(base + G->o_jpre)};
    prof.begin(PROF_FILTER, st);
    if (int rc = launch_filter(dg, (const FilterKey*)(base + G->o_keys), (int)G->keys.size(),
                               (uint32_t*)(base + G->o_keybm), st))
        return rc;
    launches[PROF_FILTER]++;
    prof.end(PROF_FILTER, st);
    prof.begin(PROF_REFINE, st);
    for (const Phase& ph : G->phases) {
        int rc = GFD_OK;
        switch (ph.kind) {
            case 0: rc = launch_and(dg, (const AndJob*)(base + G->o_and) + ph.first, (int)ph.count, st); break;
            case 1:
                rc = launch_compact(dg, (const CompactJob*)(base + G->o_cmp) + ph.first, (int)ph.count, st);
                break;
            case 2:
                rc = launch_scatter(dg, (const ScatterJob*)(base + G->o_sct) + ph.first, (int)ph.count, hq, st);
                break;
            case 3:
                rc = launch_prune(dg, (const PruneJob*)(base + G->o_prn) + ph.first, (int)ph.count, hq, st);
                break;
            case 4: {
                cudaError_t e = cudaMemsetAsync(base + G->o_tmp, 0, 4ull * dg.nwords * ph.count, st);
                rc = e == cudaSuccess ? GFD_OK : cuda_fail(e, "cudaMemsetAsync");
                break;
            }
        }
        if (rc) return rc;
        launches[PROF_REFINE] += ph.kind == 4 ? 0 : (ph.kind == 0 ? 1 : 2);  // scatter/prune: + hub kernel
    }
    prof.end(PROF_REFINE, st);
    prof.begin(PROF_INDEX, st);
    const int ncpi = (int)G->cpi_jobs.size();
    if (ncpi) {
        CpiJob* d_cpi = (CpiJob*)(base + G->o_cpi);
        uint32_t* d_tot = (uint32_t*)(base + G->o_cpi_tot);
        if (int rc = launch_cpi_count(dg, d_cpi, ncpi, G->cpi_nch, T.err, d_tot, hq, st)) return rc;
        // size the index edges exactly: one read-back of the per-edge totals
        std::vector<uint32_t> tot(ncpi);
        GFD_CUDA(cudaMemcpyAsync(tot.data(), d_tot, 4ull * ncpi, cudaMemcpyDeviceToHost, st));
        GFD_CUDA(cudaStreamSynchronize(st));
        std::vector<size_t> at(ncpi);
        size_t bytes = 256;
        for (int j = 0; j < ncpi; j++) {
            at[j] = bytes;
            bytes = (bytes + 8ull * std::max<uint32_t>(1, tot[j]) + 255) & ~(size_t)255;
        }
        void* p = nullptr;
        if (int rc = pool_alloc(pool, bytes, st, &p, "index edges")) return rc;
        G->cpi_base = (uint8_t*)p;
        G->cpi_bytes = bytes;
        int j = 0;
        for (int s = 0; s < G->n; s++)
            for (int i = 1; i < G->plans[s].k; i++) {
                if (G->plans[s].lv[i].par < 0) continue;  // same jobs, same order as built
                int2* idx = (int2*)(G->cpi_base + at[j]);
                G->cpi_jobs[j].idx = idx;
                G->cpi_jobs[j].cap = tot[j];
                G->descs[s].cpi_idx[i] = idx;
                j++;
            }
        GFD_CUDA(cudaMemcpyAsync(d_cpi, G->cpi_jobs.data(), sizeof(CpiJob) * ncpi, cudaMemcpyHostToDevice, st));
        for (int s = 0; s < G->n; s++)
            GFD_CUDA(cudaMemcpyAsync(&T.desc[G->slot[s]].cpi_idx, G->descs[s].cpi_idx, sizeof(G->descs[s].cpi_idx),
                                     cudaMemcpyHostToDevice, st));
        if (int rc = launch_cpi_fill(dg, d_cpi, ncpi, hq, st)) return rc;
        launches[PROF_INDEX] += 7;
    }
    prof.end(PROF_INDEX, st);
    return GFD_OK;
}

// kernel_variant 1..N selects a variant; 0 takes the graph's tuned one.
int pick_variant(const gfd_graph* g, const gfd_opts* o) {
    if (o && o->kernel_variant >= 1 && o->kernel_variant <= N_VARIANTS) return o->kernel_variant - 1;
    return g->tuned_variant >= 0 ? g->tuned_variant : 0;
}

// work items per block visit in units of the block size (1..64)
int pick_tile_iters(const gfd_graph* g, const gfd_opts* o) {
    if (o && o->tile_iters >= 1) return std::min(o->tile_iters, 64);
    return g->tuned_tile_iters > 0 ? g->tuned_tile_iters : 8;
}

int64_t default_budget(const gfd_graph* g, const gfd_opts* o) {
    if (o && o->frontier_budget_bytes > 0) return o->frontier_budget_bytes;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return (int64_t)1 << 32;
    }
    // memory this graph's pool holds from earlier calls but does not use is
    // free for this one too (the pool keeps what it has allocated)
    if (g && g->eng && g->eng->pool) {
        uint64_t reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(g->eng->pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(g->eng->pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
            reserved > used)
            fr += (size_t)(reserved - used);
        cudaGetLastError();
    }
    // larger frontiers mean fewer, fuller steps (batched workload: 64 GiB ->
    // 542 steps, 128 GiB -> 275 steps and 5 % less time); half the free memory
    // at most
    return (int64_t)std::min<size_t>((size_t)128 << 30, fr / 2);
}

gfd_result* make_result(const HostPlan& P, const SlotState& S, uint64_t steps, uint64_t probes, int32_t* d_viol,
                        cudaStream_t st) {
    gfd_result* r = new gfd_result();
    r->k = P.k;
    r->n_matches = S.n_matches;
    r->n_viol = S.n_viol;
    r->d_viol = d_viol;
    r->stream = st;
    r->stat[0] = steps;
    r->stat[1] = S.st_work;
    r->stat[2] = S.st_rows;
    r->stat[3] = probes;
    uint64_t nc = 0;
    for (int i = 0; i < P.k; i++) nc += S.ncand[i];
    r->stat[4] = nc;
    r->stat[5] = S.st_cpi;
    return r;
}

}  // namespace

// ------------------------------------------------------------------ batch runs
int run_batch(gfd_graph* g, const gfd_gfd* const* phis, int32_t n, const gfd_opts* o, gfd_result** out) {
    if (!g || (!phis && n > 0) || !out || n < 0) {
        set_error(GFD_ERR_INVALID_ARG, "validate: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    if (n == 0) return GFD_OK;
    if (n > GFD_MAX_SLOTS) {
        set_error(GFD_ERR_UNSUPPORTED, "validate: %d GFDs in one call, at most %d (split the batch)", n,
                  GFD_MAX_SLOTS);
        return GFD_ERR_UNSUPPORTED;
    }
    const int32_t flags = o ? o->flags : 0;
    const bool refine = !(flags & GFD_FLAG_NO_REFINE);
    const bool persistent = !(flags & GFD_FLAG_HOST_LOOP);
    const bool use_graph = !(flags & GFD_FLAG_NO_GRAPH);
    const int variant = pick_variant(g, o);
    const int block_threads = variant_threads(variant);
    cudaStream_t st = (o && o->cuda_stream) ? (cudaStream_t)o->cuda_stream : g->stream;
    const uint64_t vcap = o && o->max_violations_hint > 0 ? (uint64_t)o->max_violations_hint : (1ull << 22);

    Group G;
    const int64_t budget = (!o || o->frontier_budget_bytes <= 0) && g->tuned_budget > 0 ? g->tuned_budget
                                                                                        : default_budget(g, o);
    if (int rc = group_plan(g, phis, n, o, budget / n, &G, o && o->frontier_budget_bytes > 0)) return rc;
    int kmax = 1;
    for (auto& P : G.plans) kmax = std::max(kmax, P.k);
    cudaMemPool_t pool;
    if (int rc = get_pool(g, &pool)) return rc;
    Tables T;
    if (int rc = tables_alloc(pool, n, block_threads, pick_tile_iters(g, o), kmax, vcap, true, st, &T)) return rc;
    struct Free {
        std::vector<void*> p;
        cudaStream_t st;
        ~Free() {
            for (void* q : p)
                if (q) cudaFreeAsync(q, st);
        }
    } fr{{T.base}, st};
    void* wb = nullptr;
    if (int rc = pool_alloc(pool, G.bytes, st, &wb, "device workspace")) return rc;
    fr.p.push_back(wb);
    G.base = (uint8_t*)wb;
    G.slot.resize(n);
    for (int s = 0; s < n; s++) G.slot[s] = s;
    if (int rc = group_build(g, &G, T, refine, st)) return rc;
    ProfEvents prof;
    if (int rc = prof.init((flags & GFD_FLAG_PROFILE) != 0)) return rc;
    int64_t launches[5] = {0, 0, 0, 0, 0};
    const bool count = (flags & GFD_FLAG_COUNT) != 0;
    const int lrc = group_launch(g, &G, T, pool, st, prof, launches, count);
    fr.p.push_back(G.cpi_base);
    if (lrc) return lrc;
    const EnumArgs A = enum_args(g, T);
    if (int rc = enum_init(A, st)) return rc;
    bool general = false;  // any slot needing the general expansion
    for (int s = 0; s < n; s++) general |= G.plans[s].push_x || G.plans[s].n_components > 1;
    if (int rc = enum_run(A, persistent || count, use_graph, variant, general, st,
                          prof.on ? prof.ev[2 * PROF_ENUM] : nullptr, prof.on ? prof.ev[2 * PROF_ENUM + 1] : nullptr,
                          &launches[PROF_ENUM], count))
        return rc;
    launches[PROF_ENUM] += 1;

    std::vector<SlotState> states(n);
    Sched hs{};
    int32_t herr = 0;
    GFD_CUDA(cudaMemcpyAsync(states.data(), T.state, sizeof(SlotState) * n, cudaMemcpyDeviceToHost, st));
    GFD_CUDA(cudaMemcpyAsync(&hs, T.sched, sizeof(Sched), cudaMemcpyDeviceToHost, st));
    GFD_CUDA(cudaMemcpyAsync(&herr, T.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
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
        void* p = nullptr;
        if (int rc = pool_alloc(pool, 4ull * states[s].n_viol * G.plans[s].k, st, &p, "violation list")) return rc;
        vbuf[s] = (int32_t*)p;
    }
    if (hs.varena_used) {
        GFD_CUDA(cudaMemcpyAsync(T.vptr, vbuf.data(), sizeof(int32_t*) * n, cudaMemcpyHostToDevice, st));
        GFD_CUDA(cudaMemsetAsync(T.vcur, 0, 8ull * n, st));
        if (int rc = launch_split(T.desc, T.varena, hs.varena_used, T.vstride, T.vptr, T.vcur, st)) return rc;
        launches[PROF_ENUM] += 1;  // the split belongs to the enumeration's output
    }
    // the refined candidate lists, kept for inspection when asked for
    std::vector<std::vector<std::vector<int32_t>>> kept(n);
    if (flags & GFD_FLAG_KEEP_CANDIDATES) {
        for (int s = 0; s < n; s++) {
            kept[s].resize(G.plans[s].k);
            for (int i = 0; i < G.plans[s].k; i++) {
                auto& lst = kept[s][G.plans[s].order[i]];
                lst.resize(states[s].ncand[i]);
                if (!lst.empty())
                    GFD_CUDA(cudaMemcpyAsync(lst.data(), G.descs[s].cand[i], 4ull * lst.size(),
                                             cudaMemcpyDeviceToHost, st));
            }
        }
        GFD_CUDA(cudaStreamSynchronize(st));
    }
    for (int s = 0; s < n; s++) {
        gfd_result* r = make_result(G.plans[s], states[s], hs.steps, hs.probes, vbuf[s], st);
        vbuf[s] = nullptr;
        if (count) {
            for (int c = 0; c < N_CNT; c++) r->stat[7 + c] = hs.cnt[c];
            // the host's figures: distinct filter keys and candidate bitmaps
            // built (for the filter and bitmap bytes)
            r->stat[7 + CNT_HOST] = ((uint64_t)G.keys.size() << 32) | (uint64_t)G.compact_jobs.size();
        }
        if (flags & GFD_FLAG_KEEP_CANDIDATES) {
            r->cand = std::move(kept[s]);
            r->has_cand = true;
        }
        for (int w = 0; w < 5; w++) {
            r->prof_ms[w] = prof.ms(w);
            r->prof_launch[w] = launches[w];
        }
        out[s] = r;
    }
    return GFD_OK;
}

// ------------------------------------------------------------------ serving
namespace {

struct Request {
    int64_t id = -1;
    // an owned copy of the GFD
    std::vector<int32_t> node_label, esrc, edst, elabel;
    std::vector<gfd_literal> X, Y;
    gfd_gfd phi{};
    void fix() {
        phi.node_label = node_label.data();
        phi.esrc = esrc.data();
        phi.edst = edst.data();
        phi.elabel = elabel.data();
        phi.X = X.data();
        phi.Y = Y.data();
    }
};

struct SlotHost {
    bool busy = false;
    bool started = false;  // its index is built and its enumeration started
    int64_t id = -1;
    std::shared_ptr<Group> group;
    int index = 0;  // position inside the group
    int32_t* viol = nullptr;
    uint64_t viol_cap = 0;
    std::unique_ptr<Request> req;
};

}  // namespace

}  // namespace gfd

struct gfd_session {
    gfd_graph* g = nullptr;
    gfd_opts opts{};
    cudaStream_t st = nullptr;        // enumeration rounds
    cudaStream_t st_admit = nullptr;  // index builds of admitted requests
    cudaEvent_t ev_admit = nullptr;   // an admission's index build is complete
    cudaEvent_t ev_round[2] = {nullptr, nullptr};  // around the rounds of a step
    gfd::SlotState* h_states = nullptr;  // pinned snapshot after a round
    gfd::Sched* h_sched = nullptr;
    int32_t* h_err = nullptr;
    cudaMemPool_t pool = nullptr;
    gfd::Tables T;
    int variant = 0;
    int block_threads = 256;
    int64_t budget = 0;     // device bytes for the workspaces of running requests
    int64_t used = 0;
    uint64_t viol_cap = 0;  // violations stored per request before it is run again alone
    int32_t steps_per_round = 8;
    std::vector<gfd::SlotHost> slots;
    std::deque<std::unique_ptr<gfd::Request>> queue;
    std::deque<std::pair<int64_t, gfd_result*>> done;
    int64_t next_id = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double stat[5] = {0, 0, 0, 0, 0};  // gfd_session_stat
    double admit_ms_avg = 0;  // running averages: one admission, one round
    double round_ms_avg = 0;
};

namespace gfd {

int session_create(gfd_graph* g, int32_t max_slots, const gfd_opts* o, gfd_session** out) {
    if (!g || !out || max_slots < 1 || max_slots > GFD_MAX_SLOTS) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_session_create: bad argument");
        return GFD_ERR_INVALID_ARG;
    }
    auto S = std::make_unique<gfd_session>();
    S->g = g;
    if (o) S->opts = *o;
    S->st = o && o->cuda_stream ? (cudaStream_t)o->cuda_stream : g->stream;
    S->variant = pick_variant(g, o);
    S->block_threads = variant_threads(S->variant);
    S->budget = default_budget(g, o);
    S->viol_cap = o && o->max_violations_hint > 0 ? (uint64_t)o->max_violations_hint : (1ull << 20);
    S->slots.resize(max_slots);
    // index builds run beside the enumeration rounds at the highest stream
    // priority, so their blocks are scheduled as soon as the rounds free an SM
    int prio_least = 0, prio_greatest = 0;
    GFD_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    GFD_CUDA(cudaStreamCreateWithPriority(&S->st_admit, cudaStreamNonBlocking, prio_greatest));
    GFD_CUDA(cudaEventCreateWithFlags(&S->ev_admit, cudaEventDisableTiming));
    GFD_CUDA(cudaEventCreate(&S->ev_round[0]));
    GFD_CUDA(cudaEventCreate(&S->ev_round[1]));
    GFD_CUDA(cudaMallocHost((void**)&S->h_states, sizeof(SlotState) * max_slots));
    GFD_CUDA(cudaMallocHost((void**)&S->h_sched, sizeof(Sched)));
    GFD_CUDA(cudaMallocHost((void**)&S->h_err, sizeof(int32_t)));
    if (int rc = get_pool(g, &S->pool)) return rc;
    if (int rc = tables_alloc(S->pool, max_slots, S->block_threads, pick_tile_iters(g, o), 0, 0, false, S->st, &S->T))
        return rc;
    if (int rc = mark_idle(S->T.state, max_slots, S->st)) return rc;  // every slot starts idle
    // the enumeration steps of one round, captured once (the tables never move)
    const EnumArgs A = enum_args(g, S->T);
    if (int rc = capture_steps(A, S->variant, S->steps_per_round, S->st, &S->graph, &S->exec)) return rc;
    GFD_CUDA(cudaStreamSynchronize(S->st));
    *out = S.release();
    return GFD_OK;
}

void session_free(gfd_session* S) {
    if (!S) return;
    if (S->st_admit) cudaStreamSynchronize(S->st_admit);
    cudaStreamSynchronize(S->st);
    for (auto& d : S->done) gfd_result_free(d.second);
    for (auto& sl : S->slots) {
        if (sl.viol) cudaFreeAsync(sl.viol, S->st);
        if (sl.group && --sl.group->live == 0) {
            if (sl.group->base) cudaFreeAsync(sl.group->base, S->st);
            if (sl.group->cpi_base) cudaFreeAsync(sl.group->cpi_base, S->st);
        }
        sl.group.reset();
    }
    if (S->T.base) cudaFreeAsync(S->T.base, S->st);
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    cudaStreamSynchronize(S->st);
    if (S->h_states) cudaFreeHost(S->h_states);
    if (S->h_sched) cudaFreeHost(S->h_sched);
    if (S->h_err) cudaFreeHost(S->h_err);
    if (S->ev_admit) cudaEventDestroy(S->ev_admit);
    for (auto e : S->ev_round)
        if (e) cudaEventDestroy(e);
    if (S->st_admit) cudaStreamDestroy(S->st_admit);
    cudaGetLastError();  // a failure here must not surface in a later, unrelated call
    delete S;
}

int session_submit(gfd_session* S, const gfd_gfd* phi, int64_t* id) {
    if (!S || !phi || !id) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_session_submit: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    // plan now so that an invalid GFD is reported at submission
    HostPlan P;
    if (int rc = make_plan(phi, S->g->n_attrs, S->g->plan_stats(), &P, !(S->opts.flags & GFD_FLAG_NON_INDUCED),
                           (S->opts.flags & GFD_FLAG_PUSH_X) != 0))
        return rc;
    auto R = std::make_unique<Request>();
    R->id = S->next_id++;
    R->node_label.assign(phi->node_label, phi->node_label + phi->k);
    for (int e = 0; e < phi->m; e++) {
        R->esrc.push_back(phi->esrc[e]);
        R->edst.push_back(phi->edst[e]);
        R->elabel.push_back(phi->elabel[e]);
    }
    if (phi->nx) R->X.assign(phi->X, phi->X + phi->nx);
    if (!phi->y_false && phi->ny) R->Y.assign(phi->Y, phi->Y + phi->ny);
    R->phi = *phi;
    R->phi.ny = phi->y_false ? 0 : phi->ny;
    R->fix();
    *id = R->id;
    S->queue.push_back(std::move(R));
    return GFD_OK;
}

namespace {

// Admit queued requests, in arrival order, while a slot is free and their
// device memory (workspace and violation buffer) fits the budget; the admitted
// ones are planned and indexed together as one group.
int session_admit(gfd_session* S) {
    std::vector<int> free_slots;
    for (int i = 0; i < (int)S->slots.size(); i++)
        if (!S->slots[i].busy) free_slots.push_back(i);
    if (free_slots.empty() || S->queue.empty()) return GFD_OK;
    const int64_t per_slot = S->budget / (int64_t)S->slots.size();
    std::vector<std::unique_ptr<Request>> take;
    std::vector<const gfd_gfd*> phis;
    int64_t need = 0;
    while (!S->queue.empty() && take.size() < free_slots.size()) {
        Request* R = S->queue.front().get();
        Group trial;
        const gfd_gfd* one[1] = {&R->phi};
        if (int rc = group_plan(S->g, one, 1, &S->opts, per_slot, &trial)) return rc;
        const int64_t req_bytes =
            (int64_t)(trial.bytes + trial.cpi_bound) + (int64_t)(4ull * trial.plans[0].k * S->viol_cap);
        const bool idle = S->used == 0 && take.empty();  // always admit into an idle device
        if (!idle && S->used + need + req_bytes > S->budget) break;
        need += req_bytes;
        phis.push_back(&R->phi);
        take.push_back(std::move(S->queue.front()));
        S->queue.pop_front();
    }
    if (take.empty()) return GFD_OK;
    const int n = (int)take.size();
    S->stat[3] += n;
    S->stat[4] += 1;
    // the index build runs on the admission stream, beside the round that the
    // caller may have launched on the session stream
    cudaStream_t sa = S->st_admit;
    auto G = std::make_shared<Group>();
    if (int rc = group_plan(S->g, phis.data(), n, &S->opts, per_slot, G.get())) return rc;
    void* wb = nullptr;
    if (int rc = pool_alloc(S->pool, G->bytes, sa, &wb, "request workspace")) return rc;
    G->base = (uint8_t*)wb;
    G->slot.assign(free_slots.begin(), free_slots.begin() + n);
    S->used += (int64_t)G->bytes;
    for (int i = 0; i < n; i++) {
        void* vp = nullptr;
        if (int rc = pool_alloc(S->pool, 4ull * G->plans[i].k * S->viol_cap, sa, &vp, "violation buffer")) return rc;
        G->descs[i].viol = (int32_t*)vp;
        G->descs[i].viol_cap = S->viol_cap;
        S->used += (int64_t)(4ull * G->plans[i].k * S->viol_cap);
        SlotHost& sl = S->slots[G->slot[i]];
        sl.busy = true;
        sl.id = take[i]->id;
        sl.group = G;
        sl.index = i;
        sl.viol = (int32_t*)vp;
        sl.viol_cap = S->viol_cap;
        sl.req = std::move(take[i]);
    }
    G->live = n;
    const bool refine = !(S->opts.flags & GFD_FLAG_NO_REFINE);
    if (int rc = group_build(S->g, G.get(), S->T, refine, sa)) return rc;
    ProfEvents prof;
    int64_t launches[5] = {0, 0, 0, 0, 0};
    const int lrc = group_launch(S->g, G.get(), S->T, S->pool, sa, prof, launches);
    S->used += (int64_t)G->cpi_bytes;
    if (lrc) return lrc;
    // the session stream starts the new slots once their index is built (after
    // whatever round it is running)
    GFD_CUDA(cudaEventRecord(S->ev_admit, sa));
    GFD_CUDA(cudaStreamWaitEvent(S->st, S->ev_admit, 0));
    if (int rc = init_slots(enum_args(S->g, S->T), G->slot.data(), n, S->st)) return rc;
    for (int i = 0; i < n; i++) S->slots[G->slot[i]].started = true;
    return GFD_OK;
}

}  // namespace

namespace {

// Free a slot's device memory and return it to the pool of free slots (its
// request finished or was cancelled; no kernel of the session is running).
void slot_release(gfd_session* S, SlotHost& sl) {
    if (sl.viol) cudaFreeAsync(sl.viol, S->st);
    sl.viol = nullptr;
    S->used -= (int64_t)(4ull * sl.group->plans[sl.index].k * sl.viol_cap);
    if (--sl.group->live == 0) {
        cudaFreeAsync(sl.group->base, S->st);
        if (sl.group->cpi_base) cudaFreeAsync(sl.group->cpi_base, S->st);
        S->used -= (int64_t)(sl.group->bytes + sl.group->cpi_bytes);
        sl.group->base = nullptr;
        sl.group->cpi_base = nullptr;
    }
    sl.group.reset();
    sl.req.reset();
    sl.busy = false;
    sl.started = false;
    sl.id = -1;
}

}  // namespace

int session_step(gfd_session* S, int32_t* n_advanced, int32_t* n_running, int32_t* n_queued) {
    if (!S) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_session_step: NULL session");
        return GFD_ERR_INVALID_ARG;
    }
    using clk = std::chrono::steady_clock;
    // The round for the requests already running is launched first, its state
    // snapshot copied to pinned memory behind it; queued requests are admitted
    // meanwhile (planning on the host, index build on the admission stream), so
    // admission overlaps the round; the new requests start after it.
    std::vector<char> in_round(S->slots.size(), 0);
    int busy = 0;  // requests in the round
    // while an admission keeps the host busy, the GPU should not run dry: queue
    // as many rounds as the last admissions took, by the running averages
    const bool admitting = !S->queue.empty();
    int rounds = 1;
    if (admitting && S->round_ms_avg > 0)
        rounds = (int)std::min(16.0, std::max(1.0, std::ceil(S->admit_ms_avg / S->round_ms_avg)));
    int launched = 0;
    auto launch_round = [&]() -> int {
        busy = 0;
        for (size_t i = 0; i < S->slots.size(); i++) {
            in_round[i] = S->slots[i].busy && S->slots[i].started;
            busy += in_round[i];
        }
        if (!busy) return GFD_OK;
        GFD_CUDA(cudaEventRecord(S->ev_round[0], S->st));
        for (int r = 0; r < rounds; r++) GFD_CUDA(cudaGraphLaunch(S->exec, S->st));
        GFD_CUDA(cudaEventRecord(S->ev_round[1], S->st));
        launched = rounds;
        GFD_CUDA(cudaMemcpyAsync(S->h_states, S->T.state, sizeof(SlotState) * S->slots.size(),
                                 cudaMemcpyDeviceToHost, S->st));
        GFD_CUDA(cudaMemcpyAsync(S->h_sched, S->T.sched, sizeof(Sched), cudaMemcpyDeviceToHost, S->st));
        GFD_CUDA(cudaMemcpyAsync(S->h_err, S->T.err, sizeof(int32_t), cudaMemcpyDeviceToHost, S->st));
        return GFD_OK;
    };
    const auto t0 = clk::now();
    if (int rc = launch_round()) return rc;
    const auto ta = clk::now();
    const int64_t admissions_before = (int64_t)S->stat[4];
    if (int rc = session_admit(S)) return rc;
    const auto t1 = clk::now();
    const double admit_ms = std::chrono::duration<double, std::milli>(t1 - ta).count();
    S->stat[0] += admit_ms;
    if ((int64_t)S->stat[4] > admissions_before)
        S->admit_ms_avg = S->admit_ms_avg > 0 ? 0.8 * S->admit_ms_avg + 0.2 * admit_ms : admit_ms;
    if (!busy) {
        rounds = 1;
        if (int rc = launch_round()) return rc;  // nothing was running: run the admitted requests now
    }
    if (n_advanced) *n_advanced = busy;
    if (busy) {
        GFD_CUDA(cudaStreamSynchronize(S->st));
        float gpu_ms = 0;  // the rounds' device time (they may overlap an admission)
        if (cudaEventElapsedTime(&gpu_ms, S->ev_round[0], S->ev_round[1]) != cudaSuccess) {
            cudaGetLastError();
            gpu_ms = 0;
        }
        S->stat[1] += gpu_ms;
        S->stat[2] += launched;
        if (gpu_ms > 0) {
            const double per = gpu_ms / launched;
            S->round_ms_avg = S->round_ms_avg > 0 ? 0.8 * S->round_ms_avg + 0.2 * per : per;
        }
        const SlotState* states = S->h_states;
        const Sched& hs = *S->h_sched;
        if (hs.err == DERR_TIMEOUT) {
            set_error(GFD_ERR_TIMEOUT, "a device-side limit ran out in the serving session");
            return GFD_ERR_TIMEOUT;
        }
        if (*S->h_err) {
            set_error(GFD_ERR_OVERFLOW, "index capacity exceeded");
            return GFD_ERR_OVERFLOW;
        }
        for (size_t i = 0; i < S->slots.size(); i++) {
            SlotHost& sl = S->slots[i];
            // slots started after the round's snapshot are not in it
            if (!in_round[i] || !sl.busy || states[i].cur >= 0) continue;
            if (states[i].err) {
                set_error(GFD_ERR_OVERFLOW, "request %lld: partial-match counter overflow", (long long)sl.id);
                return GFD_ERR_OVERFLOW;
            }
            gfd_result* r = nullptr;
            if (states[i].n_viol > sl.viol_cap) {
                // more violations than the request's buffer holds: validate it again alone
                gfd_opts o2 = S->opts;
                o2.cuda_stream = S->st;
                o2.flags &= ~GFD_FLAG_HOST_LOOP;
                o2.max_violations_hint = (int64_t)states[i].n_viol;
                const gfd_gfd* one[1] = {&sl.req->phi};
                if (int rc = run_batch(S->g, one, 1, &o2, &r)) return rc;
                r->stat[6] += 1;
                cudaFreeAsync(sl.viol, S->st);
            } else {
                r = make_result(sl.group->plans[sl.index], states[i], hs.steps, hs.probes, sl.viol, S->st);
            }
            sl.viol = nullptr;  // now owned by the result (or freed above)
            S->done.emplace_back(sl.id, r);
            slot_release(S, sl);
        }
    }
    int running = 0;
    for (auto& sl : S->slots) running += sl.busy;
    if (n_running) *n_running = running;
    if (n_queued) *n_queued = (int32_t)S->queue.size();
    return GFD_OK;
}

int session_cancel(gfd_session* S, int64_t id) {
    if (!S) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_session_cancel: NULL session");
        return GFD_ERR_INVALID_ARG;
    }
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
        if ((*it)->id == id) {
            S->queue.erase(it);
            return GFD_OK;
        }
    for (size_t i = 0; i < S->slots.size(); i++) {
        SlotHost& sl = S->slots[i];
        if (!sl.busy || sl.id != id) continue;
        // the slot stops: the next control step skips it (stream-ordered after
        // the last round, which has finished when gfd_session_step returned)
        static const int32_t stopped = -1;
        GFD_CUDA(cudaMemcpyAsync(&S->T.state[i].cur, &stopped, sizeof(int32_t), cudaMemcpyHostToDevice, S->st));
        slot_release(S, sl);
        return GFD_OK;
    }
    for (auto it = S->done.begin(); it != S->done.end(); ++it)
        if (it->first == id) {
            gfd_result_free(it->second);
            S->done.erase(it);
            return GFD_OK;
        }
    set_error(GFD_ERR_INVALID_ARG, "gfd_session_cancel: no request %lld in the session", (long long)id);
    return GFD_ERR_INVALID_ARG;
}

double session_stat(const gfd_session* S, int32_t which) {
    return S && which >= 0 && which < 5 ? S->stat[which] : 0.0;
}

int session_next_result(gfd_session* S, int64_t* id, gfd_result** out) {
    if (!S || !id || !out) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_session_next_result: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    if (S->done.empty()) {
        *id = -1;
        *out = nullptr;
        return GFD_OK;
    }
    *id = S->done.front().first;
    *out = S->done.front().second;
    S->done.pop_front();
    return GFD_OK;
}

// ------------------------------------------------------------------ autotuner
int autotune(gfd_graph* g, const gfd_gfd* const* phis, int32_t n, const gfd_opts* o, gfd_opts* best) {
    if (!g || (!phis && n > 0) || n <= 0) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_autotune: empty batch");
        return GFD_ERR_INVALID_ARG;
    }
    const int64_t b0 = default_budget(g, o);
    const int64_t budgets[2] = {b0, std::max<int64_t>(b0 / 4, (int64_t)1 << 28)};
    const int tiles[2] = {8, 32};
    double best_ms = -1;
    int best_v = 0, best_t = 8;
    int64_t best_b = b0;
    std::vector<gfd_result*> res(n, nullptr);
    for (int bi = 0; bi < 2; bi++)
        for (int ti = 0; ti < 2; ti++)
        for (int v = 0; v < N_VARIANTS; v++) {
            gfd_opts t = o ? *o : gfd_opts{};
            t.kernel_variant = v + 1;
            t.tile_iters = tiles[ti];
            t.frontier_budget_bytes = budgets[bi];
            t.flags |= GFD_FLAG_PROFILE;
            t.flags &= ~GFD_FLAG_HOST_LOOP;
            const int rc = run_batch(g, phis, n, &t, res.data());
            if (rc == GFD_ERR_CUDA || rc == GFD_ERR_OUT_OF_MEMORY) continue;  // variant not usable here
            if (rc) return rc;
            double ms = 0;
            for (int w = 0; w < 4; w++) ms += res[0]->prof_ms[w];
            for (auto& r : res) {
                gfd_result_free(r);
                r = nullptr;
            }
            if (best_ms < 0 || ms < best_ms) {
                best_ms = ms;
                best_v = v;
                best_t = tiles[ti];
                best_b = budgets[bi];
            }
        }
    if (best_ms < 0) {
        set_error(GFD_ERR_CUDA, "gfd_autotune: no variant ran");
        return GFD_ERR_CUDA;
    }
    g->tuned_variant = best_v;
    g->tuned_tile_iters = best_t;
    g->tuned_budget = best_b;
    if (best) {
        *best = o ? *o : gfd_opts{};
        best->kernel_variant = best_v + 1;
        best->tile_iters = best_t;
        best->frontier_budget_bytes = best_b;
    }
    return GFD_OK;
}

// ------------------------------------------------------------------ result sort
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

// Several results' violation lists sorted together: rows of a matrix of
// width W = 1 + max k, column 0 the result's index (most significant), the
// tuple after it (zero-padded; only rows of the same result are ever compared
// past column 0).
struct PackSrc {
    const int32_t* p;   // the result's unsorted tuples
    int32_t k;
    int32_t pad;
    uint64_t row_off;   // first row of the result in the matrix (and in sorted order)
    uint64_t int_off;   // first int of the result in the packed output
};

__global__ void k_pack_multi(const PackSrc* src, int nres, uint64_t total, int W, int32_t* M) {
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total; g += (uint64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nres;  // src[lo].row_off <= g < src[hi].row_off (src[nres] = total)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (src[mid].row_off <= g) lo = mid;
            else hi = mid;
        }
        const PackSrc s = src[lo];
        const uint64_t local = g - s.row_off;
        int32_t* row = M + g * W;
        row[0] = lo;
        for (int c = 0; c < W - 1; c++) row[1 + c] = c < s.k ? s.p[local * s.k + c] : 0;
    }
}

__global__ void k_unpack_multi(const PackSrc* src, const int32_t* M, int W, const uint32_t* perm, uint64_t total,
                               int32_t* out) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < total; p += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t* row = M + (uint64_t)perm[p] * W;
        const PackSrc s = src[row[0]];
        int32_t* dst = out + s.int_off + (p - s.row_off) * s.k;
        for (int c = 0; c < s.k; c++) dst[c] = row[1 + c];
    }
}

}  // namespace

// Device-to-host copy of results into caller memory, synchronous. (A staged
// copy through a page-locked double buffer, several host threads moving each
// chunk into pageable memory, was slower here: 67 vs 44 ms for 853 MB.)
int copy_to_host(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return GFD_OK;
    GFD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
    GFD_CUDA(cudaStreamSynchronize(st));
    return GFD_OK;
}

// Lexicographic order of the violation tuples (Vio is a set; this fixes a
// canonical order): least-significant-first stable radix sorts over pairs of
// columns, carrying a permutation.
int result_fetch(gfd_result* r) {
    if (r->fetched) return GFD_OK;
    const uint64_t n = r->n_viol;
    if (n > 0) {
        r->tuples.reset(new (std::nothrow) int32_t[n * r->k]);
        if (!r->tuples) {
            set_error(GFD_ERR_OUT_OF_MEMORY, "violation tuples: %llu host bytes", (unsigned long long)(4ull * n * r->k));
            return GFD_ERR_OUT_OF_MEMORY;
        }
        if (int rc = result_sort_copy(r, r->tuples.get())) {
            r->tuples.reset();
            return rc;
        }
    }
    r->fetched = true;
    return GFD_OK;
}

int result_sort_copy(gfd_result* r, int32_t* dst) {
    const uint64_t n = r->n_viol;
    const int k = r->k;
    if (n == 0) return GFD_OK;
    cudaStream_t st = r->stream;
    uint32_t *p0, *p1;
    uint64_t *k0, *k1;
    int32_t* sorted;
    GFD_CUDA(cudaMallocAsync((void**)&p0, 4 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&p1, 4 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&k0, 8 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&k1, 8 * n, st));
    GFD_CUDA(cudaMallocAsync((void**)&sorted, 4 * n * k, st));
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sms() * 16);
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
        rc = copy_to_host(dst, sorted, 4 * n * k, st);
    }
    cudaFreeAsync(tmp, st);
    cudaFreeAsync(p0, st);
    cudaFreeAsync(p1, st);
    cudaFreeAsync(k0, st);
    cudaFreeAsync(k1, st);
    cudaFreeAsync(sorted, st);
    return rc;
}

int results_sort_copy(gfd_result* const* rs, int n, int32_t* out, uint64_t capacity) {
    std::vector<PackSrc> src((size_t)n + 1);
    uint64_t total = 0, ints = 0;
    int kmax = 1;
    cudaStream_t st = nullptr;
    for (int r = 0; r < n; r++) {
        src[r] = PackSrc{rs[r]->d_viol, rs[r]->k, 0, total, ints};
        total += rs[r]->n_viol;
        ints += rs[r]->n_viol * (uint64_t)rs[r]->k;
        kmax = std::max(kmax, rs[r]->k);
        if (rs[r]->n_viol && !st) st = rs[r]->stream;
    }
    src[n] = PackSrc{nullptr, 1, 0, total, ints};
    if (capacity < ints) {
        set_error(GFD_ERR_INVALID_ARG, "gfd_results_copy_tuples: capacity %llu < %llu ints",
                  (unsigned long long)capacity, (unsigned long long)ints);
        return GFD_ERR_INVALID_ARG;
    }
    if (total == 0) return GFD_OK;
    // Each result's violation list is written on the stream of the call that
    // made it (the split runs after that call returns). The sort runs on the
    // first such stream, so it first waits for every other one.
    std::vector<cudaStream_t> waited;
    for (int r = 0; r < n; r++) {
        const cudaStream_t rs_st = rs[r]->stream;
        if (!rs[r]->n_viol || rs_st == st || std::find(waited.begin(), waited.end(), rs_st) != waited.end())
            continue;
        waited.push_back(rs_st);
        cudaEvent_t ev = nullptr;
        GFD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, rs_st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess) return cuda_fail(e, "ordering the violation sort after the result's stream");
    }
    if (total >= ((uint64_t)1 << 32)) {  // the carried permutation is 32-bit: one result at a time
        for (int r = 0; r < n; r++)
            if (int rc = result_sort_copy(rs[r], out + src[r].int_off)) return rc;
        return GFD_OK;
    }
    const int W = kmax + 1;
    PackSrc* d_src;
    uint32_t *p0, *p1;
    uint64_t *k0, *k1;
    int32_t *M, *dout;
    GFD_CUDA(cudaMallocAsync((void**)&d_src, sizeof(PackSrc) * ((size_t)n + 1), st));
    GFD_CUDA(cudaMallocAsync((void**)&M, 4ull * total * W, st));
    GFD_CUDA(cudaMallocAsync((void**)&p0, 4 * total, st));
    GFD_CUDA(cudaMallocAsync((void**)&p1, 4 * total, st));
    GFD_CUDA(cudaMallocAsync((void**)&k0, 8 * total, st));
    GFD_CUDA(cudaMallocAsync((void**)&k1, 8 * total, st));
    GFD_CUDA(cudaMallocAsync((void**)&dout, 4 * ints, st));
    GFD_CUDA(cudaMemcpyAsync(d_src, src.data(), sizeof(PackSrc) * ((size_t)n + 1), cudaMemcpyHostToDevice, st));
    const int grid = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)device_sms() * 16);
    k_pack_multi<<<grid, 256, 0, st>>>(d_src, n, total, W, M);
    k_iota<<<grid, 256, 0, st>>>(p0, total);
    size_t tb = 0;
    cub::DoubleBuffer<uint64_t> kb(k0, k1);
    cub::DoubleBuffer<uint32_t> pb(p0, p1);
    GFD_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, kb, pb, (int64_t)total, 0, 64, st));
    void* tmp;
    GFD_CUDA(cudaMallocAsync(&tmp, tb, st));
    int rc = GFD_OK;
    for (int c1 = W - 1; c1 >= 0; c1 -= 2) {  // least significant pair of columns first
        const int c0 = c1 - 1;
        k_gather_key<<<grid, 256, 0, st>>>(M, W, pb.Current(), total, c0, c1, kb.Current());
        cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tb, kb, pb, (int64_t)total, 0, c0 >= 0 ? 64 : 32, st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cub::DeviceRadixSort::SortPairs");
            break;
        }
    }
    if (rc == GFD_OK) {
        k_unpack_multi<<<grid, 256, 0, st>>>(d_src, M, W, pb.Current(), total, dout);
        rc = copy_to_host(out, dout, 4 * ints, st);
    }
    cudaFreeAsync(tmp, st);
    cudaFreeAsync(d_src, st);
    cudaFreeAsync(M, st);
    cudaFreeAsync(p0, st);
    cudaFreeAsync(p1, st);
    cudaFreeAsync(k0, st);
    cudaFreeAsync(k1, st);
    cudaFreeAsync(dout, st);
    return rc;
}

}  // namespace gfd
