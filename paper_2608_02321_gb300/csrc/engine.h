// Host-side handles and the engine interface shared by the translation units.
#pragma once

#include <mutex>
#include <string>
#include <memory>
#include <vector>

#include "common.cuh"
#include "plan.h"

namespace gfd {
struct Engine;
}

struct gfd_graph {
    int32_t n = 0;
    int64_t m = 0;
    int32_t n_attrs = 0;
    int32_t lbits = 1;
    int64_t bytes = 0;
    gfd::DevGraph dg{};
    std::vector<void*> allocs;
    std::vector<unsigned long long> label_stats;  // [65536][count, out-degree sum, in-degree sum]
    std::vector<double> moments;                  // [65536][16], see PlanStats
    std::vector<double> moments_all;              // [16]
    std::vector<double> elabel_frac;              // [256]
    gfd::PlanStats plan_stats() const {
        gfd::PlanStats p;
        p.n_vertices = n;
        p.n_edges = m;
        p.moments = moments.data();
        p.moments_all = moments_all.data();
        p.elabel_frac = elabel_frac.data();
        return p;
    }
    cudaStream_t stream = nullptr;
    gfd::Engine* eng = nullptr;
    std::mutex mu;
    int32_t tuned_variant = -1;          // set by gfd_autotune
    int64_t tuned_budget = 0;
    int32_t tuned_tile_iters = 0;
};

struct gfd_result {
    int32_t k = 0;
    uint64_t n_matches = 0;
    uint64_t n_viol = 0;
    int32_t* d_viol = nullptr;  // device, unsorted, owned by the result
    bool fetched = false;
    std::unique_ptr<int32_t[]> tuples;  // host copy made by gfd_result_tuples
    double prof_ms[5] = {0, 0, 0, 0, 0};
    int64_t prof_launch[5] = {0, 0, 0, 0, 0};
    uint64_t stat[7 + gfd::N_CNT] = {};   // gfd_result_stat: 7 run statistics, then the counters
    cudaStream_t stream = nullptr;
    bool has_cand = false;                      // GFD_FLAG_KEEP_CANDIDATES
    std::vector<std::vector<int32_t>> cand;     // refined candidate list per pattern node
};

namespace gfd {

// ---- job descriptors of the index kernels (device memory)
struct AndJob {          // bm = src & tmp[0] & ... & tmp[ntmp-1]
    uint32_t* bm;
    const uint32_t* src;
    const uint32_t* tmp[2 * MAXK];
    int32_t ntmp;
};
struct CompactJob {      // rank and candidate list of bm
    const uint32_t* bm;
    uint32_t* rank;
    int32_t* cand;
    uint32_t* count;
    uint32_t* csum;          // per-chunk set-bit counts (scratch)
};
struct ScatterJob {      // mark vertices adjacent to the candidates of another level
    const int32_t* qcand;
    const uint32_t* qcount;
    const uint32_t* filter;  // only vertices in this bitmap are marked
    uint32_t* marks;
    int32_t scan_out;        // 1: follow out-edges of qcand, 0: in-edges
    int32_t lab;
};
struct PruneJob {        // drop candidates with no neighbour in a later level
    const int32_t* cand;
    const uint32_t* count;
    uint32_t* bm;
    int32_t ncon;
    const uint32_t* con_bm[2 * MAXK];
    int32_t con_dir[2 * MAXK];
    int32_t con_lab[2 * MAXK];
};
struct CpiJob {          // index edges of one spanning-tree edge
    const int32_t* pcand;
    const uint32_t* pcount;
    const uint32_t* cbm;
    const uint32_t* crank;
    uint32_t* off;
    int2* idx;               // (position in C(child), vertex id)
    uint64_t cap;
    int32_t out;             // 1: children are out-neighbours of the parent candidates
    int32_t lab;
    uint64_t* nnz_stat;
    uint64_t* csum;          // per-chunk count sums (scratch)
};

// Adjacency lists longer than HUB_LIST entries (hubs of a skewed degree
// distribution) are queued by the warp kernels and scanned afterwards by whole
// blocks, so that one hub does not leave a single warp running long after the
// rest of the launch; a full queue leaves the list to its warp.
constexpr uint32_t HUB_LIST = 1024;
constexpr uint32_t HUB_CAP = 1u << 19;
struct HubQueue {
    unsigned long long* item;  // (job << 40) | (constraint << 32) | candidate index
    uint32_t* n;               // items queued (may exceed cap: only cap are stored)
    uint32_t cap;
    // counting pass: [0] candidates whose adjacency was scanned, [1] adjacency
    // entries read (null: not counting)
    unsigned long long* scan;
    // room for the exclusive prefix of a launch's per-job group counts (one
    // more than the largest job table of the group)
    uint32_t* jpre;
};

// ---- index kernels (index.cu); each launch covers all jobs given
int launch_filter(const DevGraph& g, const FilterKey* d_keys, int nkeys, uint32_t* d_out, cudaStream_t st);
int launch_and(const DevGraph& g, const AndJob* d_jobs, int njobs, cudaStream_t st);
int launch_compact(const DevGraph& g, const CompactJob* d_jobs, int njobs, cudaStream_t st);
int launch_scatter(const DevGraph& g, const ScatterJob* d_jobs, int njobs, const HubQueue& hq, cudaStream_t st);
int launch_prune(const DevGraph& g, const PruneJob* d_jobs, int njobs, const HubQueue& hq, cudaStream_t st);
// Index edges in two launches: counts, offsets and per-job totals first (the
// caller reads the totals back and allocates exactly), then the fill.
int launch_cpi_count(const DevGraph& g, const CpiJob* d_jobs, int njobs, uint32_t nchunks, int32_t* d_err,
                     uint32_t* d_totals, const HubQueue& hq, cudaStream_t st);
int launch_cpi_fill(const DevGraph& g, const CpiJob* d_jobs, int njobs, const HubQueue& hq, cudaStream_t st);
uint32_t compact_chunks(const DevGraph& g);
uint32_t cpi_chunks(uint64_t max_parent_candidates);

// ---- enumeration (enumerate.cu)
struct EnumArgs {
    DevGraph g;
    const SlotDesc* slots;
    SlotState* state;
    Sched* sched;
    uint32_t* tile_base;  // [3 (n_slots + 1)]: tile prefixes of the fusing, intermediate, last-level slots
    int32_t n_slots;
    int32_t tile;         // largest number of work items per tile
    int32_t n_warps;      // warps of the expansion grid (0: unknown, tiles of `tile`)
};
int enum_init(const EnumArgs& a, cudaStream_t st);
// Mark slots [0, n) idle; start the listed slots (host ids) after their index is built.
int mark_idle(SlotState* state, int n, cudaStream_t st);
int init_slots(const EnumArgs& a, const int* host_ids, int n, cudaStream_t st);
// Capture `steps` enumeration steps (expand + control) into a CUDA graph.
int capture_steps(const EnumArgs& a, int variant, int steps, cudaStream_t st, cudaGraph_t* graph,
                  cudaGraphExec_t* exec);
// Split the violation arena (records [slot, tuple...]) into per-slot lists.
int launch_split(const SlotDesc* slots, const int32_t* arena, uint64_t n, int32_t stride, int32_t* const* lists,
                 unsigned long long* cursor, cudaStream_t st);
// Runs supersteps until every slot is finished. persistent: one cooperative
// launch; else a host loop (optionally captured into CUDA graphs). variant:
// 0 (256 threads, >= 4 blocks/SM), 1 (256, >= 6), 2 (256, >= 8), 3 (128, >= 12),
// 4 (256, >= 5), 5 (512, >= 3).
// general: some slot has a pattern component that starts after level 0 or X
// pushed down (the expansion compiled with those paths); else the leaner one.
// count: the counting instantiation (persistent, general, 256 threads), which
// also fills Sched::cnt; used untimed for the algorithmic-byte model.
int enum_run(const EnumArgs& a, bool persistent, bool use_graph, int variant, bool general, cudaStream_t st,
             cudaEvent_t ev0, cudaEvent_t ev1, int64_t* launches, bool count = false);
int variant_threads(int variant);
constexpr int N_VARIANTS = 6;

// ---- orchestration (run.cu)
// SM count of the current device (queried once per device; 1 if the query
// fails, and the next launch then reports the error).
int device_sms();

int graph_load(const gfd_graph_desc* d, const gfd_opts* o, gfd_graph** out);
void graph_free(gfd_graph* g);
void engine_free(Engine* e);
int run_batch(gfd_graph* g, const gfd_gfd* const* phis, int32_t n, const gfd_opts* o, gfd_result** out);
int session_create(gfd_graph* g, int32_t max_slots, const gfd_opts* o, gfd_session** out);
void session_free(gfd_session* s);
int session_submit(gfd_session* s, const gfd_gfd* phi, int64_t* id);
int session_step(gfd_session* s, int32_t* n_advanced, int32_t* n_running, int32_t* n_queued);
int session_next_result(gfd_session* s, int64_t* id, gfd_result** out);
int session_cancel(gfd_session* s, int64_t id);
double session_stat(const gfd_session* s, int32_t which);
int autotune(gfd_graph* g, const gfd_gfd* const* phis, int32_t n, const gfd_opts* o, gfd_opts* best);
// Sort the violation tuples on the device and copy them to dst (host memory,
// n_viol * k ints); result_fetch does this into the result's own buffer.
int result_sort_copy(gfd_result* r, int32_t* dst);
// The same for n results at once, into one host buffer: result 0's tuples,
// then result 1's, ... (one device sort keyed by (result, tuple), one copy).
int results_sort_copy(gfd_result* const* rs, int n, int32_t* out, uint64_t capacity);
int result_fetch(gfd_result* r);

}  // namespace gfd
