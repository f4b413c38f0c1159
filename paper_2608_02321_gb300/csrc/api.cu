#include <cstring>
// C-ABI entry points declared in include/gfd.h.
#include <cstdarg>
#include <cstdio>
#include <string>

#include "engine.h"

namespace gfd {

namespace {
thread_local std::string g_last_error;
}

const char* last_error_cstr() { return g_last_error.c_str(); }

void set_error(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = std::string("[code ") + std::to_string(code) + "] " + buf;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();
    set_error(GFD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return GFD_ERR_CUDA;
}

}  // namespace gfd

extern "C" {

int gfd_graph_load(const gfd_graph_desc* desc, const gfd_opts* opts, gfd_graph** out) {
    return gfd::graph_load(desc, opts, out);
}

void gfd_graph_free(gfd_graph* g) { gfd::graph_free(g); }

int32_t gfd_graph_vertices(const gfd_graph* g) { return g ? g->n : 0; }
int64_t gfd_graph_edges(const gfd_graph* g) { return g ? g->m : 0; }
int64_t gfd_graph_device_bytes(const gfd_graph* g) { return g ? g->bytes : 0; }

int gfd_validate(const gfd_graph* g, const gfd_gfd* phi, const gfd_opts* opts, gfd_result** out) {
    if (!g || !phi || !out) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_validate: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    gfd_graph* gm = const_cast<gfd_graph*>(g);
    std::lock_guard<std::mutex> lock(gm->mu);
    const gfd_gfd* one[1] = {phi};
    return gfd::run_batch(gm, one, 1, opts, out);
}

int gfd_validate_batch(const gfd_graph* g, const gfd_gfd* const* phis, int32_t n, const gfd_opts* opts,
                       gfd_result** out) {
    if (!g || !out || n < 0 || (n > 0 && !phis)) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_validate_batch: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    gfd_graph* gm = const_cast<gfd_graph*>(g);
    std::lock_guard<std::mutex> lock(gm->mu);
    return gfd::run_batch(gm, phis, n, opts, out);
}

int gfd_autotune(gfd_graph* g, const gfd_gfd* const* phis, int32_t n, const gfd_opts* opts, gfd_opts* best) {
    if (!g) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_autotune: NULL graph");
        return GFD_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g->mu);
    return gfd::autotune(g, phis, n, opts, best);
}

uint64_t gfd_result_matches(const gfd_result* r) { return r ? r->n_matches : 0; }
uint64_t gfd_result_violations(const gfd_result* r) { return r ? r->n_viol : 0; }
int32_t gfd_result_arity(const gfd_result* r) { return r ? r->k : 0; }

const int32_t* gfd_result_tuples(gfd_result* r) {
    if (!r) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_result_tuples: NULL result");
        return nullptr;
    }
    if (gfd::result_fetch(r) != GFD_OK) return nullptr;
    return r->tuples.get();
}

int gfd_results_copy_tuples(gfd_result* const* rs, int32_t n, int32_t* out, uint64_t capacity) {
    if (n < 0 || (n > 0 && !rs)) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_results_copy_tuples: NULL results or negative count");
        return GFD_ERR_INVALID_ARG;
    }
    uint64_t need = 0;
    for (int32_t i = 0; i < n; i++) {
        if (!rs[i]) {
            gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_results_copy_tuples: result %d is NULL", i);
            return GFD_ERR_INVALID_ARG;
        }
        need += rs[i]->n_viol * (uint64_t)rs[i]->k;
    }
    if (need > 0 && !out) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_results_copy_tuples: NULL output");
        return GFD_ERR_INVALID_ARG;
    }
    return gfd::results_sort_copy(rs, n, out, capacity);
}

int gfd_result_copy_tuples(gfd_result* r, int32_t* out, uint64_t capacity) {
    if (!r || (!out && r->n_viol > 0)) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_result_copy_tuples: NULL argument");
        return GFD_ERR_INVALID_ARG;
    }
    const uint64_t need = r->n_viol * (uint64_t)r->k;
    if (capacity < need) {
        gfd::set_error(GFD_ERR_INVALID_ARG, "gfd_result_copy_tuples: capacity %llu < %llu ints",
                       (unsigned long long)capacity, (unsigned long long)need);
        return GFD_ERR_INVALID_ARG;
    }
    if (need == 0) return GFD_OK;
    if (r->fetched) {
        memcpy(out, r->tuples.get(), 4 * need);
        return GFD_OK;
    }
    return gfd::result_sort_copy(r, out);
}

double gfd_result_profile(const gfd_result* r, int32_t which, int64_t* launches) {
    if (!r || which < 0 || which >= 5) {
        if (launches) *launches = 0;
        return 0.0;
    }
    if (launches) *launches = r->prof_launch[which];
    return r->prof_ms[which];
}

uint64_t gfd_result_stat(const gfd_result* r, int32_t which) {
    if (!r || which < 0 || which >= 7 + gfd::N_CNT) return 0;
    return r->stat[which];
}

int gfd_result_candidates(const gfd_result* r, int32_t node, const int32_t** list, int64_t* n) {
    if (!r || !list || !n || !r->has_cand || node < 0 || node >= (int32_t)r->cand.size()) {
        gfd::set_error(GFD_ERR_INVALID_ARG,
                       "gfd_result_candidates: NULL argument, node out of range, or no candidate lists kept "
                       "(validate with GFD_FLAG_KEEP_CANDIDATES)");
        return GFD_ERR_INVALID_ARG;
    }
    *list = r->cand[node].data();
    *n = (int64_t)r->cand[node].size();
    return GFD_OK;
}

void gfd_result_free(gfd_result* r) {
    if (!r) return;
    if (r->d_viol) cudaFree(r->d_viol);
    cudaGetLastError();  // a failure here must not surface in a later, unrelated call
    delete r;
}

int gfd_session_create(const gfd_graph* g, int32_t max_slots, const gfd_opts* opts, gfd_session** out) {
    return gfd::session_create(const_cast<gfd_graph*>(g), max_slots, opts, out);
}

int gfd_session_submit(gfd_session* s, const gfd_gfd* phi, int64_t* request_id) {
    return gfd::session_submit(s, phi, request_id);
}

int gfd_session_step(gfd_session* s, int32_t* n_advanced, int32_t* n_running, int32_t* n_queued) {
    return gfd::session_step(s, n_advanced, n_running, n_queued);
}

int gfd_session_next_result(gfd_session* s, int64_t* request_id, gfd_result** out) {
    return gfd::session_next_result(s, request_id, out);
}

int gfd_session_cancel(gfd_session* s, int64_t request_id) { return gfd::session_cancel(s, request_id); }

double gfd_session_stat(const gfd_session* s, int32_t which) { return gfd::session_stat(s, which); }

void gfd_session_free(gfd_session* s) { gfd::session_free(s); }

const char* gfd_last_error(void) { return gfd::last_error_cstr(); }

}  // extern "C"
