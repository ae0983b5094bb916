// tune.cu - push-shape autotuning of single solves, and the tuning cache.
//
// The cost unit of the paper is the elementary diffusion (Sec. 2.4); on the
// GPU the time per diffusion also depends on how frontier rows are spread
// over threads, warps and CTAs, which depends on the degree mix of the
// graph.  di_autotune times complete solves for a few push shapes and keeps
// the fastest; the result can be cached in a file of JSON lines keyed by the
// size bucket of the problem.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "di_internal.cuh"

namespace di {

di_status check_tune(const di_tune *t, const char *who) {
    if (!t) { set_error("%s: NULL tune", who); return DI_EINVAL; }
    if (t->thread_max_deg < 1 || t->thread_max_deg > 1024 || t->warp_max_deg < t->thread_max_deg ||
        t->warp_max_deg > (1 << 30) || t->push_ctas_per_sm < 0 || t->push_ctas_per_sm > 64 ||
        t->push_window < 0 || t->push_window > 1) {
        set_error("%s: bad shape (thread_max_deg %d in 1..1024, warp_max_deg %d >= it, push_ctas_per_sm %d in 0..64, "
                  "push_window %d in 0..1)",
                  who, t->thread_max_deg, t->warp_max_deg, t->push_ctas_per_sm, t->push_window);
        return DI_EINVAL;
    }
    return DI_OK;
}

// thread_max_deg in {4, 8, 16, 32} x {occupancy-maximum grid, half of it};
// ctas_per_sm = -1 marks "half" and is resolved by the caller.
int tune_candidates(di_tune *out, int cap) {
    const int tmax[4] = {4, 8, 16, 32};
    int k = 0;
    for (int half = 0; half < 2; ++half)
        for (int t : tmax) {
            if (k >= cap) return k;
            out[k++] = di_tune{t, kWarpMaxDeg, half ? -1 : 0, 0};
        }
    return k;
}

int ilog2_round(int64_t v) {
    if (v <= 1) return 0;
    return (int)std::lround(std::log2((double)v));
}

// The last line of the file whose "key" equals key.
bool tune_cache_lookup(const char *path, const char *key, di_tune *out) {
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    const std::string want = std::string("\"key\": \"") + key + "\"";
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        if (!std::strstr(line, want.c_str())) continue;
        di_tune t = {0, 0, 0, 0};
        const char *p1 = std::strstr(line, "\"thread_max_deg\":");
        const char *p2 = std::strstr(line, "\"warp_max_deg\":");
        const char *p3 = std::strstr(line, "\"push_ctas_per_sm\":");
        const char *p4 = std::strstr(line, "\"push_window\":");
        if (!p1 || !p2 || !p3) continue;
        t.thread_max_deg = (int32_t)std::strtol(p1 + 17, nullptr, 10);
        t.warp_max_deg = (int32_t)std::strtol(p2 + 15, nullptr, 10);
        t.push_ctas_per_sm = (int32_t)std::strtol(p3 + 19, nullptr, 10);
        t.push_window = p4 ? (int32_t)std::strtol(p4 + 14, nullptr, 10) : 0;
        if (check_tune(&t, "tune cache") != DI_OK) { clear_error(); continue; }
        *out = t;
        found = true;
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(const char *path, const char *key, const di_tune &t, double seconds) {
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"thread_max_deg\": %d, \"warp_max_deg\": %d, \"push_ctas_per_sm\": %d, "
                    "\"push_window\": %d, \"seconds\": %.6e}\n",
                 key, t.thread_max_deg, t.warp_max_deg, t.push_ctas_per_sm, t.push_window, seconds);
    std::fclose(f);
}

}  // namespace di

using namespace di;

extern "C" DI_API di_status di_tune_default(di_tune *t) {
    if (!t) { set_error("di_tune_default: NULL"); return DI_EINVAL; }
    *t = di_tune{kThreadMaxDeg, kWarpMaxDeg, 0, 0};
    return DI_OK;
}

extern "C" DI_API di_status di_graph_set_tune(di_graph *g, const di_tune *t) {
    clear_error();
    if (!g) { set_error("di_graph_set_tune: NULL graph"); return DI_EINVAL; }
    DI_TRY(check_tune(t, "di_graph_set_tune"));
    g->tune = *t;
    return DI_OK;
}

extern "C" DI_API di_status di_graph_get_tune(const di_graph *g, di_tune *t) {
    clear_error();
    if (!g || !t) { set_error("di_graph_get_tune: NULL argument"); return DI_EINVAL; }
    *t = g->tune;
    return DI_OK;
}

extern "C" DI_API di_status di_autotune(di_graph *g, const double *B, double d, double tol, const di_opts *opts,
                                       const char *cache_path, di_tune *best, double *best_seconds) {
    clear_error();
    if (!g || !B) { set_error("di_autotune: NULL graph or B"); return DI_EINVAL; }
    di_opts o;
    if (opts) o = *opts; else di_opts_default(&o);
    o.warm_start = 0;
    o.timing = 0;
    char key[160];
    std::snprintf(key, sizeof(key), "solve n=2^%d nnz=2^%d fp64=%d prop=%d", ilog2_round(g->n), ilog2_round(g->nnz),
                  o.fluid_fp64 ? 1 : 0, o.propagation);
    di_tune hit;
    if (tune_cache_lookup(cache_path, key, &hit)) {
        g->tune = hit;
        if (best) *best = hit;
        if (best_seconds) *best_seconds = 0.0;
        return DI_OK;
    }
    DI_TRY(ensure_workspace(g));
    double *H = nullptr;
    DI_CUDA_TRY(cudaMalloc(&H, (size_t)std::max<int64_t>(g->n, 1) * sizeof(double)));
    struct FreeH {
        double *p;
        ~FreeH() { cudaFree(p); }
    } fh{H};
    const int occ_per_sm = std::max(1, g->grid_push / std::max(1, g->num_sms));
    di_tune cand[17];
    int nc = tune_candidates(cand, 16);
    // the frontier push of propagations 3 and 7 may keep a fluid window per tile
    if (o.propagation == 3 || o.propagation == 7) cand[nc++] = di_tune{kThreadMaxDeg, kWarpMaxDeg, 0, 1};
    di_tune win = g->tune;
    double win_s = 1e300;
    for (int c = 0; c < nc; ++c) {
        di_tune t = cand[c];
        if (t.push_ctas_per_sm < 0) {
            if (occ_per_sm < 2) continue;
            t.push_ctas_per_sm = occ_per_sm / 2;
        }
        g->tune = t;
        double secs = 1e300;
        for (int rep = 0; rep < 2; ++rep) {   // the first solve rebuilds the level graph
            di_stats st;
            const di_status rc = di_solve(g, B, d, tol, H, nullptr, &o, &st);
            if (rc != DI_OK && rc != DI_ENOCONV) return rc;
            if (rep > 0) secs = st.seconds;
        }
        if (secs < win_s) { win_s = secs; win = t; }
    }
    g->tune = win;
    tune_cache_store(cache_path, key, win, win_s);
    if (best) *best = win;
    if (best_seconds) *best_seconds = win_s;
    return DI_OK;
}
