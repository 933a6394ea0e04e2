// fl_tune.cu -- launch and round-switch schedules of a graph and their
// autotuner.
//
// A schedule (fl_schedule) sets how the sketch hop lays out lanes (16 or 32
// per vertex for k <= 16), when a hop runs sparse (frontier-driven) instead
// of over every vertex, when a relaxation round (MIS sweeps, BFS) pulls
// instead of pushing, and whether the assignment BFS runs as one CUDA graph
// with its level loop on the device.  None of them changes a result.  The tuner times the
// whole path (sketches, radii, keys and MIS, assignment) on the graph itself
// under candidate schedules, by coordinate descent from the default (each
// parameter in turn over its candidates, keeping the fastest), and keeps the
// best; the choice is cached per graph signature (vertices, CSR entries, the
// sizes of the degree classes) and k, so later graphs of the same shape reuse
// it without timing.
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "fl_internal.cuh"

namespace fl {
namespace {

struct Tuned {
    fl_schedule sched;
    double ms_default, ms_tuned;
};

std::mutex g_tune_mutex;
std::map<std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t, int>, Tuned> g_tune_cache;

fl_schedule to_public(const Sched& s) {
    fl_schedule o;
    o.hop_group = s.hop_group;
    o.sparse_div = s.sparse_div;
    o.dense_div = s.dense_div;
    o.edge_div = s.edge_div;
    o.graph_bfs = s.graph_bfs;
    o.level_cap = s.level_cap;
    return o;
}

Sched from_public(const fl_schedule& s) {
    Sched o;
    o.hop_group = s.hop_group;
    o.sparse_div = s.sparse_div;
    o.dense_div = s.dense_div;
    o.edge_div = s.edge_div;
    o.graph_bfs = s.graph_bfs;
    o.level_cap = s.level_cap;
    return o;
}

bool valid(const fl_schedule& s) {
    const bool group_ok = s.hop_group == 0 || s.hop_group == 16 || s.hop_group == 32;
    auto div_ok = [](int32_t d) { return d >= 1 && d <= 1024; };
    return group_ok && div_ok(s.sparse_div) && div_ok(s.dense_div) && div_ok(s.edge_div) &&
           (s.graph_bfs == 0 || s.graph_bfs == 1) && s.level_cap >= 0;
}

// Milliseconds of one pass of the path (best of `reps`), with the graph's
// current schedule.
int time_path(fl_graph* g, int k, uint64_t seed, const double* cost, const uint8_t* client, int mem_kind, int reps,
              double* ms) {
    double best = 1e300;
    for (int r = 0; r < reps; ++r) {
        const auto t0 = std::chrono::steady_clock::now();
        FL_TRY(fl_build_sketches(g, k, seed));
        fl_solve* s = nullptr;
        FL_TRY(fl_solve_create(g, &s));
        int rc = fl_compute_radii(s, cost, client, mem_kind, nullptr);
        if (rc == FL_OK) rc = fl_open_facilities(s, nullptr, nullptr, mem_kind);
        if (rc == FL_OK) rc = fl_assign_clients(s, nullptr, nullptr, mem_kind);
        fl_solve_destroy(s);
        FL_TRY(rc);
        const double t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (t < best) best = t;
    }
    *ms = best;
    return FL_OK;
}

}  // namespace
}  // namespace fl

using namespace fl;

extern "C" {

int fl_get_schedule(const fl_graph* g, fl_schedule* out) {
    if (!g || !out) FL_FAIL(FL_EINVAL, "null argument");
    *out = to_public(g->sched);
    return FL_OK;
}

int fl_set_schedule(fl_graph* g, const fl_schedule* sched) {
    if (!g || !sched) FL_FAIL(FL_EINVAL, "null argument");
    if (!valid(*sched))
        FL_FAIL(FL_EINVAL, "bad schedule: hop_group must be 0, 16 or 32, the divisors in [1, 1024], graph_bfs 0 or 1, level_cap >= 0");
    g->sched = from_public(*sched);
    return FL_OK;
}

int fl_autotune(fl_graph* g, int k, uint64_t seed, const double* open_cost, const uint8_t* client_mask, int mem_kind,
                int max_trials, fl_schedule* chosen, double* ms_default, double* ms_tuned) {
    if (!g || !open_cost || !client_mask) FL_FAIL(FL_EINVAL, "null argument");
    if (k < 2 || k > 32) FL_FAIL(FL_EINVAL, "k must be in [2, 32]");
    if (max_trials < 1) FL_FAIL(FL_EINVAL, "max_trials must be >= 1");
    if (!g->lists_ready) {
        FL_TRY(build_work_lists(g));
        g->lists_ready = 1;
    }
    const auto key = std::make_tuple(g->n, g->nnz, g->n_hubs, g->n_small, g->n_mid, k);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            g->sched = from_public(it->second.sched);
            if (chosen) *chosen = it->second.sched;
            if (ms_default) *ms_default = it->second.ms_default;
            if (ms_tuned) *ms_tuned = it->second.ms_tuned;
            return FL_OK;
        }
    }
    const Sched base;
    g->sched = base;
    double best_ms = 0.0;
    FL_TRY(time_path(g, k, seed, open_cost, client_mask, mem_kind, 2, &best_ms));
    const double default_ms = best_ms;
    Sched best = base;
    int trials = 1;
    // coordinate descent: each parameter in turn over its candidates, the
    // ones that move the most time first (the sparse-hop cut-off sets which
    // sketch hops scan every row; the round switches set which relaxation
    // rounds pull)
    std::vector<std::pair<int Sched::*, std::vector<int>>> params;
    params.push_back({&Sched::sparse_div, {8, 32, 4, 64}});
    params.push_back({&Sched::edge_div, {8, 32, 4, 64}});
    params.push_back({&Sched::dense_div, {4, 16, 2, 32}});
    if (k <= 16) params.push_back({&Sched::hop_group, {32}});
    params.push_back({&Sched::graph_bfs, {1}});
    for (const auto& p : params) {
        for (int v : p.second) {
            if (trials >= max_trials) break;
            Sched cand = best;
            if (cand.*(p.first) == v) continue;
            cand.*(p.first) = v;
            g->sched = cand;
            double ms = 0.0;
            FL_TRY(time_path(g, k, seed, open_cost, client_mask, mem_kind, 2, &ms));
            ++trials;
            if (ms < best_ms * 0.99) {  // keep a change only for a clear gain
                best_ms = ms;
                best = cand;
            }
        }
    }
    g->sched = best;
    // leave the graph's sketches built under the chosen schedule
    FL_TRY(fl_build_sketches(g, k, seed));
    Tuned t;
    t.sched = to_public(best);
    t.ms_default = default_ms;
    t.ms_tuned = best_ms;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = t;
    }
    if (chosen) *chosen = t.sched;
    if (ms_default) *ms_default = default_ms;
    if (ms_tuned) *ms_tuned = best_ms;
    return FL_OK;
}

int fl_autotune_forget(void) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.clear();
    return FL_OK;
}

}  // extern "C"
