// k_solve.cu -- phases (ii) and (iii) plus assignment and objective:
//   radius solve (Eq. 1 at epsilon -> 0 from predicated HIP estimates),
//   key ordinals (r_f, pi_f), greedy-MIS rounds on the implicit conflict
//   graph H-bar (Section 4.3, Algorithm 6), nearest-open-facility BFS and
//   the objective (Section 3.1).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

#include "fl_internal.cuh"

namespace fl {

static int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// ------------------------------------------------------------------ frontier propagation
// A frontier is a list of vertices with a device-side count.  One round:
// snapshot (copy each frontier vertex's value, so a round moves values exactly
// one hop), then push: for every edge (v, u), X[u] = min(X[u], val(v) + add);
// u joins the next frontier the first time it decreases in the round.

__global__ void k_snapshot(const int32_t* __restrict__ fr, const unsigned long long* __restrict__ n_fr,
                           const unsigned long long* __restrict__ X, unsigned long long* __restrict__ frval,
                           unsigned long long* __restrict__ reset_next,
                           uint32_t* __restrict__ tstamp, uint32_t tval, int32_t* __restrict__ touched,
                           unsigned long long* __restrict__ n_touched) {
    const int64_t n = (int64_t)*n_fr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *reset_next = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        int64_t i = base + lane_id();
        bool fresh = false;
        int32_t v = 0;
        if (i < n) {
            v = fr[i];
            frval[i] = X[v];
            if (tstamp) fresh = atomicExch(&tstamp[v], tval) != tval;
        }
        if (tstamp) {
            long long at = warp_append(fresh, n_touched);
            if (at >= 0) touched[at] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_push(const int32_t* __restrict__ fr, const unsigned long long* __restrict__ frval,
                                              const unsigned long long* __restrict__ n_fr,
                                              const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                              unsigned long long add, unsigned long long* __restrict__ X,
                                              uint32_t* __restrict__ stamp, uint32_t sv, int32_t* __restrict__ fr_next,
                                              unsigned long long* __restrict__ n_next) {
    const int lane = lane_id();
    const int64_t n = (int64_t)*n_fr;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; w < n; w += warps) {
        const int32_t v = fr[w];
        const unsigned long long val = frval[w] + add;
        const int64_t beg = rowp[v], end = rowp[v + 1];
        for (int64_t cb = beg; cb < end; cb += 32) {
            int64_t e = cb + lane;
            bool fresh = false;
            int32_t u = 0;
            if (e < end) {
                u = cols[e];
                if (val < X[u]) {
                    unsigned long long old = atomicMin(&X[u], val);
                    if (val < old) fresh = atomicExch(&stamp[u], sv) != sv;
                }
            }
            long long at = warp_append(fresh, n_next);
            if (at >= 0) fr_next[at] = u;
        }
    }
}

// Seeds: X[s] = min(X[s], val(s)); s joins the frontier when it decreases.
// With `reach`, a seed that held no value below `limit` records reach_val.
__global__ void k_inject(const int32_t* __restrict__ src, int64_t n_src, uint8_t* __restrict__ reach,
                         uint32_t reach_val, unsigned long long limit,
                         unsigned long long hi, const uint32_t* __restrict__ lo_of, unsigned long long* __restrict__ X,
                         uint32_t* __restrict__ stamp, uint32_t sv, int32_t* __restrict__ fr,
                         unsigned long long* __restrict__ n_fr) {
    __shared__ BlockAppend<8> sh;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < n_src; bb += stride) {
        const int64_t i = bb + threadIdx.x;
        bool fresh = false;
        int32_t s = 0;
        if (i < n_src) {
            s = src[i];
            unsigned long long val = (hi << 32) | (lo_of ? lo_of[s] : (uint32_t)s);
            unsigned long long old = atomicMin(&X[s], val);
            if (val < old) {
                if (reach && old >= limit) reach[s] = (uint8_t)reach_val;
                fresh = atomicExch(&stamp[s], sv) != sv;
            }
        }
        long long at = block_append<8>(fresh, n_fr, sh);
        if (at >= 0) fr[at] = s;
    }
}

// ------------------------------------------------------------------ multi-source BFS
// Level-synchronous BFS from a source list; X[v] = (dist << 32) | label, and
// atomicMin keeps the smallest label among the sources at the smallest
// distance.  label/dist = -1 where no source is reachable.

__global__ void k_unpack_bfs(const unsigned long long* __restrict__ X, int64_t n, int32_t* __restrict__ label,
                             int32_t* __restrict__ dist) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        unsigned long long x = X[v];
        bool none = x == ~0ULL;
        if (label) label[v] = none ? -1 : (int32_t)(x & 0xffffffffULL);
        if (dist) dist[v] = none ? -1 : (int32_t)(x >> 32);
    }
}

int msbfs(fl_graph* g, const int32_t* src_list, int64_t n_src, int32_t* label, int32_t* dist, DBuf& X,
          DBuf& stampb, DBuf* fr, DBuf& frval, int cls) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    FL_TRY(dalloc(X, (size_t)n * 16));
    FL_TRY(dalloc(stampb, (size_t)n * 4));
    FL_TRY(dalloc(fr[0], (size_t)n * 4));
    FL_TRY(dalloc(fr[1], (size_t)n * 4));
    FL_TRY(dalloc(frval, (size_t)n * 8 + 64));
    Relax r;
    r.X[0] = X.as<unsigned long long>();
    r.X[1] = r.X[0] + n;
    r.fr[0] = fr[0].as<int32_t>();
    r.fr[1] = fr[1].as<int32_t>();
    r.frval = frval.as<unsigned long long>();
    r.stamp = stampb.as<uint32_t>();
    r.cnt = reinterpret_cast<unsigned long long*>(frval.as<char>() + (size_t)n * 8);
    r.h_cnt = &g->h_ctr->aux3;
    r.limit = ~0ULL;
    r.settle = true;  // level-synchronous: a vertex's first value is its final one
    FL_TRY(relax_begin(g, r));
    FL_CUDA(cudaMemsetAsync(r.X[0], 0xff, (size_t)n * 8, st));
    FL_CUDA(cudaMemsetAsync(r.stamp, 0, (size_t)n * 4, st));
    FL_CUDA(cudaMemsetAsync(r.cnt, 0, 64, st));
    if (n_src > 0) {
        // labels are the sources' rank ids: ties go to the smallest original
        // (or part-local) facility id whatever the internal numbering
        const uint32_t* label_of = g->rid.p ? g->rid.as<uint32_t>() : nullptr;
        FL_LAUNCH(cls, k_inject<<<grid_for(n_src, 256), 256, 0, st>>>(src_list, n_src, nullptr, 0u, ~0ULL, 0ULL,
                                                                      label_of, r.X[0], r.stamp, 1u, r.fr[0],
                                                                      &r.cnt[0]));
        FL_CUDA(cudaGetLastError());
    }
    r.n_front = n_src;
    r.sv_prev = 1;
    const int64_t cap = g->sched.level_cap > 0 ? g->sched.level_cap : n + 2;
    for (uint32_t level = 0; r.n_front > 0; ++level) {
        if ((int64_t)level >= cap) FL_FAIL(FL_ETIMEOUT, "BFS reached its level cap");
        FL_TRY(relax_round(g, r, 1ULL << 32, level + 2, cls));
    }
    FL_LAUNCH(cls, k_unpack_bfs<<<grid_for(n, 256), 256, 0, st>>>(r.X[r.cur], n, label, dist));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

// ------------------------------------------------------------------ BFS as one CUDA graph
// The same BFS with its level loop on the device: a CUDA graph whose
// conditional WHILE node repeats one pull level and a kernel that advances
// the level, ending the loop when a level reaches no vertex.  Values are
// updated in place: a vertex reached at level L gets stamp L, and level L
// reads only neighbours stamped L - 1, whose values are final, so no level
// sees a value written in the same level.  The level count is capped (n + 2
// levels); at the cap the loop stops with an error flag (FL_ETIMEOUT).  One
// graph launch and one synchronisation replace a launch sequence and a
// synchronisation per level.

namespace {

struct GbfsState {
    uint32_t level;
    uint32_t pad;
    unsigned long long reached;
    unsigned long long error;
};

__device__ __forceinline__ bool gbfs_front(const uint32_t* __restrict__ stamp, int32_t u, uint32_t prev) {
    return __ldg(&stamp[u]) == prev;
}

// Vertices of at most kSmallDeg neighbours: a thread each.
__global__ void __launch_bounds__(256) k_gbfs_small(const int32_t* __restrict__ list, int64_t n_list,
                                                    const int64_t* __restrict__ rowp,
                                                    const int32_t* __restrict__ cols, unsigned long long* X,
                                                    uint32_t* stamp, GbfsState* st, unsigned long long add) {
    const uint32_t L = st->level;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_list; i += stride) {
        const int32_t v = list[i];
        if (X[v] != ~0ULL) continue;
        unsigned long long m = ~0ULL;
        for (int64_t e = rowp[v]; e < rowp[v + 1]; ++e) {
            const int32_t u = __ldg(&cols[e]);
            if (gbfs_front(stamp, u, L - 1)) m = umin64(m, X[u]);
        }
        if (m != ~0ULL) {
            X[v] = m + add;
            stamp[v] = L;
            ++cnt;
        }
    }
    if (cnt) atomicAdd(&st->reached, cnt);
}

// Other vertices: a group of G lanes each (8 for the middle degrees, 32 for
// hubs), 32 / G vertices per warp; every lane of a warp runs every pass (the
// group reductions are warp shuffles).
template <int G>
__global__ void __launch_bounds__(256) k_gbfs_group(const int32_t* __restrict__ list, int64_t n_list,
                                                    const int64_t* __restrict__ rowp,
                                                    const int32_t* __restrict__ cols, unsigned long long* X,
                                                    uint32_t* stamp, GbfsState* st, unsigned long long add) {
    constexpr int kPerWarp = 32 / G;
    const uint32_t L = st->level;
    const int lane = lane_id(), sub = lane & (G - 1);
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cnt = 0;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * kPerWarp < n_list; w += warps) {
        const int64_t i = w * kPerWarp + lane / G;
        const int32_t v = i < n_list ? list[i] : 0;
        const bool work = i < n_list && X[v] == ~0ULL;
        unsigned long long m = ~0ULL;
        if (work)
            for (int64_t e = rowp[v] + sub; e < rowp[v + 1]; e += G) {
                const int32_t u = __ldg(&cols[e]);
                if (gbfs_front(stamp, u, L - 1)) m = umin64(m, X[u]);
            }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) m = umin64(m, __shfl_xor_sync(kFull, m, o, G));
        if (work && sub == 0 && m != ~0ULL) {
            X[v] = m + add;
            stamp[v] = L;
            ++cnt;
        }
    }
    if (cnt) atomicAdd(&st->reached, cnt);
}

// Sources: level 1, value = the source's label (distance 0).
__global__ void k_gbfs_sources(const int32_t* __restrict__ src, int64_t n_src, const uint32_t* __restrict__ lo_of,
                               unsigned long long* __restrict__ X, uint32_t* __restrict__ stamp) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += stride) {
        const int32_t s = src[i];
        atomicMin(&X[s], (unsigned long long)(lo_of ? lo_of[s] : (uint32_t)s));
        stamp[s] = 1u;
    }
}

// End of a level: stop when it reached no vertex (or at the level cap, with
// the error flag), else go on with the next level.
__global__ void k_gbfs_next(GbfsState* st, uint32_t cap, cudaGraphConditionalHandle h) {
    if (st->reached == 0) {
        cudaGraphSetConditional(h, 0);
        return;
    }
    if (st->level >= cap) {
        st->error = 1;
        cudaGraphSetConditional(h, 0);
        return;
    }
    st->level += 1;
    st->reached = 0;
    cudaGraphSetConditional(h, 1);
}

int graph_grid(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

void graph_bfs_release(GraphBfs* c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    dfree(c->state);
}

int msbfs_graph(fl_graph* g, const int32_t* src_list, int64_t n_src, int32_t* label, int32_t* dist, DBuf& X,
                DBuf& stampb, int cls) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    if (!g->lists_ready) {
        FL_TRY(build_work_lists(g));
        g->lists_ready = 1;
    }
    GraphBfs* c = g->gbfs;
    FL_TRY(dalloc(X, (size_t)n * 8));
    FL_TRY(dalloc(stampb, (size_t)n * 4));
    FL_TRY(dalloc(c->state, sizeof(GbfsState)));
    unsigned long long* Xp = X.as<unsigned long long>();
    uint32_t* stamp = stampb.as<uint32_t>();
    GbfsState* state = c->state.as<GbfsState>();
    const unsigned long long add = 1ULL << 32;
    const uint32_t cap = (uint32_t)std::min<int64_t>(g->sched.level_cap > 0 ? g->sched.level_cap + 1 : n + 2,
                                                     0x7fffffff);
    // (re)build the graph when its buffers or sizes changed
    const void* key[4] = {Xp, stamp, state, g->small_list.p};
    const int64_t key_n[4] = {n, g->n_small + ((int64_t)cap << 32), g->n_mid, g->n_hubs};
    bool same = c->exec != nullptr;
    for (int i = 0; i < 4; ++i) same = same && c->key[i] == key[i] && c->key_n[i] == key_n[i];
    if (!same) {
        if (c->exec) cudaGraphExecDestroy(c->exec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->exec = nullptr;
        c->graph = nullptr;
        FL_CUDA(cudaGraphCreate(&c->graph, 0));
        cudaGraphConditionalHandle h;
        FL_CUDA(cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        FL_CUDA(cudaGraphAddNode(&node, c->graph, nullptr, nullptr, 0, &p));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        cudaStream_t cs;
        FL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            const int64_t* rowp = g->rowp.as<int64_t>();
            const int32_t* cols = g->cols.as<int32_t>();
            if (g->n_small > 0)
                k_gbfs_small<<<graph_grid(g->n_small, 256), 256, 0, cs>>>(g->small_list.as<int32_t>(), g->n_small,
                                                                          rowp, cols, Xp, stamp, state, add);
            if (g->n_mid > 0)
                k_gbfs_group<8><<<graph_grid((g->n_mid + 3) / 4, 8), 256, 0, cs>>>(
                    g->mid_list.as<int32_t>(), g->n_mid, rowp, cols, Xp, stamp, state, add);
            if (g->n_hubs > 0)
                k_gbfs_group<32><<<graph_grid(g->n_hubs, 8), 256, 0, cs>>>(g->hub_list.as<int32_t>(), g->n_hubs,
                                                                           rowp, cols, Xp, stamp, state, add);
            k_gbfs_next<<<1, 1, 0, cs>>>(state, cap, h);
            cudaGraph_t captured = body;
            e = cudaStreamEndCapture(cs, &captured);
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return status_of(e, "graph BFS capture", __FILE__, __LINE__);
        FL_CUDA(cudaGraphInstantiate(&c->exec, c->graph, 0));
        for (int i = 0; i < 4; ++i) {
            c->key[i] = key[i];
            c->key_n[i] = key_n[i];
        }
    }
    FL_CUDA(cudaMemsetAsync(Xp, 0xff, (size_t)n * 8, st));
    FL_CUDA(cudaMemsetAsync(stamp, 0, (size_t)n * 4, st));
    const GbfsState init = {2u, 0u, 0ULL, 0ULL};  // sources are level 1; the loop starts at level 2
    FL_CUDA(cudaMemcpyAsync(state, &init, sizeof(init), cudaMemcpyHostToDevice, st));
    if (n_src > 0) {
        // labels are the sources' rank ids, as in msbfs
        const uint32_t* label_of = g->rid.p ? g->rid.as<uint32_t>() : nullptr;
        FL_LAUNCH(cls, k_gbfs_sources<<<grid_for(n_src, 256), 256, 0, st>>>(src_list, n_src, label_of, Xp, stamp));
        FL_CUDA(cudaGetLastError());
        cudaError_t le = cudaSuccess;
        FL_LAUNCH(cls, le = cudaGraphLaunch(c->exec, st));
        FL_CUDA(le);
    }
    FL_LAUNCH(cls, k_unpack_bfs<<<grid_for(n, 256), 256, 0, st>>>(Xp, n, label, dist));
    FL_CUDA(cudaGetLastError());
    GbfsState out;
    FL_CUDA(cudaMemcpyAsync(&out, state, sizeof(out), cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    if (out.error) FL_FAIL(FL_ETIMEOUT, "graph BFS reached its level cap");
    return FL_OK;
}

// ------------------------------------------------------------------ radius (phase ii)

__global__ void k_check_costs(const double* __restrict__ cost, int64_t n, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        double c = cost[v];
        bool ok = (c > 0.0 && c < INFINITY) || c == INFINITY;  // rejects NaN, <= 0, -inf
        if (!ok) atomicOr(&ctr->error, 1ULL);
    }
}

// Radius of facility f with opening cost c (Eq. 1 at eps -> 0), by the
// warp: W_h = (#counted client entries of the hop-h group) x weight;
// N_j = N_{j-1} + W_j; G_{j+1} = G_j + N_j; r = j + (c - G_j) / N_j at the
// first j < L with G_{j+1} >= c, else L + (c - G_L) / N_L (L = last hop of
// the ADS of f), +inf if N_L = 0.  Every operation is one IEEE-754 op in this
// order (no contraction).  The loads are issued a row at a time: the group
// words of up to 32 groups (one per lane), then the row's entry ids and their
// client flags 32 at a time; per-group client counts come from ballots, and
// the recurrence runs on registers.  Every lane returns the same value.
__device__ double facility_radius(int64_t f, double c, int64_t io, const uint8_t* __restrict__ client,
                                  const int64_t* __restrict__ gofs, const int64_t* __restrict__ eofs,
                                  const uint32_t* __restrict__ ginfo, const double* __restrict__ gwt,
                                  const int32_t* __restrict__ eid) {
    const int lane = lane_id();
    const int64_t g0 = gofs[f], ng = gofs[f + 1] - g0;
    const int L = (int)(ginfo[g0 + ng - 1] & 0xffffu);
    int64_t e = eofs[f];
    double N = 0.0, G = 0.0;
    int j = 0;
    for (int64_t gc = 0; gc < ng; gc += 32) {
        const int m = ng - gc < 32 ? (int)(ng - gc) : 32;
        const uint32_t info = lane < m ? ginfo[g0 + gc + lane] : 0u;
        const double wt = lane < m ? gwt[g0 + gc + lane] : 0.0;
        const int cnt = (int)((info >> 16) & 0xffu);
        const int counted = (int)(info >> 24);
        const int incl = warp_incl_scan(cnt);
        const int off = incl - cnt;  // first entry of group `lane` within this chunk
        const int tot = __shfl_sync(kFull, incl, 31);
        int clients = 0;             // lane g: counted client entries of group g
        for (int p = 0; p < tot; p += 32) {
            const int pos = p + lane;
            const bool is_client = pos < tot && client[io + eid[e + pos]] != 0;
            for (int gg = 0; gg < m; ++gg) {
                const int s0 = __shfl_sync(kFull, off, gg);
                const int cc = __shfl_sync(kFull, counted, gg);
                const unsigned hit = __ballot_sync(kFull, is_client && pos >= s0 && pos < s0 + cc);
                if (lane == gg) clients += __popc(hit);
            }
        }
        for (int gg = 0; gg < m; ++gg) {
            const int hop = (int)(__shfl_sync(kFull, info, gg) & 0xffffu);
            const int cl = __shfl_sync(kFull, clients, gg);
            const double w = __shfl_sync(kFull, wt, gg);
            for (; j < hop; ++j) {  // hops without new entries: W_j = 0
                if (j < L) {
                    const double Gn = __dadd_rn(G, N);
                    if (Gn >= c) return __dadd_rn((double)j, __ddiv_rn(__dsub_rn(c, G), N));
                    G = Gn;
                }
            }
            N = __dadd_rn(N, __dmul_rn((double)cl, w));
            if (j < L) {
                const double Gn = __dadd_rn(G, N);
                if (Gn >= c) return __dadd_rn((double)j, __ddiv_rn(__dsub_rn(c, G), N));
                G = Gn;
            }
            ++j;
        }
        e += tot;
    }
    return N > 0.0 ? __dadd_rn((double)L, __ddiv_rn(__dsub_rn(c, G), N)) : INFINITY;
}

// A warp per 32 consecutive vertices: one ballot finds the facilities (finite
// cost), the others get +inf, and the warp computes each facility's radius in
// turn.
//
// R > 1 (batches on one resident graph): R instances, instance i's costs,
// client mask and radii at offset i*n; the warps of one vertex block's R
// instances are adjacent, so its ADS rows are read from DRAM once.
template <bool kMulti>
__global__ void __launch_bounds__(256) k_radius(int64_t n, int64_t R, const double* __restrict__ cost,
                                                const uint8_t* __restrict__ client,
                                                const int64_t* __restrict__ gofs, const int64_t* __restrict__ eofs,
                                                const uint32_t* __restrict__ ginfo, const double* __restrict__ gwt,
                                                const int32_t* __restrict__ eid, double* __restrict__ r_out) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nb = (n + 31) >> 5;
    for (int64_t t = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; t < nb * R; t += warps) {
        const int64_t blk = kMulti ? t / R : t;
        const int64_t io = kMulti ? (t - blk * R) * n : 0;  // instance offset
        const int64_t v = (blk << 5) + lane;
        const double cv = v < n ? cost[io + v] : INFINITY;
        unsigned fac = __ballot_sync(kFull, cv < INFINITY);
        double rv = INFINITY;
        while (fac) {
            const int b = __ffs(fac) - 1;
            fac &= fac - 1;
            const double c = __shfl_sync(kFull, cv, b);
            const double res = facility_radius((blk << 5) + b, c, io, client, gofs, eofs, ginfo, gwt, eid);
            if (lane == b) rv = res;
        }
        if (v < n) r_out[io + v] = rv;
    }
}

// The solve's opening costs are finite and > 0, or +inf (not a facility).
int check_costs(fl_solve* s) {
    fl_graph* g = s->g;
    cudaStream_t st = g->stream;
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(kProfRadius, k_check_costs<<<grid_for(g->n, 256), 256, 0, st>>>(s->cost.as<double>(), g->n, g->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    if (g->h_ctr->error) FL_FAIL(FL_EINVAL, "open_cost must be finite and > 0 for facilities, +inf otherwise");
    return FL_OK;
}

int compute_radii(fl_solve* s) {
    fl_graph* g = s->g;
    cudaStream_t st = g->stream;
    FL_TRY(check_costs(s));
    FL_LAUNCH(kProfRadius, k_radius<false><<<grid_for((g->n + 31) / 32, 8), 256, 0, st>>>(g->n, 1, s->cost.as<double>(), s->client.as<uint8_t>(),
                                               g->gofs.as<int64_t>(), g->eofs.as<int64_t>(), g->ginfo.as<uint32_t>(),
                                               g->gwt.as<double>(), g->eid.as<int32_t>(), s->radii.as<double>()));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

// Radii of R instances on the built graph src (batches): cost, client and
// radii are R*n arrays, instance-major.  Runs on g's stream with g's
// counters (src is only read).
int compute_radii_multi(const fl_graph* src, fl_graph* g, int64_t R, const double* cost, const uint8_t* client,
                        double* radii) {
    cudaStream_t st = g->stream;
    const int64_t n = src->n;
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(kProfRadius, k_check_costs<<<grid_for(n * R, 256), 256, 0, st>>>(cost, n * R, g->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    if (g->h_ctr->error) FL_FAIL(FL_EINVAL, "open_cost must be finite and > 0 for facilities, +inf otherwise");
    FL_LAUNCH(kProfRadius, k_radius<true><<<grid_for((n + 31) / 32 * R, 8), 256, 0, st>>>(
                               n, R, cost, client, src->gofs.as<int64_t>(), src->eofs.as<int64_t>(),
                               src->ginfo.as<uint32_t>(), src->gwt.as<double>(), src->eid.as<int32_t>(), radii));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

// ------------------------------------------------------------------ keys (r_f, pi_f)

__global__ void k_candidates(const double* __restrict__ r, int64_t n, uint64_t seed,
                             IdMap ids, uint64_t* __restrict__ hi,
                             uint64_t* __restrict__ lo, uint32_t* __restrict__ val, uint8_t* __restrict__ state,
                             Counters* ctr) {
    // which key bits vary: OR of the words and of their complements, per
    // block in shared memory, then one global OR per block
    __shared__ unsigned long long bits[4];
    if (threadIdx.x < 4) bits[threadIdx.x] = 0;
    __syncthreads();
    __shared__ BlockAppend<8> sh;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < n; bb += stride) {
        int64_t f = bb + threadIdx.x;
        bool cand = false;
        double rf = 0.0;
        if (f < n) {
            rf = r[f];
            cand = rf < INFINITY;
            state[f] = cand ? 0 : 3;
        }
        long long at = block_append<8>(cand, &ctr->aux0, sh);
        const uint64_t h = cand ? (uint64_t)__double_as_longlong(rf) : 0;  // r >= 0: bit order = numeric order
        const uint64_t l = cand ? facility_priority(seed, rank_id(ids, f)) : 0;
        if (at >= 0) {
            hi[at] = h;
            lo[at] = l;
            val[at] = (uint32_t)f;
        }
        if (__ballot_sync(kFull, cand)) {
            const uint64_t hn = cand ? ~h : 0, ln = cand ? ~l : 0;
            uint64_t w[4] = {h, l, hn, ln};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned a = __reduce_or_sync(kFull, (unsigned)w[q]);
                const unsigned b = __reduce_or_sync(kFull, (unsigned)(w[q] >> 32));
                w[q] = ((uint64_t)b << 32) | a;
            }
            if (lane_id() == 0)
                for (int q = 0; q < 4; ++q)
                    if (w[q] & ~bits[q]) atomicOr(&bits[q], (unsigned long long)w[q]);
        }
    }
    __syncthreads();
    if (threadIdx.x < 4 && bits[threadIdx.x]) {
        unsigned long long* dst = threadIdx.x < 2 ? &ctr->key_or[threadIdx.x] : &ctr->key_orn[threadIdx.x - 2];
        atomicOr(dst, bits[threadIdx.x]);
    }
}

// Any two adjacent equal hi words (radius ties) after sorting by hi.
__global__ void k_key_ties(const uint64_t* __restrict__ hi, int64_t m, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool tie = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < m; i += stride)
        tie |= hi[i] == hi[i + 1];
    if (__any_sync(kFull, tie) && lane_id() == 0) atomicOr(&ctr->key_ties, 1ULL);
}

// Nibble digits (bit p: pass p of sort_pairs_u128_digits) of the key bits
// that vary between candidates.
static uint32_t varying_digits(const Counters& c) {
    uint32_t d = 0;
    for (int w = 0; w < 2; ++w) {
        const uint64_t var = c.key_or[w] & c.key_orn[w];
        for (int q = 0; q < 16; ++q)
            if ((var >> (4 * q)) & 15u) d |= 1u << (q + (w == 0 ? 16 : 0));
    }
    return d;
}

__global__ void k_ordinals(const uint32_t* __restrict__ sorted_f, int64_t m, const double* __restrict__ r,
                           const int32_t* __restrict__ ecc_ub, uint32_t* __restrict__ ord,
                           int32_t* __restrict__ fac_by_ord, int32_t* __restrict__ bcap, int32_t* __restrict__ ulist,
                           unsigned long long* __restrict__ bmax) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int32_t mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        int32_t f = (int32_t)sorted_f[i];
        ord[f] = (uint32_t)i;
        fac_by_ord[i] = f;
        ulist[i] = f;
        // ball radius floor(r_f), capped by an eccentricity bound (same ball)
        double fl = floor(r[f]);
        int32_t cap = ecc_ub[f];
        int32_t b = fl >= (double)cap ? cap : (int32_t)fl;
        bcap[f] = b;
        mx = max(mx, b);
    }
    // the largest ball radius: one atomic per warp
    mx = (int32_t)__reduce_max_sync(kFull, (unsigned)mx);
    if (lane_id() == 0 && mx > 0) atomicMax(bmax, (unsigned long long)mx);
}

// ------------------------------------------------------------------ MIS rounds (phase iii)

// Bucket sizes by ball radius, the largest radius, and (for a graph made of
// parts) each part's largest radius; maxima reduced per warp first.
__global__ void k_bucket_count(const int32_t* __restrict__ ulist, int64_t n_u, const int32_t* __restrict__ bcap,
                               int32_t* __restrict__ bcount, unsigned long long* __restrict__ tmax,
                               const int32_t* __restrict__ vpart, int32_t* __restrict__ part_T) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_u; base += stride) {
        const int64_t i = base + lane_id();
        const bool valid = i < n_u;
        const int32_t f = valid ? ulist[i] : 0;
        const int32_t b = valid ? bcap[f] : 0;
        const unsigned sameb = __match_any_sync(kFull, valid ? b : -1);  // one atomic per bucket and warp
        if (valid && lane_id() == __ffs(sameb) - 1) atomicAdd(&bcount[b], __popc(sameb));
        const unsigned mx = __reduce_max_sync(kFull, (unsigned)b);
        if (lane_id() == 0) atomicMax(tmax, (unsigned long long)mx);
        if (vpart) {
            const int32_t p = valid ? vpart[f] : -1;
            const unsigned same = __match_any_sync(kFull, p);
            const unsigned pm = __reduce_max_sync(same, (unsigned)b);
            if (valid && lane_id() == __ffs(same) - 1) atomicMax(&part_T[p], (int)pm);
        }
    }
}

// Facilities to their bucket's range; the lanes of a warp with the same
// bucket take consecutive places with one atomic.
__global__ void k_bucket_scatter(const int32_t* __restrict__ ulist, int64_t n_u, const int32_t* __restrict__ bcap,
                                 int32_t* __restrict__ cursor, int32_t* __restrict__ ubuck) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = lane_id();
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_u; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < n_u;
        const int32_t f = valid ? ulist[i] : 0;
        const int32_t b = valid ? bcap[f] : -1;
        const unsigned same = __match_any_sync(kFull, b);
        const int lead = __ffs(same) - 1;
        int at = 0;
        if (valid && lane == lead) at = atomicAdd(&cursor[b], __popc(same));
        at = __shfl_sync(kFull, at, lead);
        if (valid) ubuck[at + __popc(same & ((1u << lane) - 1u))] = f;
    }
}

// Gather seeds: every client covered in this round's cover sweep starts with
// 0 if already claimed, else 1 + (smallest key of an undecided facility
// covering it); mval keeps that smallest key for the claim step.
__global__ void k_gather_seed(const int32_t* __restrict__ touched, const unsigned long long* __restrict__ n_touched,
                              const uint8_t* __restrict__ client, const uint8_t* __restrict__ claimed,
                              unsigned long long hi, unsigned long long* __restrict__ X, uint32_t* __restrict__ mval,
                              uint32_t* __restrict__ stamp, uint32_t sv, int32_t* __restrict__ fr,
                              unsigned long long* __restrict__ n_fr) {
    __shared__ BlockAppend<8> sh;
    const int64_t n = (int64_t)*n_touched;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < n; bb += stride) {
        int64_t i = bb + threadIdx.x;
        bool seed = false;
        int32_t v = 0;
        if (i < n) {
            v = touched[i];
            if (client[v]) {
                uint32_t m = (uint32_t)(X[v] & 0xffffffffULL);
                mval[v] = m;
                X[v] = (hi << 32) | (claimed[v] ? 0ULL : (unsigned long long)m + 1ULL);
                stamp[v] = sv;
                seed = true;
            }
        }
        long long at = block_append<8>(seed, n_fr, sh);
        if (at >= 0) fr[at] = v;
    }
}

// Facilities whose ball radius is b read the minimum over their ball after
// b gather rounds: 0 -> a client of the ball is claimed (dead); own key + 1
// -> smallest key among all conflicting undecided facilities (joins S).
__global__ void k_decide(const int32_t* __restrict__ fl, int64_t m, const unsigned long long* __restrict__ X,
                         unsigned long long hi, const uint32_t* __restrict__ ord, uint8_t* __restrict__ state,
                         Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        int32_t f = fl[i];
        unsigned long long x = X[f];
        if ((x >> 32) != hi) {
            atomicOr(&ctr->error, 8ULL);  // a candidate's ball holds no client (cannot happen)
            continue;
        }
        uint32_t lo = (uint32_t)(x & 0xffffffffULL);
        if (lo == 0) state[f] = 2;
        else if (lo == ord[f] + 1u) state[f] = 1;
    }
}

// Clients of this round's winners' balls become claimed; with `kr`, each
// newly claimed client is a seed (kr = 1) of the round's kill sweep, and
// *n_new counts them.
__global__ void k_claim(const int32_t* __restrict__ touched, const unsigned long long* __restrict__ n_touched,
                        const uint8_t* __restrict__ client, uint8_t* __restrict__ claimed,
                        const uint32_t* __restrict__ mval, const int32_t* __restrict__ fac_by_ord,
                        const uint8_t* __restrict__ state, uint8_t* __restrict__ kr,
                        unsigned long long* __restrict__ n_new) {
    const int64_t n = (int64_t)*n_touched;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long fresh = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t i = base + lane_id();
        bool now = false;
        if (i < n) {
            const int32_t v = touched[i];
            if (client[v] && !claimed[v] && state[fac_by_ord[mval[v]]] == 1) {
                claimed[v] = 1;
                if (kr) kr[v] = 1;
                now = true;
            }
        }
        fresh += __popc(__ballot_sync(kFull, now));
    }
    if (lane_id() == 0 && fresh) atomicAdd(n_new, fresh);
}

// Kill sweep decision: an undecided facility with a client claimed in this
// round within its ball radius (kr[f] = 1 + that distance <= B_f + 1) can no
// longer join S.
__global__ void k_kill(const int32_t* __restrict__ ulist, int64_t n_u, const uint8_t* __restrict__ kr,
                       const int32_t* __restrict__ bcap, uint8_t* __restrict__ state) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_u; i += stride) {
        const int32_t f = ulist[i];
        const uint32_t k = kr[f];
        if (k != 0 && (int64_t)k <= (int64_t)bcap[f] + 1) state[f] = 2;
    }
}

__global__ void k_compact_undecided(const int32_t* __restrict__ ulist, int64_t n_u, const uint8_t* __restrict__ state,
                                    int32_t* __restrict__ out, unsigned long long* __restrict__ n_out) {
    __shared__ BlockAppend<8> sh;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < n_u; bb += stride) {
        int64_t i = bb + threadIdx.x;
        int32_t f = i < n_u ? ulist[i] : 0;
        bool keep = i < n_u && state[f] == 0;
        long long at = block_append<8>(keep, n_out, sh);
        if (at >= 0) out[at] = f;
    }
}

__global__ void k_open_list(const uint8_t* __restrict__ state, int64_t n, uint8_t* __restrict__ open,
                            int32_t* __restrict__ list, unsigned long long* __restrict__ n_list) {
    __shared__ BlockAppend<8> sh;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < n; bb += stride) {
        int64_t v = bb + threadIdx.x;
        bool is_open = v < n && state[v] == 1;
        if (v < n) open[v] = is_open ? 1 : 0;
        long long at = block_append<8>(is_open, n_list, sh);
        if (at >= 0) list[at] = (int32_t)v;
    }
}

// Candidates (finite r_f) sorted by the key (r_f, pi_f): s->key_val holds
// their ids in key order, s->state is 0 for a candidate and 3 otherwise.
int sort_candidates(fl_solve* s, int64_t* m_out) {
    fl_graph* g = s->g;
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    FL_TRY(dalloc(s->state, (size_t)n));
    DBuf& hi = s->key_hi;
    DBuf& lo = s->key_lo;
    DBuf& val = s->key_val;
    FL_TRY(dalloc(hi, (size_t)n * 8));
    FL_TRY(dalloc(lo, (size_t)n * 8));
    FL_TRY(dalloc(val, (size_t)n * 4));
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(kProfKeys, k_candidates<<<grid_for(n, 256), 256, 0, st>>>(s->radii.as<double>(), n, g->seed,
                                                   idmap_of(g), hi.as<uint64_t>(),
                                                   lo.as<uint64_t>(), val.as<uint32_t>(), s->state.as<uint8_t>(),
                                                   g->ctr.as<Counters>()));
    FL_TRY(read_counters(g));
    const int64_t m = (int64_t)g->h_ctr->aux0;
    s->n_cand = m;
    // Keys (r_f, pi_f): sort by r_f's varying digits; only when two radii are
    // equal does the order need pi_f, and then the keys are sorted again by
    // every varying digit (least significant first, so the result is the
    // order of the whole 128-bit key).
    const uint32_t digits = varying_digits(*g->h_ctr);
    FL_TRY(sort_pairs_u128_digits(hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>(), m, st, g->scratch,
                                  kProfKeys, digits & 0xffff0000u));
    if (m > 1) {
        FL_LAUNCH(kProfKeys, k_key_ties<<<grid_for(m, 256), 256, 0, st>>>(hi.as<uint64_t>(), m, g->ctr.as<Counters>()));
        FL_TRY(read_counters(g));
        if (g->h_ctr->key_ties)
            FL_TRY(sort_pairs_u128_digits(hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>(), m, st, g->scratch,
                                          kProfKeys, digits));
    }
    *m_out = m;
    return FL_OK;
}

int open_facilities(fl_solve* s) {
    fl_graph* g = s->g;
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    // -------- keys: candidates sorted by (r_f, pi_f) -> ordinals
    FL_TRY(dalloc(s->ord, (size_t)n * 4));
    FL_TRY(dalloc(s->fac_by_ord, (size_t)n * 4));
    FL_TRY(dalloc(s->bcap, (size_t)n * 4));
    FL_TRY(dalloc(s->state, (size_t)n));
    FL_TRY(dalloc(s->claimed, (size_t)n));
    FL_TRY(dalloc(s->X, (size_t)n * 16));          // two value buffers
    FL_TRY(dalloc(s->stamp, (size_t)n * 4));
    FL_TRY(dalloc(s->mval, (size_t)n * 4));
    FL_TRY(dalloc(s->fr[0], (size_t)n * 4));
    FL_TRY(dalloc(s->fr[1], (size_t)n * 4));
    FL_TRY(dalloc(s->frval, (size_t)n * 8 + 64));
    FL_TRY(dalloc(s->touched, (size_t)n * 4));
    FL_TRY(dalloc(s->ulist, (size_t)n * 4 * 2));
    FL_TRY(dalloc(s->ubuck, (size_t)n * 4));
    FL_TRY(dalloc(s->open, (size_t)n));
    FL_TRY(dalloc(s->reach, (size_t)n));
    FL_TRY(dalloc(s->kill, (size_t)n));
    s->mis_log.clear();
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(s->frval.as<char>() + (size_t)n * 8);
    // cnt[0], cnt[1]: frontier counts; cnt[2]: changed count (dense rounds);
    // cnt[3]: undecided; cnt[4]: T max; cnt[5]: open list; cnt[6]: touched
    // solve-owned, grow-only scratch: a cudaFree per solve would synchronise
    // the whole device (and stall other solves running on other streams)
    int64_t m = 0;
    FL_TRY(sort_candidates(s, &m));
    DBuf& val = s->key_val;
    int32_t* ulist[2] = {s->ulist.as<int32_t>(), s->ulist.as<int32_t>() + n};
    FL_CUDA(cudaMemsetAsync(cnt, 0, 64, st));
    if (m > 0) {
        FL_LAUNCH(kProfKeys, k_ordinals<<<grid_for(m, 256), 256, 0, st>>>(val.as<uint32_t>(), m, s->radii.as<double>(),
                                                     g->ecc_ub.as<int32_t>(), s->ord.as<uint32_t>(),
                                                     s->fac_by_ord.as<int32_t>(), s->bcap.as<int32_t>(), ulist[0],
                                                     &cnt[4]));
    }
    FL_CUDA(cudaGetLastError());
    unsigned long long bmax = 0;
    FL_CUDA(cudaMemcpyAsync(&bmax, &cnt[4], 8, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaMemsetAsync(s->claimed.p, 0, (size_t)n, st));
    FL_CUDA(cudaMemsetAsync(s->X.p, 0xff, (size_t)n * 16, st));
    FL_CUDA(cudaMemsetAsync(s->stamp.p, 0, (size_t)n * 4, st));
    FL_CUDA(cudaStreamSynchronize(st));
    DBuf& bcount_d = s->bcount;
    FL_TRY(dalloc(bcount_d, (bmax + 2) * 4 * 2));
    int32_t* bcount = bcount_d.as<int32_t>();
    int32_t* cursor = bcount + (bmax + 2);
    std::vector<int32_t> hcount(bmax + 2), hoff(bmax + 2);

    Relax r;
    r.X[0] = s->X.as<unsigned long long>();
    r.X[1] = r.X[0] + n;
    r.fr[0] = s->fr[0].as<int32_t>();
    r.fr[1] = s->fr[1].as<int32_t>();
    r.frval = s->frval.as<unsigned long long>();
    r.stamp = s->stamp.as<uint32_t>();
    r.cnt = cnt;
    r.h_cnt = &g->h_ctr->aux3;
    FL_TRY(relax_begin(g, r));
    // a graph made of parts (batches): each part's gather sweep stops after
    // its own largest ball radius
    const int32_t* vpart = g->n_parts > 0 ? g->vpart.as<int32_t>() : nullptr;
    int32_t* part_T = nullptr;
    if (vpart) {
        FL_TRY(dalloc(s->part_T, (size_t)g->n_parts * 4));
        part_T = s->part_T.as<int32_t>();
    }
    int32_t* touched = s->touched.as<int32_t>();
    uint8_t* reach = s->reach.as<uint8_t>();
    uint8_t* kill = s->kill.as<uint8_t>();
    // rows of the round log: (greedy round, kind, step, frontier in, pulled, microseconds);
    // kind 0 cover round, 1 gather round, 2 bucket size (step = ball radius), 3 greedy-round total,
    // 4 kill-sweep round (frontier = marks made)
    using clock = std::chrono::steady_clock;
    auto log_row = [&](int64_t rd, int64_t kind, int64_t step, int64_t front, int64_t dense, double us) {
        const int64_t row[6] = {rd, kind, step, front, dense, (int64_t)us};
        s->mis_log.insert(s->mis_log.end(), row, row + 6);
    };
    auto timed_round = [&](int64_t rd, int64_t kind, int64_t step, uint32_t svr) -> int {
        const int64_t front = r.n_front;
        const auto t0 = clock::now();
        FL_TRY(relax_round(g, r, 0ULL, svr, kProfMis));
        log_row(rd, kind, step, front, r.last_dense ? 1 : 0,
                std::chrono::duration<double, std::micro>(clock::now() - t0).count());
        return FL_OK;
    };
    uint32_t epoch = 0;
    uint32_t sv = 0;  // frontier stamp values, unique per round
    int64_t n_u = m;
    int cu = 0;
    int64_t rounds = 0;
    while (n_u > 0) {
        if (++rounds > m + 1) FL_FAIL(FL_ETIMEOUT, "greedy MIS did not converge");
        const auto round_t0 = clock::now();
        // bucket the undecided facilities by ball radius
        FL_CUDA(cudaMemsetAsync(bcount, 0, (bmax + 1) * 4, st));
        FL_CUDA(cudaMemsetAsync(&cnt[4], 0, 8, st));
        if (part_T) FL_CUDA(cudaMemsetAsync(part_T, 0xff, (size_t)g->n_parts * 4, st));  // -1: no undecided facility
        FL_LAUNCH(kProfMis, k_bucket_count<<<grid_for(n_u, 256), 256, 0, st>>>(
                                ulist[cu], n_u, s->bcap.as<int32_t>(), bcount, &cnt[4], vpart, part_T));
        FL_CUDA(cudaGetLastError());
        unsigned long long T64 = 0;
        FL_CUDA(cudaMemcpyAsync(&T64, &cnt[4], 8, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaMemcpyAsync(hcount.data(), bcount, (bmax + 1) * 4, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaStreamSynchronize(st));
        const int T = (int)T64;
        int32_t acc = 0;
        for (int b = 0; b <= T; ++b) {
            hoff[b] = acc;
            acc += hcount[b];
            if (hcount[b] > 0) log_row(rounds, 2, b, hcount[b], 0, 0.0);
        }
        // Gather pruning: the cover records reach = 1 + max_f (B_f - d(v, f))
        // (T minus the time its first wave arrived); gather round b needs only
        // vertices with B_f - d(v, f) >= b for some f, the others sit out.
        const bool prune = T < 255;
        if (prune) FL_CUDA(cudaMemsetAsync(reach, 0, (size_t)n, st));
        FL_CUDA(cudaMemcpyAsync(cursor, hoff.data(), (T + 1) * 4, cudaMemcpyHostToDevice, st));
        FL_LAUNCH(kProfMis, k_bucket_scatter<<<grid_for(n_u, 256), 256, 0, st>>>(
                                ulist[cu], n_u, s->bcap.as<int32_t>(), cursor, s->ubuck.as<int32_t>()));
        FL_CUDA(cudaGetLastError());
        const int32_t* ub = s->ubuck.as<int32_t>();

        // ---- cover: X[c] = smallest key of an undecided f with d(c, f) <= B_f.
        // Facility f starts at time T - B_f; all waves stop at time T.
        ++epoch;
        const unsigned long long hi_c = 0xffffffffULL - epoch;
        r.limit = (hi_c + 1) << 32;
        FL_CUDA(cudaMemsetAsync(cnt, 0, 24, st));
        r.n_front = 0;
        r.list_valid = true;
        const uint32_t sv0 = sv;
        r.sv_prev = sv0 + 1;
        r.prune = Prune();
        r.prune.reach = prune ? reach : nullptr;
        for (int t = 0; t <= T; ++t) {
            const int b = T - t;
            if (hcount[b] > 0) {
                FL_TRY(relax_prepare_list(g, r, kProfMis));
                FL_LAUNCH(kProfMis, k_inject<<<grid_for(hcount[b], 256), 256, 0, st>>>(
                                        ub + hoff[b], hcount[b], r.prune.reach, (uint32_t)b + 1u, r.limit, hi_c,
                                        s->ord.as<uint32_t>(), r.X[r.cur], r.stamp, sv0 + 1 + t, r.fr[r.fc],
                                        &r.cnt[r.fc]));
                FL_CUDA(cudaGetLastError());
                r.n_front += hcount[b];
            }
            r.prune.reach_val = (uint32_t)(T - t);  // first reached at time t + 1
            // the last round: nothing relays a value past time T, and of the
            // values at time T only the clients' are read (gather seeds and
            // claims), so the other vertices sit it out (left unreached, they
            // have the same effect on the gather and kill sweeps as slack 0)
            r.prune.only = (prune && t == T - 1) ? s->client.as<uint8_t>() : nullptr;
            if (t < T && r.n_front > 0) FL_TRY(timed_round(rounds, 0, t, sv0 + 2 + t));
            else if (t < T) r.sv_prev = sv0 + 2 + t;
        }
        r.prune = Prune();
        sv = sv0 + T + 2;
        // every vertex the cover reached (its value carries this sweep's epoch)
        FL_TRY(relax_collect_epoch(g, r.X[r.cur], hi_c, touched, &cnt[6], kProfMis));

        // ---- gather: min over Ball(f) of (claimed ? 0 : cover + 1), read at radius B_f
        ++epoch;
        const unsigned long long hi_g = 0xffffffffULL - epoch;
        r.limit = (hi_g + 1) << 32;
        FL_CUDA(cudaMemsetAsync(cnt, 0, 24, st));
        r.fc = 0;
        const uint32_t sg0 = ++sv;
        FL_LAUNCH(kProfMis, k_gather_seed<<<152 * 2, 256, 0, st>>>(touched, &cnt[6], s->client.as<uint8_t>(),
                                                                   s->claimed.as<uint8_t>(), hi_g, r.X[r.cur],
                                                                   s->mval.as<uint32_t>(), r.stamp, sg0, r.fr[0],
                                                                   &r.cnt[0]));
        FL_CUDA(cudaGetLastError());
        FL_CUDA(cudaMemcpyAsync(r.h_cnt, &r.cnt[0], 8, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaStreamSynchronize(st));
        r.n_front = (int64_t)*r.h_cnt;
        r.list_valid = true;
        r.sv_prev = sg0;
        if (hcount[0] > 0)
            FL_LAUNCH(kProfMis, k_decide<<<grid_for(hcount[0], 256), 256, 0, st>>>(
                                    ub + hoff[0], hcount[0], r.X[r.cur], hi_g, s->ord.as<uint32_t>(),
                                    s->state.as<uint8_t>(), g->ctr.as<Counters>()));
        r.part_limit = part_T;
        r.prune.need = prune ? reach : nullptr;
        for (int b = 1; b <= T; ++b) {
            r.part_round = b;
            r.prune.round = (uint32_t)b;
            if (r.n_front > 0) FL_TRY(timed_round(rounds, 1, b, sg0 + b));
            else r.sv_prev = sg0 + b;
            if (hcount[b] > 0)
                FL_LAUNCH(kProfMis, k_decide<<<grid_for(hcount[b], 256), 256, 0, st>>>(
                                        ub + hoff[b], hcount[b], r.X[r.cur], hi_g, s->ord.as<uint32_t>(),
                                        s->state.as<uint8_t>(), g->ctr.as<Counters>()));
        }
        sv = sg0 + T + 1;
        r.part_limit = nullptr;
        r.prune = Prune();
        FL_CUDA(cudaGetLastError());

        // ---- claim the balls of this round's winners; keep the undecided
        if (prune) FL_CUDA(cudaMemsetAsync(kill, 0, (size_t)n, st));
        FL_CUDA(cudaMemsetAsync(&cnt[7], 0, 8, st));
        FL_LAUNCH(kProfMis, k_claim<<<152 * 4, 256, 0, st>>>(s->touched.as<int32_t>(), &cnt[6], s->client.as<uint8_t>(),
                                         s->claimed.as<uint8_t>(), s->mval.as<uint32_t>(),
                                         s->fac_by_ord.as<int32_t>(), s->state.as<uint8_t>(),
                                         prune ? kill : nullptr, &cnt[7]));
        FL_CUDA(cudaMemsetAsync(&cnt[3], 0, 8, st));
        FL_LAUNCH(kProfMis, k_compact_undecided<<<grid_for(n_u, 256), 256, 0, st>>>(ulist[cu], n_u, s->state.as<uint8_t>(),
                                                               ulist[cu ^ 1], &cnt[3]));
        FL_CUDA(cudaGetLastError());
        unsigned long long nu = 0, n_claimed = 0;
        FL_CUDA(cudaMemcpyAsync(&nu, &cnt[3], 8, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaMemcpyAsync(&n_claimed, &cnt[7], 8, cudaMemcpyDeviceToHost, st));
        FL_TRY(read_counters(g));
        if (g->h_ctr->error) FL_FAIL(FL_ECUDA, "greedy MIS: inconsistent gather state");
        cu ^= 1;
        // ---- kill sweep: an undecided facility whose ball holds a client
        // claimed in this round is adjacent in H-bar to a facility of S and
        // can never join it.  The next round's gather would find the claim
        // too, but only after a cover sweep in which the dead facility still
        // competes; removing it now lets its neighbours decide a round earlier
        // (the result stays the lexicographically-first MIS).  A bounded
        // marking BFS from the newly claimed clients, pruned like the gather.
        if (prune && nu > 0 && n_claimed > 0) {
            for (int b = 1; b <= T; ++b) {
                const auto t0 = clock::now();
                int64_t marked = 0;
                FL_TRY(mark_round(g, r, kill, reach, (uint32_t)b, kProfMis, &marked));
                log_row(rounds, 4, b, marked, 1, std::chrono::duration<double, std::micro>(clock::now() - t0).count());
                if (marked == 0) break;
            }
            FL_LAUNCH(kProfMis, k_kill<<<grid_for((int64_t)nu, 256), 256, 0, st>>>(ulist[cu], (int64_t)nu, kill,
                                                                                  s->bcap.as<int32_t>(),
                                                                                  s->state.as<uint8_t>()));
            FL_CUDA(cudaMemsetAsync(&cnt[3], 0, 8, st));
            FL_LAUNCH(kProfMis, k_compact_undecided<<<grid_for((int64_t)nu, 256), 256, 0, st>>>(
                                    ulist[cu], (int64_t)nu, s->state.as<uint8_t>(), ulist[cu ^ 1], &cnt[3]));
            FL_CUDA(cudaGetLastError());
            FL_CUDA(cudaMemcpyAsync(&nu, &cnt[3], 8, cudaMemcpyDeviceToHost, st));
            FL_CUDA(cudaStreamSynchronize(st));
            cu ^= 1;
        }
        log_row(rounds, 3, T, n_u, n_u - (int64_t)nu,
                std::chrono::duration<double, std::micro>(clock::now() - round_t0).count());
        n_u = (int64_t)nu;
    }
    s->mis_rounds = rounds;
    // open set
    FL_CUDA(cudaMemsetAsync(&cnt[5], 0, 8, st));
    FL_LAUNCH(kProfMis, k_open_list<<<grid_for(n, 256), 256, 0, st>>>(s->state.as<uint8_t>(), n, s->open.as<uint8_t>(),
                                                  s->ulist.as<int32_t>(), &cnt[5]));
    FL_CUDA(cudaGetLastError());
    unsigned long long no = 0;
    FL_CUDA(cudaMemcpyAsync(&no, &cnt[5], 8, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    s->n_open = (int64_t)no;
    return FL_OK;
}

// ------------------------------------------------------------------ assignment + objective

int assign_clients(fl_solve* s) {
    fl_graph* g = s->g;
    FL_TRY(dalloc(s->assign, (size_t)g->n * 4));
    FL_TRY(dalloc(s->dist, (size_t)g->n * 4));
    // the open list was left in ulist by open_facilities
    if (g->sched.graph_bfs)
        return msbfs_graph(g, s->ulist.as<int32_t>(), s->n_open, s->assign.as<int32_t>(), s->dist.as<int32_t>(),
                           s->X, s->stamp, kProfBfs);
    return msbfs(g, s->ulist.as<int32_t>(), s->n_open, s->assign.as<int32_t>(), s->dist.as<int32_t>(), s->X,
                 s->stamp, s->fr, s->frval, kProfBfs);
}

constexpr int kObjBlocks = 152 * 4;

__global__ void k_objective(int64_t n, const uint8_t* __restrict__ open, const double* __restrict__ cost,
                            const uint8_t* __restrict__ client, const int32_t* __restrict__ dist,
                            double* __restrict__ partial, unsigned long long* __restrict__ sums) {
    __shared__ double red[256];
    double acc = 0.0;
    unsigned long long ds = 0, un = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (open[v]) acc += cost[v];
        if (client[v]) {
            int32_t d = dist[v];
            if (d < 0) ++un; else ds += (unsigned long long)d;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if ((int)threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (ds) atomicAdd(&sums[0], ds);
    if (un) atomicAdd(&sums[1], un);
}

int objective(fl_solve* s, double* obj, int64_t* dist_sum, int64_t* n_unserved) {
    fl_graph* g = s->g;
    cudaStream_t st = g->stream;
    DBuf& tmp = s->obj_tmp;
    FL_TRY(dalloc(tmp, kObjBlocks * 8 + 64));
    double* partial = tmp.as<double>();
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(partial + kObjBlocks);
    int rc = FL_OK;
    std::vector<double> hp(kObjBlocks);
    unsigned long long hs[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(sums, 0, 16, st);
    if (e == cudaSuccess) {
        FL_LAUNCH(kProfOther, k_objective<<<kObjBlocks, 256, 0, st>>>(g->n, s->open.as<uint8_t>(), s->cost.as<double>(),
                                                s->client.as<uint8_t>(), s->dist.as<int32_t>(), partial, sums));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), partial, kObjBlocks * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sums, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = status_of(e, "objective", __FILE__, __LINE__);

    if (rc) return rc;
    double open_cost = 0.0;
    for (int b = 0; b < kObjBlocks; ++b) open_cost += hp[b];
    *obj = open_cost + (double)hs[0];
    *dist_sum = (int64_t)hs[0];
    *n_unserved = (int64_t)hs[1];
    return FL_OK;
}

}  // namespace fl
