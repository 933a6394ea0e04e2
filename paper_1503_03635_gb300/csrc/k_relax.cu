// k_relax.cu -- synchronous min-propagation rounds over the CSR, used by the
// multi-source BFS (assignment, eccentricity bound) and by the cover / gather
// sweeps of the greedy MIS ("send to all vertices within distance d", §4.5).
//
// One round: every vertex v takes X'[v] = min(X[v], min_{u in N(v)} X[u] + add),
// reading only values of the previous round, so a value moves exactly one hop
// per round.  Only the frontier (the vertices whose value changed in the
// previous round) can lower a value.  Push rounds walk the frontier list
// (k_snap_front + k_push_low / k_push_segs, in place on one buffer, the
// frontier's values snapshotted first); pull rounds write the second buffer
// (every vertex reads its frontier neighbours, found in a bitmap; no atomics
// except per hub segment) and flag changed vertices with the next round's
// stamp.  Hub edge lists are split into kSeg-edge segments in both.
#include <algorithm>
#include <cstdio>

#include "fl_internal.cuh"

namespace fl {

namespace {

int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

__device__ __forceinline__ bool in_front(const uint32_t* __restrict__ bm, int32_t u) {
    return (__ldg(&bm[u >> 5]) >> (u & 31)) & 1u;
}


// Frontier bitmap of a pull round: bit v = (stamp[v] == sv).  Only neighbours
// whose value changed in the previous round can lower a value, so a pull
// reads the value of a neighbour only when its bit is set; the bitmap (n/8
// bytes) stays in L2 while the values do not.
//
// In a graph made of disjoint parts (batches) the frontier is also counted
// per part: a part without frontier vertices has no vertex that can change,
// and pull rounds skip it.  A part whose limit is below `round` no longer
// needs its values (nothing of it reads them any more) and sits out too.
__global__ void k_bitmap(const uint32_t* __restrict__ stamp, uint32_t sv, int64_t n, uint32_t* __restrict__ bm,
                         const int32_t* __restrict__ vpart, int32_t* __restrict__ part_cnt,
                         const int32_t* __restrict__ part_limit, int32_t round) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool in = v < n && stamp[v] == sv && !(part_limit && part_limit[vpart[v]] < round);
        const unsigned w = __ballot_sync(kFull, in);
        if (lane_id() == 0) bm[base >> 5] = w;
        if (vpart && w) {
            const int32_t p = v < n ? vpart[v] : -1;
            const unsigned same = __match_any_sync(kFull, p);
            const int lead = __ffs(same & w) - 1;  // first frontier lane of this part
            if (in && lane_id() == lead) atomicAdd(&part_cnt[p], __popc(same & w));
        }
    }
}

__device__ __forceinline__ bool part_idle(const int32_t* __restrict__ vpart, const int32_t* __restrict__ part_cnt,
                                          int32_t v) {
    return vpart && __ldg(&part_cnt[__ldg(&vpart[v])]) == 0;
}

__device__ __forceinline__ bool skipped(const Prune& pr, int32_t u) {
    return (pr.need && __ldg(&pr.need[u]) <= pr.round) || (pr.only && !__ldg(&pr.only[u]));
}

// Values >= `limit` are ignored: unset entries (BFS) or values of an earlier
// sweep (MIS sweeps stamp each sweep into the high word).  With `settle`, a
// vertex holding a value below the limit is final and is skipped.
//
// Lowest value offered by the frontier neighbours cols[e], e in [e0, e1) with
// stride `step`, four edges per lane and pass: the four bitmap loads, then
// the value loads are independent, so each lane keeps up to four dependent-
// load chains in flight; the columns of the next pass are loaded at the start
// of a pass, so their DRAM latency overlaps this pass's bitmap and value loads.
__device__ __forceinline__ unsigned long long pull_min(const int32_t* __restrict__ cols, int64_t e0, int64_t e1,
                                                       int step, const uint32_t* __restrict__ bm,
                                                       const unsigned long long* __restrict__ X,
                                                       unsigned long long add, unsigned long long limit,
                                                       unsigned long long m) {
    int32_t nx[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) nx[j] = e0 + j * step < e1 ? __ldcs(&cols[e0 + j * step]) : -1;
    for (int64_t e = e0; e < e1; e += 4 * step) {
        int32_t u[4];
        bool f[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = nx[j];
        const int64_t en = e + 4 * step;
#pragma unroll
        for (int j = 0; j < 4; ++j) nx[j] = en + j * step < e1 ? __ldcs(&cols[en + j * step]) : -1;
#pragma unroll
        for (int j = 0; j < 4; ++j) f[j] = u[j] >= 0 && in_front(bm, u[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (f[j]) {
                const unsigned long long x = __ldg(&X[u[j]]);
                if (x < limit && x + add < m) m = x + add;
            }
        }
    }
    return m;
}

// Pull round over vertices of at most kSmallDeg neighbours: a thread per
// vertex, its neighbours loaded four at a time (column, bitmap and value
// loads each independent of the others), so that a warp keeps 32 vertices'
// chains in flight.
__global__ void __launch_bounds__(256) k_pull_small(const int32_t* __restrict__ list, int64_t n_list,
                                                    const int64_t* __restrict__ rowp,
                                                    const int32_t* __restrict__ cols, unsigned long long add,
                                                    unsigned long long limit, bool settle,
                                                    const uint32_t* __restrict__ bm,
                                                    const unsigned long long* __restrict__ X,
                                                    unsigned long long* __restrict__ Xn,
                                                    uint32_t* __restrict__ stamp, uint32_t sv,
                                                    unsigned long long* __restrict__ n_changed,
                                                    const int32_t* __restrict__ vpart,
                                                    const int32_t* __restrict__ part_cnt, Prune pr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long changed = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_list; base += stride) {
        const int64_t i = base + lane_id();
        const int32_t v = i < n_list ? list[i] : 0;
        const bool have = i < n_list && !part_idle(vpart, part_cnt, v) && !skipped(pr, v);
        const unsigned long long own = have ? X[v] : ~0ULL;
        const bool work = have && !(settle && own < limit);
        const int64_t beg = work ? rowp[v] : 0, end = work ? rowp[v + 1] : 0;
        const unsigned long long m = pull_min(cols, beg, end, 1, bm, X, add, limit, own);
        const bool ch = work && m < own;
        if (ch) {
            Xn[v] = m;
            stamp[v] = sv;
            if (pr.reach && own >= limit) pr.reach[v] = (uint8_t)pr.reach_val;
        }
        changed += __popc(__ballot_sync(kFull, ch));
    }
    if (lane_id() == 0 && changed) atomicAdd(n_changed, changed);
}

// Pull round over the other non-hub vertices: four vertices per warp, eight
// lanes per vertex striding over its neighbours; the lanes meet again at the
// reduction.
__global__ void __launch_bounds__(256) k_pull_low(const int32_t* __restrict__ list, int64_t n_list,
                                                  const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                  unsigned long long add, unsigned long long limit, bool settle,
                                                  const uint32_t* __restrict__ bm,
                                                  const unsigned long long* __restrict__ X,
                                                  unsigned long long* __restrict__ Xn, uint32_t* __restrict__ stamp,
                                                  uint32_t sv, unsigned long long* __restrict__ n_changed,
                                                  const int32_t* __restrict__ vpart,
                                                  const int32_t* __restrict__ part_cnt, Prune pr) {
    const int lane = lane_id();
    const int sub = lane & 7;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long changed = 0;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 4 < n_list; w += warps) {
        const int64_t i = w * 4 + (lane >> 3);
        const int32_t v = i < n_list ? list[i] : 0;
        const bool have = i < n_list && !part_idle(vpart, part_cnt, v) && !skipped(pr, v);
        const unsigned long long own = have ? X[v] : ~0ULL;
        const bool work = have && !(settle && own < limit);
        const int64_t beg = work ? rowp[v] : 0, end = work ? rowp[v + 1] : 0;
        unsigned long long m = pull_min(cols, beg + sub, end, 8, bm, X, add, limit, own);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) m = umin64(m, __shfl_xor_sync(kFull, m, o));
        const bool ch = work && sub == 0 && m < own;
        if (ch) {
            Xn[v] = m;
            stamp[v] = sv;
            if (pr.reach && own >= limit) pr.reach[v] = (uint8_t)pr.reach_val;
        }
        changed += __popc(__ballot_sync(kFull, ch));
    }
    if (lane == 0 && changed) atomicAdd(n_changed, changed);
}

// Pull round over hubs: one warp per segment of kSeg edges.  Xn[v] starts as
// X[v]; the segments lower it with atomicMin and the one that lowers it first
// (it sees the old value) flags the hub.
__global__ void __launch_bounds__(256) k_pull_segs(const int32_t* __restrict__ seg_hub, int64_t n_seg,
                                                   const int64_t* __restrict__ hub_seg,
                                                   const int32_t* __restrict__ hub_list,
                                                   const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                   unsigned long long add, unsigned long long limit, bool settle,
                                                   const uint32_t* __restrict__ bm,
                                                   const unsigned long long* __restrict__ X,
                                                   unsigned long long* __restrict__ Xn, uint32_t* __restrict__ stamp,
                                                   uint32_t sv, unsigned long long* __restrict__ n_changed,
                                                   const int32_t* __restrict__ vpart,
                                                   const int32_t* __restrict__ part_cnt, Prune pr) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sidx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sidx < n_seg; sidx += warps) {
        const int32_t h = seg_hub[sidx];
        const int32_t v = hub_list[h];
        const unsigned long long own = X[v];
        if ((settle && own < limit) || part_idle(vpart, part_cnt, v) || skipped(pr, v)) continue;
        const int64_t e0 = rowp[v] + (sidx - hub_seg[h]) * kSeg;
        const int64_t e1 = min(e0 + (int64_t)kSeg, rowp[v + 1]);
        unsigned long long m = pull_min(cols, e0 + lane, e1, 32, bm, X, add, limit, ~0ULL);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = umin64(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0 && m < own) {
            const unsigned long long old = atomicMin(&Xn[v], m);
            if (old == own) {
                stamp[v] = sv;
                if (pr.reach && own >= limit) pr.reach[v] = (uint8_t)pr.reach_val;
                atomicAdd(n_changed, 1ULL);
            }
        }
    }
}

// Snapshot of a push frontier: frval[i] = X[fr[i]], the frontier's edge count
// into *edges, and each hub of the frontier tagged (hub_tag = tag, hub_val =
// its value) for the segment push.  hub_list is ascending.
__global__ void k_snap_front(const int32_t* __restrict__ fr, const unsigned long long* __restrict__ n_fr,
                             const unsigned long long* __restrict__ X, unsigned long long* __restrict__ frval,
                             unsigned long long* __restrict__ reset_next, const int64_t* __restrict__ rowp,
                             const int32_t* __restrict__ hub_list, int64_t n_hubs, uint32_t* __restrict__ hub_tag,
                             uint32_t tag, unsigned long long* __restrict__ hub_val,
                             unsigned long long* __restrict__ edges) {
    const int64_t n = (int64_t)*n_fr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *reset_next = 0;
    unsigned long long ed = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t v = fr[i];
        const unsigned long long x = X[v];
        frval[i] = x;
        const int64_t d = rowp[v + 1] - rowp[v];
        ed += (unsigned long long)d;
        if (d > kHubDeg) {
            int64_t lo = 0, hi = n_hubs;  // first hub_list entry >= v
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (hub_list[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            if (lo < n_hubs && hub_list[lo] == v) {
                hub_val[lo] = x;
                hub_tag[lo] = tag;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ed += __shfl_xor_sync(kFull, ed, o);
    if (lane_id() == 0 && ed) atomicAdd(edges, ed);
}

// Push from the non-hub frontier vertices: a warp per vertex, read-before-
// atomicMin on the neighbours, stamp dedupe for the next frontier.
__global__ void __launch_bounds__(256) k_push_low(const int32_t* __restrict__ fr,
                                                  const unsigned long long* __restrict__ frval,
                                                  const unsigned long long* __restrict__ n_fr,
                                                  const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                  unsigned long long add, unsigned long long limit,
                                                  unsigned long long* __restrict__ X,
                                                  uint32_t* __restrict__ stamp, uint32_t sv,
                                                  int32_t* __restrict__ fr_next, unsigned long long* __restrict__ n_next,
                                                  Prune pr) {
    const int lane = lane_id();
    const int64_t n = (int64_t)*n_fr;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; w < n; w += warps) {
        const int32_t v = fr[w];
        const int64_t beg = rowp[v], end = rowp[v + 1];
        if (end - beg > kHubDeg) continue;  // hubs: k_push_segs
        const unsigned long long val = frval[w] + add;
        for (int64_t cb = beg; cb < end; cb += 32) {
            const int64_t e = cb + lane;
            bool fresh = false;
            int32_t u = 0;
            if (e < end) {
                u = cols[e];
                if (val < X[u] && !skipped(pr, u)) {
                    const unsigned long long old = atomicMin(&X[u], val);
                    if (val < old) {
                        if (pr.reach && old >= limit) pr.reach[u] = (uint8_t)pr.reach_val;
                        fresh = atomicExch(&stamp[u], sv) != sv;
                    }
                }
            }
            const long long at = warp_append(fresh, n_next);
            if (at >= 0) fr_next[at] = u;
        }
    }
}

// Push from the frontier hubs (tagged by k_snap_front): a warp per segment.
__global__ void __launch_bounds__(256) k_push_segs(const int32_t* __restrict__ seg_hub, int64_t n_seg,
                                                   const int64_t* __restrict__ hub_seg,
                                                   const int32_t* __restrict__ hub_list,
                                                   const uint32_t* __restrict__ hub_tag, uint32_t tag,
                                                   const unsigned long long* __restrict__ hub_val,
                                                   const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                   unsigned long long add, unsigned long long limit,
                                                   unsigned long long* __restrict__ X,
                                                   uint32_t* __restrict__ stamp, uint32_t sv,
                                                   int32_t* __restrict__ fr_next, unsigned long long* __restrict__ n_next,
                                                   Prune pr) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sidx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sidx < n_seg; sidx += warps) {
        const int32_t h = seg_hub[sidx];
        if (hub_tag[h] != tag) continue;
        const int32_t v = hub_list[h];
        const unsigned long long val = hub_val[h] + add;
        const int64_t e0 = rowp[v] + (sidx - hub_seg[h]) * kSeg;
        const int64_t e1 = min(e0 + (int64_t)kSeg, rowp[v + 1]);
        for (int64_t cb = e0; cb < e1; cb += 32) {
            const int64_t e = cb + lane;
            bool fresh = false;
            int32_t u = 0;
            if (e < e1) {
                u = cols[e];
                if (val < X[u] && !skipped(pr, u)) {
                    const unsigned long long old = atomicMin(&X[u], val);
                    if (val < old) {
                        if (pr.reach && old >= limit) pr.reach[u] = (uint8_t)pr.reach_val;
                        fresh = atomicExch(&stamp[u], sv) != sv;
                    }
                }
            }
            const long long at = warp_append(fresh, n_next);
            if (at >= 0) fr_next[at] = u;
        }
    }
}

// Vertices flagged with stamp sv -> list.
__global__ void k_collect_stamped(const uint32_t* __restrict__ stamp, uint32_t sv, int64_t n,
                                  int32_t* __restrict__ out, unsigned long long* __restrict__ n_out) {
    __shared__ BlockAppend<8> sh;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < n; bb += stride) {
        const int64_t v = bb + threadIdx.x;
        const bool in = v < n && stamp[v] == sv;
        const long long at = block_append<8>(in, n_out, sh);
        if (at >= 0) out[at] = (int32_t)v;
    }
}

constexpr int64_t kPushAlways = 4096;  // smaller frontiers push without counting their edges

}  // namespace

// Vertices whose value carries high word `hi` -> list (the vertices a sweep reached).
__global__ void k_collect_epoch(const unsigned long long* __restrict__ X, unsigned long long hi, int64_t n,
                                int32_t* __restrict__ out, unsigned long long* __restrict__ n_out) {
    __shared__ BlockAppend<8> sh;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < n; bb += stride) {
        const int64_t v = bb + threadIdx.x;
        const bool in = v < n && (X[v] >> 32) == hi;
        const long long at = block_append<8>(in, n_out, sh);
        if (at >= 0) out[at] = (int32_t)v;
    }
}

int relax_collect_epoch(fl_graph* g, const unsigned long long* X, unsigned long long hi, int32_t* out,
                        unsigned long long* n_out, int cls) {
    FL_CUDA(cudaMemsetAsync(n_out, 0, 8, g->stream));
    FL_LAUNCH(cls, k_collect_epoch<<<grid_for(g->n, 256), 256, 0, g->stream>>>(X, hi, g->n, out, n_out));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

// Work lists and round scratch of g allocated ahead (so that a solve on a
// prefix view of g allocates nothing graph-owned).
int relax_reserve(fl_graph* g) {
    Relax r;
    return relax_begin(g, r);
}

int relax_begin(fl_graph* g, Relax& r) {
    if (!g->lists_ready) {
        FL_TRY(build_work_lists(g));
        g->lists_ready = 1;
    }
    r.dense_div = g->sched.dense_div;
    r.edge_div = g->sched.edge_div;
    const size_t bm_words = (size_t)(g->n + 63) / 32 + 2;
    const size_t off_tag = ((bm_words * 4 + 255) / 256) * 256;
    const size_t off_val = off_tag + (((size_t)g->n_hubs * 4 + 255) / 256) * 256;
    const size_t off_cnt = off_val + (((size_t)g->n_hubs * 8 + 255) / 256) * 256;
    const size_t off_part = off_cnt + 256;
    FL_TRY(dalloc(g->relax_aux, off_part + (size_t)(g->n_parts + 1) * 4));
    char* base = g->relax_aux.as<char>();
    r.bm = reinterpret_cast<uint32_t*>(base);
    r.hub_tag = reinterpret_cast<uint32_t*>(base + off_tag);
    r.hub_val = reinterpret_cast<unsigned long long*>(base + off_val);
    r.ecnt = reinterpret_cast<unsigned long long*>(base + off_cnt);
    r.part_cnt = reinterpret_cast<int32_t*>(base + off_part);
    if (g->n_hubs > 0) FL_CUDA(cudaMemsetAsync(r.hub_tag, 0, (size_t)g->n_hubs * 4, g->stream));
    FL_CUDA(cudaMemsetAsync(r.ecnt, 0, 256, g->stream));
    return FL_OK;
}

// One synchronous round.  The caller keeps the frontier count on the host
// (r.n_front) and, for push rounds, a valid list in r.fr[r.fc] with its count
// in r.cnt[r.fc].  `sv` is the stamp of the frontier this round produces.
// A round pushes when its frontier is small (few vertices, or few edges);
// otherwise it pulls with the frontier bitmap.
int relax_round(fl_graph* g, Relax& r, unsigned long long add, uint32_t sv, int cls) {
    cudaStream_t st = g->stream;
    const int64_t n = g->n;
    const int64_t* rowp = g->rowp.as<int64_t>();
    const int32_t* cols = g->cols.as<int32_t>();
    const int32_t* hub_list = g->hub_list.as<int32_t>();
    bool dense = r.n_front * r.dense_div >= g->n_low + g->n_hubs;
    unsigned long long* X = r.X[r.cur];
    if (!dense) {
        if (!r.list_valid) {
            // rebuild the frontier list from the stamps of the previous round
            FL_CUDA(cudaMemsetAsync(&r.cnt[r.fc], 0, 8, st));
            FL_LAUNCH(cls, k_collect_stamped<<<grid_for(n, 256), 256, 0, st>>>(r.stamp, r.sv_prev, n, r.fr[r.fc],
                                                                              &r.cnt[r.fc]));
            r.list_valid = true;
        }
        FL_CUDA(cudaMemsetAsync(r.ecnt, 0, 8, st));
        FL_LAUNCH(cls, k_snap_front<<<grid_for(r.n_front, 256), 256, 0, st>>>(
                           r.fr[r.fc], &r.cnt[r.fc], X, r.frval, &r.cnt[r.fc ^ 1], rowp, hub_list, g->n_hubs,
                           r.hub_tag, r.sv_prev, r.hub_val, r.ecnt));
        FL_CUDA(cudaGetLastError());
        if (r.n_front >= kPushAlways) {
            FL_CUDA(cudaMemcpyAsync(r.h_cnt, r.ecnt, 8, cudaMemcpyDeviceToHost, st));
            FL_CUDA(cudaStreamSynchronize(st));
            dense = (int64_t)*r.h_cnt * r.edge_div >= g->nnz;
        }
    }
    if (!dense) {
        FL_LAUNCH(cls, k_push_low<<<grid_for(r.n_front, 8), 256, 0, st>>>(r.fr[r.fc], r.frval, &r.cnt[r.fc], rowp, cols,
                                                                         add, r.limit, X, r.stamp, sv, r.fr[r.fc ^ 1],
                                                                         &r.cnt[r.fc ^ 1], r.prune));
        if (g->n_seg > 0)
            FL_LAUNCH(cls, k_push_segs<<<grid_for(g->n_seg, 8), 256, 0, st>>>(
                               g->seg_hub.as<int32_t>(), g->n_seg, g->hub_seg.as<int64_t>(), hub_list, r.hub_tag,
                               r.sv_prev, r.hub_val, rowp, cols, add, r.limit, X, r.stamp, sv, r.fr[r.fc ^ 1],
                               &r.cnt[r.fc ^ 1], r.prune));
        FL_CUDA(cudaGetLastError());
        r.fc ^= 1;
        r.list_valid = true;
        FL_CUDA(cudaMemcpyAsync(r.h_cnt, &r.cnt[r.fc], 8, cudaMemcpyDeviceToHost, st));
    } else {
        unsigned long long* Xn = r.X[r.cur ^ 1];
        const int32_t* vpart = g->n_parts > 0 ? g->vpart.as<int32_t>() : nullptr;
        if (vpart) FL_CUDA(cudaMemsetAsync(r.part_cnt, 0, (size_t)g->n_parts * 4, st));
        FL_LAUNCH(cls, k_bitmap<<<grid_for(n, 256), 256, 0, st>>>(r.stamp, r.sv_prev, n, r.bm, vpart, r.part_cnt,
                                                                  vpart ? r.part_limit : nullptr, r.part_round));
        FL_CUDA(cudaMemcpyAsync(Xn, X, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
        FL_CUDA(cudaMemsetAsync(&r.cnt[2], 0, 8, st));
        if (g->n_small > 0)
            FL_LAUNCH(cls, k_pull_small<<<grid_for(g->n_small, 256), 256, 0, st>>>(
                               g->small_list.as<int32_t>(), g->n_small, rowp, cols, add, r.limit, r.settle, r.bm, X,
                               Xn, r.stamp, sv, &r.cnt[2], vpart, r.part_cnt, r.prune));
        if (g->n_mid > 0)
            FL_LAUNCH(cls, k_pull_low<<<grid_for((g->n_mid + 3) / 4, 8), 256, 0, st>>>(
                               g->mid_list.as<int32_t>(), g->n_mid, rowp, cols, add, r.limit, r.settle, r.bm, X, Xn,
                               r.stamp, sv, &r.cnt[2], vpart, r.part_cnt, r.prune));
        if (g->n_seg > 0)
            FL_LAUNCH(cls, k_pull_segs<<<grid_for(g->n_seg, 8), 256, 0, st>>>(
                               g->seg_hub.as<int32_t>(), g->n_seg, g->hub_seg.as<int64_t>(), hub_list, rowp, cols, add,
                               r.limit, r.settle, r.bm, X, Xn, r.stamp, sv, &r.cnt[2], vpart, r.part_cnt,
                               r.prune));
        FL_CUDA(cudaGetLastError());
        r.cur ^= 1;
        r.list_valid = false;
        FL_CUDA(cudaMemcpyAsync(r.h_cnt, &r.cnt[2], 8, cudaMemcpyDeviceToHost, st));
    }
    FL_CUDA(cudaStreamSynchronize(st));
    r.n_front = (int64_t)*r.h_cnt;
    r.sv_prev = sv;
    r.last_dense = dense;
    return FL_OK;
}

// ------------------------------------------------------------------ marking rounds
// A bounded BFS that only records whether a vertex lies within distance b of
// the seeds: kr[v] = 1 + its distance, 0 while it is farther than the rounds
// run so far (seeds carry 1).  Round b marks every unmarked vertex with
// need[v] > b that has a neighbour marked in an earlier round (kr in [1, b],
// read from a bitmap); a vertex stops reading its row at the first such
// neighbour, so a dense round costs far less than a min-propagation round.

namespace {

__global__ void k_mark_bitmap(const uint8_t* __restrict__ kr, int64_t n, uint32_t b, uint32_t* __restrict__ bm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const uint32_t k = v < n ? kr[v] : 0u;
        const unsigned w = __ballot_sync(kFull, k != 0 && k <= b);
        if (lane_id() == 0) bm[base >> 5] = w;
    }
}

__device__ __forceinline__ bool unmarked_needed(const uint8_t* __restrict__ kr, const uint8_t* __restrict__ need,
                                                int32_t v, uint32_t b) {
    return kr[v] == 0 && (!need || __ldg(&need[v]) > b);
}

// Vertices of at most kSmallDeg neighbours: a thread each.
__global__ void __launch_bounds__(256) k_mark_small(const int32_t* __restrict__ list, int64_t n_list,
                                                    const int64_t* __restrict__ rowp,
                                                    const int32_t* __restrict__ cols,
                                                    const uint32_t* __restrict__ bm, uint8_t* __restrict__ kr,
                                                    const uint8_t* __restrict__ need, uint32_t b,
                                                    unsigned long long* __restrict__ n_marked) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long marked = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_list; base += stride) {
        const int64_t i = base + lane_id();
        const int32_t v = i < n_list ? list[i] : 0;
        bool hit = false;
        if (i < n_list && unmarked_needed(kr, need, v, b)) {
            const int64_t beg = rowp[v], end = rowp[v + 1];
            for (int64_t e = beg; e < end && !hit; e += 4) {
                int32_t u[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) u[j] = e + j < end ? __ldcs(&cols[e + j]) : -1;
#pragma unroll
                for (int j = 0; j < 4; ++j) hit |= u[j] >= 0 && in_front(bm, u[j]);
            }
            if (hit) kr[v] = (uint8_t)(b + 1);
        }
        marked += __popc(__ballot_sync(kFull, hit));
    }
    if (lane_id() == 0 && marked) atomicAdd(n_marked, marked);
}

// Other non-hub vertices: eight lanes each (four per warp), 32 entries of a
// row per pass; a group leaves at the first pass that finds a marked neighbour.
__global__ void __launch_bounds__(256) k_mark_low(const int32_t* __restrict__ list, int64_t n_list,
                                                  const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                  const uint32_t* __restrict__ bm, uint8_t* __restrict__ kr,
                                                  const uint8_t* __restrict__ need, uint32_t b,
                                                  unsigned long long* __restrict__ n_marked) {
    const int lane = lane_id();
    const int sub = lane & 7;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long marked = 0;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 4 < n_list; w += warps) {
        const int64_t i = w * 4 + (lane >> 3);
        const int32_t v = i < n_list ? list[i] : 0;
        bool work = i < n_list && unmarked_needed(kr, need, v, b);
        const int64_t beg = work ? rowp[v] : 0, end = work ? rowp[v + 1] : 0;
        for (int64_t at = beg;; at += 32) {
            bool hit = false;
            if (work) {
                int32_t u[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t e = at + sub + 8 * j;
                    u[j] = e < end ? __ldcs(&cols[e]) : -1;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) hit |= u[j] >= 0 && in_front(bm, u[j]);
            }
            const bool group_hit = (__ballot_sync(kFull, hit) >> (lane & ~7)) & 0xffu;
            if (work && group_hit) {
                if (sub == 0) {
                    kr[v] = (uint8_t)(b + 1);
                    ++marked;
                }
                work = false;
            }
            if (at + 32 >= end) work = false;
            if (!__any_sync(kFull, work)) break;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) marked += __shfl_xor_sync(kFull, marked, o);
    if (lane == 0 && marked) atomicAdd(n_marked, marked);
}

// Hubs: a warp per segment of kSeg entries; every segment that finds a marked
// neighbour marks the hub (the count may hold a hub more than once).
__global__ void __launch_bounds__(256) k_mark_segs(const int32_t* __restrict__ seg_hub, int64_t n_seg,
                                                   const int64_t* __restrict__ hub_seg,
                                                   const int32_t* __restrict__ hub_list,
                                                   const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                   const uint32_t* __restrict__ bm, uint8_t* __restrict__ kr,
                                                   const uint8_t* __restrict__ need, uint32_t b,
                                                   unsigned long long* __restrict__ n_marked) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sidx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sidx < n_seg; sidx += warps) {
        const int32_t h = seg_hub[sidx];
        const int32_t v = hub_list[h];
        if (!unmarked_needed(kr, need, v, b)) continue;
        const int64_t e0 = rowp[v] + (sidx - hub_seg[h]) * kSeg;
        const int64_t e1 = min(e0 + (int64_t)kSeg, rowp[v + 1]);
        for (int64_t at = e0; at < e1; at += 128) {
            bool hit = false;
            int32_t u[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t e = at + lane + 32 * j;
                u[j] = e < e1 ? __ldcs(&cols[e]) : -1;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) hit |= u[j] >= 0 && in_front(bm, u[j]);
            if (__any_sync(kFull, hit)) {
                if (lane == 0) {
                    kr[v] = (uint8_t)(b + 1);
                    atomicAdd(n_marked, 1ULL);
                }
                break;
            }
        }
    }
}

}  // namespace

int mark_round(fl_graph* g, Relax& r, uint8_t* kr, const uint8_t* need, uint32_t b, int cls, int64_t* marked) {
    cudaStream_t st = g->stream;
    const int64_t* rowp = g->rowp.as<int64_t>();
    const int32_t* cols = g->cols.as<int32_t>();
    FL_CUDA(cudaMemsetAsync(&r.cnt[2], 0, 8, st));
    FL_LAUNCH(cls, k_mark_bitmap<<<grid_for(g->n, 256), 256, 0, st>>>(kr, g->n, b, r.bm));
    if (g->n_small > 0)
        FL_LAUNCH(cls, k_mark_small<<<grid_for(g->n_small, 256), 256, 0, st>>>(
                           g->small_list.as<int32_t>(), g->n_small, rowp, cols, r.bm, kr, need, b, &r.cnt[2]));
    if (g->n_mid > 0)
        FL_LAUNCH(cls, k_mark_low<<<grid_for((g->n_mid + 3) / 4, 8), 256, 0, st>>>(
                           g->mid_list.as<int32_t>(), g->n_mid, rowp, cols, r.bm, kr, need, b, &r.cnt[2]));
    if (g->n_seg > 0)
        FL_LAUNCH(cls, k_mark_segs<<<grid_for(g->n_seg, 8), 256, 0, st>>>(
                           g->seg_hub.as<int32_t>(), g->n_seg, g->hub_seg.as<int64_t>(), g->hub_list.as<int32_t>(),
                           rowp, cols, r.bm, kr, need, b, &r.cnt[2]));
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaMemcpyAsync(r.h_cnt, &r.cnt[2], 8, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    *marked = (int64_t)*r.h_cnt;
    return FL_OK;
}

// Add vertices to the current frontier list (sources or injections): X[s] =
// min(X[s], val(s)); s joins when it decreases.  Makes the list valid first.
int relax_prepare_list(fl_graph* g, Relax& r, int cls) {
    if (r.list_valid) return FL_OK;
    cudaStream_t st = g->stream;
    FL_CUDA(cudaMemsetAsync(&r.cnt[r.fc], 0, 8, st));
    FL_LAUNCH(cls, k_collect_stamped<<<grid_for(g->n, 256), 256, 0, st>>>(r.stamp, r.sv_prev, g->n, r.fr[r.fc],
                                                                          &r.cnt[r.fc]));
    FL_CUDA(cudaGetLastError());
    r.list_valid = true;
    return FL_OK;
}

}  // namespace fl
