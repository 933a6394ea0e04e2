// k_relax.cu -- synchronous min-propagation rounds over the CSR, used by the
// multi-source BFS (assignment, eccentricity bound) and by the cover / gather
// sweeps of the greedy MIS ("send to all vertices within distance d", §3.4).
//
// One round: every vertex v takes X'[v] = min(X[v], min_{u in N(v)} X[u] + add),
// reading only values of the previous round, so a value moves exactly one hop
// per round.  Sparse rounds push from a frontier list (k_snapshot + k_push, in
// place on one buffer, the frontier's values snapshotted first); dense rounds
// pull into the second buffer (every vertex reads its neighbours; no atomics)
// and flag changed vertices with the next round's stamp.
#include <algorithm>
#include <cstdio>

#include "fl_internal.cuh"

namespace fl {

__global__ void k_snapshot(const int32_t* __restrict__ fr, const unsigned long long* __restrict__ n_fr,
                           const unsigned long long* __restrict__ X, unsigned long long* __restrict__ frval,
                           unsigned long long* __restrict__ reset_next, uint32_t* __restrict__ tstamp, uint32_t tval,
                           int32_t* __restrict__ touched, unsigned long long* __restrict__ n_touched);
__global__ void k_push(const int32_t* __restrict__ fr, const unsigned long long* __restrict__ frval,
                       const unsigned long long* __restrict__ n_fr, const int64_t* __restrict__ rowp,
                       const int32_t* __restrict__ cols, unsigned long long add, unsigned long long* __restrict__ X,
                       uint32_t* __restrict__ stamp, uint32_t sv, int32_t* __restrict__ fr_next,
                       unsigned long long* __restrict__ n_next);

namespace {

int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// Values >= `limit` are ignored: unset entries (BFS) or values of an earlier
// sweep (MIS sweeps stamp each sweep into the high word).
//
// Dense round over non-hub vertices: four vertices per warp in lockstep, eight
// lanes per vertex striding over its neighbours; the loop runs to the largest
// degree of the four so every shuffle and ballot involves the whole warp.
__global__ void __launch_bounds__(256) k_pull_low(const int32_t* __restrict__ list, int64_t n_list,
                                                  const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                  unsigned long long add, unsigned long long limit,
                                                  const unsigned long long* __restrict__ X,
                                                  unsigned long long* __restrict__ Xn, uint32_t* __restrict__ stamp,
                                                  uint32_t sv, unsigned long long* __restrict__ n_changed) {
    const int lane = lane_id();
    const int sub = lane & 7;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long changed = 0;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 4 < n_list; w += warps) {
        const int64_t i = w * 4 + (lane >> 3);
        const bool have = i < n_list;
        const int32_t v = have ? list[i] : 0;
        const int64_t beg = have ? rowp[v] : 0, end = have ? rowp[v + 1] : 0;
        const unsigned long long own = have ? X[v] : ~0ULL;
        unsigned long long m = own;
        int64_t len = end - beg;
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) len = max(len, __shfl_xor_sync(kFull, len, o));
        for (int64_t off = sub; off < len; off += 8) {
            if (beg + off < end) {
                const unsigned long long x = __ldg(&X[__ldg(&cols[beg + off])]);
                if (x < limit && x + add < m) m = x + add;
            }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) m = umin64(m, __shfl_xor_sync(kFull, m, o));
        const bool ch = have && sub == 0 && m < own;
        if (ch) {
            Xn[v] = m;
            stamp[v] = sv;
        }
        changed += __popc(__ballot_sync(kFull, ch));
    }
    if (lane == 0 && changed) atomicAdd(n_changed, changed);
}

// Dense round over hubs: one block per hub.
__global__ void __launch_bounds__(256) k_pull_hubs(const int32_t* __restrict__ hubs, int64_t n_hubs,
                                                   const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                   unsigned long long add, unsigned long long limit,
                                                   const unsigned long long* __restrict__ X,
                                                   unsigned long long* __restrict__ Xn, uint32_t* __restrict__ stamp,
                                                   uint32_t sv, unsigned long long* __restrict__ n_changed) {
    __shared__ unsigned long long red[8];
    for (int64_t h = blockIdx.x; h < n_hubs; h += gridDim.x) {
        const int32_t v = hubs[h];
        const int64_t beg = rowp[v], end = rowp[v + 1];
        unsigned long long m = ~0ULL;
        for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
            const unsigned long long x = __ldg(&X[__ldg(&cols[e])]);
            if (x < limit && x + add < m) m = x + add;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = umin64(m, __shfl_xor_sync(kFull, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = umin64(m, red[i]);
            const unsigned long long own = X[v];
            if (m < own) {
                Xn[v] = m;
                stamp[v] = sv;
                atomicAdd(n_changed, 1ULL);
            }
        }
        __syncthreads();
    }
}

// Vertices flagged with stamp sv -> list.
__global__ void k_collect_stamped(const uint32_t* __restrict__ stamp, uint32_t sv, int64_t n,
                                  int32_t* __restrict__ out, unsigned long long* __restrict__ n_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool in = v < n && stamp[v] == sv;
        const long long at = warp_append(in, n_out);
        if (at >= 0) out[at] = (int32_t)v;
    }
}

}  // namespace

// Vertices whose value carries high word `hi` -> list (the vertices a sweep reached).
__global__ void k_collect_epoch(const unsigned long long* __restrict__ X, unsigned long long hi, int64_t n,
                                int32_t* __restrict__ out, unsigned long long* __restrict__ n_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool in = v < n && (X[v] >> 32) == hi;
        const long long at = warp_append(in, n_out);
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

// One synchronous round.  The caller keeps the frontier count on the host
// (r.n_front) and, for push rounds, a valid list in r.fr[r.fc] with its count
// in r.cnt[r.fc].  `sv` is the stamp of the frontier this round produces.
int relax_round(fl_graph* g, Relax& r, unsigned long long add, uint32_t sv, int cls) {
    cudaStream_t st = g->stream;
    const int64_t n = g->n;
    const bool dense = r.n_front * r.dense_div >= g->n_low + g->n_hubs;
    unsigned long long* X = r.X[r.cur];
    if (!dense) {
        if (!r.list_valid) {
            // rebuild the frontier list from the stamps of the previous round
            FL_CUDA(cudaMemsetAsync(&r.cnt[r.fc], 0, 8, st));
            FL_LAUNCH(cls, k_collect_stamped<<<grid_for(n, 256), 256, 0, st>>>(r.stamp, r.sv_prev, n, r.fr[r.fc],
                                                                              &r.cnt[r.fc]));
        }
        FL_LAUNCH(cls, k_snapshot<<<grid_for(r.n_front, 256), 256, 0, st>>>(r.fr[r.fc], &r.cnt[r.fc], X, r.frval,
                                                                           &r.cnt[r.fc ^ 1], nullptr, 0, nullptr,
                                                                           nullptr));
        FL_LAUNCH(cls, k_push<<<grid_for(r.n_front, 8), 256, 0, st>>>(r.fr[r.fc], r.frval, &r.cnt[r.fc],
                                                                     g->rowp.as<int64_t>(), g->cols.as<int32_t>(), add,
                                                                     X, r.stamp, sv, r.fr[r.fc ^ 1], &r.cnt[r.fc ^ 1]));
        FL_CUDA(cudaGetLastError());
        r.fc ^= 1;
        r.list_valid = true;
        FL_CUDA(cudaMemcpyAsync(r.h_cnt, &r.cnt[r.fc], 8, cudaMemcpyDeviceToHost, st));
    } else {
        unsigned long long* Xn = r.X[r.cur ^ 1];
        FL_CUDA(cudaMemcpyAsync(Xn, X, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
        FL_CUDA(cudaMemsetAsync(&r.cnt[2], 0, 8, st));
        if (g->n_low > 0)
            FL_LAUNCH(cls, k_pull_low<<<grid_for((g->n_low + 3) / 4, 8), 256, 0, st>>>(
                               g->low_list.as<int32_t>(), g->n_low, g->rowp.as<int64_t>(), g->cols.as<int32_t>(), add,
                               r.limit, X, Xn, r.stamp, sv, &r.cnt[2]));
        if (g->n_hubs > 0)
            FL_LAUNCH(cls, k_pull_hubs<<<(int)std::min<int64_t>(g->n_hubs, 152 * 8), 256, 0, st>>>(
                               g->hub_list.as<int32_t>(), g->n_hubs, g->rowp.as<int64_t>(), g->cols.as<int32_t>(), add,
                               r.limit, X, Xn, r.stamp, sv, &r.cnt[2]));
        FL_CUDA(cudaGetLastError());
        r.cur ^= 1;
        r.list_valid = false;
        FL_CUDA(cudaMemcpyAsync(r.h_cnt, &r.cnt[2], 8, cudaMemcpyDeviceToHost, st));
    }
    FL_CUDA(cudaStreamSynchronize(st));
    r.n_front = (int64_t)*r.h_cnt;
    r.sv_prev = sv;
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
