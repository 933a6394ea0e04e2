// k_sketch.cu -- phase (i): bottom-k sketches and ADS by hop-synchronous
// propagation (Section 2.3, Algorithm 2 for unweighted graphs), with HIP
// weights computed where each entry joins a sketch.
//
// Data layout (k <= 32):
//   S[v*k + i]        current sketch of v, ascending ranks, kEmpty padding
//   Scnt[v]           number of ranks in S[v]
//   D[p][v*k + i]     entries v gained at the previous / current hop (ranks)
//   Dcnt[p][v]        their number (0 = v is not in the frontier)
//   staging           per hop, one group record per vertex that changed and
//                     its entry ids; compacted to a vertex-major ADS at the end
#include <algorithm>
#include <cstdio>
#include <vector>

#include "fl_internal.cuh"

namespace fl {

struct StgGroup {
    int64_t at;     // first entry in the staging entry array
    double wt;      // HIP weight of the counted entries
    int32_t v;      // vertex
    int32_t gidx;   // index of this group among v's groups
    int32_t eidx;   // index of its first entry among v's entries
    uint32_t info;  // hop | cnt << 16 | counted << 24
};

__host__ __device__ __forceinline__ uint32_t pack_info(int hop, int cnt, int counted) {
    return (uint32_t)hop | ((uint32_t)cnt << 16) | ((uint32_t)counted << 24);
}

constexpr int kMaxHops = 65535;

// ------------------------------------------------------------------ hop 0

__global__ void k_rank_init(int64_t n, int k, uint64_t seed, uint64_t* __restrict__ S,
                            uint8_t* __restrict__ Scnt, uint64_t* __restrict__ D0, uint8_t* __restrict__ Dcnt0,
                            int32_t* __restrict__ stg_ent, StgGroup* __restrict__ stg_grp,
                            int32_t* __restrict__ vg, int32_t* __restrict__ ve, Counters* ctr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint64_t r = vertex_rank(seed, v);
        if (r == kEmpty) atomicOr(&ctr->error, 1ULL);
        S[v * k] = r;
        Scnt[v] = 1;
        D0[v * k] = r;
        Dcnt0[v] = 1;
        stg_ent[v] = (int32_t)v;
        StgGroup gr;
        gr.at = v;
        gr.wt = 1.0;  // a one-vertex ball: fewer than k ranks (k >= 2)
        gr.v = (int32_t)v;
        gr.gidx = 0;
        gr.eidx = 0;
        gr.info = pack_info(0, 1, 1);
        stg_grp[v] = gr;
        vg[v] = 1;
        ve[v] = 1;
    }
}

// ------------------------------------------------------------------ one hop

// Merge a buffer of candidate ranks (one per lane, unsorted, kEmpty = none)
// into the ascending sketch list `sk` (k valid slots), keeping the k smallest
// distinct ranks.  Returns the new list; lanes >= k hold kEmpty.
__device__ __forceinline__ uint64_t merge_candidates(uint64_t sk, uint64_t buf, int k) {
    const int lane = lane_id();
    buf = warp_sort(buf);
    uint64_t prev = __shfl_up_sync(kFull, buf, 1);
    bool dup = lane > 0 && prev == buf;
    bool in_sk = warp_member(sk, buf);
    unsigned keep = __ballot_sync(kFull, buf != kEmpty && !dup && !in_sk);
    if (!keep) return sk;
    buf = warp_compact(buf, keep, kEmpty);
    uint64_t m = warp_merge_low(sk, buf);
    return lane < k ? m : kEmpty;
}

// Warp per active vertex v: S_h(v) = bottom-k(S_{h-1}(v) U union_{u in N(v)} D_{h-1}(u)).
// Candidates of up to 32 neighbours are flattened into waves of 32 loads;
// only ranks below the current k-th rank are kept in a per-lane buffer that
// is merged when full.  Then the new entries D_h(v) = S_h(v) \ S_{h-1}(v) are
// written for the next hop and staged as the hop-h ADS group of v.
__global__ void __launch_bounds__(256) k_merge_hop(
    const int32_t* __restrict__ active, const unsigned long long* __restrict__ n_active_ptr, int64_t n_active_host,
    const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols, int k, uint64_t seed, int hop,
    uint64_t* __restrict__ S, uint8_t* __restrict__ Scnt, const uint64_t* __restrict__ Dp,
    const uint8_t* __restrict__ Dcp, uint64_t* __restrict__ Dc, uint8_t* __restrict__ Dcc,
    int32_t* __restrict__ fr_next, int32_t* __restrict__ vg, int32_t* __restrict__ ve,
    int32_t* __restrict__ stg_ent, StgGroup* __restrict__ stg_grp, Counters* ctr) {
    const int lane = lane_id();
    const int64_t n_active = n_active_ptr ? (int64_t)*n_active_ptr : n_active_host;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cand_reads = 0, merging = 0;  // algorithmic-traffic counters of this warp
    for (int64_t w = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; w < n_active; w += warps) {
        const int32_t v = active[w];
        const int64_t beg = rowp[v], end = rowp[v + 1];
        const uint64_t old = lane < k ? S[(int64_t)v * k + lane] : kEmpty;
        int vtotal = 0;
        uint64_t sk = old;
        int cnt_old = Scnt[v];
        const uint64_t kth_old = __shfl_sync(kFull, sk, k - 1);
        uint64_t tau = cnt_old == k ? kth_old : kEmpty;
        uint64_t buf = kEmpty;
        int nbuf = 0;
        for (int64_t cb = beg; cb < end; cb += 32) {
            int64_t e = cb + lane;
            int32_t u = e < end ? cols[e] : 0;
            int c = e < end ? (int)Dcp[u] : 0;
            int incl = warp_incl_scan(c);
            int total = __shfl_sync(kFull, incl, 31);
            vtotal += total;
            for (int off = 0; off < total; off += 32) {
                int t = off + lane;
                // neighbour slot j holding flattened candidate t: #lanes with incl <= t
                int j = 0;
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    int y = __shfl_sync(kFull, incl, j + s - 1);
                    if (y <= t) j += s;
                }
                j = j > 31 ? 31 : j;
                int uj = __shfl_sync(kFull, u, j);
                int ij = __shfl_sync(kFull, incl, j) - __shfl_sync(kFull, c, j);
                uint64_t x = t < total ? Dp[(int64_t)uj * k + (t - ij)] : kEmpty;
                bool ok = x < tau;
                unsigned vm = __ballot_sync(kFull, ok);
                int nv = __popc(vm);
                if (nv == 0) continue;
                if (nbuf + nv > 32) {
                    sk = merge_candidates(sk, buf, k);
                    tau = __shfl_sync(kFull, sk, k - 1);
                    buf = kEmpty;
                    nbuf = 0;
                    ok = x < tau;
                    vm = __ballot_sync(kFull, ok);
                    nv = __popc(vm);
                    if (nv == 0) continue;
                }
                // append the kept candidates at buffer slots nbuf .. nbuf+nv-1
                int p = lane - nbuf;
                int src = (p >= 0 && p < nv) ? nth_set_bit(vm, p) : 0;
                uint64_t y = __shfl_sync(kFull, x, src);
                if (p >= 0 && p < nv) buf = y;
                nbuf += nv;
            }
        }
        if (nbuf) sk = merge_candidates(sk, buf, k);
        cand_reads += (unsigned long long)vtotal;
        merging += vtotal > 0 ? 1ULL : 0ULL;
        // outputs
        const bool valid = lane < k && sk != kEmpty;
        const bool was_there = warp_member(old, sk);  // every lane takes part in the shuffles
        const bool is_new = valid && !was_there;
        const unsigned newm = __ballot_sync(kFull, is_new);
        const int dcnt = __popc(newm);
        const int cnt_new = __popc(__ballot_sync(kFull, valid));
        if (dcnt == 0) continue;  // sketch unchanged (and Dc count is already 0)
        if (lane < k) S[(int64_t)v * k + lane] = sk;
        const uint64_t dv = warp_compact(sk, newm, kEmpty);
        if (lane < dcnt) Dc[(int64_t)v * k + lane] = dv;
        const int counted = cnt_new < k ? dcnt : __popc(newm & ((1u << (k - 1)) - 1u));
        const uint64_t kth = __shfl_sync(kFull, sk, k - 1);
        int64_t eat = 0;
        if (lane == 0) {
            Scnt[v] = (uint8_t)cnt_new;
            Dcc[v] = (uint8_t)dcnt;
            unsigned long long fp = atomicAdd(&ctr->frontier, 1ULL);
            fr_next[fp] = v;
            atomicAdd(&ctr->merges, (unsigned long long)(end - beg));
            eat = (int64_t)atomicAdd(&ctr->stg_entries, (unsigned long long)dcnt);
            unsigned long long gat = atomicAdd(&ctr->stg_groups, 1ULL);
            StgGroup gr;
            gr.at = eat;
            // HIP weight: 1 while the ball has fewer than k vertices, else
            // 1 / Pr[rank < k-th] = 2^64 / S_h(v)[k-1] (single IEEE division)
            gr.wt = cnt_new < k ? 1.0 : __ddiv_rn(18446744073709551616.0, __ull2double_rn(kth));
            gr.v = v;
            gr.gidx = vg[v];
            gr.eidx = ve[v];
            gr.info = pack_info(hop, dcnt, counted);
            vg[v] = gr.gidx + 1;
            ve[v] = gr.eidx + dcnt;
            stg_grp[gat] = gr;
        }
        eat = __shfl_sync(kFull, eat, 0);
        if (lane < dcnt) stg_ent[eat + lane] = (int32_t)rank_vertex(seed, dv);
    }
    if (lane == 0 && merging) {
        atomicAdd(&ctr->cand_reads, cand_reads);
        atomicAdd(&ctr->merging, merging);
    }
}

// Sparse hops: the active set is N(frontier).  Warp per frontier vertex;
// each neighbour is appended once (stamp = hop).
__global__ void k_expand(const int32_t* __restrict__ fr, int64_t n_fr, const int64_t* __restrict__ rowp,
                         const int32_t* __restrict__ cols, uint32_t* __restrict__ stamp, uint32_t hop,
                         int32_t* __restrict__ act, Counters* ctr) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; w < n_fr; w += warps) {
        const int32_t u = fr[w];
        const int64_t beg = rowp[u], end = rowp[u + 1];
        for (int64_t cb = beg; cb < end; cb += 32) {
            int64_t e = cb + lane;
            bool fresh = false;
            int32_t v = 0;
            if (e < end) {
                v = cols[e];
                fresh = atomicExch(&stamp[v], hop) != hop;
            }
            unsigned m = __ballot_sync(kFull, fresh);
            if (!m) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctr->active, (unsigned long long)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (fresh) act[base + __popc(m & ((1u << lane) - 1u))] = v;
        }
    }
}

// ------------------------------------------------------------------ ADS compaction

__global__ void k_ads_scatter(const StgGroup* __restrict__ stg_grp, int64_t n_groups,
                              const int32_t* __restrict__ stg_ent, const int64_t* __restrict__ gofs,
                              const int64_t* __restrict__ eofs, uint32_t* __restrict__ ginfo,
                              double* __restrict__ gwt, int32_t* __restrict__ eid) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_groups; i += stride) {
        StgGroup gr = stg_grp[i];
        int64_t dg = gofs[gr.v] + gr.gidx;
        int64_t de = eofs[gr.v] + gr.eidx;
        ginfo[dg] = gr.info;
        gwt[dg] = gr.wt;
        int cnt = (int)((gr.info >> 16) & 0xff);
        for (int j = 0; j < cnt; ++j) eid[de + j] = stg_ent[gr.at + j];
    }
}

// ------------------------------------------------------------------ driver

static int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

int build_sketches(fl_graph* g, int k, uint64_t seed) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    g->built = 0;
    ++g->generation;
    g->k = k;
    g->seed = seed;
    const size_t nk = (size_t)n * k;
    FL_TRY(dalloc(g->S, nk * 8));
    FL_TRY(dalloc(g->Scnt, (size_t)n));
    for (int p = 0; p < 2; ++p) {
        FL_TRY(dalloc(g->D[p], nk * 8));
        FL_TRY(dalloc(g->Dcnt[p], (size_t)n));
        FL_TRY(dalloc(g->frontier[p], (size_t)n * 4));
    }
    FL_TRY(dalloc(g->stamp, (size_t)n * 4));
    FL_TRY(dalloc(g->vg, (size_t)n * 4));
    FL_TRY(dalloc(g->ve, (size_t)n * 4));
    // staging starts at ~4 entries per vertex and grows when a hop might not fit
    size_t ent_cap = std::max<size_t>((size_t)n * 4, 1024);
    size_t grp_cap = std::max<size_t>((size_t)n * 2, 1024);
    if (g->stg_ent_cap < ent_cap) { FL_TRY(dalloc(g->stg_ent, ent_cap * 4)); g->stg_ent_cap = ent_cap; }
    if (g->stg_grp_cap < grp_cap) { FL_TRY(dalloc(g->stg_grp, grp_cap * sizeof(StgGroup))); g->stg_grp_cap = grp_cap; }
    DBuf act;  // active list of sparse hops
    FL_TRY(dalloc(act, (size_t)n * 4));

    FL_CUDA(cudaMemsetAsync(g->S.p, 0xff, nk * 8, st));
    FL_CUDA(cudaMemsetAsync(g->D[0].p, 0xff, nk * 8, st));
    FL_CUDA(cudaMemsetAsync(g->D[1].p, 0xff, nk * 8, st));
    FL_CUDA(cudaMemsetAsync(g->stamp.p, 0, (size_t)n * 4, st));
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(kProfSketchOther, k_rank_init<<<grid_for(n, 256), 256, 0, st>>>(n, k, seed, g->S.as<uint64_t>(), g->Scnt.as<uint8_t>(),
                                                   g->D[0].as<uint64_t>(), g->Dcnt[0].as<uint8_t>(),
                                                   g->stg_ent.as<int32_t>(), g->stg_grp.as<StgGroup>(),
                                                   g->vg.as<int32_t>(), g->ve.as<int32_t>(), g->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    if (g->h_ctr->error) {
        dfree(act);
        FL_FAIL(FL_EINVAL, "a vertex rank equals the reserved empty-slot value; choose another seed");
    }
    Counters init{};
    init.stg_entries = (unsigned long long)n;
    init.stg_groups = (unsigned long long)n;
    int64_t n_front = n;                // hop 0: every vertex gained its own rank
    int64_t total_merges = 0, next_merges = g->nnz;
    int64_t used_ent = n, used_grp = n;
    int hop = 1;
    int rc = FL_OK;
    for (;; ++hop) {
        if (hop > kMaxHops) { rc = FL_ETIMEOUT; set_error(rc, "more than 65535 hops"); break; }
        total_merges += next_merges;
        const int64_t hop_merges = next_merges;
        const int64_t ent_before = used_ent;
        const int pin = (hop - 1) & 1, pout = hop & 1;
        const int32_t* act_list;
        int64_t n_act;
        // dense hops run every non-isolated vertex; sparse hops expand the frontier
        bool dense = n_front * 16 >= g->n_nonisolated;
        init.frontier = 0;
        init.active = 0;
        init.merges = 0;
        init.error = 0;
        FL_CUDA(cudaMemcpyAsync(g->ctr.p, &init, sizeof(Counters), cudaMemcpyHostToDevice, st));
        if (dense) {
            act_list = g->deg_list.as<int32_t>();
            n_act = g->n_nonisolated;
        } else {
            FL_LAUNCH(kProfSketchExpand, k_expand<<<grid_for(n_front, 8), 256, 0, st>>>(g->frontier[pin].as<int32_t>(), n_front,
                                                          g->rowp.as<int64_t>(), g->cols.as<int32_t>(),
                                                          g->stamp.as<uint32_t>(), (uint32_t)hop,
                                                          act.as<int32_t>(), g->ctr.as<Counters>()));
            FL_CUDA(cudaGetLastError());
            FL_TRY(read_counters(g));
            act_list = act.as<int32_t>();
            n_act = (int64_t)g->h_ctr->active;
        }
        // staging room for the worst case of this hop (k entries per active vertex)
        if ((size_t)(used_ent + n_act * k) > g->stg_ent_cap) {
            size_t cap = std::max<size_t>((size_t)(used_ent + n_act * k), g->stg_ent_cap * 3 / 2);
            FL_TRY(dgrow(g->stg_ent, cap * 4, (size_t)used_ent * 4, st));
            g->stg_ent_cap = cap;
        }
        if ((size_t)(used_grp + n_act) > g->stg_grp_cap) {
            size_t cap = std::max<size_t>((size_t)(used_grp + n_act), g->stg_grp_cap * 3 / 2);
            FL_TRY(dgrow(g->stg_grp, cap * sizeof(StgGroup), (size_t)used_grp * sizeof(StgGroup), st));
            g->stg_grp_cap = cap;
        }
        FL_CUDA(cudaMemsetAsync(g->Dcnt[pout].p, 0, (size_t)n, st));
        if (n_act > 0) {
            FL_LAUNCH(kProfSketchMerge, k_merge_hop<<<grid_for(n_act, 8), 256, 0, st>>>(
                act_list, nullptr, n_act, g->rowp.as<int64_t>(), g->cols.as<int32_t>(), k, seed, hop,
                g->S.as<uint64_t>(), g->Scnt.as<uint8_t>(), g->D[pin].as<uint64_t>(), g->Dcnt[pin].as<uint8_t>(),
                g->D[pout].as<uint64_t>(), g->Dcnt[pout].as<uint8_t>(), g->frontier[pout].as<int32_t>(),
                g->vg.as<int32_t>(), g->ve.as<int32_t>(), g->stg_ent.as<int32_t>(), g->stg_grp.as<StgGroup>(),
                g->ctr.as<Counters>()));
            FL_CUDA(cudaGetLastError());
        }
        FL_TRY(read_counters(g));
        n_front = (int64_t)g->h_ctr->frontier;
        next_merges = (int64_t)g->h_ctr->merges;
        used_ent = (int64_t)g->h_ctr->stg_entries;
        used_grp = (int64_t)g->h_ctr->stg_groups;
        init.stg_entries = (unsigned long long)used_ent;
        init.stg_groups = (unsigned long long)used_grp;
        // algorithmic bytes of this hop's merge: active row offsets (8 B), frontier
        // columns (4 B per edge-merge), neighbour deltas (8 B per rank), own sketch
        // read + write (16k B per merging vertex), new ADS entries (id + weight, 12 B)
        {
            const double A = (double)g->h_ctr->merging, SD = (double)g->h_ctr->cand_reads;
            g->prof.bytes[kProfSketchMerge] += 8.0 * A + 4.0 * (double)hop_merges + 8.0 * SD + 16.0 * k * A +
                                               12.0 * (double)(used_ent - ent_before);
        }
        if (n_front == 0) break;
    }
    dfree(act);
    if (rc != FL_OK) return rc;
    g->hops = hop - 1;
    g->edge_merges = total_merges;
    g->n_entries = used_ent;
    g->n_groups = used_grp;

    // vertex-major ADS
    FL_TRY(dalloc(g->gofs, (size_t)(n + 1) * 8));
    FL_TRY(dalloc(g->eofs, (size_t)(n + 1) * 8));
    FL_TRY(dalloc(g->ginfo, (size_t)used_grp * 4));
    FL_TRY(dalloc(g->gwt, (size_t)used_grp * 8));
    FL_TRY(dalloc(g->eid, (size_t)used_ent * 4));
    FL_TRY(scan_exclusive_i32_to_i64(g->vg.as<int32_t>(), g->gofs.as<int64_t>(), n, st, g->scratch));
    FL_TRY(scan_exclusive_i32_to_i64(g->ve.as<int32_t>(), g->eofs.as<int64_t>(), n, st, g->scratch));
    FL_CUDA(cudaMemcpyAsync(g->gofs.as<int64_t>() + n, &g->n_groups, 8, cudaMemcpyHostToDevice, st));
    FL_CUDA(cudaMemcpyAsync(g->eofs.as<int64_t>() + n, &g->n_entries, 8, cudaMemcpyHostToDevice, st));
    FL_LAUNCH(kProfSketchOther, k_ads_scatter<<<grid_for(used_grp, 256), 256, 0, st>>>(g->stg_grp.as<StgGroup>(), used_grp,
                                                          g->stg_ent.as<int32_t>(), g->gofs.as<int64_t>(),
                                                          g->eofs.as<int64_t>(), g->ginfo.as<uint32_t>(),
                                                          g->gwt.as<double>(), g->eid.as<int32_t>()));
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaStreamSynchronize(st));
    FL_TRY(compute_ecc_bound(g));
    g->built = 1;
    return FL_OK;
}

// ------------------------------------------------------------------ eccentricity bound
// The minimum rank of a component (S[v][0] at the fixed point) names a root
// for every vertex of it; a multi-source BFS from the roots gives d(v, root)
// and ecc(root), and ecc(v) <= d(v, root) + ecc(root).

__global__ void k_roots(const uint64_t* __restrict__ S, int k, uint64_t seed, int64_t n,
                        int32_t* __restrict__ root_of, int32_t* __restrict__ roots, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        int64_t v = base + lane_id();
        bool is_root = false;
        if (v < n) {
            int32_t r = (int32_t)rank_vertex(seed, S[v * k]);
            root_of[v] = r;
            is_root = r == v;
        }
        long long at = warp_append(is_root, &ctr->aux0);
        if (at >= 0) roots[at] = (int32_t)v;
    }
}

__global__ void k_ecc_max(const int32_t* __restrict__ label, const int32_t* __restrict__ dist, int64_t n,
                          int32_t* __restrict__ eccr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        atomicMax(&eccr[label[v]], dist[v]);
}

__global__ void k_ecc_ub(const int32_t* __restrict__ label, const int32_t* __restrict__ dist,
                         const int32_t* __restrict__ eccr, int64_t n, int32_t* __restrict__ ub) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        ub[v] = dist[v] + eccr[label[v]];
}

int compute_ecc_bound(fl_graph* g) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    DBuf root_of, roots, label, dist, eccr, X, stampb, fr[2], frval;
    auto cleanup = [&]() {
        dfree(root_of); dfree(roots); dfree(label); dfree(dist); dfree(eccr);
        dfree(X); dfree(stampb); dfree(fr[0]); dfree(fr[1]); dfree(frval);
    };
    int rc = FL_OK;
    do {
        if ((rc = dalloc(root_of, (size_t)n * 4))) break;
        if ((rc = dalloc(roots, (size_t)n * 4))) break;
        if ((rc = dalloc(label, (size_t)n * 4))) break;
        if ((rc = dalloc(dist, (size_t)n * 4))) break;
        if ((rc = dalloc(eccr, (size_t)n * 4))) break;
        if ((rc = dalloc(g->ecc_ub, (size_t)n * 4))) break;
        cudaError_t e = cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(eccr.p, 0, (size_t)n * 4, st);
        if (e != cudaSuccess) { rc = status_of(e, "ecc init", __FILE__, __LINE__); break; }
        FL_LAUNCH(kProfSketchOther, k_roots<<<grid_for(n, 256), 256, 0, st>>>(g->S.as<uint64_t>(), g->k, g->seed, n, root_of.as<int32_t>(),
                                                  roots.as<int32_t>(), g->ctr.as<Counters>()));
        if ((rc = read_counters(g))) break;
        int64_t n_roots = (int64_t)g->h_ctr->aux0;
        if ((rc = msbfs(g, roots.as<int32_t>(), n_roots, label.as<int32_t>(), dist.as<int32_t>(), X, stampb,
                        fr, frval, kProfSketchOther)))
            break;
        FL_LAUNCH(kProfSketchOther, k_ecc_max<<<grid_for(n, 256), 256, 0, st>>>(label.as<int32_t>(), dist.as<int32_t>(), n,
                                                    eccr.as<int32_t>()));
        FL_LAUNCH(kProfSketchOther, k_ecc_ub<<<grid_for(n, 256), 256, 0, st>>>(label.as<int32_t>(), dist.as<int32_t>(), eccr.as<int32_t>(),
                                                   n, g->ecc_ub.as<int32_t>()));
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "ecc bound", __FILE__, __LINE__); break; }
    } while (0);
    cleanup();
    return rc;
}

}  // namespace fl
