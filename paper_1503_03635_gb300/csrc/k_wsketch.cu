// k_wsketch.cu -- sketches and ADS of a weighted graph (Section 3.3 after
// Algorithm 2; edge weights drawn uniformly in [1, 100] in Section 5).
//
// The paper's Algorithm 2 runs in BFS-order supersteps, so on a weighted
// graph a vertex can accept an entry that a closer arrival later pushes out
// of the bottom-k, and a CleanUp step removes such entries.  This build runs
// in Dijkstra order instead: level L of the loop settles every ADS entry at
// distance exactly L, so an accepted entry is final and nothing needs
// cleaning (both orders end at the ADS of the definition).  Lengths are
// positive integers, so the levels are the integers 0, 1, 2, ... up to the
// largest distance (at most 65535, the width of a group's distance field).
//
// Level L: v is active when a neighbour u gained entries at distance
// L - w(u, v); a ring of (largest length + 1) bitmaps holds the activations
// of the coming levels, and a second ring of bitmaps over the CSR entries
// marks which entries (v, u) of an active v deliver at that level (u posts
// to the entry of v's row paired with its own entry (u, v), so v reads only
// the neighbours that gained).  An active v merges into its bottom-k sketch the
// entries of each such neighbour u at distance L - w(u, v); the ranks that enter
// form v's group at distance L, with the HIP weight and counted prefix of
// the unweighted build (the sketch after the level, ties at one distance in
// ascending rank).  A vertex's entries are kept in distance order in a
// fixed-capacity row, so each edge keeps a cursor into its neighbour's row
// that only moves forward.  Entries appended at level L have distance L and
// are never read in the same level (every length is >= 1): a level reads the
// row counts as they were when it started and writes the new counts to a
// second array, which a commit pass over the active vertices copies back.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "fl_internal.cuh"

namespace fl {

namespace {

int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

struct WEnt {
    int32_t id;
    int32_t dist;
};

// One group of the log: vertex, its index among the vertex's groups, and
// the group's distance, entry count, counted prefix, weight, first entry.
struct WGroup {
    double wt;
    int32_t v, gidx;
    int32_t dist, cnt, counted, first;
};

struct WArgs {
    const int64_t* rowp;
    const int32_t* cols;
    const int32_t* wts;
    int k;
    int cap;                 // entries per vertex row
    uint64_t seed;
    uint64_t* S;             // n*k
    uint8_t* Scnt;           // n
    WEnt* ent;               // n*cap
    int32_t* ecnt;           // n: entries at the start of the level (read)
    int32_t* ecnt_n;         // n: entries after the level (written by the active vertices)
    int32_t* gcnt;           // n: groups
    int32_t* cursor;         // nnz
    WGroup* glog;            // group log
    unsigned long long* glog_n;
    unsigned long long glog_cap;
    uint32_t* ring;          // R bitmaps of `words` words
    int64_t words;
    int R;
    const uint32_t* rev;     // nnz: the entry (v, u) paired with each entry (u, v)
    uint32_t* marks;         // R bitmaps of `mwords` words over the CSR entries
    int64_t mwords;
    unsigned long long* pend;  // R activation counts
    unsigned long long* err;   // 1: a row overflowed; 2: a distance above 65535; 4: the group log overflowed
};

__device__ __forceinline__ void activate(const WArgs& a, int32_t u, int64_t level) {
    const int slot = (int)(level % a.R);
    const uint32_t bit = 1u << (u & 31);
    const uint32_t old = atomicOr(&a.ring[(int64_t)slot * a.words + (u >> 5)], bit);
    if (!(old & bit)) atomicAdd(&a.pend[slot], 1ULL);
}

// The source of CSR entry e = (u, v) gained entries that reach v at `level`:
// mark v's paired entry (v, u) and activate v.
__device__ __forceinline__ void post(const WArgs& a, int64_t e, int64_t level) {
    const int slot = (int)(level % a.R);
    const uint32_t re = a.rev[e];
    atomicOr(&a.marks[(int64_t)slot * a.mwords + (re >> 5)], 1u << (re & 31));
    activate(a, a.cols[e], level);
}

// Level 0: every vertex's own rank; its neighbours become active at the
// lengths of its edges.
__global__ void k_winit(WArgs a, int64_t n) {
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = lane_id();
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        if (lane < a.k) a.S[v * a.k + lane] = lane == 0 ? vertex_rank(a.seed, v) : kEmpty;
        if (lane == 0) {
            a.Scnt[v] = 1;
            a.ent[v * a.cap] = WEnt{(int32_t)v, 0};
            a.ecnt[v] = 1;
            a.gcnt[v] = 1;
            WGroup gr;
            gr.wt = 1.0;  // a ball of one vertex (k >= 2)
            gr.v = (int32_t)v;
            gr.gidx = 0;
            gr.dist = 0;
            gr.cnt = 1;
            gr.counted = 1;
            gr.first = 0;
            a.glog[v] = gr;
        }
        for (int64_t e = a.rowp[v] + lane; e < a.rowp[v + 1]; e += 32) {
            a.cursor[e] = 0;
            post(a, e, a.wts[e]);
        }
    }
}

// Active vertices of a level from its ring slot (the slot is cleared).
__global__ void k_wcollect(uint32_t* __restrict__ bm, int64_t words, int64_t n, int32_t* __restrict__ out,
                           unsigned long long* __restrict__ n_out) {
    __shared__ BlockAppend<8> sh;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < words * 32; bb += stride) {
        const int64_t v = bb + threadIdx.x;
        const int64_t w = v >> 5;
        const uint32_t word = w < words ? bm[w] : 0u;
        const bool in = v < n && ((word >> (v & 31)) & 1u);
        const long long at = block_append<8>(in, n_out, sh);
        if (at >= 0) out[at] = (int32_t)v;
        __syncwarp();
        if ((threadIdx.x & 31) == 0 && w < words && word) bm[w] = 0u;
    }
}

// One level: a warp per active vertex (see the file comment).
__global__ void __launch_bounds__(256) k_wlevel(WArgs a, const int32_t* __restrict__ act,
                                                const unsigned long long* __restrict__ n_act_d, int32_t L) {
    __shared__ int32_t s_stage[8][1024];      // per warp: the delivering entries of 32 mark words
    const int64_t n_act = (int64_t)*n_act_d;  // the vertices the collect pass listed
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_act; i += warps) {
        const int32_t v = act[i];
        const int cnt_old = a.Scnt[v];
        const uint64_t s_old = lane < cnt_old ? a.S[(int64_t)v * a.k + lane] : kEmpty;
        uint64_t s = s_old;
        int cnt = cnt_old;
        uint64_t kth = cnt == a.k ? __shfl_sync(kFull, s, a.k - 1) : kEmpty;
        const int64_t e0 = a.rowp[v], e1 = a.rowp[v + 1];
        const uint32_t* mk = a.marks + (int64_t)(L % a.R) * a.mwords;
        int32_t* stage = s_stage[threadIdx.x >> 5];
        const int64_t w1 = (e1 + 31) >> 5;
        for (int64_t wb = e0 >> 5; wb < w1; wb += 32) {
            // 32 words of marks at once: their set bits inside [e0, e1) are the
            // delivering entries, staged in row order (a hub's row holds
            // thousands of entries, a few of which deliver at a level)
            const int64_t wi = wb + lane;
            uint32_t bits = 0;
            if (wi < w1) {
                bits = mk[wi];
                const int64_t first = wi << 5;
                if (first < e0) bits &= ~0u << (int)(e0 - first);
                if (e1 - first < 32) bits &= (1u << (int)(e1 - first)) - 1u;
            }
            const int mine = __popc(bits);
            int pre = mine;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, pre, o);
                if (lane >= o) pre += y;
            }
            const int total = __shfl_sync(kFull, pre, 31);
            if (total == 0) continue;
            pre -= mine;
            for (uint32_t b = bits; b; b &= b - 1u) stage[pre++] = (int32_t)((wi << 5) + (__ffs(b) - 1) - e0);
            __syncwarp();
            for (int cb = 0; cb < total; cb += 32) {
                const int j = cb + lane;
                int32_t u = 0, c0 = 0, c1 = 0;
                if (j < total) {
                    const int64_t e = e0 + stage[j];
                    u = a.cols[e];
                    const int32_t x = L - a.wts[e];
                    if (x >= 0) {
                        const int32_t have = min(a.ecnt[u], a.cap);
                        const WEnt* row = a.ent + (int64_t)u * a.cap;
                        int32_t c = min(a.cursor[e], have);
                        while (c < have && row[c].dist < x) ++c;
                        c0 = c;
                        while (c < have && row[c].dist == x) ++c;
                        c1 = c;
                        a.cursor[e] = c;  // later levels ask for larger distances
                    }
                }
                // each lane offers its entry's candidates one per round
                while (__any_sync(kFull, c0 < c1)) {
                    uint64_t r = kEmpty;
                    if (c0 < c1) {
                        r = vertex_rank(a.seed, a.ent[(int64_t)u * a.cap + c0].id);
                        ++c0;
                        if (r >= kth) r = kEmpty;  // cannot enter a full sketch
                    }
                    if (warp_member(s, r)) r = kEmpty;  // already held
                    r = warp_sort(r);
                    const uint64_t prev = __shfl_up_sync(kFull, r, 1);
                    const bool keep = r != kEmpty && (lane == 0 || prev != r);
                    r = warp_compact(r, __ballot_sync(kFull, keep), kEmpty);
                    if (__ballot_sync(kFull, r != kEmpty) == 0) continue;
                    s = warp_merge_low(s, r);
                    if (lane >= a.k) s = kEmpty;
                    cnt = __popc(__ballot_sync(kFull, s != kEmpty));
                    kth = cnt == a.k ? __shfl_sync(kFull, s, a.k - 1) : kEmpty;
                }
            }
            __syncwarp();
        }
        // the entries gained at distance L: in the new sketch, not in the old
        // (every lane takes part in the membership shuffles)
        const bool held = warp_member(s_old, s);
        const bool fresh = s != kEmpty && !held;
        const unsigned fm = __ballot_sync(kFull, fresh);
        const int32_t base = a.ecnt[v];
        if (!fm) {
            if (lane == 0) a.ecnt_n[v] = base;
            continue;
        }
        const int dcnt = __popc(fm);
        if (base + dcnt > a.cap) {
            if (lane == 0) {
                a.ecnt_n[v] = base;
                atomicOr(a.err, 1ULL);
            }
            continue;
        }
        const int counted = __popc(fm & (cnt < a.k ? kFull : ((1u << (a.k - 1)) - 1u)));
        const double wt = hip_weight(cnt, a.k, __shfl_sync(kFull, s, a.k - 1));
        if (fresh) {
            const int at = base + __popc(fm & ((1u << lane) - 1u));
            a.ent[(int64_t)v * a.cap + at] = WEnt{(int32_t)rank_vertex(a.seed, s), L};
        }
        if (lane < a.k) a.S[(int64_t)v * a.k + lane] = s;
        if (lane == 0) {
            a.ecnt_n[v] = base + dcnt;
            a.Scnt[v] = (uint8_t)cnt;
            const unsigned long long gi = atomicAdd(a.glog_n, 1ULL);
            if (gi < a.glog_cap) {
                WGroup gr;
                gr.wt = wt;
                gr.v = v;
                gr.gidx = a.gcnt[v]++;
                gr.dist = L;
                gr.cnt = dcnt;
                gr.counted = counted;
                gr.first = base;
                a.glog[gi] = gr;
            } else {
                atomicOr(a.err, 4ULL);
            }
        }
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int64_t lv = (int64_t)L + a.wts[e];
            if (lv > 65535) atomicOr(a.err, 2ULL);
            else post(a, e, lv);
        }
    }
}

// End of a level: the active vertices' new row counts become current.
__global__ void k_wcommit(const int32_t* __restrict__ act, const unsigned long long* __restrict__ n_act_d,
                          const int32_t* __restrict__ ecnt_n, int32_t* __restrict__ ecnt) {
    const int64_t n_act = (int64_t)*n_act_d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_act; i += stride) {
        const int32_t v = act[i];
        ecnt[v] = ecnt_n[v];
    }
}

// Vertex-major ADS from the group log and the rows.
__global__ void k_wgroups(const WGroup* __restrict__ glog, int64_t m, const int64_t* __restrict__ gofs,
                          uint32_t* __restrict__ ginfo, double* __restrict__ gwt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const WGroup gr = glog[i];
        const int64_t at = gofs[gr.v] + gr.gidx;
        ginfo[at] = (uint32_t)gr.dist | ((uint32_t)gr.cnt << 16) | ((uint32_t)gr.counted << 24);
        gwt[at] = gr.wt;
    }
}

__global__ void k_wentries(const WEnt* __restrict__ ent, int cap, const int32_t* __restrict__ ecnt,
                           const int64_t* __restrict__ eofs, int64_t n, int32_t* __restrict__ eid) {
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps)
        for (int j = lane_id(); j < ecnt[v]; j += 32) eid[eofs[v] + j] = ent[v * cap + j].id;
}

__global__ void k_wmaxlen(const int32_t* __restrict__ w, int64_t nnz, unsigned long long* __restrict__ out,
                          unsigned long long* __restrict__ bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned mx = 0;
    bool neg = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t x = w[e];
        neg |= x < 1;
        mx = max(mx, (unsigned)max(x, 0));
    }
    mx = __reduce_max_sync(kFull, mx);
    if (lane_id() == 0) atomicMax(out, (unsigned long long)mx);
    if (__any_sync(kFull, neg) && lane_id() == 0) atomicOr(bad, 1ULL);
}

// Pairing keys of the CSR entries: (min(u, v), max(u, v)) and (length,
// direction), the entry index as payload (a warp per source vertex u).
__global__ void k_wrevkeys(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                           const int32_t* __restrict__ wts, int64_t n, uint64_t* __restrict__ hi,
                           uint64_t* __restrict__ lo, uint32_t* __restrict__ val) {
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        for (int64_t e = rowp[u] + lane_id(); e < rowp[u + 1]; e += 32) {
            const int64_t v = cols[e];
            const uint64_t a = (uint64_t)(u < v ? u : v), b = (uint64_t)(u < v ? v : u);
            hi[e] = (a << 32) | b;
            lo[e] = ((uint64_t)(uint32_t)wts[e] << 1) | (u > v ? 1u : 0u);
            val[e] = (uint32_t)e;
        }
    }
}

// First index of the sorted keys at or above (h, l).
__device__ __forceinline__ int64_t key_lower_bound(const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo,
                                                   int64_t m, uint64_t h, uint64_t l) {
    int64_t a = 0, b = m;
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        const uint64_t x = hi[mid];
        if (x < h || (x == h && lo[mid] < l)) a = mid + 1;
        else b = mid;
    }
    return a;
}

// After the sort, the entries of one edge and length form a group whose
// first half runs min -> max and second half max -> min; the i-th of each
// half pair up (a self-loop pairs with itself).  A group whose halves differ
// means a length that is not the same in both directions (bad = 1).
__global__ void k_wpair(const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo,
                        const uint32_t* __restrict__ val, int64_t m, uint32_t* __restrict__ rev,
                        unsigned long long* __restrict__ bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint64_t h = hi[i], l = lo[i];
        if ((h >> 32) == (h & 0xffffffffULL)) {
            rev[val[i]] = val[i];
            continue;
        }
        const uint64_t l0 = l & ~1ULL;  // the group: keys (h, l0) and (h, l0 | 1)
        const int64_t g0 = key_lower_bound(hi, lo, m, h, l0);
        const int64_t g1 = key_lower_bound(hi, lo, m, h, l0 + 2);
        const int64_t half = (g1 - g0) >> 1;
        if (((g1 - g0) & 1) || half < 1 || lo[g0 + half - 1] != l0 || lo[g0 + half] != (l0 | 1u)) {
            atomicOr(bad, 1ULL);
            continue;
        }
        if (l & 1u) continue;  // the second half is written by its partners
        const int64_t j = i + half;
        rev[val[i]] = val[j];
        rev[val[j]] = val[i];
    }
}

}  // namespace

// For every CSR entry (u, v) of a weighted graph, an entry (v, u) of the same
// length, paired one to one (duplicates pair in order): the weighted build
// marks the paired entry of v's row when u gains entries.  FL_EINVAL when an
// edge's lengths differ between its two directions.
int pair_reverse_edges(fl_graph* g) {
    const int64_t n = g->n, nnz = g->nnz;
    cudaStream_t st = g->stream;
    if (nnz >= (1LL << 32)) FL_FAIL(FL_EINVAL, "a weighted graph holds fewer than 2^32 CSR entries");
    FL_TRY(dalloc(g->wrev, (size_t)std::max<int64_t>(nnz, 1) * 4));
    if (nnz == 0) return FL_OK;
    DBuf hi, lo, val, flag;
    int rc = FL_OK;
    do {
        if ((rc = dalloc(hi, (size_t)nnz * 8)) || (rc = dalloc(lo, (size_t)nnz * 8)) ||
            (rc = dalloc(val, (size_t)nnz * 4)) || (rc = dalloc(flag, 16)))
            break;
        cudaError_t e = cudaMemsetAsync(flag.p, 0, 16, st);
        if (e != cudaSuccess) { rc = status_of(e, "edge pairing", __FILE__, __LINE__); break; }
        FL_LAUNCH(kProfOther, k_wrevkeys<<<grid_for(n * 32, 256), 256, 0, st>>>(
                                  g->rowp.as<int64_t>(), g->cols.as<int32_t>(), g->wts.as<int32_t>(), n,
                                  hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>()));
        // the digits that can vary: ids below n in both halves of hi, the
        // length and the direction bit in lo
        int nb = 1, wb = 1;
        while (nb < 31 && (1LL << nb) < n) ++nb;
        while (wb < 17 && (1 << wb) <= g->max_w) ++wb;
        uint32_t digits = 0;
        for (int d = 0; d * 4 < wb + 1; ++d) digits |= 1u << d;
        for (int d = 0; d * 4 < nb; ++d) digits |= (1u << (16 + d)) | (1u << (24 + d));
        if ((rc = sort_pairs_u128_digits(hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>(), nnz, st,
                                         g->scratch, kProfOther, digits)))
            break;
        FL_LAUNCH(kProfOther, k_wpair<<<grid_for(nnz, 256), 256, 0, st>>>(
                                  hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>(), nnz,
                                  g->wrev.as<uint32_t>(), flag.as<unsigned long long>()));
        unsigned long long h = 0;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag.p, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "edge pairing", __FILE__, __LINE__); break; }
        if (h) {
            rc = FL_EINVAL;
            set_error(rc, "an edge's length must be the same in both directions");
        }
    } while (0);
    dfree_after(st, {&hi, &lo, &val, &flag});
    return rc;
}

int check_weights(fl_graph* g) {
    cudaStream_t st = g->stream;
    DBuf tmp;
    FL_TRY(dalloc(tmp, 16));
    unsigned long long* d = tmp.as<unsigned long long>();
    FL_CUDA(cudaMemsetAsync(d, 0, 16, st));
    if (g->nnz > 0)
        FL_LAUNCH(kProfOther, k_wmaxlen<<<grid_for(g->nnz, 256), 256, 0, st>>>(g->wts.as<int32_t>(), g->nnz, d, d + 1));
    unsigned long long h[2] = {0, 0};
    FL_CUDA(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    dfree_after(st, {&tmp});
    if (h[1]) FL_FAIL(FL_EINVAL, "edge lengths must be positive integers");
    if (h[0] > 65535) FL_FAIL(FL_EINVAL, "edge lengths must be at most 65535");
    g->max_w = (int)h[0];
    return FL_OK;
}

int build_sketches_weighted(fl_graph* g, int k, uint64_t seed) {
    const int64_t n = g->n, nnz = g->nnz;
    cudaStream_t st = g->stream;
    const int R = g->max_w + 1;
    const int64_t words = (n + 31) / 32;
    // entries per vertex: about k (1 + ln(n / k)) expected; twice that plus a
    // margin, at most n; doubled and rebuilt on overflow
    const double expect = (double)k * (1.0 + std::log(std::max(1.0, (double)n / k)));
    int64_t cap = std::min<int64_t>(n, (int64_t)(2.0 * expect) + 64);
    const int64_t mwords = (nnz + 31) / 32;
    DBuf ent, ecnt, ecnt_n, gcnt, cursor, glog, ring, pend, act, cnt, marks;
    int rc = FL_OK;
    for (;;) {
        const unsigned long long glog_cap = (unsigned long long)n * (unsigned long long)cap;
        if ((rc = dalloc(g->S, (size_t)n * k * 8)) || (rc = dalloc(g->Scnt, (size_t)n)) ||
            (rc = dalloc(ent, (size_t)n * cap * sizeof(WEnt))) || (rc = dalloc(ecnt, (size_t)n * 4)) ||
            (rc = dalloc(ecnt_n, (size_t)n * 4)) ||
            (rc = dalloc(gcnt, (size_t)n * 4)) || (rc = dalloc(cursor, (size_t)std::max<int64_t>(nnz, 1) * 4)) ||
            (rc = dalloc(glog, (size_t)glog_cap * sizeof(WGroup))) ||
            (rc = dalloc(ring, (size_t)R * words * 4 + 16)) || (rc = dalloc(pend, (size_t)R * 8)) ||
            (rc = dalloc(act, (size_t)n * 4)) || (rc = dalloc(cnt, 64)) ||
            (rc = dalloc(marks, (size_t)R * mwords * 4 + 16)))
            break;
        WArgs a;
        a.rowp = g->rowp.as<int64_t>();
        a.cols = g->cols.as<int32_t>();
        a.wts = g->wts.as<int32_t>();
        a.k = k;
        a.cap = (int)cap;
        a.seed = seed;
        a.S = g->S.as<uint64_t>();
        a.Scnt = g->Scnt.as<uint8_t>();
        a.ent = ent.as<WEnt>();
        a.ecnt = ecnt.as<int32_t>();
        a.ecnt_n = ecnt_n.as<int32_t>();
        a.gcnt = gcnt.as<int32_t>();
        a.cursor = cursor.as<int32_t>();
        a.glog = glog.as<WGroup>();
        unsigned long long* c = cnt.as<unsigned long long>();  // [0] log size, [1] errors, [2] active
        a.glog_n = c;
        a.glog_cap = glog_cap;
        a.err = c + 1;
        a.ring = ring.as<uint32_t>();
        a.words = words;
        a.R = R;
        a.pend = pend.as<unsigned long long>();
        a.rev = g->wrev.as<uint32_t>();
        a.marks = marks.as<uint32_t>();
        a.mwords = mwords;
        cudaError_t e = cudaMemsetAsync(ring.p, 0, (size_t)R * words * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(marks.p, 0, (size_t)R * mwords * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(pend.p, 0, (size_t)R * 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, 64, st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
        const unsigned long long nlog0 = (unsigned long long)n;  // level 0 takes log slots 0..n-1
        e = cudaMemcpyAsync(c, &nlog0, 8, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
        FL_LAUNCH(kProfSketchMerge, k_winit<<<grid_for(n, 8), 256, 0, st>>>(a, n));
        std::vector<unsigned long long> hp((size_t)R);
        int64_t L = 0, last = 0, levels = 0;
        unsigned long long logged = nlog0, now = 0;
        for (;;) {
            e = cudaMemcpyAsync(hp.data(), pend.p, (size_t)R * 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&now, c, 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
            if (now > logged) {  // the level just run added groups: the largest distance so far
                last = L;
                logged = now;
            }
            int64_t next = -1;  // the next level with activations
            for (int d = 1; d <= R; ++d)
                if (hp[(size_t)((L + d) % R)]) { next = L + d; break; }
            if (next < 0) break;
            L = next;
            if (L > 65535) { rc = FL_EINVAL; set_error(rc, "a distance above 65535"); break; }
            const int slot = (int)(L % R);
            e = cudaMemsetAsync(&c[2], 0, 8, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(&a.pend[slot], 0, 8, st);
            if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
            FL_LAUNCH(kProfSketchExpand, k_wcollect<<<grid_for(words * 32, 256), 256, 0, st>>>(
                                             a.ring + (int64_t)slot * words, words, n, act.as<int32_t>(), &c[2]));
            const int64_t n_act = (int64_t)hp[(size_t)slot];  // sizes the grids; the kernels read the list's count
            FL_LAUNCH(kProfSketchMerge, k_wlevel<<<grid_for(n_act, 8), 256, 0, st>>>(a, act.as<int32_t>(), &c[2],
                                                                                       (int32_t)L));
            FL_LAUNCH(kProfSketchMerge, k_wcommit<<<grid_for(n_act, 256), 256, 0, st>>>(
                                            act.as<int32_t>(), &c[2], a.ecnt_n, a.ecnt));
            // the level's entry marks are read: the slot serves level L + R next
            e = cudaMemsetAsync(a.marks + (int64_t)slot * mwords, 0, (size_t)mwords * 4, st);
            if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
            ++levels;
        }
        if (rc != FL_OK) break;
        unsigned long long hc[2] = {0, 0};
        e = cudaMemcpyAsync(hc, c, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
        if (hc[1] & 2ULL) { rc = FL_EINVAL; set_error(rc, "a distance above 65535"); break; }
        if ((hc[1] & 5ULL) && cap < n) {  // a row overflowed: twice the capacity
            cap = std::min<int64_t>(n, cap * 2);
            continue;
        }
        if (hc[1]) { rc = FL_ECUDA; set_error(rc, "weighted build: inconsistent row capacity"); break; }
        // vertex-major ADS
        const int64_t m = (int64_t)hc[0];
        if ((rc = dalloc(g->gofs, (size_t)(n + 1) * 8)) || (rc = dalloc(g->eofs, (size_t)(n + 1) * 8))) break;
        if ((rc = scan_exclusive_i32_to_i64(gcnt.as<int32_t>(), g->gofs.as<int64_t>(), n, st, g->scratch)) ||
            (rc = scan_exclusive_i32_to_i64(ecnt.as<int32_t>(), g->eofs.as<int64_t>(), n, st, g->scratch)))
            break;
        int64_t ne = 0;
        int64_t tail_g = 0, tail_e = 0;
        e = cudaMemcpyAsync(&tail_g, g->gofs.as<int64_t>() + n - 1, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&tail_e, g->eofs.as<int64_t>() + n - 1, 8, cudaMemcpyDeviceToHost, st);
        int32_t lg = 0, le = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&lg, gcnt.as<int32_t>() + n - 1, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&le, ecnt.as<int32_t>() + n - 1, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
        g->n_groups = tail_g + lg;
        ne = tail_e + le;
        g->n_entries = ne;
        if (g->n_groups != m) { rc = FL_ECUDA; set_error(rc, "weighted build: group log and counts disagree"); break; }
        e = cudaMemcpyAsync(g->gofs.as<int64_t>() + n, &g->n_groups, 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->eofs.as<int64_t>() + n, &g->n_entries, 8, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
        if ((rc = dalloc(g->ginfo, (size_t)std::max<int64_t>(m, 1) * 4)) ||
            (rc = dalloc(g->gwt, (size_t)std::max<int64_t>(m, 1) * 8)) ||
            (rc = dalloc(g->eid, (size_t)std::max<int64_t>(ne, 1) * 4)))
            break;
        FL_LAUNCH(kProfSketchOther, k_wgroups<<<grid_for(m, 256), 256, 0, st>>>(
                                        glog.as<WGroup>(), m, g->gofs.as<int64_t>(), g->ginfo.as<uint32_t>(),
                                        g->gwt.as<double>()));
        FL_LAUNCH(kProfSketchOther, k_wentries<<<grid_for(n, 8), 256, 0, st>>>(
                                        ent.as<WEnt>(), (int)cap, ecnt.as<int32_t>(), g->eofs.as<int64_t>(), n,
                                        g->eid.as<int32_t>()));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted build", __FILE__, __LINE__); break; }
        g->hops = last;
        g->edge_merges = 0;
        g->wlevels = levels;
        break;
    }
    dfree_after(st, {&ent, &ecnt, &ecnt_n, &gcnt, &cursor, &glog, &ring, &pend, &act, &cnt, &marks});
    return rc;
}

}  // namespace fl
