// k_exact.cu -- exact neighbourhood sizes, their HIP estimates, and radii
// from exact client counts: the ground truth of the ADS accuracy study
// (Section 5.1, "Accuracy vs. k", Fig. 1) and an exact-radius mode of phase
// (ii) (Eq. 1 at epsilon -> 0 with the true number of clients at each
// distance in place of the HIP estimate).
//
// Exact sizes come from a bit-parallel breadth-first search.  One sweep
// serves 256 sources; every vertex holds 4 words of source bits for
// "visited", "frontier" and "next".  A level is one bottom-up pass: vertex v
// ORs its neighbours' frontier words, keeps the bits of running sources
// that have not reached it yet, and counts them per source (under the
// predicate).  A source stops when its question is answered -- ball sizes at
// the largest distance asked for or when its component is exhausted, a
// radius when the walk of Eq. 1 has its root -- and its bit is masked out of
// every later level, so vertices every running source has reached are
// skipped.  Rows longer than 32 entries get a whole warp (8 neighbours x 4
// words per step, stopping once every needed bit is in); shorter rows get 4
// lanes, one word each, so the 4 words of a neighbour are one 32-byte
// sector.
#include <cmath>

#include "fl_internal.cuh"

namespace fl {
namespace {

constexpr int kXW = 4;          // 64-bit words of source bits per vertex
constexpr int kXS = 64 * kXW;   // sources per sweep
constexpr int kXHeavy = 32;     // rows longer than this get a whole warp
constexpr int kXBlocks = 152 * 8;

enum XMode { kXSizes = 0, kXRadius = 1 };

// State of one sweep (device).
struct XState {
    unsigned long long active[kXW];  // sources still searching
    unsigned long long any[kXW];     // sources that reached a vertex at this level
    unsigned long long cnt[kXS];     // this level's newly reached vertices under the predicate
    long long N[kXS];                // sizes: running ball size; radius: N_j
    long long G[kXS], Gp[kXS];       // radius: G_{j+1} and G_j of the walk
    unsigned long long rows, entries;  // rows scanned and their entries read (this sweep)
};

int blocks_for(int64_t items, int64_t per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > kXBlocks) b = kXBlocks;
    return (int)b;
}

// Original ids -> internal ids, with range checks.
__global__ void k_x_map(const int32_t* __restrict__ src, int64_t n_src, const int32_t* __restrict__ inv, int64_t n,
                        int32_t* __restrict__ out, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += stride) {
        const int32_t s = src[i];
        if (s < 0 || s >= n) {
            atomicOr(&ctr->error, 1ULL);
            out[i] = 0;
        } else {
            out[i] = inv ? inv[s] : s;
        }
    }
}

// Vertices with short rows (<= kXHeavy entries, isolated ones included) and
// with long rows.
__global__ void k_x_lists(const int64_t* __restrict__ rowp, int64_t n, int32_t* __restrict__ light,
                          int32_t* __restrict__ heavy, unsigned long long* n_light, unsigned long long* n_heavy) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool valid = v < n;
        const int64_t deg = valid ? rowp[v + 1] - rowp[v] : 0;
        const long long a = warp_append(valid && deg <= kXHeavy, n_light);
        if (a >= 0) light[a] = (int32_t)v;
        const long long b = warp_append(valid && deg > kXHeavy, n_heavy);
        if (b >= 0) heavy[b] = (int32_t)v;
    }
}

// Facilities (finite cost) of an exact-radius solve; every radius starts at
// +inf; a cost that is NaN, <= 0 or -inf is an error.
__global__ void k_x_facilities(const double* __restrict__ cost, int64_t n, int32_t* __restrict__ fac,
                               double* __restrict__ radius, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool valid = v < n;
        const double c = valid ? cost[v] : INFINITY;
        if (valid) {
            const bool ok = (c > 0.0 && c < INFINITY) || c == INFINITY;
            if (!ok) atomicOr(&ctr->error, 1ULL);
            radius[v] = INFINITY;
        }
        const long long at = warp_append(valid && c > 0.0 && c < INFINITY, &ctr->aux0);
        if (at >= 0) fac[at] = (int32_t)v;
    }
}

// Start of a sweep: the sources' own bits in "visited" and "frontier"
// (which the host cleared), cleared counters.  One block of kXS threads.
__global__ void k_x_seed(const int32_t* __restrict__ src, int64_t nb, unsigned long long* __restrict__ vis,
                         unsigned long long* __restrict__ cur, XState* __restrict__ st) {
    const int s = threadIdx.x;
    if (s < nb) {
        const int32_t v = src[s];
        const unsigned long long bit = 1ULL << (s & 63);
        atomicOr(&vis[(int64_t)v * kXW + (s >> 6)], bit);
        atomicOr(&cur[(int64_t)v * kXW + (s >> 6)], bit);
    }
    st->cnt[s] = 0;
    st->N[s] = 0;
    st->G[s] = 0;
    st->Gp[s] = 0;
    if (s < kXW) {
        const int64_t m = nb - 64LL * s;  // sources in word s
        st->active[s] = m <= 0 ? 0ULL : (m >= 64 ? ~0ULL : ((1ULL << m) - 1ULL));
        st->any[s] = 0;
    }
    if (s == 0) st->rows = st->entries = 0;
}

// Per-lane counters of one word's bits -> the sweep's per-source counts
// (lane (q, w) owns bits 8j + q of word w, j = 0..7), and the OR of the new
// bits.  Every thread of the block calls.
__device__ __forceinline__ void x_flush(const unsigned (&c)[8], unsigned long long any, unsigned long long rows,
                                        unsigned long long entries, unsigned* s_cnt, unsigned long long* s_any,
                                        XState* st) {
    const int lane = lane_id();
    const int w = lane & 3, q = lane >> 2;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (c[j]) atomicAdd(&s_cnt[w * 64 + 8 * j + q], c[j]);
    any |= __shfl_xor_sync(kFull, any, 4);
    any |= __shfl_xor_sync(kFull, any, 8);
    any |= __shfl_xor_sync(kFull, any, 16);
    if (lane < kXW && any) atomicOr(&s_any[lane], any);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rows += __shfl_xor_sync(kFull, rows, o);
        entries += __shfl_xor_sync(kFull, entries, o);
    }
    if (lane == 0 && rows) {
        atomicAdd(&st->rows, rows);
        atomicAdd(&st->entries, entries);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kXS; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(&st->cnt[i], (unsigned long long)s_cnt[i]);
    if (threadIdx.x < kXW && s_any[threadIdx.x]) atomicOr(&st->any[threadIdx.x], s_any[threadIdx.x]);
}

// One level for vertices with short rows: 4 lanes per vertex (lane w holds
// word w), 8 vertices per warp.
__global__ void __launch_bounds__(256) k_x_light(const int32_t* __restrict__ list, int64_t n_list,
                                                 const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                 const unsigned long long* __restrict__ cur,
                                                 unsigned long long* __restrict__ nxt, unsigned long long* vis,
                                                 const uint8_t* __restrict__ pred, XState* __restrict__ st) {
    __shared__ unsigned s_cnt[kXS];
    __shared__ unsigned long long s_any[kXW];
    for (int i = threadIdx.x; i < kXS; i += blockDim.x) s_cnt[i] = 0;
    if (threadIdx.x < kXW) s_any[threadIdx.x] = 0;
    __syncthreads();
    const int lane = lane_id();
    const int w = lane & 3, q = lane >> 2;
    const unsigned long long act = st->active[w];
    unsigned c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long any = 0, rows = 0, entries = 0;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 2;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x) + (threadIdx.x & ~31)) >> 2; base < n_list;
         base += stride) {
        const int64_t i = base + q;
        const bool valid = i < n_list;
        const int32_t v = valid ? __ldg(&list[i]) : 0;
        const unsigned long long vw = valid ? vis[(int64_t)v * kXW + w] : ~0ULL;
        const unsigned long long need = act & ~vw;
        const unsigned nb = __ballot_sync(kFull, need != 0);
        unsigned long long nx = 0;
        if ((nb >> (lane & ~3)) & 0xFu) {  // some word of this vertex still needs bits
            int64_t e = __ldg(&rowp[v]);
            const int64_t end = __ldg(&rowp[v + 1]);
            if (w == 0) {
                ++rows;
                entries += (unsigned long long)(end - e);
            }
            unsigned long long acc = 0;
            for (; e + 1 < end; e += 2) {
                const int32_t u0 = __ldg(&cols[e]), u1 = __ldg(&cols[e + 1]);
                acc |= __ldg(&cur[(int64_t)u0 * kXW + w]) | __ldg(&cur[(int64_t)u1 * kXW + w]);
            }
            if (e < end) acc |= __ldg(&cur[(int64_t)__ldg(&cols[e]) * kXW + w]);
            nx = acc & need;
        }
        if (valid) {
            nxt[(int64_t)v * kXW + w] = nx;
            if (nx) vis[(int64_t)v * kXW + w] = vw | nx;
        }
        any |= nx;
        const unsigned long long cv = (valid && (!pred || pred[v])) ? nx : 0ULL;
        if (__ballot_sync(kFull, cv != 0)) {
            // count bit b of word w over the warp's 8 vertices: the lanes
            // holding word w are w, w+4, ..., w+28
            const unsigned wm = 0x11111111u << w;
#pragma unroll
            for (int b = 0; b < 64; ++b) {
                const unsigned bal = __ballot_sync(kFull, (cv >> b) & 1ULL);
                if (q == (b & 7)) c[b >> 3] += __popc(bal & wm);
            }
        }
    }
    x_flush(c, any, rows, entries, s_cnt, s_any, st);
}

// One level for vertices with long rows: a warp per vertex, lane (t, w)
// reads word w of neighbours t, t+8, ...; every 256 entries the warp stops
// if its OR already holds every bit the vertex needs.
__global__ void __launch_bounds__(256) k_x_heavy(const int32_t* __restrict__ list, int64_t n_list,
                                                 const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                 const unsigned long long* __restrict__ cur,
                                                 unsigned long long* __restrict__ nxt, unsigned long long* vis,
                                                 const uint8_t* __restrict__ pred, XState* __restrict__ st) {
    __shared__ unsigned s_cnt[kXS];
    __shared__ unsigned long long s_any[kXW];
    for (int i = threadIdx.x; i < kXS; i += blockDim.x) s_cnt[i] = 0;
    if (threadIdx.x < kXW) s_any[threadIdx.x] = 0;
    __syncthreads();
    const int lane = lane_id();
    const int w = lane & 3, t = lane >> 2;
    const unsigned long long act = st->active[w];
    unsigned c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long any = 0, rows = 0, entries = 0;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; i < n_list; i += warps) {
        const int32_t v = __ldg(&list[i]);
        const unsigned long long vw = vis[(int64_t)v * kXW + w];
        const unsigned long long need = act & ~vw;
        unsigned long long nx = 0;
        if (__any_sync(kFull, need != 0)) {
            const int64_t beg = __ldg(&rowp[v]), end = __ldg(&rowp[v + 1]);
            int64_t stop = end;
            unsigned long long acc = 0;
            for (int64_t b0 = beg; b0 < end; b0 += 16) {
                const int64_t e0 = b0 + t, e1 = b0 + 8 + t;
                if (e0 < end) acc |= __ldg(&cur[(int64_t)__ldg(&cols[e0]) * kXW + w]);
                if (e1 < end) acc |= __ldg(&cur[(int64_t)__ldg(&cols[e1]) * kXW + w]);
                if (((b0 - beg) & 255) == 240) {
                    unsigned long long a = acc;
                    a |= __shfl_xor_sync(kFull, a, 4);
                    a |= __shfl_xor_sync(kFull, a, 8);
                    a |= __shfl_xor_sync(kFull, a, 16);
                    if (__all_sync(kFull, (a & need) == need)) {
                        acc = a;
                        stop = b0 + 16 < end ? b0 + 16 : end;
                        break;
                    }
                }
            }
            acc |= __shfl_xor_sync(kFull, acc, 4);
            acc |= __shfl_xor_sync(kFull, acc, 8);
            acc |= __shfl_xor_sync(kFull, acc, 16);
            nx = acc & need;
            if (lane == 0) {
                ++rows;
                entries += (unsigned long long)(stop - beg);
            }
        }
        if (t == 0) {
            nxt[(int64_t)v * kXW + w] = nx;
            if (nx) vis[(int64_t)v * kXW + w] = vw | nx;
        }
        any |= nx;
        // every lane holds its word's new bits; lane (t, w) counts bits 8j + t
        const unsigned long long cv = (!pred || pred[v]) ? nx : 0ULL;
#pragma unroll
        for (int j = 0; j < 8; ++j) c[j] += (unsigned)((cv >> (8 * j + t)) & 1ULL);
    }
    x_flush(c, any, rows, entries, s_cnt, s_any, st);
}

// End of a level (one block of kXS threads, thread s = source s of the
// sweep): fold the level's counts into each running source and stop the
// sources that are answered.  Level 0 is the source itself.
//   sizes:  N += (new vertices at this distance under the predicate);
//           row[level] = N; a source stops at level D or, filling the rest
//           of its row with N, at the first level that reaches nothing.
//   radius: the walk of Eq. 1: N_j = N_{j-1} + W_j, G_{j+1} = G_j + N_j;
//           r = j + (c - G_j) / N_j at the first j with G_{j+1} >= c; a
//           level that reaches nothing means j-1 was the eccentricity L and
//           r = L + (c - G_L) / N_L (+inf when N_L = 0).  N and G are exact
//           integers; each FP64 step is one IEEE operation.
__global__ void k_x_finish(XState* __restrict__ st, int mode, int64_t level, const int32_t* __restrict__ src,
                           const uint8_t* __restrict__ pred, const double* __restrict__ cost, int64_t D,
                           int64_t* __restrict__ sizes, double* __restrict__ radius, Counters* ctr) {
    __shared__ unsigned s_bal[kXS / 32];
    const int s = threadIdx.x;
    const int w = s >> 6;
    const unsigned long long bit = 1ULL << (s & 63);
    bool act = (st->active[w] & bit) != 0;
    if (act) {
        const int32_t v = src[s];
        long long W;
        bool found;
        if (level == 0) {
            W = (!pred || pred[v]) ? 1 : 0;
            found = true;
        } else {
            W = (long long)st->cnt[s];
            found = (st->any[w] & bit) != 0;
        }
        if (mode == kXSizes) {
            const long long N = st->N[s] + W;
            st->N[s] = N;
            int64_t* row = sizes + (int64_t)s * (D + 1);
            row[level] = N;
            if (!found) {
                for (int64_t h = level + 1; h <= D; ++h) row[h] = N;
                act = false;
            } else if (level == D) {
                act = false;
            }
        } else {
            const double c = cost[v];
            double r = INFINITY;
            if (!found) {
                const long long N = st->N[s];
                if (N > 0) r = __dadd_rn((double)(level - 1), __ddiv_rn(__dsub_rn(c, (double)st->Gp[s]), (double)N));
                act = false;
            } else {
                const long long N = st->N[s] + W;
                const long long G = st->G[s];
                const long long Gn = G + N;
                st->N[s] = N;
                if ((double)Gn >= c) {
                    r = __dadd_rn((double)level, __ddiv_rn(__dsub_rn(c, (double)G), (double)N));
                    act = false;
                } else {
                    st->Gp[s] = G;
                    st->G[s] = Gn;
                }
            }
            if (!act) radius[v] = r;
        }
    }
    __syncthreads();  // every thread has read active, any and its count
    st->cnt[s] = 0;
    const unsigned bal = __ballot_sync(kFull, act);
    if (lane_id() == 0) s_bal[s >> 5] = bal;
    __syncthreads();
    if (s < kXW) {
        st->active[s] = (unsigned long long)s_bal[2 * s] | ((unsigned long long)s_bal[2 * s + 1] << 32);
        st->any[s] = 0;
    }
    if (s == 0) {
        unsigned long long tot = 0;
        for (int i = 0; i < kXS / 32; ++i) tot += __popc(s_bal[i]);
        ctr->aux0 = tot;
        ctr->scanned = st->rows;
        ctr->cand_reads = st->entries;
    }
}

// HIP estimates of the same sizes from the ADS (the predicated
// neighbourhood query of Section 2.3; the estimator of Section 3.4): a warp
// per source; out row h = sum over the groups at hop <= h, in hop order, of
// (counted entries under the predicate) x the group's weight.
__global__ void __launch_bounds__(256) k_x_estimates(const int32_t* __restrict__ src, int64_t n_src, int64_t D,
                                                     const uint8_t* __restrict__ pred,
                                                     const int64_t* __restrict__ gofs,
                                                     const int64_t* __restrict__ eofs,
                                                     const uint32_t* __restrict__ ginfo,
                                                     const double* __restrict__ gwt, const int32_t* __restrict__ eid,
                                                     double* __restrict__ out) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; s < n_src; s += warps) {
        const int32_t v = src[s];
        const int64_t g0 = gofs[v], g1 = gofs[v + 1];
        int64_t e = eofs[v];
        double* row = out + s * (D + 1);
        double N = 0.0;
        int64_t h = 0;
        for (int64_t gi = g0; gi < g1; ++gi) {
            const uint32_t info = ginfo[gi];
            const int64_t hop = (int64_t)(info & 0xffffu);
            const int cnt = (int)((info >> 16) & 0xffu);
            const int counted = (int)(info >> 24);
            if (hop > D) break;
            for (int64_t x = h + lane; x < hop; x += 32) row[x] = N;  // distances before this group
            h = hop;
            const bool in = lane < counted && (!pred || pred[eid[e + lane]]);
            const int m = __popc(__ballot_sync(kFull, in));
            N = __dadd_rn(N, __dmul_rn((double)m, gwt[gi]));
            e += cnt;
        }
        for (int64_t x = h + lane; x <= D; x += 32) row[x] = N;
    }
}

// Sweeps of kXS sources over src[0, n_src) (internal ids).
int run_sweeps(fl_graph* g, int mode, int64_t n_src, const int32_t* src, int64_t D, const uint8_t* pred,
               const double* cost, int64_t* sizes, double* radius) {
    cudaStream_t st = g->stream;
    const int64_t n = g->n;
    const int cls = kProfExact;
    const size_t words = (size_t)n * kXW;
    FL_TRY(dalloc(g->xbits, words * 8 * 3));
    const size_t lists = ((size_t)n * 8 + 255) & ~(size_t)255;
    FL_TRY(dalloc(g->xaux, lists + sizeof(XState)));
    unsigned long long* vis = g->xbits.as<unsigned long long>();
    unsigned long long* buf[2] = {vis + words, vis + 2 * words};
    int32_t* light = g->xaux.as<int32_t>();
    int32_t* heavy = light + n;
    XState* xs = reinterpret_cast<XState*>(g->xaux.as<char>() + lists);
    Counters* ctr = g->ctr.as<Counters>();
    const int64_t* rowp = g->rowp.as<int64_t>();
    const int32_t* cols = g->cols.as<int32_t>();

    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(cls, k_x_lists<<<blocks_for(n, 256), 256, 0, st>>>(rowp, n, light, heavy, &ctr->aux0, &ctr->aux3));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    const int64_t n_light = (int64_t)g->h_ctr->aux0, n_heavy = (int64_t)g->h_ctr->aux3;
    const int grid_l = blocks_for(n_light, 64);  // 8 warps x 8 vertices per block pass
    const int grid_h = blocks_for(n_heavy, 8);   // 8 warps x 1 vertex

    for (int64_t b0 = 0; b0 < n_src; b0 += kXS) {
        const int64_t nb = n_src - b0 < kXS ? n_src - b0 : kXS;
        int64_t* rows = sizes ? sizes + b0 * (D + 1) : nullptr;
        // every listed vertex rewrites its "next" words each level, so only
        // the first frontier and the visited bits need clearing
        FL_CUDA(cudaMemsetAsync(vis, 0, words * 8, st));
        FL_CUDA(cudaMemsetAsync(buf[0], 0, words * 8, st));
        int c = 0;
        FL_LAUNCH(cls, k_x_seed<<<1, kXS, 0, st>>>(src + b0, nb, vis, buf[0], xs));
        FL_LAUNCH(cls, k_x_finish<<<1, kXS, 0, st>>>(xs, mode, 0, src + b0, pred, cost, D, rows, radius, ctr));
        FL_CUDA(cudaGetLastError());
        FL_TRY(read_counters(g));
        int64_t level = 1;
        for (; g->h_ctr->aux0 > 0; ++level) {
            if (level > n + 1) FL_FAIL(FL_ETIMEOUT, "exact search did not finish");
            if (n_heavy > 0)
                FL_LAUNCH(cls, k_x_heavy<<<grid_h, 256, 0, st>>>(heavy, n_heavy, rowp, cols, buf[c], buf[c ^ 1], vis,
                                                                 pred, xs));
            if (n_light > 0)
                FL_LAUNCH(cls, k_x_light<<<grid_l, 256, 0, st>>>(light, n_light, rowp, cols, buf[c], buf[c ^ 1], vis,
                                                                 pred, xs));
            FL_LAUNCH(cls, k_x_finish<<<1, kXS, 0, st>>>(xs, mode, level, src + b0, pred, cost, D, rows, radius, ctr));
            FL_CUDA(cudaGetLastError());
            c ^= 1;
            FL_TRY(read_counters(g));
        }
        // algorithmic bytes of the sweep's levels 1..: every listed vertex
        // reads its list id and visited words and writes its next words
        // (4 + 32 + 32 B); a scanned row reads two offsets (16 B) and, per
        // entry, the column (4 B) and the neighbour's frontier words (32 B)
        g->prof.bytes[cls] += 68.0 * (double)n * (double)(level - 1) + 16.0 * (double)g->h_ctr->scanned +
                              36.0 * (double)g->h_ctr->cand_reads;
    }
    return FL_OK;
}

}  // namespace

int map_sources(fl_graph* g, const int32_t* in, int64_t n_src, int32_t* out) {
    cudaStream_t st = g->stream;
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(kProfExact, k_x_map<<<blocks_for(n_src, 256), 256, 0, st>>>(
                              in, n_src, g->relabelled ? g->inv.as<int32_t>() : nullptr, g->n, out,
                              g->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    if (g->h_ctr->error) FL_FAIL(FL_EINVAL, "source ids must lie in [0, n)");
    return FL_OK;
}

int exact_ball_sizes(fl_graph* g, int64_t n_src, const int32_t* src, int64_t D, const uint8_t* pred, int64_t* out) {
    if (n_src == 0) return FL_OK;
    return run_sweeps(g, kXSizes, n_src, src, D, pred, nullptr, out, nullptr);
}

int hip_ball_estimates(fl_graph* g, int64_t n_src, const int32_t* src, int64_t D, const uint8_t* pred, double* out) {
    if (n_src == 0) return FL_OK;
    FL_LAUNCH(kProfExact, k_x_estimates<<<blocks_for(n_src, 8), 256, 0, g->stream>>>(
                              src, n_src, D, pred, g->gofs.as<int64_t>(), g->eofs.as<int64_t>(),
                              g->ginfo.as<uint32_t>(), g->gwt.as<double>(), g->eid.as<int32_t>(), out));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

int exact_radii(fl_solve* s) {
    fl_graph* g = s->g;
    cudaStream_t st = g->stream;
    const int64_t n = g->n;
    FL_TRY(dalloc(s->ulist, (size_t)n * 4 * 2));  // facility list (the MIS reuses the buffer later)
    int32_t* fac = s->ulist.as<int32_t>();
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(kProfExact, k_x_facilities<<<blocks_for(n, 256), 256, 0, st>>>(s->cost.as<double>(), n, fac,
                                                                            s->radii.as<double>(),
                                                                            g->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    if (g->h_ctr->error) FL_FAIL(FL_EINVAL, "open_cost must be finite and > 0 for facilities, +inf otherwise");
    const int64_t m = (int64_t)g->h_ctr->aux0;
    if (m == 0) return FL_OK;
    return run_sweeps(g, kXRadius, m, fac, 0, s->client.as<uint8_t>(), s->cost.as<double>(), nullptr,
                      s->radii.as<double>());
}

}  // namespace fl
