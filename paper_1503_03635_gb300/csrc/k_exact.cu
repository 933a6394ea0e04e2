// k_exact.cu -- exact neighbourhood sizes, their HIP estimates, and radii
// from exact client counts: the ground truth of the ADS accuracy study
// (Section 5.1, "Accuracy vs. k", Fig. 1) and an exact-radius mode of phase
// (ii) (Eq. 1 at epsilon -> 0 with the true number of clients at each
// distance in place of the HIP estimate).
//
// Exact sizes come from a bit-parallel breadth-first search.  One sweep
// serves 256 sources; every vertex holds 4 words of source bits for
// "visited", "frontier" and "next".  A source stops when its question is
// answered -- ball sizes at the largest distance asked for or when its
// component is exhausted, a radius when the walk of Eq. 1 has its root --
// and its bit is masked out of every later level.  Each level runs in one of
// two directions (Beamer, Asanovic, Patterson, SC 2012), chosen from the
// frontier's row entries against the entries of rows that still need bits:
//   bottom-up: every vertex that some running source has not reached ORs
//     its neighbours' frontier words and keeps the new bits.  Rows longer
//     than 32 entries get a whole warp (8 neighbours x 4 words per step,
//     stopping once every needed bit is in); shorter rows get 4 lanes, one
//     word each, so the 4 words of a neighbour are one 32-byte sector.
//   top-down (sparse frontiers, e.g. the sources themselves): the frontier
//     rows, cut into work items of 256 entries (so a hub's row is spread
//     over many warps), OR their bits into the neighbours' next words
//     (atomicOr); one pass over all vertices then folds the new bits into
//     "visited" and counts them.
// Both directions count the new bits per source under the predicate and
// list the next frontier with its row entries.
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
    unsigned long long rows, entries;  // rows scanned and their entries read (this sweep, cumulative)
    unsigned long long n_next;       // this level: vertices listed in the next frontier
    unsigned long long fr_edges;     // this level: row entries of the next frontier
    unsigned long long rem_edges;    // bottom-up level: row entries of vertices that still need bits
};

// Per-lane sums a level kernel flushes once.
struct XSums {
    unsigned long long rows = 0, entries = 0, fr_edges = 0, rem_edges = 0;
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
// (which the host cleared), the sources as the first frontier list, cleared
// counters.  One block of kXS threads.
__global__ void k_x_seed(const int32_t* __restrict__ src, int64_t nb, const int64_t* __restrict__ rowp,
                         unsigned long long* __restrict__ vis, unsigned long long* __restrict__ cur,
                         int32_t* __restrict__ front, XState* __restrict__ st) {
    const int s = threadIdx.x;
    st->cnt[s] = 0;
    st->N[s] = 0;
    st->G[s] = 0;
    st->Gp[s] = 0;
    if (s < kXW) {
        const int64_t m = nb - 64LL * s;  // sources in word s
        st->active[s] = m <= 0 ? 0ULL : (m >= 64 ? ~0ULL : ((1ULL << m) - 1ULL));
        st->any[s] = 0;
    }
    if (s == 0) {
        st->rows = st->entries = 0;
        st->n_next = (unsigned long long)nb;
        st->fr_edges = st->rem_edges = 0;
    }
    __syncthreads();
    if (s < nb) {
        const int32_t v = src[s];
        const unsigned long long bit = 1ULL << (s & 63);
        atomicOr(&vis[(int64_t)v * kXW + (s >> 6)], bit);
        atomicOr(&cur[(int64_t)v * kXW + (s >> 6)], bit);
        front[s] = v;  // a source listed twice is harmless
        atomicAdd(&st->fr_edges, (unsigned long long)(rowp[v + 1] - rowp[v]));
    }
}


// Per-lane counters of one word's bits -> the sweep's per-source counts
// (lane (q, w) owns bits 8j + q of word w, j = 0..7), the OR of the new
// bits and the level's sums.  Every thread of the block calls.
__device__ __forceinline__ void x_flush(const unsigned (&c)[8], unsigned long long any, XSums m, unsigned* s_cnt,
                                        unsigned long long* s_any, XState* st) {
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
        m.rows += __shfl_xor_sync(kFull, m.rows, o);
        m.entries += __shfl_xor_sync(kFull, m.entries, o);
        m.fr_edges += __shfl_xor_sync(kFull, m.fr_edges, o);
        m.rem_edges += __shfl_xor_sync(kFull, m.rem_edges, o);
    }
    if (lane == 0) {
        if (m.rows) atomicAdd(&st->rows, m.rows);
        if (m.entries) atomicAdd(&st->entries, m.entries);
        if (m.fr_edges) atomicAdd(&st->fr_edges, m.fr_edges);
        if (m.rem_edges) atomicAdd(&st->rem_edges, m.rem_edges);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kXS; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(&st->cnt[i], (unsigned long long)s_cnt[i]);
    if (threadIdx.x < kXW && s_any[threadIdx.x]) atomicOr(&st->any[threadIdx.x], s_any[threadIdx.x]);
}

// Counts bit b of word w of cv over the warp's 8 vertices (lanes w, w+4,
// ..., w+28 hold word w) into the owning lanes' counters.
__device__ __forceinline__ void x_count_quads(unsigned long long cv, unsigned (&c)[8]) {
    const int lane = lane_id();
    const unsigned wm = 0x11111111u << (lane & 3);
    const int q = lane >> 2;
#pragma unroll
    for (int b = 0; b < 64; ++b) {
        const unsigned bal = __ballot_sync(kFull, (cv >> b) & 1ULL);
        if (q == (b & 7)) c[b >> 3] += __popc(bal & wm);
    }
}

// Bottom-up level for vertices with short rows: 4 lanes per vertex (lane w
// holds word w), 8 vertices per warp; each lane loads every fourth column of
// the row and the quad shares them, so 8 neighbours' words are in flight.
__global__ void __launch_bounds__(256) k_x_light(const int32_t* __restrict__ list, int64_t n_list,
                                                 const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                 const unsigned long long* __restrict__ cur,
                                                 unsigned long long* __restrict__ nxt, unsigned long long* vis,
                                                 const uint8_t* __restrict__ pred, int32_t* __restrict__ next_front,
                                                 XState* __restrict__ st) {
    __shared__ unsigned s_cnt[kXS];
    __shared__ unsigned long long s_any[kXW];
    for (int i = threadIdx.x; i < kXS; i += blockDim.x) s_cnt[i] = 0;
    if (threadIdx.x < kXW) s_any[threadIdx.x] = 0;
    __syncthreads();
    const int lane = lane_id();
    const int w = lane & 3, q = lane >> 2;
    const unsigned qm = 0xFu << (lane & ~3);
    const unsigned long long act = st->active[w];
    unsigned c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long any = 0;
    XSums m;
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
        int64_t deg = 0;
        if ((nb >> (lane & ~3)) & 0xFu) {  // some word of this vertex still needs bits
            const int64_t beg = __ldg(&rowp[v]), end = __ldg(&rowp[v + 1]);
            deg = end - beg;
            if (w == 0) {
                ++m.rows;
                m.entries += (unsigned long long)deg;
            }
            unsigned long long acc = 0;
            for (int64_t e0 = beg; e0 < end; e0 += 8) {
                const int64_t ea = e0 + w, eb = e0 + 4 + w;
                const int32_t ua = ea < end ? __ldg(&cols[ea]) : -1;
                const int32_t ub = eb < end ? __ldg(&cols[eb]) : -1;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t x = __shfl_sync(qm, ua, j, 4);
                    const int32_t y = __shfl_sync(qm, ub, j, 4);
                    if (x >= 0) acc |= __ldg(&cur[(int64_t)x * kXW + w]);
                    if (y >= 0) acc |= __ldg(&cur[(int64_t)y * kXW + w]);
                }
            }
            nx = acc & need;
        }
        if (valid) {
            nxt[(int64_t)v * kXW + w] = nx;
            if (nx) vis[(int64_t)v * kXW + w] = vw | nx;
        }
        any |= nx;
        // the vertex joins the next frontier; or still needs bits afterwards
        const bool got = (__ballot_sync(kFull, nx != 0) >> (lane & ~3)) & 0xFu;
        const bool left = (__ballot_sync(kFull, (need & ~nx) != 0) >> (lane & ~3)) & 0xFu;
        const long long at = warp_append(w == 0 && got, &st->n_next);
        if (at >= 0) {
            next_front[at] = v;
            m.fr_edges += (unsigned long long)deg;
        }
        if (w == 0 && left) m.rem_edges += (unsigned long long)deg;
        const unsigned long long cv = (valid && (!pred || pred[v])) ? nx : 0ULL;
        if (__ballot_sync(kFull, cv != 0)) x_count_quads(cv, c);
    }
    x_flush(c, any, m, s_cnt, s_any, st);
}

// Bottom-up level for vertices with long rows: a warp per vertex, lane
// (t, w) reads word w of neighbours t, t+8, ...; every 256 entries the warp
// stops if its OR already holds every bit the vertex needs.
__global__ void __launch_bounds__(256) k_x_heavy(const int32_t* __restrict__ list, int64_t n_list,
                                                 const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                                 const unsigned long long* __restrict__ cur,
                                                 unsigned long long* __restrict__ nxt, unsigned long long* vis,
                                                 const uint8_t* __restrict__ pred, int32_t* __restrict__ next_front,
                                                 XState* __restrict__ st) {
    __shared__ unsigned s_cnt[kXS];
    __shared__ unsigned long long s_any[kXW];
    for (int i = threadIdx.x; i < kXS; i += blockDim.x) s_cnt[i] = 0;
    if (threadIdx.x < kXW) s_any[threadIdx.x] = 0;
    __syncthreads();
    const int lane = lane_id();
    const int w = lane & 3, t = lane >> 2;
    const unsigned long long act = st->active[w];
    unsigned c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long any = 0;
    XSums m;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; i < n_list; i += warps) {
        const int32_t v = __ldg(&list[i]);
        const unsigned long long vw = vis[(int64_t)v * kXW + w];
        const unsigned long long need = act & ~vw;
        unsigned long long nx = 0;
        int64_t deg = 0;
        if (__any_sync(kFull, need != 0)) {
            const int64_t beg = __ldg(&rowp[v]), end = __ldg(&rowp[v + 1]);
            deg = end - beg;
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
                ++m.rows;
                m.entries += (unsigned long long)(stop - beg);
            }
        }
        if (t == 0) {
            nxt[(int64_t)v * kXW + w] = nx;
            if (nx) vis[(int64_t)v * kXW + w] = vw | nx;
        }
        any |= nx;
        const bool got = __any_sync(kFull, nx != 0);
        const bool left = __any_sync(kFull, (need & ~nx) != 0);
        const long long at = warp_append(lane == 0 && got, &st->n_next);
        if (at >= 0) {
            next_front[at] = v;
            m.fr_edges += (unsigned long long)deg;
        }
        if (lane == 0 && left) m.rem_edges += (unsigned long long)deg;
        // every lane holds its word's new bits; lane (t, w) counts bits 8j + t
        const unsigned long long cv = (!pred || pred[v]) ? nx : 0ULL;
#pragma unroll
        for (int j = 0; j < 8; ++j) c[j] += (unsigned)((cv >> (8 * j + t)) & 1ULL);
    }
    x_flush(c, any, m, s_cnt, s_any, st);
}

// Top-down level, step 1: the frontier rows as work items of at most
// kXSeg entries (vertex << 32 | segment), so that a hub's row is spread over
// many warps.  A vertex without running bits gives none.
constexpr int kXSeg = 256;

__global__ void k_x_td_items(const int32_t* __restrict__ front, int64_t n_front, const int64_t* __restrict__ rowp,
                             const unsigned long long* __restrict__ cur, unsigned long long* __restrict__ items,
                             XState* __restrict__ st) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = lane_id();
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_front; base += stride) {
        const int64_t i = base + lane;
        int segs = 0;
        int32_t u = 0;
        if (i < n_front) {
            u = __ldg(&front[i]);
            const int64_t o = (int64_t)u * kXW;
            const bool live = ((__ldg(&cur[o]) & st->active[0]) | (__ldg(&cur[o + 1]) & st->active[1]) |
                               (__ldg(&cur[o + 2]) & st->active[2]) | (__ldg(&cur[o + 3]) & st->active[3])) != 0;
            const int64_t deg = __ldg(&rowp[u + 1]) - __ldg(&rowp[u]);
            segs = live ? (int)((deg + kXSeg - 1) / kXSeg) : 0;
        }
        const int incl = warp_incl_scan(segs);
        const int total = __shfl_sync(kFull, incl, 31);
        unsigned long long at = 0;
        if (lane == 31 && total) at = atomicAdd(&st->n_next, (unsigned long long)total);
        at = __shfl_sync(kFull, at, 31) + (unsigned long long)(incl - segs);
        for (int j = 0; j < segs; ++j) items[at + j] = ((unsigned long long)(uint32_t)u << 32) | (unsigned)j;
    }
}

// Step 2: a warp per work item, lane (t, w) takes word w of the row owner's
// running bits to entries t, t+8, ...: the bits a neighbour has not visited
// go into its next words (atomicOr; the host cleared them).
__global__ void __launch_bounds__(256) k_x_td(const unsigned long long* __restrict__ items,
                                              const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                                              const unsigned long long* __restrict__ cur,
                                              unsigned long long* __restrict__ nxt,
                                              const unsigned long long* __restrict__ vis, XState* __restrict__ st) {
    const int lane = lane_id();
    const int w = lane & 3, t = lane >> 2;
    const unsigned long long act = st->active[w];
    const int64_t n_items = (int64_t)st->n_next;
    unsigned long long rows = 0, entries = 0;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; i < n_items; i += warps) {
        const unsigned long long it = __ldg(&items[i]);
        const int32_t u = (int32_t)(it >> 32);
        const int64_t seg = (int64_t)(it & 0xffffffffULL);
        const unsigned long long bits = __ldg(&cur[(int64_t)u * kXW + w]) & act;
        const int64_t row_end = __ldg(&rowp[u + 1]);
        const int64_t beg = __ldg(&rowp[u]) + seg * kXSeg;
        const int64_t end = beg + kXSeg < row_end ? beg + kXSeg : row_end;
        if (lane == 0) {
            rows += seg == 0 ? 1 : 0;
            entries += (unsigned long long)(end - beg);
        }
#pragma unroll 4
        for (int64_t b0 = beg; b0 < end; b0 += 8) {
            const int64_t e = b0 + t;
            if (e < end) {
                const int32_t v = __ldg(&cols[e]);
                const unsigned long long nb = bits & ~__ldg(&vis[(int64_t)v * kXW + w]);
                if (nb) atomicOr(&nxt[(int64_t)v * kXW + w], nb);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rows += __shfl_xor_sync(kFull, rows, o);
        entries += __shfl_xor_sync(kFull, entries, o);
    }
    if (lane == 0 && rows) {
        atomicAdd(&st->rows, rows);
        atomicAdd(&st->entries, entries);
    }
}

// Step 3, over every vertex (4 lanes per vertex): fold the new bits into
// "visited", count them, list the next frontier and its row entries.
__global__ void __launch_bounds__(256) k_x_td_finish(int64_t n, const int64_t* __restrict__ rowp,
                                                     const unsigned long long* __restrict__ nxt,
                                                     unsigned long long* vis, const uint8_t* __restrict__ pred,
                                                     int32_t* __restrict__ next_front, XState* __restrict__ st) {
    __shared__ unsigned s_cnt[kXS];
    __shared__ unsigned long long s_any[kXW];
    for (int i = threadIdx.x; i < kXS; i += blockDim.x) s_cnt[i] = 0;
    if (threadIdx.x < kXW) s_any[threadIdx.x] = 0;
    __syncthreads();
    const int lane = lane_id();
    const int w = lane & 3, q = lane >> 2;
    unsigned c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long any = 0;
    XSums m;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 2;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x) + (threadIdx.x & ~31)) >> 2; base < n; base += stride) {
        const int64_t v = base + q;
        const bool valid = v < n;
        const unsigned long long nx = valid ? nxt[v * kXW + w] : 0ULL;
        if (nx) vis[v * kXW + w] |= nx;
        any |= nx;
        const bool got = (__ballot_sync(kFull, nx != 0) >> (lane & ~3)) & 0xFu;
        const long long at = warp_append(w == 0 && got, &st->n_next);
        if (at >= 0) {
            next_front[at] = (int32_t)v;
            m.fr_edges += (unsigned long long)(__ldg(&rowp[v + 1]) - __ldg(&rowp[v]));
        }
        const unsigned long long cv = (valid && (!pred || pred[v])) ? nx : 0ULL;
        if (__ballot_sync(kFull, cv != 0)) x_count_quads(cv, c);
    }
    x_flush(c, any, m, s_cnt, s_any, st);
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
        ctr->frontier = st->n_next;
        ctr->merges = st->fr_edges;
        ctr->aux3 = st->rem_edges;
        st->n_next = st->fr_edges = st->rem_edges = 0;
    }
}

// HIP estimates of the same sizes from the ADS (the predicated
// neighbourhood query of Section 3.3; the estimator of Section 4.5): a warp
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
    const int64_t n = g->n, nnz = g->nnz;
    const int cls = kProfExact;
    const size_t words = (size_t)n * kXW;
    FL_TRY(dalloc(g->xbits, words * 8 * 3));
    // int32 lists: light rows (n), heavy rows (n), two frontiers (n + kXS
    // each: the first frontier lists the sweep's sources, repeats included);
    // then the top-down work items (uint64, one per kXSeg entries of a
    // frontier row: at most n + kXS + nnz / kXSeg) and the sweep state
    const size_t lists = ((size_t)(4 * n + 2 * kXS) * 4 + 255) & ~(size_t)255;
    const size_t n_items = (size_t)(n + kXS + nnz / kXSeg + 1);
    const size_t items_b = (n_items * 8 + 255) & ~(size_t)255;
    FL_TRY(dalloc(g->xaux, lists + items_b + sizeof(XState)));
    unsigned long long* vis = g->xbits.as<unsigned long long>();
    unsigned long long* buf[2] = {vis + words, vis + 2 * words};
    int32_t* light = g->xaux.as<int32_t>();
    int32_t* heavy = light + n;
    int32_t* front[2] = {light + 2 * n, light + 3 * n + kXS};
    unsigned long long* items = reinterpret_cast<unsigned long long*>(g->xaux.as<char>() + lists);
    XState* xs = reinterpret_cast<XState*>(g->xaux.as<char>() + lists + items_b);
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
        // a bottom-up level rewrites the next words of every vertex; a
        // top-down level gets them cleared first
        FL_CUDA(cudaMemsetAsync(vis, 0, words * 8, st));
        FL_CUDA(cudaMemsetAsync(buf[0], 0, words * 8, st));
        int c = 0, fc = 0;
        FL_LAUNCH(cls, k_x_seed<<<1, kXS, 0, st>>>(src + b0, nb, rowp, vis, buf[0], front[0], xs));
        FL_LAUNCH(cls, k_x_finish<<<1, kXS, 0, st>>>(xs, mode, 0, src + b0, pred, cost, D, rows, radius, ctr));
        FL_CUDA(cudaGetLastError());
        FL_TRY(read_counters(g));
        int64_t n_front = (int64_t)g->h_ctr->frontier;
        int64_t fr_edges = (int64_t)g->h_ctr->merges;
        int64_t rem = nnz;  // entries of rows that may still need bits
        unsigned long long rows_prev = 0, entries_prev = 0;
        for (int64_t level = 1; g->h_ctr->aux0 > 0; ++level) {
            if (level > n + 1) FL_FAIL(FL_ETIMEOUT, "exact search did not finish");
            // top-down when the frontier's rows are much shorter than the
            // rows bottom-up would scan, and their work items fit
            const bool td = 2 * fr_edges < rem && n_front + fr_edges / kXSeg + 1 <= (int64_t)n_items;
            if (td) {
                FL_CUDA(cudaMemsetAsync(buf[c ^ 1], 0, words * 8, st));
                // work items (their count in st->n_next), then the pushes;
                // k_x_td_finish restarts n_next for the next frontier
                FL_LAUNCH(cls, k_x_td_items<<<blocks_for(n_front, 256), 256, 0, st>>>(front[fc], n_front, rowp,
                                                                                     buf[c], items, xs));
                const int64_t most = n_front + fr_edges / kXSeg;  // work items at most
                FL_LAUNCH(cls, k_x_td<<<blocks_for(most, 8), 256, 0, st>>>(items, rowp, cols, buf[c], buf[c ^ 1], vis,
                                                                           xs));
                FL_CUDA(cudaMemsetAsync(&xs->n_next, 0, 8, st));
                FL_LAUNCH(cls, k_x_td_finish<<<blocks_for(n, 64), 256, 0, st>>>(n, rowp, buf[c ^ 1], vis, pred,
                                                                                front[fc ^ 1], xs));
            } else {
                if (n_heavy > 0)
                    FL_LAUNCH(cls, k_x_heavy<<<grid_h, 256, 0, st>>>(heavy, n_heavy, rowp, cols, buf[c], buf[c ^ 1],
                                                                     vis, pred, front[fc ^ 1], xs));
                if (n_light > 0)
                    FL_LAUNCH(cls, k_x_light<<<grid_l, 256, 0, st>>>(light, n_light, rowp, cols, buf[c], buf[c ^ 1],
                                                                     vis, pred, front[fc ^ 1], xs));
            }
            FL_LAUNCH(cls, k_x_finish<<<1, kXS, 0, st>>>(xs, mode, level, src + b0, pred, cost, D, rows, radius, ctr));
            FL_CUDA(cudaGetLastError());
            c ^= 1;
            fc ^= 1;
            FL_TRY(read_counters(g));
            const int64_t touched = (int64_t)g->h_ctr->frontier;
            // algorithmic bytes of the level.  Bottom-up: every listed vertex
            // reads its list id and visited words and writes its next words
            // (4 + 32 + 32 B); a scanned row reads two offsets (16 B) and, per
            // entry, the column and the neighbour's frontier words (4 + 32 B).
            // Top-down: a frontier vertex reads its list id, frontier words
            // and offsets (4 + 32 + 16 B); per entry the column and the
            // neighbour's visited words (4 + 32 B); every vertex reads its
            // next words (32 B) and a newly reached one reads and writes its
            // visited words, reads its offsets and is listed (32 + 32 + 16 + 4 B).
            const double d_rows = (double)(g->h_ctr->scanned - rows_prev);
            const double d_entries = (double)(g->h_ctr->cand_reads - entries_prev);
            rows_prev = g->h_ctr->scanned;
            entries_prev = g->h_ctr->cand_reads;
            g->prof.bytes[cls] += td ? 52.0 * (double)n_front + 36.0 * d_entries + 32.0 * (double)n +
                                           84.0 * (double)touched
                                     : 68.0 * (double)n + 16.0 * d_rows + 36.0 * d_entries;
            n_front = touched;
            fr_edges = (int64_t)g->h_ctr->merges;
            if (!td) rem = (int64_t)g->h_ctr->aux3;
        }
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
