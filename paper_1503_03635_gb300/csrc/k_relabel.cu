// k_relabel.cu -- internal vertex numbering by descending degree.
//
// R-MAT-like graphs send most CSR entries to few vertices: at scale 24 the 6 %
// of vertices with the largest degree are the endpoint of 86 % of the entries.
// Numbering vertices by descending degree puts the per-vertex values those
// entries read (sketch deltas, propagation values) side by side, so a cache
// sector holds several hot values instead of one hot value and three cold
// ones.  Ranks, priorities and reported facility ids keep the original ids
// (IdMap), so every result is the one of the original numbering; inputs and
// outputs indexed by vertex are permuted at the boundary.
#include <algorithm>

#include "fl_internal.cuh"

namespace fl {

namespace {

int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// Sort keys: descending degree (a 31-bit key), then ascending id (the input
// order, kept by the stable sort).
// *max_key_span: the largest degree (capped like the key), so that the sort
// can leave out the key digits above it, equal in every key.
__global__ void k_degree_keys(const int64_t* __restrict__ rowp, int64_t n, uint64_t* __restrict__ hi,
                              uint64_t* __restrict__ lo, uint32_t* __restrict__ val,
                              unsigned long long* __restrict__ max_deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned mx = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = rowp[v + 1] - rowp[v];
        const uint64_t dc = (uint64_t)(d < 0x7fffffffLL ? d : 0x7fffffffLL);
        hi[v] = 0x7fffffffULL - dc;
        lo[v] = (uint64_t)v;
        val[v] = (uint32_t)v;
        mx = max(mx, (unsigned)dc);
    }
    mx = __reduce_max_sync(kFull, mx);
    if (lane_id() == 0 && mx) atomicMax(max_deg, (unsigned long long)mx);
}

// perm (new -> original) to rid and inv, and the degrees in the new order.
__global__ void k_perm_maps(const uint32_t* __restrict__ perm, const int64_t* __restrict__ rowp, int64_t n,
                            int32_t* __restrict__ rid, int32_t* __restrict__ inv, int32_t* __restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t o = (int32_t)perm[i];
        rid[i] = o;
        inv[o] = (int32_t)i;
        deg[i] = (int32_t)(rowp[o + 1] - rowp[o]);
    }
}

// ---- the relabelled CSR, its rows sorted
// Row i of the new CSR is the row of original vertex rid[i], its ids mapped
// by inv and sorted ascending (new ids: descending degree first).  Sorting
// does not change any result (every step is order-independent); it makes a
// vertex meet its high-degree neighbours first, whose sketch entries are the
// smallest ranks and tighten its filter, and lets early-exit scans stop
// sooner.  Rows are numbered by descending length, so each length class is a
// contiguous range of rows with a kernel of its own: a thread per row of at
// most 8 entries (a sorting network in registers), a warp per row of 9-32
// (a bitonic network of shuffles), a warp per row of 33-kSortMax (a bitonic
// network over values held m/32 per lane, in registers and shuffles), and for
// the longer rows (hubs, kept in their input order) a warp per kSeg entries
// of the new CSR.
constexpr int kSortMax = 2048;
constexpr int32_t kSortPad = 0x7fffffff;  // above every vertex id

__device__ __forceinline__ int32_t warp_sort32(int32_t x) {
    const int lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int32_t y = __shfl_xor_sync(kFull, x, stride);
            const bool up = ((lane & size) == 0) || size == 32;
            const bool low = (lane & stride) == 0;
            x = (low == up) ? min(x, y) : max(x, y);
        }
    }
    return x;
}

// Rows [i0, i1) of 1-8 entries: a thread each.
__global__ void k_rows_small(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                             const int32_t* __restrict__ rid, const int32_t* __restrict__ inv,
                             const int64_t* __restrict__ rowp_new, int64_t i0, int64_t i1,
                             int32_t* __restrict__ cols_new) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += stride) {
        const int32_t o = rid[i];
        const int64_t b = rowp[o];
        const int len = (int)(rowp[o + 1] - b);
        int32_t x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = j < len ? __ldg(&inv[__ldcs(&cols[b + j])]) : kSortPad;
#pragma unroll
        for (int r = 0; r < 8; ++r) {  // odd-even transposition: 8 rounds sort 8 values
#pragma unroll
            for (int j = r & 1; j + 1 < 8; j += 2) {
                const int32_t lo = min(x[j], x[j + 1]), hi = max(x[j], x[j + 1]);
                x[j] = lo;
                x[j + 1] = hi;
            }
        }
        const int64_t d = rowp_new[i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < len) cols_new[d + j] = x[j];
    }
}

// Rows [i0, i1) of 9-32 entries: a warp each.
__global__ void k_rows_warp(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                            const int32_t* __restrict__ rid, const int32_t* __restrict__ inv,
                            const int64_t* __restrict__ rowp_new, int64_t i0, int64_t i1,
                            int32_t* __restrict__ cols_new) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = i0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < i1; i += warps) {
        const int32_t o = rid[i];
        const int64_t b = rowp[o];
        const int len = (int)(rowp[o + 1] - b);
        const int32_t x = warp_sort32(lane < len ? __ldg(&inv[__ldcs(&cols[b + lane])]) : kSortPad);
        if (lane < len) cols_new[rowp_new[i] + lane] = x;
    }
}

// Bitonic sort of 32 * Q values held Q per lane (lane L holds positions
// L*Q .. L*Q + Q - 1): pairs closer than Q are compared in registers, farther
// pairs exchange through shuffles.  Ascending when done.
template <int Q>
__device__ __forceinline__ void warp_bitonic(int32_t (&x)[Q]) {
    const int lane = lane_id();
    constexpr int N = 32 * Q;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= Q) {
                const int ls = stride / Q;
                const bool keep_min = ((lane & ls) == 0) == (((lane * Q) & size) == 0);
#pragma unroll
                for (int r = 0; r < Q; ++r) {
                    const int32_t y = __shfl_xor_sync(kFull, x[r], ls);
                    x[r] = keep_min ? min(x[r], y) : max(x[r], y);
                }
            } else {
#pragma unroll
                for (int r = 0; r < Q; ++r) {
                    if ((r & stride) == 0) {
                        const bool asc = ((lane * Q + r) & size) == 0;
                        const int32_t a = x[r], b = x[r + stride];
                        x[r] = asc ? min(a, b) : max(a, b);
                        x[r + stride] = asc ? max(a, b) : min(a, b);
                    }
                }
            }
        }
    }
}

// One row of len <= 32*Q entries: the ids loaded striped (the column loads,
// then the id loads, independent, in batches), sorted, written blocked to
// out[0 .. lim) (lim = len, or 32*Q to keep the padding).
template <int Q>
__device__ __forceinline__ void sort_row(const int32_t* __restrict__ cols, const int32_t* __restrict__ inv,
                                         int64_t b, int len, int32_t* __restrict__ out, int lim) {
    const int lane = lane_id();
    int32_t x[Q];
    constexpr int kBatch = Q < 16 ? Q : 16;  // loads in flight per lane, bounded to keep registers
#pragma unroll
    for (int r0 = 0; r0 < Q; r0 += kBatch) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int j = 32 * (r0 + u) + lane;
            x[r0 + u] = j < len ? __ldcs(&cols[b + j]) : -1;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) x[r0 + u] = x[r0 + u] >= 0 ? __ldg(&inv[x[r0 + u]]) : kSortPad;
    }
    warp_bitonic<Q>(x);
#pragma unroll
    for (int r = 0; r < Q; ++r) {
        const int j = lane * Q + r;
        if (j < lim) out[j] = x[r];
    }
}

// How many of the first d outputs of the stable merge of sorted A and B
// (A's element first on ties) come from A; both runs have length L.
__device__ __forceinline__ int merge_split(const int32_t* A, const int32_t* B, int L, int d) {
    int lo = max(0, d - L), hi = min(d, L);
    while (lo < hi) {
        const int i = (lo + hi) >> 1;
        if (A[i] <= B[d - 1 - i]) lo = i + 1;
        else hi = i;
    }
    return lo;
}

// Rows [i0, i1) of 33-kSortMax entries: a warp each.  kBig selects the rows
// above 512 entries: up to 1024 one Q = 32 sort; longer ones sort their two
// halves of 1024 that way into shared memory and merge them (each lane
// writes 64 outputs from its merge-path split).  The other rows take
// Q = 2..16, so that the register arrays of the long rows do not limit the
// occupancy of the short ones.
constexpr int kBigWarps = 4;

template <bool kBig>
__global__ void __launch_bounds__(kBig ? 32 * kBigWarps : 256, kBig ? 4 : 3) k_rows_sort(
    const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols, const int32_t* __restrict__ rid,
    const int32_t* __restrict__ inv, const int64_t* __restrict__ rowp_new, int64_t i0, int64_t i1,
    int32_t* __restrict__ cols_new) {
    __shared__ int32_t halves[kBig ? kBigWarps : 1][kBig ? kSortMax : 1];
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = i0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < i1; i += warps) {
        const int32_t o = rid[i];
        const int64_t b = rowp[o];
        const int len = (int)(rowp[o + 1] - b);
        int32_t* out = cols_new + rowp_new[i];
        if (kBig) {
            if (len > 1024) {
                int32_t* A = halves[threadIdx.x >> 5];
                int32_t* B = A + 1024;
                sort_row<32>(cols, inv, b, 1024, A, 1024);
                sort_row<32>(cols, inv, b + 1024, len - 1024, B, 1024);
                __syncwarp();
                const int d = lane * 64;
                int ia = merge_split(A, B, 1024, d), ib = d - ia;
                for (int k = 0; k < 64; ++k) {
                    const bool take_a = ib >= 1024 || (ia < 1024 && A[ia] <= B[ib]);
                    const int32_t v = take_a ? A[ia++] : B[ib++];
                    if (d + k < len) out[d + k] = v;
                }
                __syncwarp();
            } else {
                sort_row<32>(cols, inv, b, len, out, len);
            }
        } else {
            if (len > 256) sort_row<16>(cols, inv, b, len, out, len);
            else if (len > 128) sort_row<8>(cols, inv, b, len, out, len);
            else if (len > 64) sort_row<4>(cols, inv, b, len, out, len);
            else sort_row<2>(cols, inv, b, len, out, len);
        }
    }
}

// Rows [0, i1) (hubs, more than kSortMax entries, kept in input order): a
// warp per kSeg consecutive entries of the new CSR; a chunk spans at most two
// rows (every hub row is longer than kSeg).
__global__ void k_rows_hub(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                           const int32_t* __restrict__ rid, const int32_t* __restrict__ inv,
                           const int64_t* __restrict__ rowp_new, int64_t i1, int32_t* __restrict__ cols_new) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = rowp_new[i1];
    for (int64_t c0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kSeg; c0 < total;
         c0 += warps * kSeg) {
        int64_t lo = 0, hi = i1 - 1;  // the row holding entry c0: last r with rowp_new[r] <= c0
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (rowp_new[mid] <= c0) lo = mid;
            else hi = mid - 1;
        }
        const int64_t r0 = lo, r1 = lo + 1 < i1 ? lo + 1 : lo;
        const int64_t s0 = rowp_new[r0], s1 = rowp_new[r0 + 1];
        const int64_t o0 = rowp[rid[r0]], o1 = rowp[rid[r1]];
        const int64_t c1 = c0 + kSeg < total ? c0 + kSeg : total;
        for (int64_t p = c0 + lane; p < c1; p += 32) {
            const int64_t src = p < s1 ? o0 + (p - s0) : o1 + (p - s1);
            cols_new[p] = __ldg(&inv[__ldcs(&cols[src])]);
        }
    }
}

// First row of each length class: bounds[t] = the first i with deg[i] <=
// lim[t] (deg is non-increasing), left at n when there is none.
__global__ void k_class_bounds(const int32_t* __restrict__ deg, int64_t n, int64_t* __restrict__ bounds) {
    const int32_t lim[5] = {kSortMax, 512, 32, 8, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t d = deg[i], dp = i > 0 ? deg[i - 1] : 0x7fffffff;
#pragma unroll
        for (int t = 0; t < 5; ++t)
            if (d <= lim[t] && dp > lim[t]) bounds[t] = i;
    }
}

// out[r*n + i] = in[r*n + map[i]] for each of `reps` consecutive blocks of n.
template <class T>
__global__ void k_gather_map(const T* __restrict__ in, const int32_t* __restrict__ map, int64_t n, int64_t reps,
                             T* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * reps; t += stride) {
        const int64_t r = t / n, i = t - r * n;
        out[t] = in[r * n + map[i]];
    }
}

// Sketch rows in original order: out[o*k + j] = S[inv[o]*k + j].
__global__ void k_gather_rows(const uint64_t* __restrict__ S, const int32_t* __restrict__ inv, int64_t n, int k,
                              uint64_t* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += stride) {
        const int64_t o = t / k, j = t - o * k;
        out[t] = S[(int64_t)inv[o] * k + j];
    }
}

__global__ void k_ads_counts(const int64_t* __restrict__ gofs, const int64_t* __restrict__ eofs,
                             const int32_t* __restrict__ inv, int64_t n, int64_t* __restrict__ gc,
                             int64_t* __restrict__ ec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += stride) {
        const int32_t v = inv[o];
        gc[o] = gofs[v + 1] - gofs[v];
        ec[o] = eofs[v + 1] - eofs[v];
    }
}

// ADS rows in original vertex order, entry ids as original ids.
__global__ void k_ads_reorder(const int64_t* __restrict__ gofs, const int64_t* __restrict__ eofs,
                              const uint32_t* __restrict__ ginfo, const double* __restrict__ gwt,
                              const int32_t* __restrict__ eid, const int32_t* __restrict__ inv,
                              const int32_t* __restrict__ rid, int64_t n, const int64_t* __restrict__ gofs_o,
                              const int64_t* __restrict__ eofs_o, uint32_t* __restrict__ ginfo_o,
                              double* __restrict__ gwt_o, int32_t* __restrict__ eid_o) {
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < n; o += warps) {
        const int32_t v = inv[o];
        const int64_t g0 = gofs[v], ng = gofs[v + 1] - g0, go = gofs_o[o];
        for (int64_t j = lane_id(); j < ng; j += 32) {
            ginfo_o[go + j] = ginfo[g0 + j];
            gwt_o[go + j] = gwt[g0 + j];
        }
        const int64_t e0 = eofs[v], ne = eofs[v + 1] - e0, eo = eofs_o[o];
        for (int64_t j = lane_id(); j < ne; j += 32) eid_o[eo + j] = rid[eid[e0 + j]];
    }
}

}  // namespace

int relabel_graph(fl_graph* g) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    DBuf hi, lo, val, deg, rowp_new, cols_new;
    int rc = FL_OK;
    do {
        if ((rc = dalloc(hi, (size_t)n * 8)) || (rc = dalloc(lo, (size_t)n * 8)) || (rc = dalloc(val, (size_t)n * 4 + 64)) ||
            (rc = dalloc(deg, (size_t)n * 4 + 96)) || (rc = dalloc(rowp_new, (size_t)(n + 1) * 8)) ||
            (rc = dalloc(cols_new, (size_t)std::max<int64_t>(g->nnz, 1) * 4)) ||
            (rc = dalloc(g->rid, (size_t)n * 4)) || (rc = dalloc(g->inv, (size_t)n * 4)))
            break;
        unsigned long long* max_deg = reinterpret_cast<unsigned long long*>(val.as<char>() + (((size_t)n * 4 + 15) & ~(size_t)15));
        cudaError_t e = cudaMemsetAsync(max_deg, 0, 8, st);
        if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
        FL_LAUNCH(kProfOther, k_degree_keys<<<grid_for(n, 256), 256, 0, st>>>(
                                  g->rowp.as<int64_t>(), n, hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>(),
                                  max_deg));
        unsigned long long hmax = 0;
        e = cudaMemcpyAsync(&hmax, max_deg, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
        // keys lie in [2^31 - 1 - max, 2^31 - 1]: digits above the highest bit
        // where the two ends differ are equal in every key
        const uint64_t span = 0x7fffffffULL ^ (0x7fffffffULL - hmax);
        uint32_t digits = 0;
        for (int q = 0; q < 8 && (span >> (4 * q)) != 0; ++q) digits |= 1u << (16 + q);
        if ((rc = sort_pairs_u128_digits(hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>(), n, st, g->scratch,
                                         kProfOther, digits)))
            break;
        FL_LAUNCH(kProfOther, k_perm_maps<<<grid_for(n, 256), 256, 0, st>>>(
                                  val.as<uint32_t>(), g->rowp.as<int64_t>(), n, g->rid.as<int32_t>(),
                                  g->inv.as<int32_t>(), deg.as<int32_t>()));
        if ((rc = scan_exclusive_i32_to_i64(deg.as<int32_t>(), rowp_new.as<int64_t>(), n, st, g->scratch, kProfOther)))
            break;
        e = cudaMemcpyAsync(rowp_new.as<int64_t>() + n, g->rowp.as<int64_t>() + n, 8,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
        if (g->nnz > 0) {
            // four int64 after deg, 16-byte aligned
            int64_t* bounds = reinterpret_cast<int64_t*>(deg.as<char>() + (((size_t)n * 4 + 15) & ~(size_t)15));
            int64_t hb[5] = {n, n, n, n, n};
            e = cudaMemcpyAsync(bounds, hb, sizeof(hb), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
            FL_LAUNCH(kProfOther, k_class_bounds<<<grid_for(n, 256), 256, 0, st>>>(deg.as<int32_t>(), n, bounds));
            e = cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
            const int64_t c_mid = hb[0], c_lo = std::max(hb[1], c_mid), c_warp = std::max(hb[2], c_lo),
                          c_small = std::max(hb[3], c_warp), c_none = std::max(hb[4], c_small);
            const int64_t* rp = g->rowp.as<int64_t>();
            const int32_t* cl = g->cols.as<int32_t>();
            const int32_t* rid = g->rid.as<int32_t>();
            const int32_t* inv = g->inv.as<int32_t>();
            const int64_t* rpn = rowp_new.as<int64_t>();
            int32_t* cn = cols_new.as<int32_t>();
            if (c_mid > 0) {
                const int64_t chunks = (g->nnz + kSeg - 1) / kSeg;  // an upper bound of the hub chunks
                FL_LAUNCH(kProfOther, k_rows_hub<<<grid_for(chunks, 8), 256, 0, st>>>(rp, cl, rid, inv, rpn, c_mid, cn));
            }
            if (c_lo > c_mid)
                FL_LAUNCH(kProfOther, k_rows_sort<true><<<grid_for(c_lo - c_mid, kBigWarps), 32 * kBigWarps, 0, st>>>(
                                          rp, cl, rid, inv, rpn, c_mid, c_lo, cn));
            if (c_warp > c_lo)
                FL_LAUNCH(kProfOther, k_rows_sort<false><<<grid_for(c_warp - c_lo, 8), 256, 0, st>>>(
                                          rp, cl, rid, inv, rpn, c_lo, c_warp, cn));
            if (c_small > c_warp)
                FL_LAUNCH(kProfOther, k_rows_warp<<<grid_for(c_small - c_warp, 8), 256, 0, st>>>(
                                          rp, cl, rid, inv, rpn, c_warp, c_small, cn));
            if (c_none > c_small)
                FL_LAUNCH(kProfOther, k_rows_small<<<grid_for(c_none - c_small, 256), 256, 0, st>>>(
                                          rp, cl, rid, inv, rpn, c_small, c_none, cn));
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
        std::swap(g->rowp, rowp_new);
        std::swap(g->cols, cols_new);
        g->relabelled = true;
    } while (0);
    dfree_after(st, {&hi, &lo, &val, &deg, &rowp_new, &cols_new});
    return rc;
}

// Per-vertex arrays between original and internal order (reps blocks of n):
// to_internal: out[i] = in[rid[i]];  to_original: out[o] = in[inv[o]].
template <class T>
int permute_vertices(const fl_graph* g, const T* in, T* out, int64_t reps, bool to_internal, cudaStream_t st) {
    const int32_t* map = to_internal ? g->rid.as<int32_t>() : g->inv.as<int32_t>();
    FL_LAUNCH(kProfOther, k_gather_map<T><<<grid_for(g->n * reps, 256), 256, 0, st>>>(in, map, g->n, reps, out));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}
template int permute_vertices<double>(const fl_graph*, const double*, double*, int64_t, bool, cudaStream_t);
template int permute_vertices<uint8_t>(const fl_graph*, const uint8_t*, uint8_t*, int64_t, bool, cudaStream_t);
template int permute_vertices<int32_t>(const fl_graph*, const int32_t*, int32_t*, int64_t, bool, cudaStream_t);

int sketch_rows_original(const fl_graph* g, uint64_t* out) {
    FL_LAUNCH(kProfOther, k_gather_rows<<<grid_for(g->n * g->k, 256), 256, 0, g->stream>>>(
                              g->S.as<uint64_t>(), g->inv.as<int32_t>(), g->n, g->k, out));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

// The ADS in original vertex order (offsets, packed group info, weights,
// entry ids) into caller-provided device buffers.
int ads_original(fl_graph* g, int64_t* gofs_o, int64_t* eofs_o, uint32_t* ginfo_o, double* gwt_o, int32_t* eid_o) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    DBuf gc, ec;
    int rc = FL_OK;
    do {
        if ((rc = dalloc(gc, (size_t)n * 8)) || (rc = dalloc(ec, (size_t)n * 8))) break;
        FL_LAUNCH(kProfOther, k_ads_counts<<<grid_for(n, 256), 256, 0, st>>>(
                                  g->gofs.as<int64_t>(), g->eofs.as<int64_t>(), g->inv.as<int32_t>(), n,
                                  gc.as<int64_t>(), ec.as<int64_t>()));
        if ((rc = scan_exclusive_i64(gc.as<int64_t>(), gofs_o, n, st, g->scratch, kProfOther)) ||
            (rc = scan_exclusive_i64(ec.as<int64_t>(), eofs_o, n, st, g->scratch, kProfOther)))
            break;
        cudaError_t e = cudaMemcpyAsync(gofs_o + n, &g->n_groups, 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(eofs_o + n, &g->n_entries, 8, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { rc = status_of(e, "ADS export", __FILE__, __LINE__); break; }
        FL_LAUNCH(kProfOther, k_ads_reorder<<<grid_for(n, 8), 256, 0, st>>>(
                                  g->gofs.as<int64_t>(), g->eofs.as<int64_t>(), g->ginfo.as<uint32_t>(),
                                  g->gwt.as<double>(), g->eid.as<int32_t>(), g->inv.as<int32_t>(),
                                  g->rid.as<int32_t>(), n, gofs_o, eofs_o, ginfo_o, gwt_o, eid_o));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = status_of(e, "ADS export", __FILE__, __LINE__);
    } while (0);
    dfree_after(st, {&gc, &ec});
    return rc;
}

}  // namespace fl
