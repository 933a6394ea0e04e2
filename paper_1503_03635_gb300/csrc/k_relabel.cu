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
__global__ void k_degree_keys(const int64_t* __restrict__ rowp, int64_t n, uint64_t* __restrict__ hi,
                              uint64_t* __restrict__ lo, uint32_t* __restrict__ val) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = rowp[v + 1] - rowp[v];
        hi[v] = 0x7fffffffULL - (uint64_t)(d < 0x7fffffffLL ? d : 0x7fffffffLL);
        lo[v] = (uint64_t)v;
        val[v] = (uint32_t)v;
    }
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

// Row i of the new CSR: the row of original vertex rid[i], ids mapped by inv.
__global__ void k_relabel_rows(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols,
                               const int32_t* __restrict__ rid, const int32_t* __restrict__ inv,
                               const int64_t* __restrict__ rowp_new, int64_t n, int32_t* __restrict__ cols_new) {
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int32_t o = rid[i];
        const int64_t b = rowp[o], len = rowp[o + 1] - b, d = rowp_new[i];
        for (int64_t j = lane_id(); j < len; j += 32) cols_new[d + j] = __ldg(&inv[__ldg(&cols[b + j])]);
    }
}

// Rows of at most kSortMax entries sorted ascending (new ids: descending
// degree first), one warp per row through a shared-memory bitonic sort.
// Hub rows keep their order.  Sorting does not change any result (every step
// is order-independent); it makes a vertex meet its high-degree neighbours
// first, whose sketch entries are the smallest ranks and tighten its filter.
constexpr int kSortMax = 2048;
constexpr int kSortWarps = 4;

__global__ void __launch_bounds__(32 * kSortWarps) k_sort_rows(const int64_t* __restrict__ rowp, int64_t n,
                                                                 int32_t* __restrict__ cols) {
    __shared__ int32_t buf[kSortWarps][kSortMax];
    int32_t* a = buf[threadIdx.x >> 5];
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const int64_t b = rowp[v];
        const int len = (int)(rowp[v + 1] - b);
        if (len < 2 || len > kSortMax) continue;  // warp-uniform
        if (len <= 32) {
            // one entry per lane: bitonic network through shuffles
            int32_t x = lane < len ? cols[b + lane] : 0x7fffffff;
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
            if (lane < len) cols[b + lane] = x;
            continue;
        }
        int m = 2;
        while (m < len) m <<= 1;
        for (int j = lane; j < m; j += 32) a[j] = j < len ? cols[b + j] : 0x7fffffff;
        __syncwarp();
        for (int size = 2; size <= m; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = lane; i < m; i += 32) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const bool asc = (i & size) == 0;
                        const int32_t x = a[i], y = a[j];
                        if ((x > y) == asc) {
                            a[i] = y;
                            a[j] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int j = lane; j < len; j += 32) cols[b + j] = a[j];
        __syncwarp();
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
        if ((rc = dalloc(hi, (size_t)n * 8)) || (rc = dalloc(lo, (size_t)n * 8)) || (rc = dalloc(val, (size_t)n * 4)) ||
            (rc = dalloc(deg, (size_t)n * 4)) || (rc = dalloc(rowp_new, (size_t)(n + 1) * 8)) ||
            (rc = dalloc(cols_new, (size_t)std::max<int64_t>(g->nnz, 1) * 4)) ||
            (rc = dalloc(g->rid, (size_t)n * 4)) || (rc = dalloc(g->inv, (size_t)n * 4)))
            break;
        FL_LAUNCH(kProfOther, k_degree_keys<<<grid_for(n, 256), 256, 0, st>>>(
                                  g->rowp.as<int64_t>(), n, hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>()));
        if ((rc = sort_pairs_u128(hi.as<uint64_t>(), lo.as<uint64_t>(), val.as<uint32_t>(), n, st, g->scratch,
                                  kProfOther, 16, 24)))  // the low 32 bits of hi
            break;
        FL_LAUNCH(kProfOther, k_perm_maps<<<grid_for(n, 256), 256, 0, st>>>(
                                  val.as<uint32_t>(), g->rowp.as<int64_t>(), n, g->rid.as<int32_t>(),
                                  g->inv.as<int32_t>(), deg.as<int32_t>()));
        if ((rc = scan_exclusive_i32_to_i64(deg.as<int32_t>(), rowp_new.as<int64_t>(), n, st, g->scratch, kProfOther)))
            break;
        cudaError_t e = cudaMemcpyAsync(rowp_new.as<int64_t>() + n, g->rowp.as<int64_t>() + n, 8,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
        if (g->nnz > 0)
            FL_LAUNCH(kProfOther, k_relabel_rows<<<grid_for(n, 8), 256, 0, st>>>(
                                      g->rowp.as<int64_t>(), g->cols.as<int32_t>(), g->rid.as<int32_t>(),
                                      g->inv.as<int32_t>(), rowp_new.as<int64_t>(), n, cols_new.as<int32_t>()));
        if (g->nnz > 0)
            FL_LAUNCH(kProfOther, k_sort_rows<<<grid_for(n, kSortWarps), 32 * kSortWarps, 0, st>>>(
                                      rowp_new.as<int64_t>(), n, cols_new.as<int32_t>()));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "relabel", __FILE__, __LINE__); break; }
        std::swap(g->rowp, rowp_new);
        std::swap(g->cols, cols_new);
        g->relabelled = true;
    } while (0);
    dfree(hi); dfree(lo); dfree(val); dfree(deg); dfree(rowp_new); dfree(cols_new);
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
    dfree(gc); dfree(ec);
    return rc;
}

}  // namespace fl
