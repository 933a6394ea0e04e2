// k_batch.cu -- many facility-location instances solved in one pass.
//
// A batch is one graph U whose connected parts are the instances, so every
// phase (sketch hops, radii, keys, MIS sweeps, BFS) runs once over all of
// them, with the launch and synchronisation costs of one instance:
//   * a union batch: independent graphs placed side by side (graph i holds
//     vertices [off_i, off_{i+1}) of U); U's sketches are built per solve;
//   * a replica batch: R instances (own costs and client sets) on one
//     resident graph G whose sketches are built once.  U is R copies of G's
//     CSR; the instances share G's ADS: radii of all R instances are read
//     off it in one kernel, and only keys, MIS and BFS run on U.
// Ranks and priorities use part-local ids (fl_graph::vbase), so each part
// is solved exactly as it would be alone (Sections 3.1 and 4.1: the instances share no
// client, facility or edge).
#include <algorithm>
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

// Part i's CSR, already copied into U (its first n_i row offsets at voff,
// its columns at eoff), shifted to U's numbering.
__global__ void k_place_part(int part, int64_t n_i, int64_t nnz_i, int64_t voff, int64_t eoff,
                             int64_t* __restrict__ rowp, int32_t* __restrict__ cols, int32_t* __restrict__ vbase,
                             int32_t* __restrict__ vpart, int32_t* __restrict__ rid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_i || t < nnz_i; t += stride) {
        if (t < n_i) {
            rowp[voff + t] += eoff;
            vbase[voff + t] = (int32_t)voff;
            vpart[voff + t] = part;
            rid[voff + t] = (int32_t)t;
        }
        if (t < nnz_i) cols[eoff + t] += (int32_t)voff;
    }
}

// Every CSR entry stays inside its vertex's part.
__global__ void k_check_parts(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols, int64_t n,
                              const int32_t* __restrict__ vbase, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t b = vbase[v];
        for (int64_t e = rowp[v]; e < rowp[v + 1]; ++e)
            if (vbase[cols[e]] != b) {
                atomicOr(&ctr->error, 1ULL);
                break;
            }
    }
}

// U = R copies of G: vertex i*n + v, entries i*nnz + e.
__global__ void k_replicate_csr(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols, int64_t n,
                                int64_t nnz, int64_t R, int64_t* __restrict__ Urowp, int32_t* __restrict__ Ucols,
                                int32_t* __restrict__ vbase, int32_t* __restrict__ vpart,
                                const int32_t* __restrict__ base_rid, int32_t* __restrict__ rid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t total_e = R * nnz, total_v = R * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total_e || t <= total_v; t += stride) {
        if (t < total_e) {
            const int64_t i = t / nnz, e = t - i * nnz;
            Ucols[t] = (int32_t)(i * n + cols[e]);
        }
        if (t < total_v) {
            const int64_t i = t / n, v = t - i * n;
            Urowp[t] = i * nnz + rowp[v];
            vbase[t] = (int32_t)(i * n);
            vpart[t] = (int32_t)i;
            rid[t] = base_rid ? base_rid[v] : (int32_t)v;
        } else if (t == total_v) {
            Urowp[t] = total_e;
        }
    }
}

__global__ void k_replicate_i32(const int32_t* __restrict__ a, int64_t n, int64_t R, int32_t* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * R; t += stride) out[t] = a[t % n];
}

// Per instance (one block each): opening cost of its open facilities summed
// in a fixed tree order, open count, distance sum and unserved clients.
__global__ void __launch_bounds__(256) k_batch_objective(const int64_t* __restrict__ off, int n_inst,
                                                         const uint8_t* __restrict__ open,
                                                         const double* __restrict__ cost,
                                                         const uint8_t* __restrict__ client,
                                                         const int32_t* __restrict__ dist, double* __restrict__ obj,
                                                         long long* __restrict__ n_open,
                                                         long long* __restrict__ dist_sum,
                                                         long long* __restrict__ unserved) {
    __shared__ double rc[256];
    __shared__ long long ro[256], rd[256], ru[256];
    for (int i = blockIdx.x; i < n_inst; i += gridDim.x) {
        double acc = 0.0;
        long long no = 0, ds = 0, un = 0;
        for (int64_t v = off[i] + threadIdx.x; v < off[i + 1]; v += blockDim.x) {
            if (open[v]) {
                acc += cost[v];
                ++no;
            }
            if (client[v]) {
                const int32_t d = dist[v];
                if (d < 0) ++un;
                else ds += d;
            }
        }
        rc[threadIdx.x] = acc;
        ro[threadIdx.x] = no;
        rd[threadIdx.x] = ds;
        ru[threadIdx.x] = un;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) {
                rc[threadIdx.x] += rc[threadIdx.x + s];
                ro[threadIdx.x] += ro[threadIdx.x + s];
                rd[threadIdx.x] += rd[threadIdx.x + s];
                ru[threadIdx.x] += ru[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            obj[i] = rc[0] + (double)rd[0];
            n_open[i] = ro[0];
            dist_sum[i] = rd[0];
            unserved[i] = ru[0];
        }
        __syncthreads();
    }
}

}  // namespace


int batch_place_parts(fl_graph* U, const std::vector<int64_t>& voff, const std::vector<int64_t>& eoff) {
    cudaStream_t st = U->stream;
    const int n_parts = (int)voff.size() - 1;
    for (int i = 0; i < n_parts; ++i) {
        const int64_t n_i = voff[i + 1] - voff[i], nnz_i = eoff[i + 1] - eoff[i];
        FL_LAUNCH(kProfOther, k_place_part<<<grid_for(std::max(n_i, nnz_i), 256), 256, 0, st>>>(
                                  i, n_i, nnz_i, voff[i], eoff[i], U->rowp.as<int64_t>(), U->cols.as<int32_t>(),
                                  U->vbase.as<int32_t>(), U->vpart.as<int32_t>(), U->rid.as<int32_t>()));
    }
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

int batch_check_parts(fl_graph* U) {
    cudaStream_t st = U->stream;
    FL_CUDA(cudaMemsetAsync(U->ctr.p, 0, sizeof(Counters), st));
    FL_LAUNCH(kProfOther, k_check_parts<<<grid_for(U->n, 256), 256, 0, st>>>(
                              U->rowp.as<int64_t>(), U->cols.as<int32_t>(), U->n, U->vbase.as<int32_t>(),
                              U->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(U));
    if (U->h_ctr->error) FL_FAIL(FL_EINVAL, "a CSR entry leaves its graph (column outside [0, n_i))");
    return FL_OK;
}

int batch_replicate(const fl_graph* G, int64_t R, fl_graph* U) {
    cudaStream_t st = U->stream;
    FL_LAUNCH(kProfOther, k_replicate_csr<<<grid_for(std::max(R * G->nnz, R * G->n + 1), 256), 256, 0, st>>>(
                              G->rowp.as<int64_t>(), G->cols.as<int32_t>(), G->n, G->nnz, R, U->rowp.as<int64_t>(),
                              U->cols.as<int32_t>(), U->vbase.as<int32_t>(), U->vpart.as<int32_t>(),
                              G->rid.p ? G->rid.as<int32_t>() : nullptr, U->rid.as<int32_t>()));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

int batch_replicate_ecc(const fl_graph* G, int64_t R, fl_graph* U) {
    FL_TRY(dalloc(U->ecc_ub, (size_t)U->n * 4));
    FL_LAUNCH(kProfOther, k_replicate_i32<<<grid_for(U->n, 256), 256, 0, U->stream>>>(
                              G->ecc_ub.as<int32_t>(), G->n, R, U->ecc_ub.as<int32_t>()));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

int batch_objective(fl_solve* s, const int64_t* off_d, int n_inst, double* obj, long long* n_open,
                    long long* dist_sum, long long* unserved) {
    fl_graph* g = s->g;
    FL_LAUNCH(kProfOther, k_batch_objective<<<std::min(n_inst, 152 * 8), 256, 0, g->stream>>>(
                              off_d, n_inst, s->open.as<uint8_t>(), s->cost.as<double>(), s->client.as<uint8_t>(),
                              s->dist.as<int32_t>(), obj, n_open, dist_sum, unserved));
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}


}  // namespace fl
