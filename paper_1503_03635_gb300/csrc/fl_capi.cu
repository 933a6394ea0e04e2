// fl_capi.cu -- the extern "C" entry points declared in include/fl.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fl_internal.cuh"

namespace fl {
int last_error(char* buf, size_t len);
}

using namespace fl;

namespace {

cudaMemcpyKind kind_in(int mem_kind) {
    return mem_kind == FL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_out(int mem_kind) {
    return mem_kind == FL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}
bool bad_kind(int mem_kind) { return mem_kind != FL_MEM_HOST && mem_kind != FL_MEM_DEVICE; }

int copy_out(void* dst, const void* src, size_t bytes, int mem_kind, cudaStream_t st) {
    if (!dst || bytes == 0) return FL_OK;
    FL_CUDA(cudaMemcpyAsync(dst, src, bytes, kind_out(mem_kind), st));
    return FL_OK;
}

void destroy_graph(fl_graph* g) {
    cudaStreamSynchronize(g->stream);  // its buffers go to the idle-block cache
    DBuf* bufs[] = {&g->rowp, &g->cols, &g->wts, &g->wrev, &g->low_list, &g->small_list, &g->mid_list, &g->hub_list, &g->hub_seg, &g->seg_hub, &g->part,
                    &g->S, &g->Scnt, &g->D[0], &g->D[1], &g->Dcnt[0], &g->Dcnt[1], &g->frontier[0],
                    &g->frontier[1], &g->stamp, &g->vg, &g->ve, &g->stg_ent, &g->stg_grp, &g->gofs, &g->eofs,
                    &g->ginfo, &g->gwt, &g->eid, &g->ecc_ub, &g->ctr, &g->scratch,
                    &g->relax_aux, &g->U, &g->DM[0], &g->DM[1], &g->PM, &g->seg_flag, &g->PH, &g->F[0], &g->F[1], &g->H[0],
                    &g->H[1], &g->W, &g->fbm, &g->URid, &g->vbase, &g->vpart, &g->rid,
                    &g->inv, &g->xbits, &g->xaux, &g->xio};
    for (DBuf* b : bufs) dfree_idle(*b);
    if (g->gbfs) {
        graph_bfs_release(g->gbfs);
        delete g->gbfs;
        g->gbfs = nullptr;
    }
    for (cudaEvent_t e : g->prof.ev) cudaEventDestroy(e);
    for (cudaEvent_t e : g->hop_ev)
        if (e) cudaEventDestroy(e);
    if (g->h_ctr) cudaFreeHost(g->h_ctr);
    delete g;
}

void destroy_solve(fl_solve* s) {
    if (s->g) cudaStreamSynchronize(s->g->stream);
    DBuf* bufs[] = {&s->cost, &s->client, &s->radii, &s->ord, &s->fac_by_ord, &s->bcap, &s->state, &s->claimed,
                    &s->X, &s->stamp, &s->mval, &s->fr[0], &s->fr[1], &s->frval, &s->touched, &s->ulist,
                    &s->ubuck, &s->bcount, &s->open, &s->assign, &s->dist, &s->key_hi, &s->key_lo,
                    &s->key_val, &s->obj_tmp, &s->part_T, &s->io, &s->eps, &s->eps_tab, &s->eps_r,
                    &s->eps_c};
    for (DBuf* b : bufs) dfree_idle(*b);
    delete s;
}

// Routes the launch accounting of the kernels of one API call to the
// handle's profiler; when kernel timing is on, drains the recorded events
// (after a stream sync) when the call returns.
struct ProfScope {
    fl_graph* g;
    explicit ProfScope(fl_graph* gg) : g(gg) { set_current_prof(g ? &g->prof : nullptr, g ? g->stream : nullptr); }
    ~ProfScope() {
        if (g && g->prof.on && g->prof.used) {
            cudaStreamSynchronize(g->stream);
            prof_drain(&g->prof);
        }
        set_current_prof(nullptr, nullptr);
    }
};

int check_solve(fl_solve* s) {
    if (!s || !s->g) FL_FAIL(FL_EINVAL, "null solve handle");
    if (!s->g->built || s->generation != s->g->generation)
        FL_FAIL(FL_ESTATE, "the graph's sketches were rebuilt after this solve was created");
    return FL_OK;
}

// Opening costs and client mask (original order) into the solve (internal order).
int load_solve_inputs(fl_solve* s, const double* open_cost, const uint8_t* client_mask, int mem_kind) {
    fl_graph* g = s->g;
    cudaStream_t st = g->stream;
    if (g->relabelled) {
        FL_TRY(dalloc(s->io, (size_t)g->n * 9));
        uint8_t* io = s->io.as<uint8_t>();
        FL_CUDA(cudaMemcpyAsync(io, open_cost, (size_t)g->n * 8, kind_in(mem_kind), st));
        FL_CUDA(cudaMemcpyAsync(io + (size_t)g->n * 8, client_mask, (size_t)g->n, kind_in(mem_kind), st));
        FL_TRY(permute_vertices<double>(g, reinterpret_cast<double*>(io), s->cost.as<double>(), 1, true, st));
        FL_TRY(permute_vertices<uint8_t>(g, io + (size_t)g->n * 8, s->client.as<uint8_t>(), 1, true, st));
    } else {
        FL_CUDA(cudaMemcpyAsync(s->cost.p, open_cost, (size_t)g->n * 8, kind_in(mem_kind), st));
        FL_CUDA(cudaMemcpyAsync(s->client.p, client_mask, (size_t)g->n, kind_in(mem_kind), st));
    }
    return FL_OK;
}

// The solve's radii (internal order) to radii_out (original order, or
// nothing when NULL); waits for the stream.
int copy_radii_out(fl_solve* s, double* radii_out, int mem_kind) {
    fl_graph* g = s->g;
    if (radii_out && g->relabelled) {
        FL_TRY(dalloc(s->io, (size_t)g->n * 9));
        FL_TRY(permute_vertices<double>(g, s->radii.as<double>(), s->io.as<double>(), 1, false, g->stream));
        FL_TRY(copy_out(radii_out, s->io.p, (size_t)g->n * 8, mem_kind, g->stream));
    } else {
        FL_TRY(copy_out(radii_out, s->radii.p, (size_t)g->n * 8, mem_kind, g->stream));
    }
    FL_CUDA(cudaStreamSynchronize(g->stream));
    return FL_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Stages a neighbourhood query in g->xio: the sources mapped to internal
// ids, the predicate in internal order (NULL stays NULL) and an output of
// n_src * (D + 1) elements of `elem` bytes.
int stage_query(fl_graph* g, int64_t n_src, const int32_t* src, int64_t D, const uint8_t* pred, int mem_kind,
                size_t elem, int32_t** src_d, uint8_t** pred_d, void** out_d) {
    cudaStream_t st = g->stream;
    if ((double)n_src * (double)(D + 1) * (double)elem > 9.0e15) FL_FAIL(FL_ENOMEM, "query output too large");
    const size_t a = up256((size_t)n_src * 4), p = pred ? up256((size_t)g->n) : 0;
    const size_t o = (size_t)n_src * (size_t)(D + 1) * elem;
    FL_TRY(dalloc(g->xio, 2 * a + 2 * p + o));
    char* base = g->xio.as<char>();
    int32_t* raw = reinterpret_cast<int32_t*>(base);
    *src_d = reinterpret_cast<int32_t*>(base + a);
    FL_CUDA(cudaMemcpyAsync(raw, src, (size_t)n_src * 4, kind_in(mem_kind), st));
    FL_TRY(map_sources(g, raw, n_src, *src_d));
    *pred_d = nullptr;
    if (pred) {
        uint8_t* p0 = reinterpret_cast<uint8_t*>(base + 2 * a);
        uint8_t* p1 = p0 + p;
        FL_CUDA(cudaMemcpyAsync(p0, pred, (size_t)g->n, kind_in(mem_kind), st));
        if (g->relabelled) {
            FL_TRY(permute_vertices<uint8_t>(g, p0, p1, 1, true, st));
            *pred_d = p1;
        } else {
            *pred_d = p0;
        }
    }
    *out_d = base + 2 * a + 2 * p;
    return FL_OK;
}

}  // namespace

extern "C" {

const char* fl_status_str(int status) {
    switch (status) {
        case FL_OK: return "ok";
        case FL_EINVAL: return "invalid argument";
        case FL_ESTATE: return "call out of order";
        case FL_ENOMEM: return "out of memory";
        case FL_ECUDA: return "CUDA error";
        case FL_ETIMEOUT: return "iteration limit reached";
        default: return "unknown status";
    }
}

int fl_last_error(char* buf, size_t len) { return fl::last_error(buf, len); }

int fl_graph_create(int64_t n, const int64_t* row_off, const int32_t* cols, int64_t nnz, int mem_kind,
                    void* stream, fl_graph** out) {
    if (!out) FL_FAIL(FL_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 2147483647LL) FL_FAIL(FL_EINVAL, "n must be in [1, 2^31-1]");
    if (nnz < 0 || !row_off || (nnz > 0 && !cols)) FL_FAIL(FL_EINVAL, "bad CSR arrays");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    fl_graph* g = new (std::nothrow) fl_graph();
    if (!g) FL_FAIL(FL_ENOMEM, "host allocation failed");
    ProfScope ps(nullptr);
    g->n = n;
    g->nnz = nnz;
    g->stream = static_cast<cudaStream_t>(stream);
    int rc = FL_OK;
    do {
        cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&g->h_ctr), sizeof(Counters));
        if (e != cudaSuccess) { rc = status_of(e, "cudaMallocHost", __FILE__, __LINE__); break; }
        if ((rc = dalloc(g->ctr, sizeof(Counters)))) break;
        if ((rc = dalloc(g->rowp, (size_t)(n + 1) * 8))) break;
        if ((rc = dalloc(g->cols, (size_t)(nnz > 0 ? nnz : 1) * 4))) break;
        e = cudaMemcpyAsync(g->rowp.p, row_off, (size_t)(n + 1) * 8, kind_in(mem_kind), g->stream);
        if (e == cudaSuccess && nnz > 0)
            e = cudaMemcpyAsync(g->cols.p, cols, (size_t)nnz * 4, kind_in(mem_kind), g->stream);
        if (e != cudaSuccess) { rc = status_of(e, "CSR upload", __FILE__, __LINE__); break; }
        set_current_prof(&g->prof, g->stream);
        if ((rc = validate_csr(g))) break;
        if ((rc = relabel_graph(g))) break;
    } while (0);
    if (rc != FL_OK) {
        destroy_graph(g);
        return rc;
    }
    *out = g;
    return FL_OK;
}

int fl_graph_create_weighted(int64_t n, const int64_t* row_off, const int32_t* cols, const int32_t* lengths,
                             int64_t nnz, int mem_kind, void* stream, fl_graph** out) {
    if (!out) FL_FAIL(FL_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 2147483647LL) FL_FAIL(FL_EINVAL, "n must be in [1, 2^31-1]");
    if (nnz < 0 || !row_off || (nnz > 0 && (!cols || !lengths))) FL_FAIL(FL_EINVAL, "bad CSR arrays");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    fl_graph* g = new (std::nothrow) fl_graph();
    if (!g) FL_FAIL(FL_ENOMEM, "host allocation failed");
    ProfScope ps(nullptr);
    g->n = n;
    g->nnz = nnz;
    g->stream = static_cast<cudaStream_t>(stream);
    int rc = FL_OK;
    do {
        cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&g->h_ctr), sizeof(Counters));
        if (e != cudaSuccess) { rc = status_of(e, "cudaMallocHost", __FILE__, __LINE__); break; }
        if ((rc = dalloc(g->ctr, sizeof(Counters)))) break;
        if ((rc = dalloc(g->rowp, (size_t)(n + 1) * 8))) break;
        if ((rc = dalloc(g->cols, (size_t)(nnz > 0 ? nnz : 1) * 4))) break;
        if ((rc = dalloc(g->wts, (size_t)(nnz > 0 ? nnz : 1) * 4))) break;
        e = cudaMemcpyAsync(g->rowp.p, row_off, (size_t)(n + 1) * 8, kind_in(mem_kind), g->stream);
        if (e == cudaSuccess && nnz > 0)
            e = cudaMemcpyAsync(g->cols.p, cols, (size_t)nnz * 4, kind_in(mem_kind), g->stream);
        if (e == cudaSuccess && nnz > 0)
            e = cudaMemcpyAsync(g->wts.p, lengths, (size_t)nnz * 4, kind_in(mem_kind), g->stream);
        if (e != cudaSuccess) { rc = status_of(e, "CSR upload", __FILE__, __LINE__); break; }
        set_current_prof(&g->prof, g->stream);
        if ((rc = validate_csr(g))) break;
        if ((rc = check_weights(g))) break;
        if ((rc = pair_reverse_edges(g))) break;
        // kept in the caller's numbering: the lengths stay aligned with the columns
    } while (0);
    if (rc != FL_OK) {
        destroy_graph(g);
        return rc;
    }
    *out = g;
    return FL_OK;
}

int fl_graph_destroy(fl_graph* g) {
    if (!g) return FL_OK;
    cudaStreamSynchronize(g->stream);
    destroy_graph(g);
    return FL_OK;
}

int fl_build_sketches(fl_graph* g, int k, uint64_t seed) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (k < 2 || k > 32) FL_FAIL(FL_EINVAL, "k must be in [2, 32]");
    ProfScope ps(g);
    return build_sketches(g, k, seed);
}

int fl_sketch_stats(const fl_graph* g, int64_t* hops, int64_t* edge_merges, int64_t* ads_entries,
                    int64_t* ads_groups) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (!g->built) FL_FAIL(FL_ESTATE, "sketches not built");
    if (hops) *hops = g->hops;
    if (edge_merges) *edge_merges = g->edge_merges;
    if (ads_entries) *ads_entries = g->n_entries;
    if (ads_groups) *ads_groups = g->n_groups;
    return FL_OK;
}

int fl_hop_stats(const fl_graph* g, int64_t cap, int64_t* n_hops, int64_t* scanned, int64_t* mask,
                 int64_t* changed, double* ms) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (!g->built) FL_FAIL(FL_ESTATE, "sketches not built");
    if (cap < 0) FL_FAIL(FL_EINVAL, "negative capacity");
    const int64_t H = (int64_t)g->hop_scanned.size();
    if (n_hops) *n_hops = H;
    for (int64_t i = 0; i < std::min(H, cap); ++i) {
        if (scanned) scanned[i] = g->hop_scanned[i];
        if (mask) mask[i] = g->hop_mask[i];
        if (changed) changed[i] = g->hop_changed[i];
        if (ms) ms[i] = g->hop_ms[i];
    }
    return FL_OK;
}

int fl_hop_model(const fl_graph* g, int64_t cap, int64_t* n_hops, int64_t* edge_merges, int64_t* merging,
                 int64_t* delta_read, int64_t* delta_sum, int64_t* new_entries) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (!g->built) FL_FAIL(FL_ESTATE, "sketches not built");
    if (cap < 0) FL_FAIL(FL_EINVAL, "negative capacity");
    const int64_t H = (int64_t)g->hop_E.size();
    if (n_hops) *n_hops = H;
    for (int64_t i = 0; i < std::min(H, cap); ++i) {
        if (edge_merges) edge_merges[i] = g->hop_E[i];
        if (merging) merging[i] = g->hop_A[i];
        if (delta_read) delta_read[i] = g->hop_R[i];
        if (delta_sum) delta_sum[i] = g->hop_SD[i];
        if (new_entries) new_entries[i] = g->hop_new[i];
    }
    return FL_OK;
}

__global__ void k_export_sketch(const uint64_t* __restrict__ S, const uint8_t* __restrict__ Scnt, int64_t n,
                                int32_t* __restrict__ cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) cnt[v] = Scnt[v];
}

__global__ void k_unpack_ginfo(const uint32_t* __restrict__ ginfo, int64_t m, int32_t* __restrict__ hop,
                               int32_t* __restrict__ cnt, int32_t* __restrict__ counted) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint32_t x = ginfo[i];
        if (hop) hop[i] = (int32_t)(x & 0xffffu);
        if (cnt) cnt[i] = (int32_t)((x >> 16) & 0xffu);
        if (counted) counted[i] = (int32_t)(x >> 24);
    }
}

int fl_export_sketches(fl_graph* g, uint64_t* S, int32_t* cnt, int mem_kind) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (!g->built) FL_FAIL(FL_ESTATE, "sketches not built");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    ProfScope ps(g);
    cudaStream_t st = g->stream;
    if (S && g->relabelled) {
        DBuf tmp;
        FL_TRY(dalloc(tmp, (size_t)g->n * g->k * 8));
        int rc = sketch_rows_original(g, tmp.as<uint64_t>());
        if (!rc) rc = copy_out(S, tmp.p, (size_t)g->n * g->k * 8, mem_kind, st);
        cudaError_t e = cudaStreamSynchronize(st);
        dfree(tmp);
        if (rc) return rc;
        if (e != cudaSuccess) return status_of(e, "export sketches", __FILE__, __LINE__);
    } else {
        FL_TRY(copy_out(S, g->S.p, (size_t)g->n * g->k * 8, mem_kind, st));
    }
    if (cnt) {
        DBuf tmp;
        FL_TRY(dalloc(tmp, (size_t)g->n * 8));
        FL_LAUNCH(kProfOther, k_export_sketch<<<152 * 4, 256, 0, st>>>(g->S.as<uint64_t>(), g->Scnt.as<uint8_t>(), g->n,
                                                 tmp.as<int32_t>()));
        int32_t* src = tmp.as<int32_t>();
        int rc = FL_OK;
        if (g->relabelled) {
            rc = permute_vertices<int32_t>(g, src, src + g->n, 1, false, g->stream);
            src += g->n;
        }
        if (!rc) rc = copy_out(cnt, src, (size_t)g->n * 4, mem_kind, st);
        cudaError_t e = cudaStreamSynchronize(st);
        dfree(tmp);
        if (rc) return rc;
        if (e != cudaSuccess) return status_of(e, "export sketches", __FILE__, __LINE__);
    }
    FL_CUDA(cudaStreamSynchronize(st));
    return FL_OK;
}

int fl_export_ads(fl_graph* g, int64_t* gofs, int64_t* eofs, int32_t* ghop, int32_t* gcnt, int32_t* gcounted,
                  double* gwt, int32_t* eid, int mem_kind) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (!g->built) FL_FAIL(FL_ESTATE, "sketches not built");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    ProfScope ps(g);
    cudaStream_t st = g->stream;
    const size_t n1 = (size_t)(g->n + 1), m = (size_t)g->n_groups, ne = (size_t)g->n_entries;
    // a relabelled graph's ADS in original vertex order and ids (device copy)
    DBuf orig;
    const int64_t* src_gofs = g->gofs.as<int64_t>();
    const int64_t* src_eofs = g->eofs.as<int64_t>();
    const uint32_t* src_ginfo = g->ginfo.as<uint32_t>();
    const double* src_gwt = g->gwt.as<double>();
    const int32_t* src_eid = g->eid.as<int32_t>();
    if (g->relabelled) {
        FL_TRY(dalloc(orig, n1 * 16 + m * 12 + ne * 4 + 64));
        int64_t* go = orig.as<int64_t>();
        int64_t* eo = go + n1;
        double* wt = reinterpret_cast<double*>(eo + n1);
        uint32_t* gi = reinterpret_cast<uint32_t*>(wt + m);
        int32_t* ei = reinterpret_cast<int32_t*>(gi + m);
        int rc = ads_original(g, go, eo, gi, wt, ei);
        if (rc) {
            dfree(orig);
            return rc;
        }
        src_gofs = go;
        src_eofs = eo;
        src_ginfo = gi;
        src_gwt = wt;
        src_eid = ei;
    }
    int rc0 = copy_out(gofs, src_gofs, n1 * 8, mem_kind, st);
    if (!rc0) rc0 = copy_out(eofs, src_eofs, n1 * 8, mem_kind, st);
    if (!rc0) rc0 = copy_out(gwt, src_gwt, m * 8, mem_kind, st);
    if (!rc0) rc0 = copy_out(eid, src_eid, ne * 4, mem_kind, st);
    if (rc0) {
        dfree(orig);
        return rc0;
    }
    if (ghop || gcnt || gcounted) {
        DBuf tmp;
        FL_TRY(dalloc(tmp, m * 12 + 16));
        int32_t* h = tmp.as<int32_t>();
        FL_LAUNCH(kProfOther, k_unpack_ginfo<<<152 * 4, 256, 0, st>>>(src_ginfo, (int64_t)m, h, h + m, h + 2 * m));
        int rc = copy_out(ghop, h, m * 4, mem_kind, st);
        if (!rc) rc = copy_out(gcnt, h + m, m * 4, mem_kind, st);
        if (!rc) rc = copy_out(gcounted, h + 2 * m, m * 4, mem_kind, st);
        cudaError_t e = cudaStreamSynchronize(st);
        dfree(tmp);
        if (rc || e != cudaSuccess) {
            dfree(orig);
            return rc ? rc : status_of(e, "export ADS", __FILE__, __LINE__);
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    dfree(orig);
    if (e != cudaSuccess) return status_of(e, "export ADS", __FILE__, __LINE__);
    return FL_OK;
}

int fl_solve_create(fl_graph* g, fl_solve** out) {
    if (!out) FL_FAIL(FL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (!g->built) FL_FAIL(FL_ESTATE, "build the sketches before creating a solve");
    fl_solve* s = new (std::nothrow) fl_solve();
    if (!s) FL_FAIL(FL_ENOMEM, "host allocation failed");
    s->g = g;
    s->generation = g->generation;
    int rc = dalloc(s->cost, (size_t)g->n * 8);
    if (!rc) rc = dalloc(s->client, (size_t)g->n);
    if (!rc) rc = dalloc(s->radii, (size_t)g->n * 8);
    if (rc) {
        destroy_solve(s);
        return rc;
    }
    *out = s;
    return FL_OK;
}

int fl_solve_destroy(fl_solve* s) {
    if (!s) return FL_OK;
    if (s->g) cudaStreamSynchronize(s->g->stream);
    destroy_solve(s);
    return FL_OK;
}

int fl_compute_radii(fl_solve* s, const double* open_cost, const uint8_t* client_mask, int mem_kind,
                     double* radii_out) {
    FL_TRY(check_solve(s));
    if (!open_cost || !client_mask) FL_FAIL(FL_EINVAL, "open_cost and client_mask are required");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    ProfScope ps(s->g);
    s->have_radii = s->have_open = s->have_assign = 0;
    FL_TRY(load_solve_inputs(s, open_cost, client_mask, mem_kind));
    FL_TRY(compute_radii(s));
    FL_TRY(copy_radii_out(s, radii_out, mem_kind));
    s->have_radii = 1;
    return FL_OK;
}

// The epsilon > 0 phase, exact ball sizes and batches are built for
// unweighted graphs; on a weighted graph they return FL_ESTATE (sketches, ADS,
// radii, the selection and the assignment are built for both).
static int unweighted_only(const fl_graph* g, const char* what) {
    if (g && g->wts.p) FL_FAIL(FL_ESTATE, std::string(what) + " is not built for weighted graphs");
    return FL_OK;
}

int fl_compute_radii_exact(fl_solve* s, const double* open_cost, const uint8_t* client_mask, int mem_kind,
                           double* radii_out) {
    FL_TRY(check_solve(s));
    FL_TRY(unweighted_only(s->g, "fl_compute_radii_exact"));
    if (!open_cost || !client_mask) FL_FAIL(FL_EINVAL, "open_cost and client_mask are required");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    ProfScope ps(s->g);
    s->have_radii = s->have_open = s->have_assign = 0;
    FL_TRY(load_solve_inputs(s, open_cost, client_mask, mem_kind));
    FL_TRY(exact_radii(s));
    FL_TRY(copy_radii_out(s, radii_out, mem_kind));
    s->have_radii = 1;
    return FL_OK;
}

int fl_open_facilities(fl_solve* s, uint8_t* open_out, int64_t* n_open, int mem_kind) {
    FL_TRY(check_solve(s));
    if (!s->have_radii) FL_FAIL(FL_ESTATE, "compute radii first");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    s->have_open = s->have_assign = 0;
    ProfScope ps(s->g);
    FL_TRY(s->g->wts.p ? open_facilities_weighted(s) : open_facilities(s));
    if (open_out && s->g->relabelled) {
        FL_TRY(dalloc(s->io, (size_t)s->g->n * 9));
        FL_TRY(permute_vertices<uint8_t>(s->g, s->open.as<uint8_t>(), s->io.as<uint8_t>(), 1, false, s->g->stream));
        FL_TRY(copy_out(open_out, s->io.p, (size_t)s->g->n, mem_kind, s->g->stream));
    } else {
        FL_TRY(copy_out(open_out, s->open.p, (size_t)s->g->n, mem_kind, s->g->stream));
    }
    FL_CUDA(cudaStreamSynchronize(s->g->stream));
    if (n_open) *n_open = s->n_open;
    s->have_open = 1;
    return FL_OK;
}

int fl_open_facilities_eps(fl_solve* s, double eps, const double* open_cost, const uint8_t* client_mask,
                           int mem_kind, uint8_t* open_out, int64_t* n_open, int32_t* fac_iter_out,
                           int32_t* cli_iter_out) {
    FL_TRY(check_solve(s));
    FL_TRY(unweighted_only(s->g, "fl_open_facilities_eps"));
    if (!(eps > 0.0) || !(eps <= 1.0e6)) FL_FAIL(FL_EINVAL, "eps must be in (0, 1e6]");
    if (!open_cost || !client_mask) FL_FAIL(FL_EINVAL, "open_cost and client_mask are required");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    ProfScope ps(s->g);
    fl_graph* g = s->g;
    cudaStream_t st = g->stream;
    s->have_radii = s->have_open = s->have_assign = s->have_eps = 0;
    FL_TRY(load_solve_inputs(s, open_cost, client_mask, mem_kind));
    FL_TRY(check_costs(s));
    FL_TRY(open_facilities_eps(s, eps));
    if (open_out && g->relabelled) {
        FL_TRY(dalloc(s->io, (size_t)g->n * 9));
        FL_TRY(permute_vertices<uint8_t>(g, s->open.as<uint8_t>(), s->io.as<uint8_t>(), 1, false, st));
        FL_TRY(copy_out(open_out, s->io.p, (size_t)g->n, mem_kind, st));
    } else {
        FL_TRY(copy_out(open_out, s->open.p, (size_t)g->n, mem_kind, st));
    }
    for (int c = 0; c < 2; ++c) {
        int32_t* out = c ? cli_iter_out : fac_iter_out;
        if (!out) continue;
        const int32_t* it = eps_iterations_of(s, c == 1);
        if (g->relabelled) {
            FL_TRY(dalloc(s->io, (size_t)g->n * 9));
            FL_TRY(permute_vertices<int32_t>(g, it, s->io.as<int32_t>(), 1, false, st));
            it = s->io.as<int32_t>();
        }
        FL_TRY(copy_out(out, it, (size_t)g->n * 4, mem_kind, st));
        FL_CUDA(cudaStreamSynchronize(st));
    }
    FL_CUDA(cudaStreamSynchronize(st));
    if (n_open) *n_open = s->n_open;
    s->have_open = 1;
    s->have_eps = 1;
    return FL_OK;
}

int fl_eps_stats(const fl_solve* s, double* gamma, double* alpha0, int64_t* iterations, int64_t* events,
                 int64_t* groups) {
    if (!s) FL_FAIL(FL_EINVAL, "null solve handle");
    if (!s->have_eps) FL_FAIL(FL_ESTATE, "no epsilon phase has run on this solve");
    if (gamma) *gamma = s->eps_gamma;
    if (alpha0) *alpha0 = s->eps_alpha0;
    if (iterations) *iterations = s->eps_iterations;
    if (events) *events = s->eps_events;
    if (groups) *groups = s->eps_groups;
    return FL_OK;
}

int fl_assign_clients(fl_solve* s, int32_t* assign_out, int32_t* dist_out, int mem_kind) {
    FL_TRY(check_solve(s));
    if (!s->have_open) FL_FAIL(FL_ESTATE, "open facilities first");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    ProfScope ps(s->g);
    FL_TRY(s->g->wts.p ? assign_weighted(s) : assign_clients(s));
    const int32_t* a = s->assign.as<int32_t>();
    const int32_t* d = s->dist.as<int32_t>();
    if (s->g->relabelled && (assign_out || dist_out)) {  // facility ids are already original ids
        FL_TRY(dalloc(s->io, (size_t)s->g->n * 9));
        int32_t* io = s->io.as<int32_t>();
        FL_TRY(permute_vertices<int32_t>(s->g, a, io, 1, false, s->g->stream));
        FL_TRY(permute_vertices<int32_t>(s->g, d, io + s->g->n, 1, false, s->g->stream));
        a = io;
        d = io + s->g->n;
    }
    FL_TRY(copy_out(assign_out, a, (size_t)s->g->n * 4, mem_kind, s->g->stream));
    FL_TRY(copy_out(dist_out, d, (size_t)s->g->n * 4, mem_kind, s->g->stream));
    FL_CUDA(cudaStreamSynchronize(s->g->stream));
    s->have_assign = 1;
    return FL_OK;
}

int fl_objective(fl_solve* s, double* obj, int64_t* dist_sum, int64_t* n_unserved) {
    FL_TRY(check_solve(s));
    if (!s->have_assign) FL_FAIL(FL_ESTATE, "assign clients first");
    double o = 0.0;
    int64_t ds = 0, un = 0;
    ProfScope ps(s->g);
    FL_TRY(objective(s, &o, &ds, &un));
    if (obj) *obj = o;
    if (dist_sum) *dist_sum = ds;
    if (n_unserved) *n_unserved = un;
    return FL_OK;
}


int fl_ball_sizes(fl_graph* g, int64_t n_src, const int32_t* src, int32_t max_dist, const uint8_t* pred,
                  int mem_kind, int64_t* out) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    FL_TRY(unweighted_only(g, "fl_ball_sizes"));
    if (n_src < 0 || max_dist < 0) FL_FAIL(FL_EINVAL, "n_src and max_dist must be >= 0");
    if (n_src > 0 && (!src || !out)) FL_FAIL(FL_EINVAL, "src and out are required");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    if (n_src == 0) return FL_OK;
    ProfScope ps(g);
    int32_t* src_d;
    uint8_t* pred_d;
    void* out_d;
    FL_TRY(stage_query(g, n_src, src, max_dist, pred, mem_kind, 8, &src_d, &pred_d, &out_d));
    FL_TRY(exact_ball_sizes(g, n_src, src_d, max_dist, pred_d, static_cast<int64_t*>(out_d)));
    FL_TRY(copy_out(out, out_d, (size_t)n_src * (size_t)(max_dist + 1) * 8, mem_kind, g->stream));
    FL_CUDA(cudaStreamSynchronize(g->stream));
    return FL_OK;
}

int fl_ball_estimates(fl_graph* g, int64_t n_src, const int32_t* src, int32_t max_dist, const uint8_t* pred,
                      int mem_kind, double* out) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (!g->built) FL_FAIL(FL_ESTATE, "sketches not built");
    if (n_src < 0 || max_dist < 0) FL_FAIL(FL_EINVAL, "n_src and max_dist must be >= 0");
    if (n_src > 0 && (!src || !out)) FL_FAIL(FL_EINVAL, "src and out are required");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    if (n_src == 0) return FL_OK;
    ProfScope ps(g);
    int32_t* src_d;
    uint8_t* pred_d;
    void* out_d;
    FL_TRY(stage_query(g, n_src, src, max_dist, pred, mem_kind, 8, &src_d, &pred_d, &out_d));
    FL_TRY(hip_ball_estimates(g, n_src, src_d, max_dist, pred_d, static_cast<double*>(out_d)));
    FL_TRY(copy_out(out, out_d, (size_t)n_src * (size_t)(max_dist + 1) * 8, mem_kind, g->stream));
    FL_CUDA(cudaStreamSynchronize(g->stream));
    return FL_OK;
}

// ------------------------------------------------------------------ batches

}  // extern "C"

struct fl_batch {
    int kind = 0;                  // 1: union of graphs, 2: replicas of a resident graph
    fl_graph* base = nullptr;      // replicas: the resident graph (not owned)
    fl_graph* U = nullptr;         // the batch graph (owned)
    fl_solve* s = nullptr;         // its solve state (owned)
    int64_t n_inst = 0;
    std::vector<int64_t> off;      // host: first vertex of each instance, n_inst + 1 entries
    fl::DBuf off_d;                // device copy
    fl::DBuf res;                  // per instance: double obj, int64 n_open, dist_sum, unserved; int32 assign[N]
    uint64_t ecc_generation = ~0ULL;  // replicas: the base build whose eccentricity bounds U holds
};

namespace {

void destroy_batch(fl_batch* b) {
    if (!b) return;
    if (b->s) destroy_solve(b->s);
    if (b->U) destroy_graph(b->U);
    dfree_idle(b->off_d);
    dfree_idle(b->res);
    delete b;
}

// An empty graph handle of n vertices and nnz entries on `stream` (CSR and
// part bases allocated, contents unset).
int new_graph(int64_t n, int64_t nnz, cudaStream_t stream, fl_graph** out) {
    fl_graph* g = new (std::nothrow) fl_graph();
    if (!g) FL_FAIL(FL_ENOMEM, "host allocation failed");
    g->n = n;
    g->nnz = nnz;
    g->stream = stream;
    int rc = FL_OK;
    do {
        cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&g->h_ctr), sizeof(Counters));
        if (e != cudaSuccess) { rc = status_of(e, "cudaMallocHost", __FILE__, __LINE__); break; }
        if ((rc = dalloc(g->ctr, sizeof(Counters)))) break;
        if ((rc = dalloc(g->rowp, (size_t)(n + 1) * 8))) break;
        if ((rc = dalloc(g->cols, (size_t)(nnz > 0 ? nnz : 1) * 4))) break;
        if ((rc = dalloc(g->vbase, (size_t)n * 4))) break;
        if ((rc = dalloc(g->vpart, (size_t)n * 4))) break;
        if ((rc = dalloc(g->rid, (size_t)n * 4))) break;
    } while (0);
    if (rc != FL_OK) {
        destroy_graph(g);
        return rc;
    }
    *out = g;
    return FL_OK;
}

// The batch's solve state and per-instance result buffers.
int batch_finish(fl_batch* b) {
    const int64_t N = b->U->n;
    fl_solve* s = new (std::nothrow) fl_solve();
    if (!s) FL_FAIL(FL_ENOMEM, "host allocation failed");
    b->s = s;
    s->g = b->U;
    FL_TRY(dalloc(s->cost, (size_t)N * 8));
    FL_TRY(dalloc(s->client, (size_t)N));
    FL_TRY(dalloc(s->radii, (size_t)N * 8));
    FL_TRY(dalloc(b->off_d, (size_t)(b->n_inst + 1) * 8));
    FL_TRY(dalloc(b->res, (size_t)b->n_inst * 32 + (size_t)N * 4 + 64));
    FL_CUDA(cudaMemcpyAsync(b->off_d.p, b->off.data(), (size_t)(b->n_inst + 1) * 8, cudaMemcpyHostToDevice,
                            b->U->stream));
    FL_CUDA(cudaStreamSynchronize(b->U->stream));
    return FL_OK;
}

}  // namespace

extern "C" {

int fl_batch_create_union(int n_graphs, const int64_t* n_of, const int64_t* nnz_of, const int64_t* const* row_off,
                          const int32_t* const* cols, int mem_kind, void* stream, fl_batch** out) {
    if (!out) FL_FAIL(FL_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_graphs < 1 || !n_of || !nnz_of || !row_off || !cols) FL_FAIL(FL_EINVAL, "bad arguments");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    std::vector<int64_t> voff(n_graphs + 1, 0), eoff(n_graphs + 1, 0);
    for (int i = 0; i < n_graphs; ++i) {
        if (n_of[i] < 1 || nnz_of[i] < 0 || !row_off[i] || (nnz_of[i] > 0 && !cols[i]))
            FL_FAIL(FL_EINVAL, "bad CSR arrays of a graph");
        voff[i + 1] = voff[i] + n_of[i];
        eoff[i + 1] = eoff[i] + nnz_of[i];
        if (voff[i + 1] > 2147483647LL) FL_FAIL(FL_EINVAL, "more than 2^31-1 vertices in the batch");
    }
    fl_batch* b = new (std::nothrow) fl_batch();
    if (!b) FL_FAIL(FL_ENOMEM, "host allocation failed");
    b->kind = 1;
    b->n_inst = n_graphs;
    b->off = voff;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope ps(nullptr);
    int rc = new_graph(voff[n_graphs], eoff[n_graphs], st, &b->U);
    if (rc == FL_OK) {
        fl_graph* U = b->U;
        U->n_parts = n_graphs;
        set_current_prof(&U->prof, st);
        for (int i = 0; i < n_graphs && rc == FL_OK; ++i) {
            // each graph's offsets must run from 0 to its nnz
            int64_t ends[2] = {-1, -1};
            cudaError_t e = cudaSuccess;
            if (mem_kind == FL_MEM_HOST) {
                ends[0] = row_off[i][0];
                ends[1] = row_off[i][n_of[i]];
            } else {
                e = cudaMemcpyAsync(&ends[0], row_off[i], 8, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(&ends[1], row_off[i] + n_of[i], 8, cudaMemcpyDeviceToHost, st);
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(U->rowp.as<int64_t>() + voff[i], row_off[i], (size_t)n_of[i] * 8,
                                    kind_in(mem_kind), st);
            if (e == cudaSuccess && nnz_of[i] > 0)
                e = cudaMemcpyAsync(U->cols.as<int32_t>() + eoff[i], cols[i], (size_t)nnz_of[i] * 4,
                                    kind_in(mem_kind), st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = status_of(e, "batch CSR upload", __FILE__, __LINE__);
            else if (ends[0] != 0 || ends[1] != nnz_of[i]) {
                set_error(FL_EINVAL, "a graph's row offsets must run from 0 to its nnz");
                rc = FL_EINVAL;
            }
        }
        const int64_t total = eoff[n_graphs];
        if (rc == FL_OK) rc = batch_place_parts(U, voff, eoff);
        if (rc == FL_OK) {
            cudaError_t e = cudaMemcpyAsync(U->rowp.as<int64_t>() + U->n, &total, 8, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = status_of(e, "batch CSR", __FILE__, __LINE__);
        }
        if (rc == FL_OK) rc = validate_csr(U);
        if (rc == FL_OK) rc = batch_check_parts(U);
        if (rc == FL_OK) rc = batch_finish(b);
    }
    if (rc != FL_OK) {
        destroy_batch(b);
        return rc;
    }
    *out = b;
    return FL_OK;
}

int fl_batch_create_replicas(fl_graph* g, int n_inst, void* stream, fl_batch** out) {
    if (!out) FL_FAIL(FL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    FL_TRY(unweighted_only(g, "a batch"));
    if (!g->built) FL_FAIL(FL_ESTATE, "build the sketches before creating a replica batch");
    if (n_inst < 1) FL_FAIL(FL_EINVAL, "n_inst must be >= 1");
    if ((int64_t)n_inst * g->n > 2147483647LL) FL_FAIL(FL_EINVAL, "n_inst * n exceeds 2^31-1 vertices");
    fl_batch* b = new (std::nothrow) fl_batch();
    if (!b) FL_FAIL(FL_ENOMEM, "host allocation failed");
    b->kind = 2;
    b->base = g;
    b->n_inst = n_inst;
    b->off.resize(n_inst + 1);
    for (int i = 0; i <= n_inst; ++i) b->off[i] = (int64_t)i * g->n;
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : g->stream;
    ProfScope ps(nullptr);
    int rc = FL_OK;
    // g's stream may be another one: its pending work (the build) must be done
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) rc = status_of(cudaGetLastError(), "sync", __FILE__, __LINE__);
    if (rc == FL_OK) rc = new_graph((int64_t)n_inst * g->n, (int64_t)n_inst * g->nnz, st, &b->U);
    if (rc == FL_OK) {
        b->U->n_parts = n_inst;
        set_current_prof(&b->U->prof, st);
        rc = batch_replicate(g, n_inst, b->U);
    }
    if (rc == FL_OK) {
        rc = build_work_lists(b->U);
        b->U->lists_ready = rc == FL_OK;
    }
    if (rc == FL_OK) rc = relax_reserve(b->U);
    if (rc == FL_OK) rc = batch_finish(b);
    if (rc != FL_OK) {
        destroy_batch(b);
        return rc;
    }
    *out = b;
    return FL_OK;
}

int fl_batch_solve(fl_batch* b, int n_active, int k, uint64_t seed, const double* cost, const uint8_t* client,
                   uint8_t* open_out, int32_t* assign_out, int32_t* dist_out, int64_t* n_open, double* objective,
                   int64_t* dist_sum, int64_t* n_unserved, int mem_kind) {
    if (!b || !b->U || !b->s) FL_FAIL(FL_EINVAL, "null batch handle");
    if (!cost || !client) FL_FAIL(FL_EINVAL, "cost and client are required");
    if (bad_kind(mem_kind)) FL_FAIL(FL_EINVAL, "bad mem_kind");
    if (k < 2 || k > 32) FL_FAIL(FL_EINVAL, "k must be in [2, 32]");
    if (n_active < 1 || n_active > b->n_inst) FL_FAIL(FL_EINVAL, "n_active must be in [1, n_inst]");
    if (b->kind == 1 && n_active != b->n_inst) FL_FAIL(FL_EINVAL, "a union batch solves all its instances");
    fl_graph* U = b->U;
    fl_solve* s = b->s;
    const int64_t N = b->off[n_active];
    cudaStream_t st = U->stream;
    ProfScope ps(U);
    s->have_radii = s->have_open = s->have_assign = 0;
    if (b->kind == 1) {
        FL_TRY(build_sketches(U, k, seed));
    } else {
        fl_graph* G = b->base;
        if (!G->built || G->k != k || G->seed != seed)
            FL_FAIL(FL_ESTATE, "the resident graph's sketches were not built with this k and seed");
        if (b->ecc_generation != G->generation) {
            FL_TRY(batch_replicate_ecc(G, b->n_inst, U));
            b->ecc_generation = G->generation;
        }
        U->k = k;
        U->seed = seed;
        U->built = 1;
    }
    // the first n_active instances: a prefix view of U (vertices, CSR entries
    // and work lists of the leading replicas; the lists are sorted by id)
    fl_graph view = *U;
    if (b->kind == 2) {
        const int64_t R = b->n_inst;
        view.n = N;
        view.nnz = n_active * b->base->nnz;
        view.n_low = U->n_low / R * n_active;
        view.n_small = U->n_small / R * n_active;
        view.n_mid = U->n_mid / R * n_active;
        view.n_hubs = U->n_hubs / R * n_active;
        view.n_seg = U->n_seg / R * n_active;
    }
    s->g = &view;
    s->generation = view.generation;
    // replicas of a relabelled graph: per-instance arrays in original order
    const fl_graph* P = (b->kind == 2 && b->base->relabelled) ? b->base : nullptr;
    auto run = [&]() -> int {
        if (P) {
            FL_TRY(dalloc(s->io, (size_t)b->U->n * 9));
            uint8_t* io = s->io.as<uint8_t>();
            FL_CUDA(cudaMemcpyAsync(io, cost, (size_t)N * 8, kind_in(mem_kind), st));
            FL_CUDA(cudaMemcpyAsync(io + (size_t)N * 8, client, (size_t)N, kind_in(mem_kind), st));
            FL_TRY(permute_vertices<double>(P, reinterpret_cast<double*>(io), s->cost.as<double>(), n_active, true, st));
            FL_TRY(permute_vertices<uint8_t>(P, io + (size_t)N * 8, s->client.as<uint8_t>(), n_active, true, st));
        } else {
            FL_CUDA(cudaMemcpyAsync(s->cost.p, cost, (size_t)N * 8, kind_in(mem_kind), st));
            FL_CUDA(cudaMemcpyAsync(s->client.p, client, (size_t)N, kind_in(mem_kind), st));
        }
        if (b->kind == 1)
            FL_TRY(compute_radii(s));
        else
            FL_TRY(compute_radii_multi(b->base, &view, n_active, s->cost.as<double>(), s->client.as<uint8_t>(),
                                       s->radii.as<double>()));
        FL_TRY(open_facilities(s));
        FL_TRY(assign_clients(s));
        double* obj_d = b->res.as<double>();
        long long* cnt_d = reinterpret_cast<long long*>(obj_d + b->n_inst);
        int32_t* asg_d = reinterpret_cast<int32_t*>(cnt_d + 3 * b->n_inst);
        FL_TRY(batch_objective(s, b->off_d.as<int64_t>(), n_active, obj_d, cnt_d, cnt_d + b->n_inst,
                               cnt_d + 2 * b->n_inst));
        // facility labels are rank ids already: part-local (unions) or
        // original ids of the resident graph (replicas)
        const uint8_t* op = s->open.as<uint8_t>();
        const int32_t* as = s->assign.as<int32_t>();
        const int32_t* ds = s->dist.as<int32_t>();
        if (P) {
            FL_TRY(dalloc(s->io, (size_t)b->U->n * 9));
            uint8_t* io = s->io.as<uint8_t>();
            if (open_out) FL_TRY(permute_vertices<uint8_t>(P, op, io, n_active, false, st));
            if (assign_out) FL_TRY(permute_vertices<int32_t>(P, as, asg_d, n_active, false, st));
            if (dist_out) FL_TRY(permute_vertices<int32_t>(P, ds, reinterpret_cast<int32_t*>(io + N), n_active, false, st));
            op = io;
            as = asg_d;
            ds = reinterpret_cast<int32_t*>(io + N);
        }
        FL_TRY(copy_out(open_out, op, (size_t)N, mem_kind, st));
        FL_TRY(copy_out(assign_out, as, (size_t)N * 4, mem_kind, st));
        FL_TRY(copy_out(dist_out, ds, (size_t)N * 4, mem_kind, st));
        std::vector<double> h_obj(n_active);
        std::vector<long long> h_cnt(3 * b->n_inst);
        FL_CUDA(cudaMemcpyAsync(h_obj.data(), obj_d, (size_t)n_active * 8, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaMemcpyAsync(h_cnt.data(), cnt_d, (size_t)b->n_inst * 24, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < n_active; ++i) {
            if (objective) objective[i] = h_obj[i];
            if (n_open) n_open[i] = h_cnt[i];
            if (dist_sum) dist_sum[i] = h_cnt[b->n_inst + i];
            if (n_unserved) n_unserved[i] = h_cnt[2 * b->n_inst + i];
        }
        return FL_OK;
    };
    const int rc = run();
    // graph-owned buffers the solve may have (re)allocated through the view
    // (scan/sort scratch, round scratch; work lists are built at creation)
    U->scratch = view.scratch;
    U->relax_aux = view.relax_aux;
    s->g = U;
    return rc;
}

int fl_batch_info(const fl_batch* b, int64_t* n_inst, int64_t* n_total) {
    if (!b || !b->U) FL_FAIL(FL_EINVAL, "null batch handle");
    if (n_inst) *n_inst = b->n_inst;
    if (n_total) *n_total = b->U->n;
    return FL_OK;
}

int fl_batch_set_schedule(fl_batch* b, const fl_schedule* sched) {
    if (!b) FL_FAIL(FL_EINVAL, "null batch handle");
    return fl_set_schedule(b->U, sched);
}

int fl_batch_destroy(fl_batch* b) {
    if (!b) return FL_OK;
    if (b->U) cudaStreamSynchronize(b->U->stream);
    destroy_batch(b);
    return FL_OK;
}

int fl_profile_enable(fl_graph* g, int on) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (on < 0 || on > 2) FL_FAIL(FL_EINVAL, "on must be 0, 1 or 2");
    g->prof.on = on;
    return FL_OK;
}

int fl_profile_reset(fl_graph* g) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    FL_CUDA(cudaStreamSynchronize(g->stream));
    g->prof.used = 0;
    for (int i = 0; i < kProfClasses; ++i) {
        g->prof.launches[i] = 0;
        g->prof.ms[i] = 0.0;
        g->prof.bytes[i] = 0.0;
    }
    return FL_OK;
}

int fl_profile_query(const fl_graph* g, int kernel_class, int64_t* launches, double* ms, double* alg_bytes) {
    if (!g) FL_FAIL(FL_EINVAL, "null graph handle");
    if (kernel_class < -1 || kernel_class >= kProfClasses) FL_FAIL(FL_EINVAL, "bad kernel class");
    int64_t l = 0;
    double t = 0.0, b = 0.0;
    for (int i = 0; i < kProfClasses; ++i) {
        if (kernel_class != -1 && i != kernel_class) continue;
        l += g->prof.launches[i];
        t += g->prof.ms[i];
        b += g->prof.bytes[i];
    }
    if (launches) *launches = l;
    if (ms) *ms = t;
    if (alg_bytes) *alg_bytes = b;
    return FL_OK;
}

int fl_solve_stats(const fl_solve* s, int64_t* mis_rounds, int64_t* candidates) {
    if (!s) FL_FAIL(FL_EINVAL, "null solve handle");
    if (mis_rounds) *mis_rounds = s->mis_rounds;
    if (candidates) *candidates = s->n_cand;
    return FL_OK;
}

int fl_mis_log(const fl_solve* s, int64_t cap, int64_t* n_rows, int64_t* rows) {
    if (!s || !n_rows) FL_FAIL(FL_EINVAL, "null argument");
    if (cap < 0) FL_FAIL(FL_EINVAL, "cap must be >= 0");
    const int64_t total = (int64_t)s->mis_log.size() / 6;
    *n_rows = total;
    if (rows && cap > 0) {
        const int64_t k = std::min(cap, total);
        std::copy(s->mis_log.begin(), s->mis_log.begin() + 6 * k, rows);
    }
    return FL_OK;
}

}  // extern "C"
