// k_eps.cu -- the opening phase with eps > 0 (Section 4.1, Algorithm 3;
// Section 4.2, Algorithms 4 and 5 with Eq. 2/3) and the selection of
// Algorithm 6 (Section 4.3).
//
// The phase runs on a grid of radii alpha_j = alpha_{j-1} (1 + eps) from
// alpha_0 = gamma (1 + eps) / m^2, m = |F||C|, gamma = max over clients that
// reach a facility of min_f (c(f) + d(c, f)).  In iteration j every unopened
// facility whose q(f) reaches c(f) opens (alpha(f) = alpha_j), then every
// unfrozen client with an open facility within (1 + eps) alpha_j freezes
// (alpha(c) = alpha_j).  q(f) is what Eq. 2 (first iteration) and Eq. 3
// (later ones) add up to: per client c of f's ADS (HIP-weighted), with d_c
// the smallest grid value >= d(c, f),
//     [d_c <= alpha(c)] ((1 + eps) alpha(c) - d_c),
// alpha(c) the current radius for unfrozen clients, else the one at which c
// froze; it is summed in ADS order with one IEEE operation per step.
//
// Nothing changes between iterations without an opening or a freezing, so the
// GPU jumps from event to event: for fixed frozen clients q(f) is
// non-decreasing in j (each rounded step is monotone), so the first
// iteration at which f opens is found by binary search over the grid, and the
// first at which a client freezes by binary search over (1 + eps) alpha_j.
// The next event is the smallest of them; its openings and freezings are
// applied and the search repeats.  The result is the iteration-by-iteration
// loop's.
//
// Selection: H joins a client c to an open facility f iff alpha(c) =
// alpha(f) and d(c, f) <= (1 + eps) alpha(c), so facilities opened in
// different iterations never share a client.  Each iteration's facilities
// are selected by the lexicographically-first MIS under pi, with balls of
// floor((1 + eps) alpha_j) hops over the clients frozen in that iteration:
// the MIS machinery of the epsilon -> 0 path, run once per iteration that
// opened two or more facilities.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
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

constexpr int64_t kMaxGrid = 1 << 22;      // the grid of radii, at most
constexpr int32_t kNever = 0x7fffffff;

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long x) { return __longlong_as_double((long long)x); }

// Facilities, clients and the largest finite opening cost.
__global__ void k_eps_counts(const double* __restrict__ cost, const uint8_t* __restrict__ client, int64_t n,
                             unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long nf = 0, nc = 0, mx = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double c = cost[v];
        if (c < INFINITY) {
            ++nf;
            mx = max(mx, dbits(c));  // positive doubles order as their bits
        }
        nc += client[v] ? 1ULL : 0ULL;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nf += __shfl_xor_sync(kFull, nf, o);
        nc += __shfl_xor_sync(kFull, nc, o);
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if (lane_id() == 0) {
        if (nf) atomicAdd(&out[0], nf);
        if (nc) atomicAdd(&out[1], nc);
        if (mx) atomicMax(&out[2], mx);
    }
}

// gamma, step d: M[v] = the smallest cost of a facility within d hops of v
// (as bits: positive doubles order as their bits, +inf for none); a client's
// gamma_c = min over d of fl(M + d), which equals min over facilities of
// fl(c(f) + d(c, f)) because rounded addition is monotone in each operand.
__global__ void k_eps_min_pull(const int64_t* __restrict__ rowp, const int32_t* __restrict__ cols, int64_t n,
                               const unsigned long long* __restrict__ M, unsigned long long* __restrict__ Mn,
                               unsigned long long* __restrict__ changed) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long ch = 0;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const unsigned long long own = M[v];
        unsigned long long m = own;
        for (int64_t e = rowp[v] + lane; e < rowp[v + 1]; e += 32) m = min(m, __ldg(&M[cols[e]]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0) {
            Mn[v] = m;
            ch += m < own ? 1ULL : 0ULL;
        }
    }
    if (lane == 0 && ch) atomicAdd(changed, ch);
}

__global__ void k_eps_gamma_step(const unsigned long long* __restrict__ M, const uint8_t* __restrict__ client,
                                 int64_t n, double d, double* __restrict__ gam) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!client[v]) continue;
        const double m = bitsd(M[v]);
        if (!(m < INFINITY)) continue;
        const double t = __dadd_rn(m, d);
        if (t < gam[v]) gam[v] = t;
    }
}

// gamma = max over clients with a facility in reach; their number.
__global__ void k_eps_gamma_max(const double* __restrict__ gam, const uint8_t* __restrict__ client, int64_t n,
                                unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long mx = 0, cnt = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (client[v] && gam[v] < INFINITY) {
            mx = max(mx, dbits(gam[v]));
            ++cnt;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        cnt += __shfl_xor_sync(kFull, cnt, o);
    }
    if (lane_id() == 0) {
        if (mx) atomicMax(&out[0], mx);
        if (cnt) atomicAdd(&out[1], cnt);
    }
}

struct EpsADS {
    const int64_t* __restrict__ gofs;
    const int64_t* __restrict__ eofs;
    const uint32_t* __restrict__ ginfo;
    const double* __restrict__ gwt;
    const int32_t* __restrict__ eid;
};

// q_j(f) by the closed form (see the top of this file).
__device__ double eps_q(const EpsADS& a, int64_t f, int32_t j, const double* __restrict__ grid, double onepe,
                        const int32_t* __restrict__ shell, int32_t nshell, const uint8_t* __restrict__ client,
                        const int32_t* __restrict__ cli_iter) {
    double q = 0.0;
    int64_t e = a.eofs[f];
    for (int64_t gi = a.gofs[f]; gi < a.gofs[f + 1]; ++gi) {
        const uint32_t info = a.ginfo[gi];
        const int hop = (int)(info & 0xffffu), cnt = (int)((info >> 16) & 0xffu), counted = (int)(info >> 24);
        const double wt = a.gwt[gi];
        const int32_t sj = hop < nshell ? shell[hop] : kNever;
        for (int i = 0; i < counted; ++i) {
            const int32_t w = a.eid[e + i];
            if (!client[w]) continue;
            const int32_t jw = cli_iter[w] >= 0 ? cli_iter[w] : j;
            if (sj > jw) continue;  // the client's shell is beyond its radius
            q = __dadd_rn(q, __dmul_rn(wt, __dsub_rn(__dmul_rn(onepe, grid[jw]), grid[sj])));
        }
        e += cnt;
    }
    return q;
}

// First iteration in (jcur, J] at which each unopened facility opens, given
// the current frozen clients (kNever: none); the smallest into *jmin.
__global__ void k_eps_next_open(const int32_t* __restrict__ fac, int64_t n_fac, const int32_t* __restrict__ fac_iter,
                                const double* __restrict__ cost, EpsADS a, const double* __restrict__ grid,
                                double onepe, const int32_t* __restrict__ shell, int32_t nshell,
                                const uint8_t* __restrict__ client, const int32_t* __restrict__ cli_iter, int32_t jcur,
                                int32_t J, int32_t* __restrict__ nxt, int32_t* __restrict__ jmin) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_fac; i += stride) {
        const int32_t f = fac[i];
        if (fac_iter[f] >= 0) continue;
        const double c = cost[f];
        int32_t res = kNever;
        if (jcur < J && eps_q(a, f, J, grid, onepe, shell, nshell, client, cli_iter) >= c) {
            int32_t lo = jcur + 1, hi = J;
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (eps_q(a, f, mid, grid, onepe, shell, nshell, client, cli_iter) >= c) hi = mid;
                else lo = mid + 1;
            }
            res = lo;
            atomicMin(jmin, res);
        }
        nxt[f] = res;
    }
}

// First iteration in (jcur, J] at which each unfrozen client that reaches a
// facility freezes, given the distances to the open facilities.
__global__ void k_eps_next_freeze(const uint8_t* __restrict__ client, const double* __restrict__ gam,
                                  const int32_t* __restrict__ cli_iter, const int32_t* __restrict__ dist, int64_t n,
                                  const double* __restrict__ reach, int32_t jcur, int32_t J,
                                  int32_t* __restrict__ jmin) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!client[v] || cli_iter[v] >= 0 || !(gam[v] < INFINITY) || dist[v] < 0 || jcur >= J) continue;
        const double d = (double)dist[v];
        if (!(reach[J] >= d)) continue;
        int32_t lo = jcur + 1, hi = J;
        while (lo < hi) {
            const int32_t mid = lo + (hi - lo) / 2;
            if (reach[mid] >= d) hi = mid;
            else lo = mid + 1;
        }
        atomicMin(jmin, lo);
    }
}

// Open the facilities of iteration j; list every open facility (for the
// distances to the open set).
__global__ void k_eps_open(const int32_t* __restrict__ fac, int64_t n_fac, const int32_t* __restrict__ nxt, int32_t j,
                           int32_t* __restrict__ fac_iter, int32_t* __restrict__ open_list,
                           unsigned long long* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_fac; base += stride) {
        const int64_t i = base + lane_id();
        const int32_t f = i < n_fac ? fac[i] : 0;
        bool is_open = false, opened = false;
        if (i < n_fac) {
            if (fac_iter[f] < 0 && nxt[f] == j) {
                fac_iter[f] = j;
                opened = true;
            }
            is_open = fac_iter[f] >= 0;
        }
        const long long at = warp_append(is_open, &cnt[0]);
        if (at >= 0) open_list[at] = f;
        const unsigned m = __ballot_sync(kFull, opened);
        if (lane_id() == 0 && m) atomicAdd(&cnt[1], (unsigned long long)__popc(m));
    }
}

// Freeze the unfrozen clients with an open facility within (1 + eps) alpha_j.
__global__ void k_eps_freeze(const uint8_t* __restrict__ client, const double* __restrict__ gam,
                             int32_t* __restrict__ cli_iter, const int32_t* __restrict__ dist, int64_t n, double reach_j,
                             int32_t j, unsigned long long* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!client[v] || cli_iter[v] >= 0 || !(gam[v] < INFINITY) || dist[v] < 0) continue;
        if ((double)dist[v] <= reach_j) {
            cli_iter[v] = j;
            ++c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane_id() == 0 && c) atomicAdd(cnt, c);
}

// The facility list (finite costs).
__global__ void k_eps_facilities(const double* __restrict__ cost, int64_t n, int32_t* __restrict__ fac,
                                 unsigned long long* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool in = v < n && cost[v] < INFINITY;
        const long long at = warp_append(in, cnt);
        if (at >= 0) fac[at] = (int32_t)v;
    }
}

// Inputs of one iteration's selection: radius (1 + eps) alpha_j for its
// facilities (+inf for the others), its frozen clients as the client mask;
// facilities alone in their iteration are selected directly.
__global__ void k_eps_group(const int32_t* __restrict__ fac_iter, const int32_t* __restrict__ cli_iter, int64_t n,
                            int32_t j, double r, double* __restrict__ radii, uint8_t* __restrict__ gclient) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        radii[v] = fac_iter[v] == j ? r : INFINITY;
        gclient[v] = cli_iter[v] == j ? 1 : 0;
    }
}

__global__ void k_eps_or(const uint8_t* __restrict__ open, int64_t n, uint8_t* __restrict__ acc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (open[v]) acc[v] = 1;
}

__global__ void k_eps_single(const int32_t* __restrict__ fac_iter, int64_t n, const uint8_t* __restrict__ multi,
                             uint8_t* __restrict__ acc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (fac_iter[v] >= 0 && !multi[fac_iter[v]]) acc[v] = 1;
}

// Final open set and its list (for the assignment).
__global__ void k_eps_finish(const uint8_t* __restrict__ acc, int64_t n, uint8_t* __restrict__ open,
                             int32_t* __restrict__ list, unsigned long long* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const bool o = v < n && acc[v] != 0;
        if (v < n) open[v] = o ? 1 : 0;
        const long long at = warp_append(o, cnt);
        if (at >= 0) list[at] = (int32_t)v;
    }
}

__global__ void k_eps_fill(double* __restrict__ a, int64_t n, double x) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) a[v] = x;
}

int read_u64(const unsigned long long* d, unsigned long long* h, int cnt, cudaStream_t st) {
    FL_CUDA(cudaMemcpyAsync(h, d, (size_t)cnt * 8, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    return FL_OK;
}

}  // namespace

int open_facilities_eps(fl_solve* s, double eps) {
    fl_graph* g = s->g;
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    const double onepe = 1.0 + eps;
    const double* cost = s->cost.as<double>();
    const uint8_t* client = s->client.as<uint8_t>();
    // scratch: fac_iter, cli_iter, nxt, facility list, open list, dist, label
    // (int32); gamma (double); M[2] (uint64); selected (uint8); counters
    DBuf& E = s->eps;
    const size_t i32n = (size_t)n * 4;
    const size_t off_gam = ((i32n * 7 + 255) / 256) * 256;  // 8-byte values start aligned
    const size_t off_M = off_gam + (size_t)n * 8, off_acc = off_M + (size_t)n * 16;
    const size_t off_ctr = ((off_acc + (size_t)n + 255) / 256) * 256;
    FL_TRY(dalloc(E, off_ctr + 256));
    char* base = E.as<char>();
    int32_t* fac_iter = reinterpret_cast<int32_t*>(base);
    int32_t* cli_iter = fac_iter + n;
    int32_t* nxt = cli_iter + n;
    int32_t* fac = nxt + n;
    int32_t* open_list = fac + n;
    int32_t* dist = open_list + n;
    int32_t* label = dist + n;
    double* gam = reinterpret_cast<double*>(base + off_gam);
    unsigned long long* M[2] = {reinterpret_cast<unsigned long long*>(base + off_M),
                                reinterpret_cast<unsigned long long*>(base + off_M) + n};
    uint8_t* acc = reinterpret_cast<uint8_t*>(base + off_acc);
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(base + off_ctr);
    int32_t* jmin = reinterpret_cast<int32_t*>(ctr + 16);
    FL_CUDA(cudaMemsetAsync(fac_iter, 0xff, i32n * 2, st));
    FL_CUDA(cudaMemsetAsync(dist, 0xff, i32n, st));
    FL_CUDA(cudaMemsetAsync(acc, 0, (size_t)n, st));
    FL_CUDA(cudaMemsetAsync(ctr, 0, 256, st));
    s->eps_gamma = -1.0;
    s->eps_alpha0 = 0.0;
    s->eps_iterations = 0;
    s->eps_events = 0;
    s->eps_groups = 0;
    unsigned long long h[4] = {0, 0, 0, 0};

    // the selected set -> s->open and its list -> s->ulist (for the assignment)
    auto finish = [&]() -> int {
        FL_TRY(dalloc(s->open, (size_t)n));
        FL_TRY(dalloc(s->ulist, (size_t)n * 8));
        FL_CUDA(cudaMemsetAsync(&ctr[8], 0, 8, st));
        FL_LAUNCH(kProfMis, k_eps_finish<<<grid_for(n, 256), 256, 0, st>>>(acc, n, s->open.as<uint8_t>(),
                                                                             s->ulist.as<int32_t>(), &ctr[8]));
        unsigned long long no = 0;
        FL_TRY(read_u64(&ctr[8], &no, 1, st));
        s->n_open = (int64_t)no;
        return FL_OK;
    };

    // |F|, |C|, the largest finite cost
    FL_LAUNCH(kProfMis, k_eps_counts<<<grid_for(n, 256), 256, 0, st>>>(cost, client, n, ctr));
    FL_TRY(read_u64(ctr, h, 3, st));
    const int64_t nF = (int64_t)h[0], nC = (int64_t)h[1];
    double max_cost = 0.0;
    std::memcpy(&max_cost, &h[2], 8);
    if (nF == 0 || nC == 0) return finish();

    // gamma: rounds of min-propagation of the costs
    FL_LAUNCH(kProfMis, k_eps_fill<<<grid_for(n, 256), 256, 0, st>>>(gam, n, INFINITY));
    FL_CUDA(cudaMemcpyAsync(M[0], cost, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
    FL_LAUNCH(kProfMis, k_eps_gamma_step<<<grid_for(n, 256), 256, 0, st>>>(M[0], client, n, 0.0, gam));
    int cur = 0;
    for (int64_t d = 1;; ++d) {
        if (d > n + 1) FL_FAIL(FL_ETIMEOUT, "epsilon phase: cost propagation did not settle");
        FL_CUDA(cudaMemsetAsync(&ctr[3], 0, 8, st));
        FL_LAUNCH(kProfMis, k_eps_min_pull<<<grid_for(n, 8), 256, 0, st>>>(
                                g->rowp.as<int64_t>(), g->cols.as<int32_t>(), n, M[cur], M[cur ^ 1], &ctr[3]));
        FL_LAUNCH(kProfMis, k_eps_gamma_step<<<grid_for(n, 256), 256, 0, st>>>(M[cur ^ 1], client, n, (double)d,
                                                                                 gam));
        cur ^= 1;
        FL_TRY(read_u64(&ctr[3], h, 1, st));
        if (h[0] == 0) break;
    }
    FL_CUDA(cudaMemsetAsync(&ctr[4], 0, 16, st));
    FL_LAUNCH(kProfMis, k_eps_gamma_max<<<grid_for(n, 256), 256, 0, st>>>(gam, client, n, &ctr[4]));
    FL_TRY(read_u64(&ctr[4], h, 2, st));
    if (h[1] == 0) return finish();  // no client reaches a facility
    double gamma = 0.0;
    std::memcpy(&gamma, &h[0], 8);
    int64_t unfrozen = (int64_t)h[1];
    s->eps_gamma = gamma;

    // the grid of radii, (1 + eps) alpha_j, and the shell of every hop distance
    const double m = (double)nF * (double)nC;
    const double alpha0 = (gamma * onepe) / (m * m);
    s->eps_alpha0 = alpha0;
    const double bound = 2.0 * (max_cost + (double)n + 1.0);
    std::vector<double> grid(1, alpha0);
    while (grid.back() < bound) {
        if ((int64_t)grid.size() >= kMaxGrid) FL_FAIL(FL_EINVAL, "eps too small: the grid of radii exceeds 2^22 values");
        grid.push_back(grid.back() * onepe);
    }
    const int32_t J = (int32_t)grid.size() - 1;
    std::vector<double> reach(grid.size());
    for (size_t j = 0; j < grid.size(); ++j) reach[j] = onepe * grid[j];
    const int32_t nshell = (int32_t)g->hops + 1;
    std::vector<int32_t> shell(nshell);
    for (int32_t hop = 0; hop < nshell; ++hop)
        shell[hop] = (int32_t)(std::lower_bound(grid.begin(), grid.end(), (double)hop) - grid.begin());
    FL_TRY(dalloc(s->eps_tab, grid.size() * 17 + (size_t)nshell * 4 + 64));
    double* grid_d = s->eps_tab.as<double>();
    double* reach_d = grid_d + grid.size();
    int32_t* shell_d = reinterpret_cast<int32_t*>(reach_d + grid.size());
    uint8_t* multi_d = reinterpret_cast<uint8_t*>(shell_d + nshell);
    FL_CUDA(cudaMemcpyAsync(grid_d, grid.data(), grid.size() * 8, cudaMemcpyHostToDevice, st));
    FL_CUDA(cudaMemcpyAsync(reach_d, reach.data(), reach.size() * 8, cudaMemcpyHostToDevice, st));
    FL_CUDA(cudaMemcpyAsync(shell_d, shell.data(), (size_t)nshell * 4, cudaMemcpyHostToDevice, st));

    // the facilities
    FL_CUDA(cudaMemsetAsync(&ctr[6], 0, 8, st));
    FL_LAUNCH(kProfMis, k_eps_facilities<<<grid_for(n, 256), 256, 0, st>>>(cost, n, fac, &ctr[6]));
    EpsADS ads;
    ads.gofs = g->gofs.as<int64_t>();
    ads.eofs = g->eofs.as<int64_t>();
    ads.ginfo = g->ginfo.as<uint32_t>();
    ads.gwt = g->gwt.as<double>();
    ads.eid = g->eid.as<int32_t>();

    // events: the next iteration at which a facility opens or a client freezes
    int64_t unopened = nF;
    int32_t jcur = 0;
    std::vector<std::pair<int32_t, int64_t>> openings;  // (iteration, facilities opened)
    while (unopened > 0 && unfrozen > 0) {
        if (s->eps_events > (int64_t)J + 1) FL_FAIL(FL_ETIMEOUT, "epsilon phase: more events than iterations");
        const int32_t never = kNever;
        FL_CUDA(cudaMemcpyAsync(jmin, &never, 4, cudaMemcpyHostToDevice, st));
        FL_LAUNCH(kProfMis, k_eps_next_open<<<grid_for(nF, 128), 128, 0, st>>>(
                                fac, nF, fac_iter, cost, ads, grid_d, onepe, shell_d, nshell, client, cli_iter, jcur,
                                J, nxt, jmin));
        FL_LAUNCH(kProfMis, k_eps_next_freeze<<<grid_for(n, 256), 256, 0, st>>>(client, gam, cli_iter, dist, n,
                                                                                  reach_d, jcur, J, jmin));
        int32_t js = kNever;
        FL_CUDA(cudaMemcpyAsync(&js, jmin, 4, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaStreamSynchronize(st));
        if (js == kNever) {
            jcur = J;  // nothing changes any more up to the last radius of the grid
            break;
        }
        ++s->eps_events;
        FL_CUDA(cudaMemsetAsync(&ctr[9], 0, 24, st));
        FL_LAUNCH(kProfMis, k_eps_open<<<grid_for(nF, 256), 256, 0, st>>>(fac, nF, nxt, js, fac_iter, open_list,
                                                                            &ctr[9]));
        FL_TRY(read_u64(&ctr[9], h, 2, st));
        const int64_t n_open_all = (int64_t)h[0], opened = (int64_t)h[1];
        if (opened > 0) {
            unopened -= opened;
            openings.push_back({js, opened});
            FL_TRY(msbfs(g, open_list, n_open_all, label, dist, s->X, s->stamp, s->fr, s->frval, kProfMis));
        }
        FL_LAUNCH(kProfMis, k_eps_freeze<<<grid_for(n, 256), 256, 0, st>>>(client, gam, cli_iter, dist, n,
                                                                             reach[js], js, &ctr[11]));
        FL_TRY(read_u64(&ctr[11], h, 1, st));
        unfrozen -= (int64_t)h[0];
        jcur = js;
    }
    s->eps_iterations = jcur;

    // selection: one lexicographically-first MIS per iteration that opened
    // two or more facilities; the others' facilities are selected directly
    std::vector<uint8_t> multi(grid.size(), 0);
    for (const auto& o : openings)
        if (o.second >= 2) multi[o.first] = 1;
    FL_CUDA(cudaMemcpyAsync(multi_d, multi.data(), multi.size(), cudaMemcpyHostToDevice, st));
    FL_LAUNCH(kProfMis, k_eps_single<<<grid_for(n, 256), 256, 0, st>>>(fac_iter, n, multi_d, acc));
    FL_TRY(dalloc(s->eps_r, (size_t)n * 8));
    FL_TRY(dalloc(s->eps_c, (size_t)n));
    for (const auto& o : openings) {
        if (o.second < 2) continue;
        ++s->eps_groups;
        FL_LAUNCH(kProfMis, k_eps_group<<<grid_for(n, 256), 256, 0, st>>>(fac_iter, cli_iter, n, o.first,
                                                                            reach[o.first], s->eps_r.as<double>(),
                                                                            s->eps_c.as<uint8_t>()));
        std::swap(s->radii, s->eps_r);
        std::swap(s->client, s->eps_c);
        const int rc = open_facilities(s);
        std::swap(s->radii, s->eps_r);
        std::swap(s->client, s->eps_c);
        FL_TRY(rc);
        FL_LAUNCH(kProfMis, k_eps_or<<<grid_for(n, 256), 256, 0, st>>>(s->open.as<uint8_t>(), n, acc));
    }
    FL_CUDA(cudaGetLastError());
    return finish();
}

// The iteration at which each vertex opened (as a facility) and froze (as a
// client) in the last epsilon phase of s (-1: never), internal numbering.
const int32_t* eps_iterations_of(const fl_solve* s, bool clients) {
    const int32_t* fi = s->eps.as<int32_t>();
    return clients ? fi + s->g->n : fi;
}

}  // namespace fl
