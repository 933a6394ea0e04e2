// k_wsolve.cu -- the greedy MIS (phase iii) and the assignment on a weighted
// graph: balls and nearest facilities by weighted distance (Section 3.1 with
// the edge lengths of Section 3.3).
//
// Ball(f) = the clients within distance B_f = floor(r_f) of f.  The MIS is
// the lexicographically-first one under the keys (r_f, pi_f), as on an
// unweighted graph, found in greedy rounds: in each round every client gets
// the smallest key among the undecided facilities whose ball holds it (the
// cover), a facility whose ball holds only clients carrying its own key
// joins S (the gather), its clients are claimed, and every undecided facility
// whose ball holds a newly claimed client drops out (the kill).  The round's
// smallest undecided key always joins, and a facility joins exactly when
// every facility before it in key order that shares a client with it has
// dropped out, so the rounds end at the sequential greedy's set.
//
// Each of the three steps is a sweep over integer time: a value leaving
// vertex u at time t reaches neighbour v at time t + w(u, v).  A ring of
// R = (largest length + 1) slots holds the arrivals of the coming times: slot
// t mod R keeps, per vertex, the smallest value arriving at time t, and the
// list of vertices that have one.  Step t drains its slot into the labels
// (a vertex whose label drops joins the step's frontier) and the frontier
// pushes its labels along its edges into later slots.
//   cover:  facility f enters at time H - B_f with its key ordinal (H = the
//           largest B_f), so every wave ends at H and the label of v at H is
//           the smallest key whose ball holds v;
//   gather: each covered client enters at time 0 with its cover label, and f
//           reads its label at time B_f: the smallest cover label over its
//           ball (a deadline per vertex);
//   kill:   each newly claimed client enters at time 0, and f drops out when
//           anything has reached it by time B_f.
// The assignment is the same sweep with every open facility entering at
// time 0 with its id, where a vertex keeps its first arrival: the distance
// to the nearest open facility and, among those at that distance, the
// smallest id (the slot keeps the minimum of the values arriving together).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <vector>

#include "fl_internal.cuh"

namespace fl {

namespace {

constexpr uint32_t kNone = 0xffffffffu;
constexpr int kChunk = 16;  // time steps between two looks at the ring's counts

int grid_for(int64_t items, int per_block, int cap = 152 * 4) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

struct WSweep {
    const int64_t* rowp;
    const int32_t* cols;
    const int32_t* wts;
    int64_t n;
    int R;
    uint32_t* pend;             // R*n: smallest value arriving at each vertex at the slot's time (kNone: none)
    int32_t* plist;             // R*n: vertices with an arrival, per slot
    unsigned long long* pcnt;   // R
    int32_t* fr[2];             // frontier of the even / odd steps (2n each)
    unsigned long long* fcnt;   // 2
    unsigned long long* err;    // bit 1: a decision saw an impossible value
    uint32_t* lab;              // current label (kNone: none)
    const int32_t* dl;          // deadline: the label at this time is kept in dlab (or NULL)
    uint32_t* dlab;             // smallest arrival up to the deadline
    int32_t* dist;              // first-arrival mode: arrival time
    uint8_t* past;              // first-arrival mode: 1 where a push went past the horizon
    int32_t* ft;                // (cover) time of each vertex's first arrival, or NULL
    const int32_t* fts;         // (gather, kill) the cover's first arrivals: prune by slack, or NULL
    int first;                  // 1: a vertex keeps its first arrival; 0: the minimum
};

// One arrival of x at v at time t; true when v joins the step's frontier.
__device__ __forceinline__ bool arrive(const WSweep& a, int32_t v, uint32_t x, int64_t t) {
    if (a.dl && t <= (int64_t)a.dl[v] && x < a.dlab[v]) a.dlab[v] = x;
    const uint32_t old = a.lab[v];
    if (a.first) {
        if (old != kNone) return false;
        a.dist[v] = (int32_t)t;
    } else if (x >= old) {
        return false;
    }
    if (a.ft && old == kNone) a.ft[v] = (int32_t)t;
    a.lab[v] = x;
    return true;
}

// First index i in [0, m) with bs[i] >= b (m when none), bs non-decreasing.
// All 32 lanes call it and get the answer: each pass probes 32 evenly spaced
// positions of the remaining range at once (log32 m dependent loads).
__device__ int64_t warp_lower_bound(const int32_t* __restrict__ bs, int64_t m, int64_t b) {
    int64_t lo = 0, hi = m;  // the answer lies in [lo, hi]
    while (lo < hi) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t p = lo + step * lane_id();
        const bool below = p < hi && (int64_t)bs[p] < b;
        const int c = __popc(__ballot_sync(kFull, below));  // the probes below b are a prefix
        if (c == 0) break;                                  // bs[lo] >= b
        const int64_t first_not = lo + step * c;
        lo += step * (c - 1) + 1;
        hi = first_not < hi ? first_not : hi;
    }
    return lo;
}

// Appends the lanes' vertices with `want` to list (all 32 lanes call it).
__device__ __forceinline__ void warp_append(bool want, int32_t v, int32_t* list, unsigned long long* cnt) {
    const unsigned mask = __ballot_sync(kFull, want);
    if (!mask) return;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane_id() == leader) base = atomicAdd(cnt, (unsigned long long)__popc(mask));
    base = __shfl_sync(kFull, base, leader);
    if (want) list[base + __popc(mask & ((1u << lane_id()) - 1u))] = v;
}

// Step t, part 1: the arrivals of slot t mod R.
__global__ void k_wdrain(WSweep a, int64_t t) {
    const int s = (int)(t % a.R);
    const int p = (int)(t & 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.fcnt[p ^ 1] = 0;  // the next step's frontier
    const int64_t cnt = (int64_t)a.pcnt[s];
    uint32_t* pend = a.pend + (int64_t)s * a.n;
    const int32_t* list = a.plist + (int64_t)s * a.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < cnt; base += stride) {
        const int64_t i = base + lane_id();
        bool join = false;
        int32_t v = 0;
        if (i < cnt) {
            v = list[i];
            const uint32_t x = pend[v];
            pend[v] = kNone;
            join = arrive(a, v, x, t);
        }
        warp_append(join, v, a.fr[p], &a.fcnt[p]);
    }
}

// Step t, part 2 (cover): the undecided facilities with B_f = H - t enter.
// Candidates in key order have non-decreasing B_f (bsort[i] = B of the i-th),
// so they are one range of fac_by_ord, found by search; a candidate's value
// is its ordinal.
__global__ void k_winject(WSweep a, const int32_t* __restrict__ fac_by_ord, const int32_t* __restrict__ bsort,
                          const uint8_t* __restrict__ state, int64_t m, int64_t H, int64_t t) {
    __shared__ int64_t range[2];
    if (threadIdx.x < 64) {  // warp 0: first B >= H - t; warp 1: first B > H - t
        const int64_t at = warp_lower_bound(bsort, m, H - t + (int64_t)(threadIdx.x >> 5));
        if (lane_id() == 0) range[threadIdx.x >> 5] = at;
    }
    __syncthreads();
    const int p = (int)(t & 1);
    const int64_t end = range[1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = range[0] + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < end;
         base += stride) {
        const int64_t i = base + lane_id();
        bool join = false;
        int32_t f = 0;
        if (i < end) {
            f = fac_by_ord[i];
            if (state[f] == 0) join = arrive(a, f, (uint32_t)i, t);
        }
        warp_append(join, f, a.fr[p], &a.fcnt[p]);
    }
}

// Time 0 of a sweep: every vertex with mask[v] (all when NULL) enters with
// val[v] (its id when val is NULL), unless that is kNone.
__global__ void k_wseed(WSweep a, const uint32_t* __restrict__ val, const uint8_t* __restrict__ mask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n; base += stride) {
        const int64_t v = base + lane_id();
        bool join = false;
        if (v < a.n && (!mask || mask[v])) {
            const uint32_t x = val ? val[v] : (uint32_t)v;
            if (x != kNone) join = arrive(a, (int32_t)v, x, 0);
        }
        warp_append(join, (int32_t)v, a.fr[0], &a.fcnt[0]);
    }
}

// Step t, part 3: the frontier's labels go out along its edges (a warp per
// frontier vertex).  An arrival that cannot lower v's label is not sent: v's
// label already holds a value at most x from an arrival at or before t, and
// that arrival was also kept by v's deadline whenever this one would be.
__global__ void __launch_bounds__(256) k_wpush(WSweep a, int64_t t, int64_t H) {
    const int s = (int)(t % a.R);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.pcnt[s] = 0;  // drained; no push of this step targets it
    const int p = (int)(t & 1);
    const int64_t cnt = (int64_t)a.fcnt[p];
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < cnt; i += warps) {
        const int32_t u = a.fr[p][i];
        const uint32_t x = a.lab[u];
        const int64_t e1 = a.rowp[u + 1];
        for (int64_t e = a.rowp[u] + lane; e < e1; e += 32) {
            const int32_t v = a.cols[e];
            const uint32_t lv = a.lab[v];
            if (a.first ? lv != kNone : lv <= x) continue;
            const int64_t t2 = t + a.wts[e];
            if (a.fts) {  // v relays nothing useful after its slack H - (first cover arrival)
                const int32_t fv = a.fts[v];
                if (fv < 0 || t2 > H - (int64_t)fv) continue;
            }
            if (t2 > H) {
                if (a.first) a.past[v] = 1;
                continue;
            }
            const int64_t s2 = t2 % a.R;
            const uint32_t old = atomicMin(&a.pend[s2 * a.n + v], x);
            if (old == kNone) {
                const unsigned long long at = atomicAdd(&a.pcnt[s2], 1ULL);
                a.plist[s2 * a.n + (int64_t)at] = v;
            }
        }
    }
}

// The earliest time >= t at which a candidate enters the cover (H - B_f for
// the largest B_f <= H - t, decided or not), or ~0 when none does (one warp).
__global__ void k_wnext(const int32_t* __restrict__ bsort, int64_t m, int64_t H, int64_t t,
                        unsigned long long* __restrict__ out) {
    const int64_t lo = warp_lower_bound(bsort, m, H - t + 1);
    if (lane_id() == 0) *out = lo == 0 ? ~0ULL : (unsigned long long)(H - (int64_t)bsort[lo - 1]);
}

// Ordinals and ball radii of the sorted candidates: ord[f] = position in key
// order, B_f = floor(r_f) (at most 2^31 - 1).
__global__ void k_wordinals(const uint32_t* __restrict__ sorted_f, int64_t m, const double* __restrict__ r,
                            uint32_t* __restrict__ ord, int32_t* __restrict__ fac_by_ord, int32_t* __restrict__ bcap,
                            int32_t* __restrict__ bsort) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t f = (int32_t)sorted_f[i];
        ord[f] = (uint32_t)i;
        fac_by_ord[i] = f;
        const double fl = floor(r[f]);
        const int32_t b = fl >= 2147483647.0 ? 2147483647 : (int32_t)fl;
        bcap[f] = b;
        bsort[i] = b;
    }
}

// Undecided facilities: count, largest and smallest B_f.
__global__ void k_wundecided(const int32_t* __restrict__ fac_by_ord, const int32_t* __restrict__ bcap,
                             const uint8_t* __restrict__ state, int64_t m, unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0, bmax = 0, bmin = ~0ULL;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < m; base += stride) {
        const int64_t i = base + lane_id();
        if (i < m) {
            const int32_t f = fac_by_ord[i];
            if (state[f] == 0) {
                const unsigned long long b = (unsigned long long)bcap[f];
                ++c;
                bmax = b > bmax ? b : bmax;
                bmin = b < bmin ? b : bmin;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(kFull, c, o);
        const unsigned long long x = __shfl_xor_sync(kFull, bmax, o), y = __shfl_xor_sync(kFull, bmin, o);
        bmax = x > bmax ? x : bmax;
        bmin = y < bmin ? y : bmin;
    }
    if (lane_id() == 0 && c) {
        atomicAdd(&out[0], c);
        atomicMax(&out[1], bmax);
        atomicMin(&out[2], bmin);
    }
}

// Gather decision: an undecided f whose ball's smallest cover label is its
// own ordinal (or whose ball holds no client) joins S.  A smaller label means
// an undecided facility before f shares a client with it; a larger one
// cannot happen (f's own wave labels every client of its ball).
__global__ void k_wdecide(const int32_t* __restrict__ fac_by_ord, int64_t m, const uint32_t* __restrict__ dlab,
                          uint8_t* __restrict__ state, unsigned long long* __restrict__ joined,
                          unsigned long long* __restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t f = fac_by_ord[i];
        if (state[f] != 0) continue;
        const uint32_t g = dlab[f];
        if (g == kNone || g == (uint32_t)i) {
            state[f] = 1;
            ++c;
        } else if (g > (uint32_t)i) {
            atomicOr(err, 1ULL);
        }
    }
    if (c) atomicAdd(joined, c);
}

// Claims: a covered client whose cover label belongs to a facility that
// joined S is claimed and seeds the kill sweep.
__global__ void k_wclaim(int64_t n, const uint8_t* __restrict__ client, const uint32_t* __restrict__ cover,
                         const int32_t* __restrict__ fac_by_ord, const uint8_t* __restrict__ state,
                         uint8_t* __restrict__ claimed, uint8_t* __restrict__ seed,
                         unsigned long long* __restrict__ n_new) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint8_t sd = 0;
        const uint32_t o = cover[v];
        if (client[v] && o != kNone && state[fac_by_ord[o]] == 1) {
            claimed[v] = 1;
            sd = 1;
            ++c;
        }
        seed[v] = sd;
    }
    if (c) atomicAdd(n_new, c);
}

// Kill decision: an undecided facility reached by a newly claimed client
// within its ball radius drops out.
__global__ void k_wkill(const int32_t* __restrict__ fac_by_ord, int64_t m, const uint32_t* __restrict__ dlab,
                        uint8_t* __restrict__ state) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t f = fac_by_ord[i];
        if (state[f] == 0 && dlab[f] != kNone) state[f] = 2;
    }
}

__global__ void k_wopen(const uint8_t* __restrict__ state, int64_t n, uint8_t* __restrict__ open,
                        unsigned long long* __restrict__ n_open) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint8_t o = state[v] == 1 ? 1 : 0;
        open[v] = o;
        c += o;
    }
    if (c) atomicAdd(n_open, c);
}

// A vertex that a push past the horizon would have reached but that no
// arrival settled lies farther than the horizon.
__global__ void k_wbeyond(int64_t n, const uint8_t* __restrict__ past, const uint32_t* __restrict__ lab,
                          unsigned long long* __restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (past[v] && lab[v] == kNone) atomicOr(err, 2ULL);
}

// Device state of the sweeps of one call: the ring, the frontiers, counters.
struct WRing {
    DBuf pend, plist, fr, cnt;
    int R = 0;
    int64_t n = 0;
    unsigned long long* c = nullptr;  // [0, R): slot counts; R, R+1: frontier counts; R+2: errors;
                                      // R+3: next entry time; R+4..R+6: undecided count, max B, min B;
                                      // R+7: joined; R+8: claimed; R+9: open
    int alloc(fl_graph* g) {
        R = g->max_w + 1;
        n = g->n;
        FL_TRY(dalloc(pend, (size_t)R * n * 4));
        FL_TRY(dalloc(plist, (size_t)R * n * 4));
        FL_TRY(dalloc(fr, (size_t)n * 16));
        FL_TRY(dalloc(cnt, (size_t)(R + 16) * 8));
        c = cnt.as<unsigned long long>();
        FL_CUDA(cudaMemsetAsync(pend.p, 0xff, (size_t)R * n * 4, g->stream));
        FL_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(R + 16) * 8, g->stream));
        return FL_OK;
    }
    WSweep sweep(const fl_graph* g) const {
        WSweep a;
        a.rowp = g->rowp.as<int64_t>();
        a.cols = g->cols.as<int32_t>();
        a.wts = g->wts.as<int32_t>();
        a.n = n;
        a.R = R;
        a.pend = pend.as<uint32_t>();
        a.plist = plist.as<int32_t>();
        a.pcnt = c;
        a.fr[0] = fr.as<int32_t>();
        a.fr[1] = fr.as<int32_t>() + 2 * n;
        a.fcnt = c + R;
        a.err = c + R + 2;
        a.lab = nullptr;
        a.dl = nullptr;
        a.dlab = nullptr;
        a.dist = nullptr;
        a.past = nullptr;
        a.ft = nullptr;
        a.fts = nullptr;
        a.first = 0;
        return a;
    }
    // Before a sweep's sources enter: both frontiers empty (the slots are
    // empty after every sweep).
    int begin(cudaStream_t st) const {
        cudaError_t e = cudaMemsetAsync(c + R, 0, 16, st);
        return e == cudaSuccess ? FL_OK : status_of(e, "weighted sweep", __FILE__, __LINE__);
    }
    void release(cudaStream_t st) { dfree_after(st, {&pend, &plist, &fr, &cnt}); }
};

// The cover's entering facilities (NULL for sweeps whose sources all enter
// at time 0 through k_wseed).
struct Entry {
    const int32_t* fac_by_ord;
    const int32_t* bsort;
    const uint8_t* state;
    int64_t m;
    int64_t t_last;  // no facility enters after this time
};

// Runs steps 0..H of a sweep whose time-0 sources have entered.  Between
// chunks of steps the host reads the ring's counts: when nothing is pending
// it jumps to the next entry time, or stops.  *t_end = the last step run,
// *steps = the steps run.
int run_sweep(fl_graph* g, WRing& ring, const WSweep& a, int64_t H, const Entry* entry, int cls, int64_t* t_end,
              int64_t* steps) {
    cudaStream_t st = g->stream;
    const int R = ring.R;
    const int gd = grid_for(a.n, 256);
    const int gp = grid_for(a.n * 32, 256);
    const int gi = entry ? grid_for(entry->m, 256, 152) : 1;
    std::vector<unsigned long long> hc((size_t)R + 4);
    int64_t t = 0, ran = 0, last = 0;
    for (;;) {
        for (int j = 0; j < kChunk && t <= H; ++j, ++t) {
            FL_LAUNCH(cls, k_wdrain<<<gd, 256, 0, st>>>(a, t));
            if (entry && t <= entry->t_last)
                FL_LAUNCH(cls, k_winject<<<gi, 256, 0, st>>>(a, entry->fac_by_ord, entry->bsort, entry->state,
                                                              entry->m, H, t));
            FL_LAUNCH(cls, k_wpush<<<gp, 256, 0, st>>>(a, t, H));
            last = t;
            ++ran;
        }
        FL_CUDA(cudaGetLastError());
        if (t > H) break;
        if (entry && t <= entry->t_last)
            FL_LAUNCH(cls, k_wnext<<<1, 32, 0, st>>>(entry->bsort, entry->m, H, t, ring.c + R + 3));
        FL_CUDA(cudaMemcpyAsync(hc.data(), ring.c, (size_t)(R + 4) * 8, cudaMemcpyDeviceToHost, st));
        FL_CUDA(cudaStreamSynchronize(st));
        unsigned long long pending = 0;
        for (int s2 = 0; s2 < R; ++s2) pending += hc[(size_t)s2];
        if (pending) continue;
        // nothing in flight: the next entry, or the end
        if (!entry || t > entry->t_last || hc[(size_t)R + 3] == ~0ULL) break;
        const int64_t next = (int64_t)hc[(size_t)R + 3];
        if (next > t) {
            FL_CUDA(cudaMemsetAsync(ring.c + R, 0, 16, st));  // both frontiers are empty
            t = next;
        }
    }
    *t_end = last;
    *steps = ran;
    return FL_OK;
}

}  // namespace

int open_facilities_weighted(fl_solve* s) {
    fl_graph* g = s->g;
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    using clock = std::chrono::steady_clock;
    s->mis_log.clear();
    int64_t m = 0;
    FL_TRY(sort_candidates(s, &m));
    FL_TRY(dalloc(s->ord, (size_t)n * 4));
    FL_TRY(dalloc(s->fac_by_ord, (size_t)std::max<int64_t>(m, 1) * 4));
    FL_TRY(dalloc(s->bcap, (size_t)n * 4));
    FL_TRY(dalloc(s->claimed, (size_t)n));
    FL_TRY(dalloc(s->kill, (size_t)n));
    FL_TRY(dalloc(s->open, (size_t)n));
    FL_TRY(dalloc(s->X, (size_t)n * 16));  // cover labels, sweep labels, deadline labels, first arrivals
    FL_TRY(dalloc(s->ubuck, (size_t)std::max<int64_t>(m, 1) * 4));
    uint32_t* cover = s->X.as<uint32_t>();
    uint32_t* lab = cover + n;
    uint32_t* dlab = cover + 2 * n;
    int32_t* ft = reinterpret_cast<int32_t*>(cover + 3 * n);
    int32_t* bsort = s->ubuck.as<int32_t>();
    int32_t* fac_by_ord = s->fac_by_ord.as<int32_t>();
    int32_t* bcap = s->bcap.as<int32_t>();
    uint8_t* state = s->state.as<uint8_t>();
    FL_CUDA(cudaMemsetAsync(s->bcap.p, 0xff, (size_t)n * 4, st));
    FL_CUDA(cudaMemsetAsync(s->claimed.p, 0, (size_t)n, st));
    if (m > 0)
        FL_LAUNCH(kProfKeys, k_wordinals<<<grid_for(m, 256), 256, 0, st>>>(s->key_val.as<uint32_t>(), m,
                                                                          s->radii.as<double>(), s->ord.as<uint32_t>(),
                                                                          fac_by_ord, bcap, bsort));
    FL_CUDA(cudaGetLastError());
    WRing ring;
    int rc = ring.alloc(g);
    const int R = ring.R;
    unsigned long long* c = ring.c;
    int64_t rounds = 0;
    while (rc == FL_OK) {
        const auto round_t0 = clock::now();
        unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
        cudaError_t e = cudaMemsetAsync(c + R + 4, 0, 16, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c + R + 6, 0xff, 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c + R + 7, 0, 16, st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted MIS", __FILE__, __LINE__); break; }
        if (m > 0)
            FL_LAUNCH(kProfMis, k_wundecided<<<grid_for(m, 256), 256, 0, st>>>(fac_by_ord, bcap, state, m, c + R + 4));
        e = cudaMemcpyAsync(h, c + R + 2, 48, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted MIS", __FILE__, __LINE__); break; }
        if (h[0]) { rc = FL_ECUDA; set_error(rc, "weighted MIS: a ball's smallest label is above its own key"); break; }
        const int64_t nu = (int64_t)h[2];
        if (nu == 0) break;
        if (++rounds > m + 1) { rc = FL_ETIMEOUT; set_error(rc, "weighted MIS did not converge"); break; }
        const int64_t H = (int64_t)h[3];
        Entry entry{fac_by_ord, bsort, state, m, H - (int64_t)h[4]};
        auto timed = [&](int kind, int64_t t_end, int64_t steps, clock::time_point t0) {
            const double us = std::chrono::duration<double, std::micro>(clock::now() - t0).count();
            s->mis_log.insert(s->mis_log.end(), {rounds, (int64_t)kind, t_end, steps, 0, (int64_t)us});
        };
        int64_t t_end = 0, steps = 0;
        // cover
        auto t0 = clock::now();
        WSweep a = ring.sweep(g);
        a.lab = cover;
        a.ft = ft;
        e = cudaMemsetAsync(cover, 0xff, (size_t)n * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ft, 0xff, (size_t)n * 4, st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted MIS", __FILE__, __LINE__); break; }
        if ((rc = ring.begin(st)) || (rc = run_sweep(g, ring, a, H, &entry, kProfMis, &t_end, &steps))) break;
        timed(0, t_end, steps, t0);
        // gather
        t0 = clock::now();
        a.lab = lab;
        a.dl = bcap;
        a.dlab = dlab;
        a.ft = nullptr;
        a.fts = ft;
        e = cudaMemsetAsync(lab, 0xff, (size_t)n * 8, st);  // lab and dlab
        if (e != cudaSuccess) { rc = status_of(e, "weighted MIS", __FILE__, __LINE__); break; }
        if ((rc = ring.begin(st))) break;
        FL_LAUNCH(kProfMis, k_wseed<<<grid_for(n, 256), 256, 0, st>>>(a, cover, s->client.as<uint8_t>()));
        if ((rc = run_sweep(g, ring, a, H, nullptr, kProfMis, &t_end, &steps))) break;
        timed(1, t_end, steps, t0);
        if (m > 0)
            FL_LAUNCH(kProfMis, k_wdecide<<<grid_for(m, 256), 256, 0, st>>>(fac_by_ord, m, dlab, state, c + R + 7,
                                                                            c + R + 2));
        FL_LAUNCH(kProfMis, k_wclaim<<<grid_for(n, 256), 256, 0, st>>>(n, s->client.as<uint8_t>(), cover, fac_by_ord,
                                                                       state, s->claimed.as<uint8_t>(),
                                                                       s->kill.as<uint8_t>(), c + R + 8));
        e = cudaMemcpyAsync(h, c + R + 7, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "weighted MIS", __FILE__, __LINE__); break; }
        const int64_t joined = (int64_t)h[0], claimed = (int64_t)h[1];
        if (joined == 0) { rc = FL_ECUDA; set_error(rc, "weighted MIS: a round decided nothing"); break; }
        // kill
        if (nu > joined && claimed > 0) {
            t0 = clock::now();
            e = cudaMemsetAsync(lab, 0xff, (size_t)n * 8, st);
            if (e != cudaSuccess) { rc = status_of(e, "weighted MIS", __FILE__, __LINE__); break; }
            if ((rc = ring.begin(st))) break;
            FL_LAUNCH(kProfMis, k_wseed<<<grid_for(n, 256), 256, 0, st>>>(a, nullptr, s->kill.as<uint8_t>()));
            if ((rc = run_sweep(g, ring, a, H, nullptr, kProfMis, &t_end, &steps))) break;
            timed(4, t_end, steps, t0);
            FL_LAUNCH(kProfMis, k_wkill<<<grid_for(m, 256), 256, 0, st>>>(fac_by_ord, m, dlab, state));
        }
        s->mis_log.insert(s->mis_log.end(),
                          {rounds, 3, H, nu, joined,
                           (int64_t)std::chrono::duration<double, std::micro>(clock::now() - round_t0).count()});
    }
    if (rc == FL_OK) {
        unsigned long long no = 0;
        cudaError_t e = cudaMemsetAsync(c + R + 9, 0, 8, st);
        if (e == cudaSuccess) {
            FL_LAUNCH(kProfMis, k_wopen<<<grid_for(n, 256), 256, 0, st>>>(state, n, s->open.as<uint8_t>(), c + R + 9));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&no, c + R + 9, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = status_of(e, "weighted MIS", __FILE__, __LINE__);
        s->n_open = (int64_t)no;
        s->mis_rounds = rounds;
    }
    ring.release(st);
    return rc;
}

int assign_weighted(fl_solve* s) {
    fl_graph* g = s->g;
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    FL_TRY(dalloc(s->assign, (size_t)n * 4));
    FL_TRY(dalloc(s->dist, (size_t)n * 4));
    FL_TRY(dalloc(s->kill, (size_t)n));
    FL_CUDA(cudaMemsetAsync(s->assign.p, 0xff, (size_t)n * 4, st));
    FL_CUDA(cudaMemsetAsync(s->dist.p, 0xff, (size_t)n * 4, st));
    FL_CUDA(cudaMemsetAsync(s->kill.p, 0, (size_t)n, st));
    WRing ring;
    int rc = ring.alloc(g);
    if (rc == FL_OK) {
        WSweep a = ring.sweep(g);
        a.lab = s->assign.as<uint32_t>();  // facility id; kNone reads as -1
        a.dist = s->dist.as<int32_t>();
        a.past = s->kill.as<uint8_t>();
        a.first = 1;
        int64_t t_end = 0, steps = 0;
        rc = ring.begin(st);
        if (rc == FL_OK) {
            FL_LAUNCH(kProfBfs, k_wseed<<<grid_for(n, 256), 256, 0, st>>>(a, nullptr, s->open.as<uint8_t>()));
            rc = run_sweep(g, ring, a, 2147483647LL, nullptr, kProfBfs, &t_end, &steps);
        }
        unsigned long long err = 0;
        if (rc == FL_OK) {
            FL_LAUNCH(kProfBfs, k_wbeyond<<<grid_for(n, 256), 256, 0, st>>>(n, s->kill.as<uint8_t>(), a.lab,
                                                                           ring.c + ring.R + 2));
            cudaError_t e = cudaMemcpyAsync(&err, ring.c + ring.R + 2, 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = status_of(e, "weighted assignment", __FILE__, __LINE__);
        }
        if (rc == FL_OK && (err & 2ULL)) {
            rc = FL_EINVAL;
            set_error(rc, "weighted assignment: a distance above 2^31 - 1");
        }
    }
    ring.release(st);
    return rc;
}

}  // namespace fl
