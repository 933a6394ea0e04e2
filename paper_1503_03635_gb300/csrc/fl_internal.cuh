// fl_internal.cuh -- shared internals of libflgpu (handles, errors, warp primitives).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <initializer_list>
#include <vector>

#include "../../include/fl.h"

namespace fl {

// ----------------------------------------------------------------- errors

void set_error(int status, const std::string& msg);
int status_of(cudaError_t e, const char* what, const char* file, int line);

#define FL_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e__ = (call);                                                  \
        if (e__ != cudaSuccess) return ::fl::status_of(e__, #call, __FILE__, __LINE__); \
    } while (0)

#define FL_TRY(expr)                 \
    do {                             \
        int s__ = (expr);            \
        if (s__ != FL_OK) return s__; \
    } while (0)

#define FL_FAIL(code, msg)               \
    do {                                 \
        ::fl::set_error((code), (msg));  \
        return (code);                   \
    } while (0)

// ----------------------------------------------------------------- device buffers

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

int dalloc(DBuf& b, size_t bytes);            // free + allocate (no copy)
int dgrow(DBuf& b, size_t bytes, size_t keep, cudaStream_t st);  // grow keeping `keep` bytes
void dfree(DBuf& b);
void dfree_idle(DBuf& b);                     // to the idle-block cache (no pending work uses b)
// A call's temporaries: to the idle-block cache once `st` has finished with them.
void dfree_after(cudaStream_t st, std::initializer_list<DBuf*> bufs);

// ----------------------------------------------------------------- constants

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;   // SplitMix64 increment
constexpr uint64_t kMul1 = 0xbf58476d1ce4e5b9ULL;
constexpr uint64_t kMul2 = 0x94d049bb133111ebULL;
constexpr uint64_t kEmpty = ~0ULL;                   // empty sketch slot

// Vertex ids.  Kernels work on internal ids.  A graph may relabel its
// vertices (by descending degree, so that the values of high-degree vertices,
// read by most edges, share cache sectors) or be a disjoint union of parts
// (batches).  The rank id of a vertex is the id that ranks, priorities and
// reported facility labels use: the original id of a relabelled graph, the
// part-local id in a union, else the id itself.
struct IdMap {
    const int32_t* rid = nullptr;    // rank id of each internal vertex (NULL: the id itself)
    const int32_t* inv = nullptr;    // relabelled graph: internal id of each original id
    const int32_t* vbase = nullptr;  // union: first internal id of each vertex's part
};

__device__ __forceinline__ int64_t rank_id(const IdMap& m, int64_t v) {
    return m.rid ? (int64_t)__ldg(&m.rid[v]) : v;
}

// Internal id of the vertex with rank id r, in the part of vertex v.
__device__ __forceinline__ int64_t internal_of(const IdMap& m, int64_t r, int64_t v) {
    return m.inv ? (int64_t)__ldg(&m.inv[r]) : (m.vbase ? r + (int64_t)__ldg(&m.vbase[v]) : r);
}

__host__ __device__ constexpr uint64_t inv_odd(uint64_t a) {
    // Newton iteration for the inverse of an odd number mod 2^64
    uint64_t x = a;
    for (int i = 0; i < 6; ++i) x *= 2 - a * x;
    return x;
}

// SplitMix64 finaliser and its inverse (each step is a bijection on 64 bits).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * kMul1;
    z = (z ^ (z >> 27)) * kMul2;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t unmix64(uint64_t y) {
    y = y ^ (y >> 31) ^ (y >> 62);
    y *= inv_odd(kMul2);
    y = y ^ (y >> 27) ^ (y >> 54);
    y *= inv_odd(kMul1);
    return y ^ (y >> 30) ^ (y >> 60);
}
// r(v): SplitMix64 output v+1 from state `seed`.
__host__ __device__ __forceinline__ uint64_t vertex_rank(uint64_t seed, int64_t v) {
    return mix64(seed + (uint64_t)(v + 1) * kGamma);
}
// the vertex whose rank is x (ranks are a bijection of the counter)
__host__ __device__ __forceinline__ int64_t rank_vertex(uint64_t seed, uint64_t x) {
    return (int64_t)((unmix64(x) - seed) * inv_odd(kGamma) - 1);
}
// pi(f): SplitMix64 output f+1 from the state given by the first output for `seed`.
__host__ __device__ __forceinline__ uint64_t facility_priority(uint64_t seed, int64_t f) {
    uint64_t stream = mix64(seed + kGamma);
    return mix64(stream + (uint64_t)(f + 1) * kGamma);
}

// ----------------------------------------------------------------- warp primitives
// A "lane list" holds up to 32 uint64 values, one per lane, ascending by lane,
// padded with kEmpty.

constexpr unsigned kFull = 0xffffffffu;

// Vertices with more than kHubDeg neighbours are hubs; their edge lists are
// processed in segments of kSeg edges, one group of lanes per segment.
constexpr int kHubDeg = 2048;
constexpr int kSeg = 2048;
// Non-hub vertices with at most kSmallDeg neighbours are pulled by one thread each.
constexpr int kSmallDeg = 8;
// Width of the small-rank universe of the sketch hops (the kUW smallest
// ranks of a graph; a saturated sketch is a kUW-bit mask over them).
constexpr int kUW = 1024;
constexpr int kUSlices = kUW / 256;  // a mask is read and merged in 256-bit slices
constexpr int kUWords = kUW / 64;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// Bitonic sort of one value per lane, ascending across lanes.
__device__ __forceinline__ uint64_t warp_sort(uint64_t x) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint64_t y = __shfl_xor_sync(kFull, x, j);
            bool up = (lane & k) == 0 || k == 32;
            bool low = (lane & j) == 0;
            x = (low == up) ? umin64(x, y) : umax64(x, y);
        }
    }
    return x;
}

// The 32 smallest of two ascending lane lists, ascending (bitonic merge).
__device__ __forceinline__ uint64_t warp_merge_low(uint64_t a, uint64_t b) {
    const int lane = lane_id();
    uint64_t br = __shfl_sync(kFull, b, 31 - lane);
    uint64_t c = umin64(a, br);
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        uint64_t y = __shfl_xor_sync(kFull, c, j);
        c = (lane & j) ? umax64(c, y) : umin64(c, y);
    }
    return c;
}

// Number of entries of ascending lane list L that are < x (0..32).
__device__ __forceinline__ int warp_lower_bound(uint64_t L, uint64_t x) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        uint64_t y = __shfl_sync(kFull, L, pos + s - 1);
        if (y < x) pos += s;
    }
    uint64_t last = __shfl_sync(kFull, L, 31);
    if (pos == 31 && last < x) pos = 32;
    return pos;
}

// Is x one of the entries of ascending lane list L?
__device__ __forceinline__ bool warp_member(uint64_t L, uint64_t x) {
    int pos = warp_lower_bound(L, x);
    uint64_t y = __shfl_sync(kFull, L, pos & 31);
    return pos < 32 && y == x;
}

// HIP weight of a group whose ball holds cnt ranks with k-th smallest kth:
// 1 while the ball has fewer than k vertices, else 1 / Pr[rank < k-th] =
// 2^64 / kth (one IEEE division).
__device__ __forceinline__ double hip_weight(int cnt, int k, uint64_t kth) {
    return cnt < k ? 1.0 : __ddiv_rn(18446744073709551616.0, __ull2double_rn(kth));
}

// Position of the n-th (0-based) set bit of m (m must have > n set bits).
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        unsigned low = m & ((1u << s) - 1u);
        int c = __popc(low);
        if (n >= c) {
            n -= c;
            m >>= s;
            pos += s;
        } else {
            m = low;
        }
    }
    return pos;
}

// Gather the values of lanes in `keep` to lanes 0..popc(keep)-1 (order kept),
// the rest get `fill`.
__device__ __forceinline__ uint64_t warp_compact(uint64_t x, unsigned keep, uint64_t fill) {
    const int lane = lane_id();
    int total = __popc(keep);
    int src = lane < total ? nth_set_bit(keep, lane) : 0;
    uint64_t y = __shfl_sync(kFull, x, src);
    return lane < total ? y : fill;
}

__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = lane_id();
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        int y = __shfl_up_sync(kFull, x, s);
        if (lane >= s) x += y;
    }
    return x;
}

// Warp-aggregated append: every lane with `pred` gets a distinct slot index
// from `counter` (one atomic per warp); lanes without it get -1.  All 32
// lanes must call it.
__device__ __forceinline__ long long warp_append(bool pred, unsigned long long* counter) {
    const int lane = lane_id();
    unsigned m = __ballot_sync(kFull, pred);
    if (!m) return -1;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    return pred ? (long long)(base + __popc(m & ((1u << lane) - 1u))) : -1LL;
}

// Append with one global atomic per block and call: the block's warps take
// consecutive places.  Every thread of the block calls it the same number of
// times (a block-uniform loop); blockDim.x = 32 * W.  Which places a block
// gets depends on the order of the blocks' atomics, like warp_append.
template <int W>
struct BlockAppend {
    unsigned cnt[W];
    unsigned long long off[W];
};

template <int W>
__device__ __forceinline__ long long block_append(bool pred, unsigned long long* counter, BlockAppend<W>& sh) {
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(kFull, pred);
    if (lane == 0) sh.cnt[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long total = 0;
        for (int w = 0; w < W; ++w) {
            sh.off[w] = total;
            total += sh.cnt[w];
        }
        const unsigned long long base = total ? atomicAdd(counter, total) : 0ULL;
        for (int w = 0; w < W; ++w) sh.off[w] += base;
    }
    __syncthreads();
    return pred ? (long long)(sh.off[warp] + __popc(m & ((1u << lane) - 1u))) : -1LL;
}

// ----------------------------------------------------------------- group primitives
// A group is G consecutive lanes of a warp (G = 16 or 32) that works on one
// vertex; a G-lane list holds up to G uint64 values, one per lane, ascending,
// padded with kEmpty.  All sync intrinsics use the group's own lane mask, so
// the two half-warp groups of a warp may diverge.

template <int G>
struct Grp {
    unsigned mask;
    int l;      // lane within the group
    int shift;  // position of the group's bits in a warp ballot
    __device__ __forceinline__ Grp() {
        const int lane = lane_id();
        l = lane & (G - 1);
        shift = (G == 32) ? 0 : (lane & 16);
        mask = (G == 32) ? kFull : (0xffffu << shift);
    }
    __device__ __forceinline__ unsigned ballot(bool p) const {
        unsigned b = __ballot_sync(mask, p);
        return (G == 32) ? b : ((b >> shift) & 0xffffu);
    }
    template <class T>
    __device__ __forceinline__ T shfl(T x, int src) const { return __shfl_sync(mask, x, src, G); }
    template <class T>
    __device__ __forceinline__ T shfl_xor(T x, int m) const { return __shfl_xor_sync(mask, x, m, G); }
    template <class T>
    __device__ __forceinline__ T shfl_up(T x, int d) const { return __shfl_up_sync(mask, x, d, G); }
};

// Bitonic sort of a G-lane list (ascending).
template <int G>
__device__ __forceinline__ uint64_t grp_sort(const Grp<G>& g, uint64_t x) {
#pragma unroll
    for (int k = 2; k <= G; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint64_t y = g.shfl_xor(x, j);
            bool up = (g.l & k) == 0 || k == G;
            bool low = (g.l & j) == 0;
            x = (low == up) ? umin64(x, y) : umax64(x, y);
        }
    }
    return x;
}

// The G smallest of two ascending G-lane lists, ascending.
template <int G>
__device__ __forceinline__ uint64_t grp_merge_low(const Grp<G>& g, uint64_t a, uint64_t b) {
    uint64_t c = umin64(a, g.shfl(b, G - 1 - g.l));
#pragma unroll
    for (int j = G / 2; j > 0; j >>= 1) {
        uint64_t y = g.shfl_xor(c, j);
        c = (g.l & j) ? umax64(c, y) : umin64(c, y);
    }
    return c;
}

// Is x an entry of the ascending G-lane list L?  (every lane of the group calls)
template <int G>
__device__ __forceinline__ bool grp_member(const Grp<G>& g, uint64_t L, uint64_t x) {
    int pos = 0;
#pragma unroll
    for (int s = G / 2; s > 0; s >>= 1) {
        uint64_t y = g.shfl(L, pos + s - 1);
        if (y < x) pos += s;
    }
    uint64_t last = g.shfl(L, G - 1);
    if (pos == G - 1 && last < x) pos = G;
    uint64_t y = g.shfl(L, pos & (G - 1));
    return pos < G && y == x;
}

// Gather the lanes in `keep` (group-relative bits) to lanes 0.., order kept.
template <int G>
__device__ __forceinline__ uint64_t grp_compact(const Grp<G>& g, uint64_t x, unsigned keep, uint64_t fill) {
    int total = __popc(keep);
    int src = g.l < total ? nth_set_bit(keep, g.l) : 0;
    uint64_t y = g.shfl(x, src);
    return g.l < total ? y : fill;
}

// ----------------------------------------------------------------- device counters

// Small block of device counters read back by the host between launches.
struct Counters {
    unsigned long long frontier;     // vertices appended to the next frontier
    unsigned long long active;       // vertices in the active list of a hop
    unsigned long long stg_entries;  // ADS staging entries used
    unsigned long long stg_groups;   // ADS staging groups used
    unsigned long long merges;       // edge-merges of the next hop (sum of deg of frontier)
    unsigned long long error;        // nonzero: a kernel detected a bad input
    unsigned long long aux0;         // general purpose
    unsigned long long cand_reads;   // merge: neighbour-delta ranks read (sum of |D_{h-1}(u)| over frontier edges)
    unsigned long long merging;      // merge: vertices with at least one frontier neighbour
    unsigned long long aux3;
    unsigned long long scanned;      // hop census: CSR entries read this hop
    unsigned long long mask_scanned; // hop census: of those, read by the mask merge
    unsigned long long delta_next;   // merge: sum of deg(u) * |D_h(u)| over changed u (delta ranks of the next hop's edge-merges)
    unsigned long long new_entries;  // merge: entries gained this hop (sum of |D_h(v)|)
    unsigned long long key_or[2];    // keys: OR of the candidates' (hi, lo) key words
    unsigned long long key_orn[2];   // keys: OR of their complements (a bit set in both varies)
    unsigned long long key_ties;     // keys: adjacent equal hi words after sorting by hi
};

// ----------------------------------------------------------------- profiling
// Kernel classes for launch counts and CUDA-event timings.
enum ProfClass {
    kProfSketchMerge = 0,  // k_merge_hop
    kProfSketchExpand = 1, // k_expand
    kProfSketchOther = 2,  // rank init, ADS compaction, scans, eccentricity bound
    kProfRadius = 3,
    kProfKeys = 4,         // candidates, radix sort, ordinals
    kProfMis = 5,          // greedy-MIS rounds
    kProfBfs = 6,          // assignment BFS
    kProfOther = 7,        // validation, exports, objective
    kProfExact = 8,        // exact ball sizes, their HIP estimates, exact-count radii
    kProfClasses = 9
};

struct Prof {
    int on = 0;
    int64_t launches[kProfClasses] = {};
    double ms[kProfClasses] = {};
    double bytes[kProfClasses] = {};
    std::vector<cudaEvent_t> ev;   // pool of (start, stop) pairs
    std::vector<int> cls;          // class of each recorded pair
    size_t used = 0;
};

// The profiler of the handle whose API call is running on this thread.
Prof* current_prof();
void set_current_prof(Prof* p, cudaStream_t st);
int prof_begin(int cls);           // counts the launch; records a start event when on
void prof_end(int slot);           // records the stop event
int prof_drain(Prof* p);           // after a stream sync: accumulate elapsed times

// Launch a kernel statement and account it to a class.
#define FL_LAUNCH(cls, ...)                      \
    do {                                         \
        int slot__ = ::fl::prof_begin(cls);      \
        __VA_ARGS__;                             \
        ::fl::prof_end(slot__);                  \
    } while (0)

// ----------------------------------------------------------------- schedules
// Launch and round-switch parameters of a graph: they change how fast the
// path runs, never what it computes.
struct Sched {
    int hop_group = 0;    // lanes per vertex in the sketch hop for k <= 16 (16 or 32; 0: 16)
    int sparse_div = 16;  // a hop runs sparse when frontier * sparse_div < listed vertices
    int dense_div = 8;    // a relaxation round pulls when frontier * dense_div >= listed vertices
    int edge_div = 16;    // ... or when frontier edges * edge_div >= nnz
    int graph_bfs = 0;    // 1: the assignment BFS runs as one CUDA graph (a device-side level loop)
    int level_cap = 0;    // BFS levels at most (0: n + 2); beyond it FL_ETIMEOUT
};

// ----------------------------------------------------------------- graph BFS
// A level-synchronous BFS run as one CUDA graph (k_solve.cu): its
// instantiation, cached per graph handle (prefix views of a batch share it)
// and rebuilt when the buffers or sizes it was built for change.
struct GraphBfs {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t key_n[4] = {0, 0, 0, 0};
    DBuf state;  // level (uint32), vertices reached this level, error flag
};

// ----------------------------------------------------------------- handles

}  // namespace fl

struct fl_graph {
    int64_t n = 0, nnz = 0;
    cudaStream_t stream = nullptr;
    fl::DBuf rowp, cols;           // int64[n+1], int32[nnz]
    fl::DBuf wts;                  // int32[nnz]: edge lengths of a weighted graph, else empty
    fl::DBuf wrev;                 // uint32[nnz]: (weighted) the entry (v, u) paired with each entry (u, v)
    int max_w = 0;                 // largest edge length
    int64_t wlevels = 0;           // distance levels with active vertices in the last weighted build
    // static work lists: non-hub non-isolated vertices, hubs, hub segments
    int lists_ready = 0;
    fl::DBuf low_list, hub_list;   // int32[n_low], int32[n_hubs]
    // the non-hub vertices split by degree for the relaxation rounds: at most
    // kSmallDeg neighbours (a thread each), more (a group of lanes each)
    fl::DBuf small_list, mid_list; // int32[n_small], int32[n_mid]
    int64_t n_small = 0, n_mid = 0;
    fl::DBuf hub_seg;              // int64[n_hubs+1]: first segment of each hub
    fl::DBuf seg_hub;              // int32[n_seg]: hub of each segment
    int64_t n_low = 0, n_hubs = 0, n_seg = 0;
    fl::DBuf part;                 // uint64[n_seg*k]: partial bottom-k of each hub segment (scratch)
    // A graph that is a disjoint union of parts (batched instances): vertex v
    // of the part starting at vbase[v] has local id v - vbase[v], and ranks
    // and priorities are those of the local id, so every part is solved
    // exactly as it would be alone.  Empty for an ordinary graph.
    fl::DBuf vbase;                // int32[n] or empty
    fl::DBuf vpart;                // int32[n]: part of each vertex (with vbase)
    // relabelled graphs (see IdMap): rid = original id of each internal
    // vertex, inv = internal id of each original id; unions keep rid = local id
    fl::DBuf rid, inv;             // int32[n] or empty
    bool relabelled = false;
    int64_t n_parts = 0;           // 0: not a union
    fl::DBuf U;                    // uint64[kUW]: the kUW smallest ranks, ascending (kEmpty padded)
    uint64_t ulim = 0;             // largest entry of U
    fl::DBuf DM[2];                // uint64[kUSlices][n][4]: hop delta masks over U, slice-major
    fl::DBuf PM;                   // uint64[n_seg*kUWords]: partial masks of hub segments (scratch)
    fl::DBuf seg_flag;             // uint8[n_seg]: the segment had a neighbour that gained entries (scratch)
    fl::DBuf PH;                   // uint64[n_seg]: OR of the segment's neighbours' delta heads (scratch)
    fl::DBuf F[2], H[2];           // uint64[n]: smallest new rank of the hop (kEmpty: none), delta bits over U[0..63]
    fl::DBuf W;                    // uint64[n]: own sketch's mask over U[0..63] of head vertices, else 0
    fl::DBuf fbm;                  // uint32[n/32+1]: frontier bitmap of the previous hop
    fl::DBuf URid;                 // int32[kUW]: rank id of the vertex of each entry of U
    uint64_t hlim = 0;             // U[min(63, |U| - 1)]
    // sketches
    int k = 0;
    uint64_t seed = 0;
    int built = 0;
    uint64_t generation = 0;       // bumped by every build
    fl::DBuf S, Scnt;              // uint64[n*k], uint8[n]
    fl::DBuf D[2], Dcnt[2];        // hop deltas (ranks), counts
    fl::DBuf frontier[2];          // int32[n]
    fl::DBuf stamp;                // uint32[n]
    fl::DBuf vg, ve;               // int32[n] per-vertex running group / entry counts
    fl::DBuf stg_ent;              // int32 staging entries (k per slot)
    fl::DBuf stg_grp;              // staging group records (one per slot)
    size_t stg_grp_cap = 0;        // slots
    int stg_k = 0;
    // ADS (vertex-major)
    fl::DBuf gofs, eofs;           // int64[n+1]
    fl::DBuf ginfo, gwt, eid;      // uint32[G], double[G], int32[E]
    int64_t hops = 0, edge_merges = 0, n_entries = 0, n_groups = 0;
    // per-vertex eccentricity upper bound (caps ball radii; balls unchanged)
    fl::DBuf ecc_ub;               // int32[n]
    // counters + scratch
    fl::DBuf ctr;                  // Counters
    fl::Counters* h_ctr = nullptr; // pinned host mirror
    fl::DBuf scratch;              // general scratch (scans, sorts)
    fl::DBuf relax_aux;            // bitmap, hub frontier tags/values, edge counter of the rounds
    fl::Prof prof;                 // launch counts and kernel timings
    fl::Sched sched;               // launch and round-switch schedule (fl_set_schedule, fl_autotune)
    fl::GraphBfs* gbfs = new fl::GraphBfs();  // the CUDA-graph BFS of this handle (shared by prefix views)
    // per-hop counters of the last build (index h-1)
    std::vector<int64_t> hop_scanned, hop_mask, hop_changed;
    std::vector<double> hop_ms;
    // per-hop terms of the algorithmic-bytes model of a hop: edge-merges E_h,
    // merging vertices A_h, neighbour-delta ranks the kernels read R_h, the
    // delta ranks of the edge-merges sum |D_{h-1}(u)| over E_h, new entries |D_h|
    std::vector<int64_t> hop_E, hop_A, hop_R, hop_SD, hop_new;
    cudaEvent_t hop_ev[2] = {nullptr, nullptr};
    // exact sizes and radii: source bits (visited, two frontiers), row-length
    // lists and sweep state, staged query inputs and outputs
    fl::DBuf xbits, xaux, xio;
};

namespace fl {
inline IdMap idmap_of(const fl_graph* g) {
    IdMap m;
    m.rid = g->rid.p ? g->rid.as<int32_t>() : nullptr;
    m.inv = g->relabelled ? g->inv.as<int32_t>() : nullptr;
    m.vbase = (!g->relabelled && g->vbase.p) ? g->vbase.as<int32_t>() : nullptr;
    return m;
}
}  // namespace fl

struct fl_solve {
    fl_graph* g = nullptr;
    uint64_t generation = 0;
    int have_radii = 0, have_open = 0, have_assign = 0;
    fl::DBuf cost, client;         // double[n], uint8[n]
    fl::DBuf radii;                // double[n]
    fl::DBuf ord, fac_by_ord, bcap, state, claimed;  // MIS state
    fl::DBuf reach;                // uint8[n]: 1 + slack of a vertex in the current cover (gather pruning)
    fl::DBuf kill;                 // uint8[n]: 1 + distance to a client claimed in the current round
    std::vector<int64_t> mis_log;  // rows of 6: the rounds of the last MIS (fl_mis_log)
    fl::DBuf X, stamp, mval, fr[2], frval, touched, ulist, ubuck, bcount;
    fl::DBuf key_hi, key_lo, key_val, obj_tmp;  // key sort and objective scratch
    fl::DBuf part_T;               // int32[n_parts]: largest ball radius of a part's undecided facilities
    fl::DBuf io;                   // per-vertex inputs/outputs in original order (relabelled graphs)
    fl::DBuf open;                 // uint8[n]
    fl::DBuf assign, dist;         // int32[n]
    int64_t n_cand = 0, n_open = 0, mis_rounds = 0;
    // opening phase with eps > 0: per-vertex iterations and scratch, the grid
    // tables, one iteration's selection inputs, statistics of the last run
    fl::DBuf eps, eps_tab, eps_r, eps_c;
    double eps_gamma = -1.0, eps_alpha0 = 0.0;
    int64_t eps_iterations = 0, eps_events = 0, eps_groups = 0;
    int have_eps = 0;
};

namespace fl {

// ----------------------------------------------------------------- kernel launchers
// (implemented in the .cu files; all run on g->stream)

int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, DBuf& tmp,
                       int cls = kProfSketchOther);
int scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st, DBuf& tmp,
                              int cls = kProfSketchOther);
// Stable LSD radix sort of (hi, lo) pairs with a payload, 4 bits per pass:
// passes 0-15 take lo's digits, 16-31 hi's; [pass_begin, pass_end) (an even
// count) may skip digits known to be equal.
int sort_pairs_u128(uint64_t* hi, uint64_t* lo, uint32_t* val, int64_t n, cudaStream_t st, DBuf& tmp,
                    int cls = kProfKeys, int pass_begin = 0, int pass_end = 32);
// The same sort over the digits whose bit is set in `digits` (bit p: pass p
// of the full sort, 0-15 lo's digits, 16-31 hi's), least significant first.
// Leaving out digits that are equal in every key changes nothing: a pass
// over such a digit is the identity.
int sort_pairs_u128_digits(uint64_t* hi, uint64_t* lo, uint32_t* val, int64_t n, cudaStream_t st, DBuf& tmp,
                           int cls, uint32_t digits);

int validate_csr(fl_graph* g);
int build_work_lists(fl_graph* g);
int build_sketches(fl_graph* g, int k, uint64_t seed);
// weighted graphs (k_wsketch.cu): length check, and the build in Dijkstra order
int check_weights(fl_graph* g);
int pair_reverse_edges(fl_graph* g);
int build_sketches_weighted(fl_graph* g, int k, uint64_t seed);
int compute_ecc_bound(fl_graph* g);

int check_costs(fl_solve* s);
int compute_radii(fl_solve* s);
int sort_candidates(fl_solve* s, int64_t* m_out);
int open_facilities(fl_solve* s);
// the greedy MIS and the assignment by weighted distance (k_wsolve.cu)
int open_facilities_weighted(fl_solve* s);
int assign_weighted(fl_solve* s);
int msbfs(fl_graph* g, const int32_t* src_list, int64_t n_src, int32_t* label, int32_t* dist,
          DBuf& X, DBuf& stampb, DBuf* fr, DBuf& frval, int cls);
int msbfs_graph(fl_graph* g, const int32_t* src_list, int64_t n_src, int32_t* label, int32_t* dist, DBuf& X,
                DBuf& stampb, int cls);
void graph_bfs_release(GraphBfs* c);

// Per-vertex pruning of the rounds of a sweep (the MIS cover and gather
// sweeps).  A round that first gives v a value below the limit records
// reach[v] = reach_val; a round skips every v with need[v] <= round, and
// every v with only[v] == 0: it does not lower v's value, and a push does
// not offer v one.
struct Prune {
    uint8_t* reach = nullptr;
    const uint8_t* need = nullptr;
    const uint8_t* only = nullptr;
    uint32_t reach_val = 0, round = 0;
};

// State of a sequence of synchronous min-propagation rounds (k_relax.cu).
struct Relax {
    unsigned long long* X[2] = {nullptr, nullptr};  // value buffers; X[cur] is current
    int cur = 0;
    int32_t* fr[2] = {nullptr, nullptr};            // frontier lists; fr[fc] is current
    int fc = 0;
    unsigned long long* frval = nullptr;            // snapshot of frontier values
    uint32_t* stamp = nullptr;                      // frontier stamps / changed flags
    unsigned long long* cnt = nullptr;              // device: [0], [1] list sizes, [2] changed count
    unsigned long long* h_cnt = nullptr;            // pinned host word
    int64_t n_front = 0;                            // host copy of the frontier size
    bool list_valid = true;                         // fr[fc] lists the frontier
    uint32_t sv_prev = 0;                           // stamp of the current frontier
    unsigned long long limit = ~0ULL;               // values >= limit are ignored by pulls
    int dense_div = 8;                              // pull when frontier * dense_div >= vertices
    int edge_div = 16;                              // pull when frontier edges * edge_div >= nnz
    bool settle = false;                            // a value < limit is final (level-synchronous BFS)
    // set by relax_begin (graph-owned scratch)
    uint32_t* bm = nullptr;                         // frontier bitmap of a pull round (n bits)
    uint32_t* hub_tag = nullptr;                    // uint32[n_hubs]: round whose push frontier holds the hub
    unsigned long long* hub_val = nullptr;          // uint64[n_hubs]: the hub's snapshotted value
    unsigned long long* ecnt = nullptr;             // device: frontier edge count
    int32_t* part_cnt = nullptr;                    // device int32[n_parts]: frontier vertices per part
    const int32_t* part_limit = nullptr;            // device int32[n_parts] or NULL: a part whose limit is
    int32_t part_round = 0;                         //   below part_round sits the pull rounds out
    Prune prune;                                    // per-vertex reach / need of the sweep
    bool last_dense = false;                        // the last round pulled
};
// Binds the graph-owned scratch of the rounds to r; call once per sweep
// family, after r.stamp values of earlier users may have been reused.
int relax_begin(fl_graph* g, Relax& r);
int relax_round(fl_graph* g, Relax& r, unsigned long long add, uint32_t sv, int cls);
int relax_prepare_list(fl_graph* g, Relax& r, int cls);
// One round of a bounded marking BFS over g (k_relax.cu): kr[v] = b + 1 for
// every unmarked v with need[v] > b (need may be NULL) and a neighbour whose
// kr is in [1, b]; *marked = the marks made (hubs may count more than once).
int mark_round(fl_graph* g, Relax& r, uint8_t* kr, const uint8_t* need, uint32_t b, int cls, int64_t* marked);
int relax_collect_epoch(fl_graph* g, const unsigned long long* X, unsigned long long hi, int32_t* out,
                        unsigned long long* n_out, int cls);
int assign_clients(fl_solve* s);
// the opening phase with eps > 0 and the selection of Algorithm 6 (k_eps.cu)
int open_facilities_eps(fl_solve* s, double eps);
const int32_t* eps_iterations_of(const fl_solve* s, bool clients);
// exact neighbourhood sizes, their HIP estimates, exact-count radii (k_exact.cu)
int map_sources(fl_graph* g, const int32_t* in, int64_t n_src, int32_t* out);
int exact_ball_sizes(fl_graph* g, int64_t n_src, const int32_t* src, int64_t D, const uint8_t* pred, int64_t* out);
int hip_ball_estimates(fl_graph* g, int64_t n_src, const int32_t* src, int64_t D, const uint8_t* pred, double* out);
int exact_radii(fl_solve* s);
int objective(fl_solve* s, double* obj, int64_t* dist_sum, int64_t* n_unserved);

int read_counters(fl_graph* g);
// batches (k_batch.cu)
int batch_place_parts(fl_graph* U, const std::vector<int64_t>& voff, const std::vector<int64_t>& eoff);
int batch_check_parts(fl_graph* U);
int batch_replicate(const fl_graph* G, int64_t R, fl_graph* U);
int batch_replicate_ecc(const fl_graph* G, int64_t R, fl_graph* U);
int batch_objective(fl_solve* s, const int64_t* off_d, int n_inst, double* obj, long long* n_open,
                    long long* dist_sum, long long* unserved);
int compute_radii_multi(const fl_graph* src, fl_graph* g, int64_t R, const double* cost, const uint8_t* client,
                        double* radii);
int relax_reserve(fl_graph* g);
// vertex numbering by descending degree (k_relabel.cu)
int relabel_graph(fl_graph* g);
template <class T>
int permute_vertices(const fl_graph* g, const T* in, T* out, int64_t reps, bool to_internal, cudaStream_t st);
int sketch_rows_original(const fl_graph* g, uint64_t* out);
int ads_original(fl_graph* g, int64_t* gofs_o, int64_t* eofs_o, uint32_t* ginfo_o, double* gwt_o, int32_t* eid_o);

}  // namespace fl
