// k_sketch.cu -- phase (i): bottom-k sketches and ADS by hop-synchronous
// propagation (Section 3.3, Algorithm 2 for unweighted graphs), with HIP
// weights computed where each entry joins a sketch.
//
// Data layout (k <= 32):
//   S[v*k + i]        current sketch of v, ascending ranks, kEmpty padding
//   Scnt[v]           number of ranks in S[v]
//   D[p][v*k + i]     entries v gained at the previous / current hop (ranks)
//   Dcnt[p][v]        their number (0 = v is not in the frontier)
//   staging           one group slot per work item of every hop (v, hop, HIP
//                     weight, counts) and k entry slots; compacted into the
//                     vertex-major ADS after the last hop
//
// Work decomposition of one hop.  A group of G lanes (G = 16 when k <= 16,
// else 32) owns one vertex: lane i holds S[v][i].  Non-hub vertices are
// processed directly (k_hop_vertices).  Hubs (degree > kHubDeg) are cut into
// segments of kSeg edges; each segment yields a partial bottom-k of its
// candidates in scratch (k_hop_hub_segments), and one group per hub merges
// the partials into the hub's sketch (k_hop_hubs).  Bottom-k of a union is the
// bottom-k of the union of bottom-k's, so the split does not change results.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "fl_internal.cuh"

namespace fl {

struct StgGroup {
    double wt;      // HIP weight of the counted entries
    int32_t v;      // vertex
    int32_t gidx;   // index of this group among v's groups
    int32_t eidx;   // index of its first entry among v's entries
    uint32_t info;  // hop | cnt << 16 | counted << 24; 0 = empty slot
};

__host__ __device__ __forceinline__ uint32_t pack_info(int hop, int cnt, int counted) {
    return (uint32_t)hop | ((uint32_t)cnt << 16) | ((uint32_t)counted << 24);
}

constexpr int kMaxHops = 65535;

// ------------------------------------------------------------------ small-rank masks
// U = the kUW smallest ranks of the graph, ascending.  Every rank <= U[last]
// is an entry of U, so once a sketch is full and its k-th rank is <= U[last]
// ("saturated"), all its entries and every candidate that can still enter it
// are entries of U: the sketch is a kUW-bit mask over U, and one hop is
// S_h(v) = lowest k bits of (S_{h-1}(v) | OR_{u in N(v)} D_{h-1}(u)), with
// D_{h-1}(u) kept as a mask beside its list.  Candidates above U[last] are
// above the k-th rank and drop out either way, so the mask update is the
// list merge exactly.  Masks are merged in 256-bit slices from the smallest
// ranks up, stopping once k bits are kept: a sketch whose k-th rank lies in
// the first slice reads 32 bytes per neighbour.

struct Mask4 {  // one 256-bit slice
    uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    __device__ __forceinline__ void set(int i) {
        const uint64_t b = 1ULL << (i & 63);
        const int q = i >> 6;
        w0 |= q == 0 ? b : 0ULL;
        w1 |= q == 1 ? b : 0ULL;
        w2 |= q == 2 ? b : 0ULL;
        w3 |= q == 3 ? b : 0ULL;
    }
    __device__ __forceinline__ void load(const uint64_t* __restrict__ p) {
        const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(p));
        const ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2*>(p) + 1);
        w0 |= a.x;
        w1 |= a.y;
        w2 |= b.x;
        w3 |= b.y;
    }
    __device__ __forceinline__ void add(const Mask4& o) {
        w0 |= o.w0;
        w1 |= o.w1;
        w2 |= o.w2;
        w3 |= o.w3;
    }
    __device__ __forceinline__ uint64_t word(int q) const {
        return q == 0 ? w0 : (q == 1 ? w1 : (q == 2 ? w2 : w3));
    }
    __device__ __forceinline__ bool operator==(const Mask4& o) const {
        return w0 == o.w0 && w1 == o.w1 && w2 == o.w2 && w3 == o.w3;
    }
    __device__ __forceinline__ bool empty() const { return (w0 | w1 | w2 | w3) == 0; }
    __device__ __forceinline__ int count() const {
        return __popcll(w0) + __popcll(w1) + __popcll(w2) + __popcll(w3);
    }
};

// Lowest m set bits of x (m < popcount(x)).
__device__ __forceinline__ uint64_t keep_lowest64(uint64_t x, int m) {
    const unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
    const int c = __popc(lo);
    const int p = m < c ? nth_set_bit(lo, m) : 32 + nth_set_bit(hi, m - c);
    return x & ((1ULL << p) - 1ULL);
}

__device__ __forceinline__ uint64_t lowest_word(uint64_t x, int& left) {
    const int c = __popcll(x);
    const uint64_t r = left <= 0 ? 0ULL : (c > left ? keep_lowest64(x, left) : x);
    left -= c;
    return r;
}

// Keep the lowest k set bits of the slice.
__device__ __forceinline__ void mask_lowest(Mask4& m, int k) {
    int left = k;
    m.w0 = lowest_word(m.w0, left);
    m.w1 = lowest_word(m.w1, left);
    m.w2 = lowest_word(m.w2, left);
    m.w3 = lowest_word(m.w3, left);
}

// Index of the j-th set bit (0-based) of the slice; j < count().
__device__ __forceinline__ int mask_nth(const Mask4& m, int j) {
    const int c0 = __popcll(m.w0), c1 = __popcll(m.w1), c2 = __popcll(m.w2);
    int q = 0;
    uint64_t x = m.w0;
    if (j >= c0) { j -= c0; q = 1; x = m.w1;
        if (j >= c1) { j -= c1; q = 2; x = m.w2;
            if (j >= c2) { j -= c2; q = 3; x = m.w3; } } }
    const unsigned lo = (unsigned)x;
    const int c = __popc(lo);
    const int p = j < c ? nth_set_bit(lo, j) : 32 + nth_set_bit((unsigned)(x >> 32), j - c);
    return q * 64 + p;
}

// Position of rank x in U (-1 when x > ulim: not an entry).
__device__ __forceinline__ int u_pos(const uint64_t* sU, uint64_t ulim, uint64_t x) {
    if (x > ulim) return -1;
    int pos = 0;
#pragma unroll
    for (int s = kUW / 2; s > 0; s >>= 1)
        if (sU[pos + s - 1] < x) pos += s;
    return pos;
}

template <int G>
__device__ __forceinline__ void grp_or(const Grp<G>& g, Mask4& m) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        m.w0 |= g.shfl_xor(m.w0, o);
        m.w1 |= g.shfl_xor(m.w1, o);
        m.w2 |= g.shfl_xor(m.w2, o);
        m.w3 |= g.shfl_xor(m.w3, o);
    }
}

// Slice q of the mask of the lanes' U positions (-1 = none).
template <int G>
__device__ __forceinline__ Mask4 slice_mask(const Grp<G>& g, int idx, int q) {
    Mask4 m;
    if (idx >= 0 && (idx >> 8) == q) m.set(idx & 255);
    grp_or(g, m);
    return m;
}

// Saturated merge, slice by slice from the smallest ranks: first = the OR of
// the candidates' slice 0, src(q) gives it for q >= 1; idx is the lane's old
// entry's U position.  Lanes j < k receive the new sketch in sk_new; returns
// whether it changed.
template <int G, class Src>
__device__ __forceinline__ bool merge_slices(const Grp<G>& g, int k, const uint64_t* sU, int idx, const Mask4& first,
                                             Src src, uint64_t& sk_new) {
    int left = k, base = 0, own_seen = 0;
    bool changed = false;
    sk_new = kEmpty;
    for (int q = 0; q < kUSlices && left > 0; ++q) {
        const Mask4 own = slice_mask(g, idx, q);
        Mask4 m = q == 0 ? first : src(q);
        m.add(own);
        mask_lowest(m, left);
        changed |= !(m == own);
        own_seen += own.count();
        const int c = m.count();
        if (g.l >= base && g.l < base + c) sk_new = sU[q * 256 + mask_nth(m, g.l - base)];
        base += c;
        left -= c;
    }
    return changed || own_seen < k;
}

// Per-group hop counters in shared memory, one slot per group, updated by
// the group's lane 0 without atomics and flushed once at the end of a kernel
// (the hop kernels run at the register limit; counters in registers cost
// spills in the merge loops).  32-bit: a group adds at most 32 * kHubDeg
// per vertex it processes (hub degrees go to the global counters directly)
// and, with the grids of the hop kernels, processes at most 2^31 / 77824 <
// 2^16 work items.
enum { kCFront, kCMerges, kCMerging, kCDelta, kCNew, kNCtr };
__shared__ unsigned s_hop_ctr[256 / 16][kNCtr];

struct HopCounters {
    unsigned long long cand = 0;  // per lane: neighbour-delta words read
};

template <int G>
__device__ __forceinline__ void hop_ctr_init(const Grp<G>& g) {
    if (g.l == 0)
        for (int i = 0; i < kNCtr; ++i) s_hop_ctr[threadIdx.x / G][i] = 0;
}
// lane 0 of the group only
template <int G>
__device__ __forceinline__ void hop_ctr_add(int field, unsigned x) {
    s_hop_ctr[threadIdx.x / G][field] += x;
}

// Per-hop inputs and outputs of the merge kernels (p = previous hop's
// buffers, read-only during a hop; c = this hop's).  Besides each vertex's
// delta list D and delta mask DM, two dense per-vertex words make the
// per-edge reads small and cache-friendly:
//   F[u]  the smallest rank u gained at the hop (kEmpty: none), the filter of
//         the list and slice merges: a neighbour whose F is not below the
//         vertex's k-th rank cannot change its sketch;
//   H[u]  the bits of u's delta mask over U[0..63] (word 0 of DM);
// and W[v], the mask over U[0..63] of v's own sketch once the sketch is full
// and its k-th rank is at most U[63] ("head" vertices; 0 otherwise).  A head
// vertex takes S_h(v) = lowest k bits of (W[v] | OR_u H[u]): every candidate
// that can still enter is among U[0..63], so this is the list merge's result.
// Frontier membership for the counters comes from a bitmap of the previous
// hop's frontier (n/8 bytes, cache-resident).
struct HopIO {
    const int64_t* __restrict__ rowp;
    const int32_t* __restrict__ cols;
    int k;
    int hop;
    uint64_t seed;
    uint64_t* __restrict__ S;
    uint8_t* __restrict__ Scnt;
    const uint64_t* __restrict__ Dp;
    const uint8_t* __restrict__ Dcp;
    uint64_t* __restrict__ Dc;
    uint8_t* __restrict__ Dcc;
    const uint64_t* __restrict__ Fp;
    uint64_t* __restrict__ Fc;
    const uint64_t* __restrict__ Hp;
    uint64_t* __restrict__ Hc;
    uint64_t* __restrict__ W;
    const uint32_t* __restrict__ bm;
    const uint64_t* __restrict__ DMp;  // slice-major: slice q of vertex v at [(q * n + v) * 4]
    uint64_t* __restrict__ DMc;
    int64_t n;
    int32_t* __restrict__ vg;
    int32_t* __restrict__ ve;
    int32_t* __restrict__ stg_ent;
    StgGroup* __restrict__ stg_grp;
    const uint64_t* __restrict__ U;
    const int32_t* __restrict__ URid;  // rank id of the vertex of each U rank
    uint64_t ulim;                     // U's largest entry
    uint64_t hlim;                     // U[min(63, |U| - 1)]: the head's largest rank
    IdMap ids;
    Counters* ctr;
};

__device__ __forceinline__ bool in_bitmap(const uint32_t* __restrict__ bm, int32_t u) {
    return (__ldg(&bm[u >> 5]) >> (u & 31)) & 1u;
}

// Position of the n-th (0-based) set bit of a 64-bit word (n < popcount).
__device__ __forceinline__ int nth_bit64(uint64_t x, int n) {
    const unsigned lo = (unsigned)x;
    const int c = __popc(lo);
    return n < c ? nth_set_bit(lo, n) : 32 + nth_set_bit((unsigned)(x >> 32), n - c);
}

// The lowest k set bits of x.
__device__ __forceinline__ uint64_t lowest_k64(uint64_t x, int k) {
    return __popcll(x) <= k ? x : keep_lowest64(x, k);
}

template <int G>
__device__ __forceinline__ uint64_t grp_or64(const Grp<G>& g, uint64_t x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x |= g.shfl_xor(x, o);
    return x;
}

// Index of word w of vertex v's delta mask in the slice-major layout (each
// 256-bit slice of all vertices is one dense array, so that the hot slices
// of high-degree vertices share cache lines).
__device__ __forceinline__ int64_t dm_word(int64_t n, int64_t v, int w) {
    return ((int64_t)(w >> 2) * n + v) * 4 + (w & 3);
}

// Slice q of the OR of the delta masks of the neighbours in [e0, e1) that
// gained entries at the previous hop (frontier bitmap; lane-parallel, four
// columns per lane in flight, then reduced over the group); `front` tells
// whether there is such a neighbour.
template <int G>
__device__ __forceinline__ Mask4 gather_masks(const Grp<G>& g, const HopIO& io, int64_t e0, int64_t e1, int q,
                                              bool& front, unsigned long long& cand) {
    Mask4 acc;
    bool f = false;
    const uint64_t* __restrict__ slice = io.DMp + (int64_t)q * io.n * 4;
    for (int64_t e = e0 + g.l; e < e1; e += 4 * G) {
        int32_t u[4];
        bool in[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = e + j * G < e1 ? __ldcs(&io.cols[e + j * G]) : -1;
#pragma unroll
        for (int j = 0; j < 4; ++j) in[j] = u[j] >= 0 && in_bitmap(io.bm, u[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (in[j]) {
                acc.load(slice + (int64_t)u[j] * 4);
                f = true;
                cand += 4ULL;
            }
        }
    }
    grp_or(g, acc);
    front = g.ballot(f) != 0;
    return acc;
}

// OR of the delta heads H[u] of the neighbours in [e0, e1) that are in the
// previous hop's frontier (four columns per lane in flight); `front` tells
// whether there is such a neighbour.
template <int G>
__device__ __forceinline__ uint64_t gather_heads(const Grp<G>& g, const HopIO& io, int64_t e0, int64_t e1,
                                                 bool& front, unsigned long long& cand) {
    uint64_t acc = 0;
    bool f = false;
    for (int64_t e = e0 + g.l; e < e1; e += 4 * G) {
        int32_t u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = e + j * G < e1 ? __ldcs(&io.cols[e + j * G]) : -1;
        bool in[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) in[j] = u[j] >= 0 && in_bitmap(io.bm, u[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (in[j]) {
                acc |= __ldg(&io.Hp[u[j]]);
                f = true;
                cand += 1ULL;
            }
        }
    }
    front = g.ballot(f) != 0;
    return grp_or64(g, acc);
}

// ------------------------------------------------------------------ hop 0

// Hop 0: S_0(v) = {r(v)} and v's ADS group at distance 0.  (Hop 1 recomputes
// the neighbours' ranks from their ids, so no hop-0 delta list or mask is
// stored; the group's single entry is v itself, written by the compaction.)
__global__ void k_rank_init(int64_t n, int k, uint64_t seed, uint64_t* __restrict__ S,
                            uint8_t* __restrict__ Scnt, StgGroup* __restrict__ stg_grp,
                            int32_t* __restrict__ vg, int32_t* __restrict__ ve, IdMap ids, Counters* ctr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint64_t r = vertex_rank(seed, rank_id(ids, v));
        if (r == kEmpty) atomicOr(&ctr->error, 1ULL);
        S[v * k] = r;
        Scnt[v] = 1;
        StgGroup gr;
        gr.wt = 1.0;  // a one-vertex ball: fewer than k ranks (k >= 2)
        gr.v = (int32_t)v;
        gr.gidx = 0;
        gr.eidx = 0;
        gr.info = pack_info(0, 1, 1);
        stg_grp[v] = gr;
        vg[v] = 1;
        ve[v] = 1;
    }
}

// ------------------------------------------------------------------ group sketch updates

// Running sketch of one group: list `sk` (k valid lanes), its size `cnt` and
// the filter `tau` (= sk[k-1] when full, else `tau_base`: kEmpty for a
// vertex's own sketch, the vertex's old k-th rank for a hub partial).
template <int G>
struct Sketch {
    uint64_t sk;
    int cnt;
    uint64_t tau;
    uint64_t tau_base;
    __device__ __forceinline__ void retau(const Grp<G>& g, int k) {
        uint64_t kth = g.shfl(sk, k - 1);
        tau = cnt == k ? kth : tau_base;
    }
};

// Insert one rank x (uniform over the group, x < tau) unless present.
template <int G>
__device__ __forceinline__ void insert_one(const Grp<G>& g, int k, uint64_t x, Sketch<G>& s) {
    if (g.ballot(s.sk == x)) return;
    int p = __popc(g.ballot(s.sk < x));
    uint64_t up = g.shfl_up(s.sk, 1);
    s.sk = (g.l > p) ? up : ((g.l == p) ? x : s.sk);
    if (g.l >= k) s.sk = kEmpty;
    if (s.cnt < k) ++s.cnt;
    s.retau(g, k);
}

// Merge a batch of candidates (one per lane, kEmpty = none; unsorted, may
// repeat or already be in the sketch) keeping the k smallest distinct ranks.
template <int G>
__device__ __forceinline__ void merge_batch(const Grp<G>& g, int k, uint64_t buf, Sketch<G>& s) {
    buf = grp_sort(g, buf);
    uint64_t prev = g.shfl_up(buf, 1);
    bool dup = g.l > 0 && prev == buf;
    bool in_sk = grp_member(g, s.sk, buf);
    unsigned keep = g.ballot(buf != kEmpty && !dup && !in_sk);
    if (!keep) return;
    buf = grp_compact(g, buf, keep, kEmpty);
    uint64_t m = grp_merge_low(g, s.sk, buf);
    s.sk = g.l < k ? m : kEmpty;
    s.cnt = __popc(g.ballot(s.sk != kEmpty));
    s.retau(g, k);
}

// Merge an ascending list of distinct candidates (lanes 0.., kEmpty after)
// into the sketch: drop the ones already present, then one bitonic merge.
template <int G>
__device__ __forceinline__ void merge_sorted(const Grp<G>& g, int k, uint64_t x, Sketch<G>& s) {
    const bool in_sk = grp_member(g, s.sk, x);
    const unsigned have = g.ballot(x != kEmpty);
    const unsigned keep = g.ballot(x != kEmpty && !in_sk);
    if (!keep) return;
    if (keep != have) x = grp_compact(g, x, keep, kEmpty);
    const uint64_t m = grp_merge_low(g, s.sk, x);
    s.sk = g.l < k ? m : kEmpty;
    s.cnt = __popc(g.ballot(s.sk != kEmpty));
    s.retau(g, k);
}

// Absorb one batch of candidates: filter by tau, then insert one by one when
// few survive, else merge the whole batch.
template <int G>
__device__ __forceinline__ void absorb(const Grp<G>& g, int k, uint64_t x, Sketch<G>& s) {
    unsigned m = g.ballot(x < s.tau);
    if (!m) return;
    if (__popc(m) <= 2) {
        while (m) {
            int j = __ffs(m) - 1;
            m &= m - 1;
            uint64_t xj = g.shfl(x, j);
            if (xj < s.tau) insert_one(g, k, xj, s);
        }
    } else {
        merge_batch(g, k, x < s.tau ? x : kEmpty, s);
    }
}

// Absorb the candidates of CSR entries [e0, e1): at hop 1 the neighbours' own
// ranks (recomputed from their ids), later the entries each neighbour gained
// at the previous hop.  Lane j of the group owns neighbour j of a chunk of G
// neighbours and loads its smallest new rank F[u] (independent loads into a
// dense array that also filter whole lists).  Each neighbour whose smallest
// new rank is below the filter then has its list loaded across the group;
// the entries below the filter form an ascending prefix, absorbed by 1-2
// insertions or one bitonic merge.  `front`: some neighbour gained entries.
template <int G>
__device__ __forceinline__ void gather_range(const Grp<G>& g, const HopIO& io, int64_t e0, int64_t e1,
                                             Sketch<G>& s, bool& front, unsigned long long& cand) {
    const int k = io.k;
    bool fr = false;
    // the next chunk's columns are loaded while this chunk merges
    int32_t u_next = e0 + g.l < e1 ? __ldcs(&io.cols[e0 + g.l]) : 0;
    for (int64_t cb = e0; cb < e1; cb += G) {
        const int64_t e = cb + g.l;
        const bool in = e < e1;
        const int32_t u = u_next;
        u_next = e + G < e1 ? __ldcs(&io.cols[e + G]) : 0;
        if (io.hop == 1) {
            absorb(g, k, in ? vertex_rank(io.seed, rank_id(io.ids, u)) : kEmpty, s);
            continue;
        }
        const uint64_t first = in ? __ldg(&io.Fp[u]) : kEmpty;
        fr |= first != kEmpty;
        cand += first != kEmpty ? 1ULL : 0ULL;
        // list lengths of the neighbours that pass the filter, loaded together
        const int c = first < s.tau ? (int)__ldg(&io.Dcp[u]) : 0;
        unsigned live = g.ballot(first < s.tau);
        while (live) {
            const int j = __ffs(live) - 1;
            live &= live - 1;
            const int cj = g.shfl(c, j);
            const uint64_t fj = g.shfl(first, j);
            if (!(fj < s.tau)) continue;  // the filter tightened since the first loads
            if (cj == 1) {
                insert_one(g, k, fj, s);
                continue;
            }
            const int uj = g.shfl(u, j);
            uint64_t x = (g.l > 0 && g.l < cj) ? __ldg(&io.Dp[(int64_t)uj * k + g.l]) : kEmpty;
            cand += (g.l > 0 && g.l < cj) ? 1ULL : 0ULL;
            if (g.l == 0) x = fj;
            const unsigned pm = g.ballot(x < s.tau);  // an ascending prefix of the list
            if (__popc(pm) <= 2) {
                insert_one(g, k, fj, s);
                if (pm & 2u) {
                    const uint64_t x1 = g.shfl(x, 1);
                    if (x1 < s.tau) insert_one(g, k, x1, s);
                }
            } else {
                merge_sorted(g, k, x < s.tau ? x : kEmpty, s);
            }
        }
    }
    front = io.hop == 1 || g.ballot(fr) != 0;
}

// Record a changed vertex's ADS group in staging slot `slot` and count it
// (lane 0 of the group).
template <int G>
__device__ __forceinline__ void stage_group(const HopIO& io, int32_t v, int64_t deg, int64_t slot, int dcnt,
                                            int counted, double wt) {
    StgGroup gr;
    gr.wt = wt;
    gr.v = v;
    gr.gidx = io.vg[v];
    gr.eidx = io.ve[v];
    gr.info = pack_info(io.hop, dcnt, counted);
    io.vg[v] = gr.gidx + 1;
    io.ve[v] = gr.eidx + dcnt;
    io.stg_grp[slot] = gr;
    hop_ctr_add<G>(kCFront, 1u);
    hop_ctr_add<G>(kCNew, (unsigned)dcnt);
    if (deg <= kHubDeg) {
        hop_ctr_add<G>(kCMerges, (unsigned)deg);
        hop_ctr_add<G>(kCDelta, (unsigned)(deg * dcnt));
    }
}


// Write the results of vertex v after a list or slice merge: new sketch, the
// entries it gained (list, mask, head word, smallest one, for the next hop),
// its own head mask once the sketch is a head sketch, and its staged ADS
// group in work slot `slot`.  Returns the number of entries gained (0: the
// sketch is unchanged).
template <int G>
__device__ __forceinline__ int finish_vertex(const Grp<G>& g, const HopIO& io, int32_t v, int64_t deg, uint64_t old,
                                             const Sketch<G>& s, int64_t slot, const uint64_t* sU) {
    const int k = io.k;
    const bool valid = g.l < k && s.sk != kEmpty;
    const bool was_there = grp_member(g, old, s.sk);
    const unsigned newm = g.ballot(valid && !was_there);
    const int dcnt = __popc(newm);
    if (dcnt == 0) {
        if (g.l == 0) io.stg_grp[slot].info = 0;  // empty slot
        return 0;
    }
    const int cnt_new = __popc(g.ballot(valid));
    if (g.l < k) io.S[(int64_t)v * k + g.l] = s.sk;
    const uint64_t dv = grp_compact(g, s.sk, newm, kEmpty);
    if (g.l < dcnt) {
        io.Dc[(int64_t)v * k + g.l] = dv;
        io.stg_ent[slot * k + g.l] = (int32_t)internal_of(io.ids, (int64_t)rank_vertex(io.seed, dv), v);
    }
    // delta mask over U: lane w < kUWords builds word w
    const int di = g.l < dcnt ? u_pos(sU, io.ulim, dv) : -1;
    uint64_t word = 0;
    for (int j = 0; j < dcnt; ++j) {
        const int ij = g.shfl(di, j);
        if (ij >= 0 && (ij >> 6) == g.l) word |= 1ULL << (ij & 63);
    }
    if (g.l < kUWords) io.DMc[dm_word(io.n, v, g.l)] = word;
    const uint64_t kth = g.shfl(s.sk, k - 1);
    // a full sketch whose k-th rank is in U's head becomes a head vertex
    if (cnt_new == k && kth <= io.hlim) {
        const int p = g.l < k ? u_pos(sU, io.ulim, s.sk) : -1;
        const uint64_t own = grp_or64(g, p >= 0 ? 1ULL << p : 0ULL);
        if (g.l == 0) io.W[v] = own;
    }
    if (g.l == 0) {
        io.Fc[v] = dv;    // lane 0 holds the smallest new rank
        io.Hc[v] = word;  // lane 0 built word 0
        io.Scnt[v] = (uint8_t)cnt_new;
        io.Dcc[v] = (uint8_t)dcnt;
        const int counted = cnt_new < k ? dcnt : __popc(newm & ((1u << (k - 1)) - 1u));
        stage_group<G>(io, v, deg, slot, dcnt, counted, hip_weight(cnt_new, k, kth));
    }
    return dcnt;
}

// Write the results of head vertex v whose new sketch is the mask nw over
// U[0..63] (k bits) with gained bits delta (nonzero); the same outputs as
// finish_vertex.
template <int G>
__device__ __forceinline__ void finish_head(const Grp<G>& g, const HopIO& io, int32_t v, int64_t deg, uint64_t nw,
                                            uint64_t delta, int64_t slot, const uint64_t* sU,
                                            const int32_t* sURid) {
    const int k = io.k;
    const int dcnt = __popcll(delta);
    if (g.l < k) io.S[(int64_t)v * k + g.l] = sU[nth_bit64(nw, g.l)];
    if (g.l < dcnt) {
        const int p = nth_bit64(delta, g.l);
        io.Dc[(int64_t)v * k + g.l] = sU[p];
        io.stg_ent[slot * k + g.l] = (int32_t)internal_of(io.ids, (int64_t)sURid[p], v);
    }
    if (g.l < kUWords) io.DMc[dm_word(io.n, v, g.l)] = g.l == 0 ? delta : 0ULL;
    if (g.l == 0) {
        const int top = 63 - __clzll(nw);  // the k-th smallest rank's position
        io.W[v] = nw;
        io.Fc[v] = sU[__ffsll(delta) - 1];
        io.Hc[v] = delta;
        io.Dcc[v] = (uint8_t)dcnt;
        const int counted = dcnt - (int)((delta >> top) & 1ULL);
        stage_group<G>(io, v, deg, slot, dcnt, counted, hip_weight(k, k, sU[top]));
    }
}

template <int G>
__device__ __forceinline__ void flush_counters(const Grp<G>& g, HopCounters hc, Counters* ctr) {
    // candidate reads are counted per lane; the other counters by lane 0
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) hc.cand += g.shfl_xor(hc.cand, o);
    if (g.l == 0) {
        const unsigned* c = s_hop_ctr[threadIdx.x / G];
        if (hc.cand) atomicAdd(&ctr->cand_reads, hc.cand);
        if (c[kCFront]) atomicAdd(&ctr->frontier, (unsigned long long)c[kCFront]);
        if (c[kCMerges]) atomicAdd(&ctr->merges, (unsigned long long)c[kCMerges]);
        if (c[kCMerging]) atomicAdd(&ctr->merging, (unsigned long long)c[kCMerging]);
        if (c[kCDelta]) atomicAdd(&ctr->delta_next, (unsigned long long)c[kCDelta]);
        if (c[kCNew]) atomicAdd(&ctr->new_entries, (unsigned long long)c[kCNew]);
    }
}

// U and the rank ids of its entries, staged in shared memory by every hop kernel.
__device__ __forceinline__ void load_tables(uint64_t* sU, int32_t* sURid, const HopIO& io) {
    for (int i = threadIdx.x; i < kUW; i += blockDim.x) {
        sU[i] = io.U[i];
        sURid[i] = io.URid[i];
    }
    __syncthreads();
}

// ------------------------------------------------------------------ hop kernels

// Non-hub vertices: S_h(v) = bottom-k(S_{h-1}(v) U union_{u in N(v)} D_{h-1}(u)),
// by the head merge (head vertices), the mask merge (other saturated
// sketches) or the list merge.
template <int G>
__global__ void __launch_bounds__(256, 4) k_hop_vertices(const int32_t* __restrict__ list, int64_t n_list, HopIO io) {
    __shared__ uint64_t sU[kUW];
    __shared__ int32_t sURid[kUW];
    load_tables(sU, sURid, io);
    const Grp<G> g;
    const int k = io.k;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    HopCounters hc;
    hop_ctr_init(g);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < n_list; i += groups) {
        const int32_t v = list[i];
        const int64_t beg = io.rowp[v], end = io.rowp[v + 1];
        const uint64_t wv = io.hop > 1 ? io.W[v] : 0ULL;
        bool front = false;
        if (wv != 0) {
            // head vertex: the head merge
            const uint64_t acc = gather_heads(g, io, beg, end, front, hc.cand);
            if (g.l == 0 && front) hop_ctr_add<G>(kCMerging, 1u);
            const uint64_t nw = lowest_k64(wv | acc, k);
            const uint64_t delta = nw & ~wv;
            if (delta == 0) {
                if (g.l == 0) io.stg_grp[i].info = 0;  // unchanged: empty slot
                continue;
            }
            finish_head(g, io, v, end - beg, nw, delta, i, sU, sURid);
            continue;
        }
        const uint64_t old = g.l < k ? io.S[(int64_t)v * k + g.l] : kEmpty;
        Sketch<G> s;
        s.sk = old;
        s.cnt = io.Scnt[v];
        s.tau_base = kEmpty;
        s.retau(g, k);
        const bool sat = io.hop > 1 && s.cnt == k && s.tau <= io.ulim;
        if (sat) {
            // saturated: mask merge over the neighbours whose smallest new
            // rank is below the k-th rank
            const Mask4 first = gather_masks(g, io, beg, end, 0, front, hc.cand);
            if (g.l == 0 && front) hop_ctr_add<G>(kCMerging, 1u);
            if (!front) {
                if (g.l == 0) io.stg_grp[i].info = 0;  // unchanged: empty slot
                continue;
            }
            const int idx = g.l < k ? u_pos(sU, io.ulim, old) : -1;
            uint64_t sk_new;
            bool fq;
            const bool changed = merge_slices(
                g, k, sU, idx, first, [&](int q) { return gather_masks(g, io, beg, end, q, fq, hc.cand); },
                sk_new);
            if (!changed) {
                if (g.l == 0) io.stg_grp[i].info = 0;  // unchanged: empty slot
                continue;
            }
            s.sk = sk_new;
            s.cnt = k;
        } else {
            gather_range(g, io, beg, end, s, front, hc.cand);
            if (g.l == 0 && front) hop_ctr_add<G>(kCMerging, 1u);
        }
        finish_vertex(g, io, v, end - beg, old, s, i, sU);
    }
    flush_counters(g, hc, io.ctr);
}

// Hub segments: partial results of one segment, written per segment -- the
// OR of its neighbours' delta heads (head hubs), the slices of their delta
// masks up to the hub's k-th rank (other saturated hubs), or the bottom-k of
// its candidates below the hub's old k-th rank (list hubs).
template <int G>
__global__ void __launch_bounds__(256) k_hop_hub_segments(const int32_t* __restrict__ hubs,
                                                          const int64_t* __restrict__ hub_seg,
                                                          const int32_t* __restrict__ seg_hub, int64_t n_seg,
                                                          uint64_t* __restrict__ part, uint64_t* __restrict__ PM,
                                                          uint64_t* __restrict__ PH, uint8_t* __restrict__ seg_flag,
                                                          const uint32_t* __restrict__ hub_stamp, uint32_t sparse_hop,
                                                          HopIO io) {
    __shared__ uint64_t sU[kUW];
    __shared__ int32_t sURid[kUW];
    load_tables(sU, sURid, io);
    const Grp<G> g;
    const int k = io.k;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    HopCounters hc;
    hop_ctr_init(g);
    for (int64_t sidx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; sidx < n_seg; sidx += groups) {
        const int32_t h = seg_hub[sidx];
        const int32_t v = hubs[h];
        if (sparse_hop && hub_stamp[v] != sparse_hop) {
            // sparse hop: no neighbour of this hub gained entries
            if (g.l == 0) seg_flag[sidx] = 0;
            continue;
        }
        const int64_t e0 = io.rowp[v] + (sidx - hub_seg[h]) * kSeg;
        const int64_t e1 = min(e0 + (int64_t)kSeg, io.rowp[v + 1]);
        bool front = false;
        if (io.hop > 1 && io.W[v] != 0) {
            const uint64_t acc = gather_heads(g, io, e0, e1, front, hc.cand);
            if (g.l == 0) {
                PH[sidx] = acc;
                seg_flag[sidx] = front ? 1 : 0;
            }
            continue;
        }
        const uint64_t kth_old = io.S[(int64_t)v * k + k - 1];
        const bool sat = io.hop > 1 && io.Scnt[v] == k && kth_old <= io.ulim;
        if (sat) {
            // saturated hub: partial masks of the segment, the slices up to
            // the one holding the hub's k-th rank (the merge stops there)
            const int top = u_pos(sU, io.ulim, kth_old) >> 8;
            for (int q = 0; q <= top; ++q) {
                bool fq;
                const Mask4 m = gather_masks(g, io, e0, e1, q, fq, hc.cand);
                if (q == 0) front = fq;
                if (g.l < 4) PM[sidx * kUWords + q * 4 + g.l] = m.word(g.l);
            }
            if (g.l == 0) seg_flag[sidx] = front ? 1 : 0;
            continue;
        }
        Sketch<G> s;
        s.sk = kEmpty;
        s.cnt = 0;
        s.tau_base = io.Scnt[v] == k ? kth_old : kEmpty;
        s.tau = s.tau_base;
        gather_range(g, io, e0, e1, s, front, hc.cand);
        if (g.l < k) part[sidx * k + g.l] = s.sk;
        if (g.l == 0) seg_flag[sidx] = front ? 1 : 0;
    }
    flush_counters(g, hc, io.ctr);
}

// Did some segment of hub h have a neighbour that gained entries?
template <int G>
__device__ __forceinline__ bool hub_merged(const Grp<G>& g, const int64_t* __restrict__ hub_seg,
                                           const uint8_t* __restrict__ seg_flag, int64_t h) {
    bool any = false;
    for (int64_t sidx = hub_seg[h] + g.l; sidx < hub_seg[h + 1]; sidx += G) any |= seg_flag[sidx] != 0;
    return g.ballot(any) != 0;
}

// Hubs: merge the partial results of all segments into the hub's sketch.
template <int G>
__global__ void __launch_bounds__(256) k_hop_hubs(const int32_t* __restrict__ hubs, int64_t n_hubs,
                                                  const int64_t* __restrict__ hub_seg,
                                                  const uint64_t* __restrict__ part, const uint64_t* __restrict__ PM,
                                                  const uint64_t* __restrict__ PH,
                                                  const uint8_t* __restrict__ seg_flag,
                                                  const uint32_t* __restrict__ hub_stamp, uint32_t sparse_hop,
                                                  int64_t slot0, HopIO io) {
    __shared__ uint64_t sU[kUW];
    __shared__ int32_t sURid[kUW];
    load_tables(sU, sURid, io);
    const Grp<G> g;
    const int k = io.k;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    HopCounters hc;
    hop_ctr_init(g);
    for (int64_t h = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; h < n_hubs; h += groups) {
        const int32_t v = hubs[h];
        const int64_t slot = slot0 + h;
        if (sparse_hop && hub_stamp[v] != sparse_hop) {
            if (g.l == 0) io.stg_grp[slot].info = 0;  // unchanged: empty slot
            continue;
        }
        const int64_t deg = io.rowp[v + 1] - io.rowp[v];
        const bool any = hub_merged(g, hub_seg, seg_flag, h);
        if (g.l == 0 && any) hop_ctr_add<G>(kCMerging, 1u);
        const uint64_t wv = io.hop > 1 ? io.W[v] : 0ULL;
        int dc = 0;
        if (wv != 0) {
            uint64_t acc = 0;
            for (int64_t sidx = hub_seg[h] + g.l; sidx < hub_seg[h + 1]; sidx += G) acc |= PH[sidx];
            acc = grp_or64(g, acc);
            const uint64_t nw = lowest_k64(wv | acc, k);
            const uint64_t delta = nw & ~wv;
            if (delta != 0) {
                finish_head(g, io, v, deg, nw, delta, slot, sU, sURid);
                dc = __popcll(delta);
            } else if (g.l == 0) {
                io.stg_grp[slot].info = 0;  // unchanged: empty slot
            }
        } else {
            const uint64_t old = g.l < k ? io.S[(int64_t)v * k + g.l] : kEmpty;
            Sketch<G> s;
            s.sk = old;
            s.cnt = io.Scnt[v];
            s.tau_base = kEmpty;
            s.retau(g, k);
            bool changed = true;
            if (io.hop > 1 && s.cnt == k && s.tau <= io.ulim) {
                // saturated hub: OR of the segments' partial masks
                const int idx = g.l < k ? u_pos(sU, io.ulim, old) : -1;
                auto part_slice = [&](int q) {
                    Mask4 m;
                    for (int64_t sidx = hub_seg[h] + g.l; sidx < hub_seg[h + 1]; sidx += G)
                        m.load(PM + sidx * kUWords + q * 4);
                    grp_or(g, m);
                    return m;
                };
                uint64_t sk_new;
                changed = merge_slices(g, k, sU, idx, part_slice(0), part_slice, sk_new);
                s.sk = sk_new;
                s.cnt = k;
            } else {
                for (int64_t sidx = hub_seg[h]; sidx < hub_seg[h + 1]; ++sidx) {
                    const uint64_t x = g.l < k ? part[sidx * k + g.l] : kEmpty;
                    absorb(g, k, x, s);
                }
            }
            if (changed) {
                dc = finish_vertex(g, io, v, deg, old, s, slot, sU);
            } else if (g.l == 0) {
                io.stg_grp[slot].info = 0;  // unchanged: empty slot
            }
        }
        if (dc && g.l == 0) {
            atomicAdd(&io.ctr->merges, (unsigned long long)deg);
            atomicAdd(&io.ctr->delta_next, (unsigned long long)(deg * dc));
        }
    }
    flush_counters(g, hc, io.ctr);
}

// Sparse hops: the non-hub part of N(frontier).  Warp per frontier vertex;
// each neighbour is appended once (stamp = hop); hubs in N(frontier) get
// stamp = hop too, and the hub kernels skip the others.
__global__ void k_expand(const int32_t* __restrict__ fr, int64_t n_fr, const int64_t* __restrict__ rowp,
                         const int32_t* __restrict__ cols, uint32_t* __restrict__ stamp, uint32_t hop,
                         int32_t* __restrict__ act, Counters* ctr) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (((int64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; w < n_fr; w += warps) {
        const int32_t u = fr[w];
        const int64_t beg = rowp[u], end = rowp[u + 1];
        for (int64_t cb = beg; cb < end; cb += 32) {
            int64_t e = cb + lane;
            bool fresh = false;
            int32_t v = 0;
            if (e < end) {
                v = cols[e];
                if (rowp[v + 1] - rowp[v] <= kHubDeg)
                    fresh = atomicExch(&stamp[v], hop) != hop;
                else
                    stamp[v] = hop;  // a hub with a frontier neighbour: its segments run this hop
            }
            long long at = warp_append(fresh, &ctr->active);
            if (at >= 0) act[at] = v;
        }
    }
}

// Vertices of a work list that gained entries this hop (the next frontier).
__global__ void k_collect_frontier(const int32_t* __restrict__ list, int64_t n, const uint8_t* __restrict__ Dcc,
                                   int32_t* __restrict__ fr, unsigned long long* __restrict__ n_fr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        int64_t i = base + lane_id();
        int32_t v = i < n ? list[i] : 0;
        bool in = i < n && Dcc[v] > 0;
        long long at = warp_append(in, n_fr);
        if (at >= 0) fr[at] = v;
    }
}

// ------------------------------------------------------------------ ADS compaction

// Staged groups -> vertex-major ADS.  kp = k rounded up to a power of two; a
// thread per (slot, entry) pair, so that a slot's entries are copied by
// adjacent threads (coalesced); the first thread of a slot writes the group.
// In the hop-0 region the single entry of slot v is v itself.
__global__ void k_ads_scatter(const StgGroup* __restrict__ stg_grp, int64_t n_slots, int64_t slot_base, int k,
                              int log2_kp, bool hop0, const int32_t* __restrict__ stg_ent,
                              const int64_t* __restrict__ gofs, const int64_t* __restrict__ eofs,
                              uint32_t* __restrict__ ginfo, double* __restrict__ gwt, int32_t* __restrict__ eid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = n_slots << log2_kp;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t i = t >> log2_kp;
        const int j = (int)(t & ((1 << log2_kp) - 1));
        const StgGroup gr = stg_grp[slot_base + i];
        if (gr.info == 0) continue;
        const int cnt = (int)((gr.info >> 16) & 0xff);
        if (j >= cnt) continue;
        const int64_t de = eofs[gr.v] + gr.eidx;
        if (j == 0) {
            const int64_t dg = gofs[gr.v] + gr.gidx;
            ginfo[dg] = gr.info;
            gwt[dg] = gr.wt;
        }
        eid[de + j] = hop0 ? gr.v : stg_ent[(slot_base + i) * k + j];
    }
}

// ------------------------------------------------------------------ graph work lists

__global__ void k_flag_degree(const int64_t* __restrict__ rowp, int64_t n, int32_t* __restrict__ low,
                              int32_t* __restrict__ hub, int32_t* __restrict__ nseg, int32_t* __restrict__ small) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = rowp[v + 1] - rowp[v];
        low[v] = (d > 0 && d <= kHubDeg) ? 1 : 0;
        hub[v] = d > kHubDeg ? 1 : 0;
        nseg[v] = d > kHubDeg ? (int32_t)((d + kSeg - 1) / kSeg) : 0;
        small[v] = (d > 0 && d <= kSmallDeg) ? 1 : 0;
    }
}

// Split the non-hub vertices by degree (ids ascending in both lists).
__global__ void k_scatter_by_degree(const int32_t* __restrict__ low, const int32_t* __restrict__ small,
                                    const int64_t* __restrict__ small_pos, const int64_t* __restrict__ low_pos,
                                    int64_t n, int32_t* __restrict__ small_list, int32_t* __restrict__ mid_list) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (small[v]) small_list[small_pos[v]] = (int32_t)v;
        else if (low[v]) mid_list[low_pos[v] - small_pos[v]] = (int32_t)v;
    }
}

__global__ void k_scatter_lists(const int32_t* __restrict__ low, const int32_t* __restrict__ hub,
                                const int64_t* __restrict__ low_pos, const int64_t* __restrict__ hub_pos,
                                const int64_t* __restrict__ seg_pos, int64_t n, int32_t* __restrict__ low_list,
                                int32_t* __restrict__ hub_list, int64_t* __restrict__ hub_seg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (low[v]) low_list[low_pos[v]] = (int32_t)v;
        if (hub[v]) {
            hub_list[hub_pos[v]] = (int32_t)v;
            hub_seg[hub_pos[v]] = seg_pos[v];
        }
    }
}

__global__ void k_seg_owner(const int64_t* __restrict__ hub_seg, int64_t n_hubs, int32_t* __restrict__ seg_hub) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_hubs; h += stride)
        for (int64_t s = hub_seg[h]; s < hub_seg[h + 1]; ++s) seg_hub[s] = (int32_t)h;
}

static int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// Last element of an exclusive scan plus the last input = the total.
static int scan_total(const int64_t* pos, const int32_t* flag, int64_t n, cudaStream_t st, int64_t* total) {
    int64_t p = 0;
    int32_t f = 0;
    FL_CUDA(cudaMemcpyAsync(&p, pos + n - 1, 8, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaMemcpyAsync(&f, flag + n - 1, 4, cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    *total = p + f;
    return FL_OK;
}

// Static work lists of a graph: non-hub non-isolated vertices, hubs and the
// segment table of the hubs.
int build_work_lists(fl_graph* g) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    DBuf low, hub, nseg, low_pos, hub_pos, seg_pos, small, small_pos;
    int rc = FL_OK;
    do {
        if ((rc = dalloc(low, (size_t)n * 4)) || (rc = dalloc(hub, (size_t)n * 4)) ||
            (rc = dalloc(nseg, (size_t)n * 4)) || (rc = dalloc(low_pos, (size_t)n * 8)) ||
            (rc = dalloc(hub_pos, (size_t)n * 8)) || (rc = dalloc(seg_pos, (size_t)n * 8)) ||
            (rc = dalloc(small, (size_t)n * 4)) || (rc = dalloc(small_pos, (size_t)n * 8)))
            break;
        FL_LAUNCH(kProfOther, k_flag_degree<<<grid_for(n, 256), 256, 0, st>>>(
                                  g->rowp.as<int64_t>(), n, low.as<int32_t>(), hub.as<int32_t>(), nseg.as<int32_t>(),
                                  small.as<int32_t>()));
        if ((rc = scan_exclusive_i32_to_i64(low.as<int32_t>(), low_pos.as<int64_t>(), n, st, g->scratch, kProfOther)) ||
            (rc = scan_exclusive_i32_to_i64(hub.as<int32_t>(), hub_pos.as<int64_t>(), n, st, g->scratch, kProfOther)) ||
            (rc = scan_exclusive_i32_to_i64(nseg.as<int32_t>(), seg_pos.as<int64_t>(), n, st, g->scratch, kProfOther)) ||
            (rc = scan_exclusive_i32_to_i64(small.as<int32_t>(), small_pos.as<int64_t>(), n, st, g->scratch,
                                            kProfOther)))
            break;
        if ((rc = scan_total(low_pos.as<int64_t>(), low.as<int32_t>(), n, st, &g->n_low)) ||
            (rc = scan_total(hub_pos.as<int64_t>(), hub.as<int32_t>(), n, st, &g->n_hubs)) ||
            (rc = scan_total(seg_pos.as<int64_t>(), nseg.as<int32_t>(), n, st, &g->n_seg)) ||
            (rc = scan_total(small_pos.as<int64_t>(), small.as<int32_t>(), n, st, &g->n_small)))
            break;
        g->n_mid = g->n_low - g->n_small;
        if ((rc = dalloc(g->small_list, (size_t)std::max<int64_t>(g->n_small, 1) * 4)) ||
            (rc = dalloc(g->mid_list, (size_t)std::max<int64_t>(g->n_mid, 1) * 4)))
            break;
        FL_LAUNCH(kProfOther, k_scatter_by_degree<<<grid_for(n, 256), 256, 0, st>>>(
                                  low.as<int32_t>(), small.as<int32_t>(), small_pos.as<int64_t>(),
                                  low_pos.as<int64_t>(), n, g->small_list.as<int32_t>(), g->mid_list.as<int32_t>()));
        if ((rc = dalloc(g->low_list, (size_t)std::max<int64_t>(g->n_low, 1) * 4)) ||
            (rc = dalloc(g->hub_list, (size_t)std::max<int64_t>(g->n_hubs, 1) * 4)) ||
            (rc = dalloc(g->hub_seg, (size_t)(g->n_hubs + 1) * 8)) ||
            (rc = dalloc(g->seg_hub, (size_t)std::max<int64_t>(g->n_seg, 1) * 4)))
            break;
        FL_LAUNCH(kProfOther, k_scatter_lists<<<grid_for(n, 256), 256, 0, st>>>(
                                  low.as<int32_t>(), hub.as<int32_t>(), low_pos.as<int64_t>(), hub_pos.as<int64_t>(),
                                  seg_pos.as<int64_t>(), n, g->low_list.as<int32_t>(), g->hub_list.as<int32_t>(),
                                  g->hub_seg.as<int64_t>()));
        cudaError_t e = cudaMemcpyAsync(g->hub_seg.as<int64_t>() + g->n_hubs, &g->n_seg, 8, cudaMemcpyHostToDevice, st);
        if (e) { rc = status_of(e, "work lists", __FILE__, __LINE__); break; }
        if (g->n_hubs > 0)
            FL_LAUNCH(kProfOther, k_seg_owner<<<grid_for(g->n_hubs, 256), 256, 0, st>>>(
                                      g->hub_seg.as<int64_t>(), g->n_hubs, g->seg_hub.as<int32_t>()));
        e = cudaStreamSynchronize(st);
        if (e) { rc = status_of(e, "work lists", __FILE__, __LINE__); break; }
    } while (0);
    dfree_after(st, {&low, &hub, &nseg, &low_pos, &hub_pos, &seg_pos, &small, &small_pos});
    return rc;
}

// Census of a hop's work list (profiling): CSR entries of the listed
// vertices, and of those whose sketch is saturated (read by the mask merge).
// Runs before the hop kernels change the sketches.
__global__ void k_hop_census(const int32_t* __restrict__ list, int64_t n_list, const int64_t* __restrict__ rowp,
                             const uint64_t* __restrict__ S, const uint8_t* __restrict__ Scnt, int k, int hop,
                             uint64_t ulim, const uint32_t* __restrict__ stamp, uint32_t sparse_hop, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long sc = 0, mk = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_list; i += stride) {
        const int32_t v = list[i];
        if (sparse_hop && stamp[v] != sparse_hop) continue;  // a hub the hop skips
        const unsigned long long d = (unsigned long long)(rowp[v + 1] - rowp[v]);
        sc += d;
        if (hop > 1 && Scnt[v] == k && S[(int64_t)v * k + k - 1] <= ulim) mk += d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(kFull, sc, o);
        mk += __shfl_xor_sync(kFull, mk, o);
    }
    if (lane_id() == 0) {
        if (sc) atomicAdd(&ctr->scanned, sc);
        if (mk) atomicAdd(&ctr->mask_scanned, mk);
    }
}

// ------------------------------------------------------------------ small-rank table

constexpr int kSelCap = 4096;  // candidates sorted in one block

// Ranks below T -> buf (first kSelCap of them); their number -> *cnt.
__global__ void k_small_ranks(int64_t n, uint64_t seed, uint64_t T, IdMap ids,
                              uint64_t* __restrict__ buf, unsigned long long* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const uint64_t r = v < n ? vertex_rank(seed, rank_id(ids, v)) : kEmpty;
        const long long at = warp_append(v < n && r < T, cnt);
        if (at >= 0 && at < kSelCap) buf[at] = r;
    }
}

// Sort the m <= kSelCap candidates (bitonic, one block) and keep the w smallest.
__global__ void __launch_bounds__(1024) k_sort_small(const uint64_t* __restrict__ buf, int m, int w,
                                                     uint64_t* __restrict__ U) {
    __shared__ uint64_t a[kSelCap];
    for (int i = threadIdx.x; i < kSelCap; i += blockDim.x) a[i] = i < m ? buf[i] : kEmpty;
    __syncthreads();
    for (int size = 2; size <= kSelCap; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < kSelCap; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool asc = (i & size) == 0;
                    const uint64_t x = a[i], y = a[j];
                    if ((x > y) == asc) {
                        a[i] = y;
                        a[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < kUW; i += blockDim.x) U[i] = i < w ? a[i] : kEmpty;
}

// Rank id of the vertex of each rank of U (-1 for padding).
__global__ void k_rank_ids(const uint64_t* __restrict__ U, int w, uint64_t seed, int32_t* __restrict__ URid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kUW) URid[i] = i < w ? (int32_t)rank_vertex(seed, U[i]) : -1;
}

// The frontier of the previous hop as a bitmap: bit v = (Dcnt[v] > 0).
__global__ void k_front_bitmap(const uint8_t* __restrict__ Dcnt, int64_t n, uint32_t* __restrict__ bm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t v = base + lane_id();
        const unsigned w = __ballot_sync(kFull, v < n && Dcnt[v] > 0);
        if (lane_id() == 0) bm[base >> 5] = w;
    }
}

// U = the min(kUW, n) smallest vertex ranks: collect the ranks below a
// threshold expected to pass about 2048 of them (ranks are uniform), widen or
// narrow it until between min(kUW, n) and kSelCap pass, then sort them.
static int select_small_ranks(fl_graph* g) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    const int w = (int)std::min<int64_t>(kUW, n);
    DBuf buf;
    FL_TRY(dalloc(buf, (size_t)kSelCap * 8 + 256));
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(buf.as<char>() + (size_t)kSelCap * 8);
    uint64_t T = n <= kSelCap / 2 ? kEmpty : (kEmpty / (uint64_t)n) * 2048ULL;
    unsigned long long c = 0;
    int rc = FL_OK;
    for (int it = 0;; ++it) {
        if (it > 130) { rc = FL_ECUDA; set_error(rc, "small-rank selection did not converge"); break; }
        cudaError_t e = cudaMemsetAsync(cnt, 0, 8, st);
        if (e != cudaSuccess) { rc = status_of(e, "small ranks", __FILE__, __LINE__); break; }
        FL_LAUNCH(kProfSketchOther, k_small_ranks<<<grid_for(n, 256), 256, 0, st>>>(
                                        n, g->seed, T, idmap_of(g),
                                        buf.as<uint64_t>(), cnt));
        e = cudaMemcpyAsync(&c, cnt, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "small ranks", __FILE__, __LINE__); break; }
        if ((int64_t)c < w) {
            T = T > kEmpty / 2 ? kEmpty : T * 2;
            continue;
        }
        if (c > (unsigned long long)kSelCap) {
            T = T / 4 * 3;
            continue;
        }
        break;
    }
    if (rc == FL_OK) {
        FL_LAUNCH(kProfSketchOther, k_sort_small<<<1, 1024, 0, st>>>(buf.as<uint64_t>(), (int)c, w,
                                                                     g->U.as<uint64_t>()));
        FL_LAUNCH(kProfSketchOther, k_rank_ids<<<(kUW + 255) / 256, 256, 0, st>>>(
                                        g->U.as<uint64_t>(), w, g->seed, g->URid.as<int32_t>()));
        cudaError_t e = cudaMemcpyAsync(&g->ulim, g->U.as<uint64_t>() + (w - 1), 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&g->hlim, g->U.as<uint64_t>() + (std::min(w, 64) - 1), 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = status_of(e, "small ranks", __FILE__, __LINE__);
    }
    dfree_after(st, {&buf});
    return rc;
}

// ------------------------------------------------------------------ driver

template <int G>
static int launch_hop(fl_graph* g, int hop, const int32_t* list, int64_t n_list, int pin, int pout,
                      int64_t slot_base, bool sparse) {
    cudaStream_t st = g->stream;
    const int k = g->k;
    const int per_block = 256 / G;
    const uint32_t sparse_hop = sparse ? (uint32_t)hop : 0u;
    HopIO io;
    io.rowp = g->rowp.as<int64_t>();
    io.cols = g->cols.as<int32_t>();
    io.k = k;
    io.hop = hop;
    io.seed = g->seed;
    io.S = g->S.as<uint64_t>();
    io.Scnt = g->Scnt.as<uint8_t>();
    io.Dp = g->D[pin].as<uint64_t>();
    io.Dcp = g->Dcnt[pin].as<uint8_t>();
    io.Dc = g->D[pout].as<uint64_t>();
    io.Dcc = g->Dcnt[pout].as<uint8_t>();
    io.Fp = g->F[pin].as<uint64_t>();
    io.Fc = g->F[pout].as<uint64_t>();
    io.Hp = g->H[pin].as<uint64_t>();
    io.Hc = g->H[pout].as<uint64_t>();
    io.W = g->W.as<uint64_t>();
    io.bm = g->fbm.as<uint32_t>();
    io.DMp = g->DM[pin].as<uint64_t>();
    io.DMc = g->DM[pout].as<uint64_t>();
    io.n = g->n;
    io.vg = g->vg.as<int32_t>();
    io.ve = g->ve.as<int32_t>();
    io.stg_ent = g->stg_ent.as<int32_t>() + slot_base * k;
    io.stg_grp = g->stg_grp.as<StgGroup>() + slot_base;
    io.U = g->U.as<uint64_t>();
    io.URid = g->URid.as<int32_t>();
    io.ulim = g->ulim;
    io.hlim = g->hlim;
    io.ids = idmap_of(g);
    io.ctr = g->ctr.as<Counters>();
    if (n_list > 0)
        FL_LAUNCH(kProfSketchMerge, k_hop_vertices<G><<<grid_for(n_list, per_block), 256, 0, st>>>(list, n_list, io));
    if (g->n_hubs > 0) {
        FL_LAUNCH(kProfSketchMerge, k_hop_hub_segments<G><<<grid_for(g->n_seg, per_block), 256, 0, st>>>(
                                        g->hub_list.as<int32_t>(), g->hub_seg.as<int64_t>(), g->seg_hub.as<int32_t>(),
                                        g->n_seg, g->part.as<uint64_t>(), g->PM.as<uint64_t>(), g->PH.as<uint64_t>(),
                                        g->seg_flag.as<uint8_t>(), g->stamp.as<uint32_t>(), sparse_hop, io));
        FL_LAUNCH(kProfSketchMerge, k_hop_hubs<G><<<grid_for(g->n_hubs, per_block), 256, 0, st>>>(
                                        g->hub_list.as<int32_t>(), g->n_hubs, g->hub_seg.as<int64_t>(),
                                        g->part.as<uint64_t>(), g->PM.as<uint64_t>(), g->PH.as<uint64_t>(),
                                        g->seg_flag.as<uint8_t>(), g->stamp.as<uint32_t>(), sparse_hop, n_list, io));
    }
    FL_CUDA(cudaGetLastError());
    return FL_OK;
}

int build_sketches(fl_graph* g, int k, uint64_t seed) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    g->built = 0;
    ++g->generation;
    g->k = k;
    g->seed = seed;
    if (g->wts.p) {  // a weighted graph: levels in Dijkstra order (k_wsketch.cu)
        g->hop_scanned.clear();
        g->hop_mask.clear();
        g->hop_changed.clear();
        g->hop_ms.clear();
        for (auto* vec : {&g->hop_E, &g->hop_A, &g->hop_R, &g->hop_SD, &g->hop_new}) vec->clear();
        FL_TRY(build_sketches_weighted(g, k, seed));
        g->built = 1;
        return FL_OK;
    }
    if (!g->lists_ready) {
        FL_TRY(build_work_lists(g));
        g->lists_ready = 1;
    }
    const size_t nk = (size_t)n * k;
    FL_TRY(dalloc(g->S, nk * 8));
    FL_TRY(dalloc(g->Scnt, (size_t)n));
    for (int p = 0; p < 2; ++p) {
        FL_TRY(dalloc(g->D[p], nk * 8));
        FL_TRY(dalloc(g->Dcnt[p], (size_t)n));
        FL_TRY(dalloc(g->frontier[p], (size_t)n * 4));
    }
    FL_TRY(dalloc(g->stamp, (size_t)n * 4));
    FL_TRY(dalloc(g->vg, (size_t)n * 4));
    FL_TRY(dalloc(g->ve, (size_t)n * 4));
    FL_TRY(dalloc(g->part, (size_t)std::max<int64_t>(g->n_seg, 1) * k * 8));
    FL_TRY(dalloc(g->U, (size_t)kUW * 8));
    FL_TRY(dalloc(g->DM[0], (size_t)n * kUWords * 8));
    FL_TRY(dalloc(g->DM[1], (size_t)n * kUWords * 8));
    FL_TRY(dalloc(g->PM, (size_t)std::max<int64_t>(g->n_seg, 1) * kUWords * 8));
    FL_TRY(dalloc(g->PH, (size_t)std::max<int64_t>(g->n_seg, 1) * 8));
    FL_TRY(dalloc(g->seg_flag, (size_t)std::max<int64_t>(g->n_seg, 1)));
    for (int p = 0; p < 2; ++p) {
        FL_TRY(dalloc(g->F[p], (size_t)n * 8));
        FL_TRY(dalloc(g->H[p], (size_t)n * 8));
    }
    FL_TRY(dalloc(g->W, (size_t)n * 8));
    FL_TRY(dalloc(g->fbm, ((size_t)(n + 31) / 32 + 1) * 4));
    FL_TRY(dalloc(g->URid, (size_t)kUW * 4));
    // staging: slots 0..n-1 for hop 0, then one slot per work item of each hop
    const int64_t per_dense = g->n_low + g->n_hubs;
    size_t slot_cap = (size_t)n + (size_t)per_dense * 8 + 1024;
    if (g->stg_grp_cap < slot_cap || g->stg_k != k) {
        slot_cap = std::max(slot_cap, g->stg_grp_cap);
        FL_TRY(dalloc(g->stg_grp, slot_cap * sizeof(StgGroup)));
        FL_TRY(dalloc(g->stg_ent, slot_cap * k * 4));
        g->stg_grp_cap = slot_cap;
        g->stg_k = k;
    }
    DBuf act;  // active list of sparse hops
    FL_TRY(dalloc(act, (size_t)n * 4));

    FL_CUDA(cudaMemsetAsync(g->S.p, 0xff, nk * 8, st));
    FL_CUDA(cudaMemsetAsync(g->W.p, 0, (size_t)n * 8, st));
    FL_CUDA(cudaMemsetAsync(g->stamp.p, 0, (size_t)n * 4, st));
    FL_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st));
    {
        int rc0 = select_small_ranks(g);
        if (rc0 != FL_OK) {
            dfree_after(st, {&act});
            return rc0;
        }
    }
    FL_LAUNCH(kProfSketchOther, k_rank_init<<<grid_for(n, 256), 256, 0, st>>>(
                                    n, k, seed, g->S.as<uint64_t>(), g->Scnt.as<uint8_t>(), g->stg_grp.as<StgGroup>(),
                                    g->vg.as<int32_t>(), g->ve.as<int32_t>(), idmap_of(g), g->ctr.as<Counters>()));
    FL_CUDA(cudaGetLastError());
    FL_TRY(read_counters(g));
    if (g->h_ctr->error) {
        dfree_after(st, {&act});
        FL_FAIL(FL_EINVAL, "a vertex rank equals the reserved empty-slot value; choose another seed");
    }
    g->hop_scanned.clear();
    g->hop_mask.clear();
    g->hop_changed.clear();
    g->hop_ms.clear();
    for (auto* vec : {&g->hop_E, &g->hop_A, &g->hop_R, &g->hop_SD, &g->hop_new}) vec->clear();
    const bool time_hops = g->prof.on != 0;
    const bool census = g->prof.on >= 2;  // per-hop scanned / mask counts (extra kernels)
    if (time_hops && !g->hop_ev[0]) {
        FL_CUDA(cudaEventCreate(&g->hop_ev[0]));
        FL_CUDA(cudaEventCreate(&g->hop_ev[1]));
    }
    std::vector<std::pair<int64_t, int64_t>> regions;  // (slot base, slots) of each hop
    regions.push_back({0, n});
    int64_t used_slots = n;
    int64_t n_front = n;  // hop 0: every vertex gained its own rank
    bool fr_list_ready = false;
    // hop 1: every vertex gained its own rank at hop 0, so each CSR entry is
    // an edge-merge carrying one delta rank
    int64_t total_merges = 0, next_merges = g->nnz, next_delta = g->nnz;
    int hop = 1;
    int rc = FL_OK;
    for (;; ++hop) {
        if (hop > kMaxHops) { rc = FL_ETIMEOUT; set_error(rc, "more than 65535 hops"); break; }
        total_merges += next_merges;
        const int64_t hop_merges = next_merges, hop_delta = next_delta;
        const int pin = (hop - 1) & 1, pout = hop & 1;
        const int32_t* list;
        int64_t n_list;
        // dense hops run every non-isolated vertex; sparse hops expand the frontier
        const bool dense = !fr_list_ready;
        Counters init{};
        FL_CUDA(cudaMemcpyAsync(g->ctr.p, &init, sizeof(Counters), cudaMemcpyHostToDevice, st));
        if (dense) {
            list = g->low_list.as<int32_t>();
            n_list = g->n_low;
        } else {
            FL_LAUNCH(kProfSketchExpand, k_expand<<<grid_for(n_front, 8), 256, 0, st>>>(
                                             g->frontier[pin].as<int32_t>(), n_front, g->rowp.as<int64_t>(),
                                             g->cols.as<int32_t>(), g->stamp.as<uint32_t>(), (uint32_t)hop,
                                             act.as<int32_t>(), g->ctr.as<Counters>()));
            FL_CUDA(cudaGetLastError());
            FL_TRY(read_counters(g));
            list = act.as<int32_t>();
            n_list = (int64_t)g->h_ctr->active;
        }
        const int64_t slots = n_list + g->n_hubs;
        if ((size_t)(used_slots + slots) > g->stg_grp_cap) {
            size_t cap = std::max<size_t>((size_t)(used_slots + slots), g->stg_grp_cap * 3 / 2);
            FL_TRY(dgrow(g->stg_grp, cap * sizeof(StgGroup), (size_t)used_slots * sizeof(StgGroup), st));
            FL_TRY(dgrow(g->stg_ent, cap * k * 4, (size_t)used_slots * k * 4, st));
            g->stg_grp_cap = cap;
        }
        // this hop's outputs read "no new entries" for every vertex that does not change
        FL_CUDA(cudaMemsetAsync(g->Dcnt[pout].p, 0, (size_t)n, st));
        FL_CUDA(cudaMemsetAsync(g->F[pout].p, 0xff, (size_t)n * 8, st));
        FL_CUDA(cudaMemsetAsync(g->H[pout].p, 0, (size_t)n * 8, st));
        if (hop > 1)
            FL_LAUNCH(kProfSketchOther, k_front_bitmap<<<grid_for(n, 256), 256, 0, st>>>(
                                            g->Dcnt[pin].as<uint8_t>(), n, g->fbm.as<uint32_t>()));
        if (census) {
            if (n_list > 0)
                FL_LAUNCH(kProfSketchOther, k_hop_census<<<grid_for(n_list, 256), 256, 0, st>>>(
                                                list, n_list, g->rowp.as<int64_t>(), g->S.as<uint64_t>(),
                                                g->Scnt.as<uint8_t>(), k, hop, g->ulim, nullptr, 0u,
                                                g->ctr.as<Counters>()));
            if (g->n_hubs > 0)
                FL_LAUNCH(kProfSketchOther, k_hop_census<<<grid_for(g->n_hubs, 256), 256, 0, st>>>(
                                                g->hub_list.as<int32_t>(), g->n_hubs, g->rowp.as<int64_t>(),
                                                g->S.as<uint64_t>(), g->Scnt.as<uint8_t>(), k, hop, g->ulim,
                                                g->stamp.as<uint32_t>(), dense ? 0u : (uint32_t)hop,
                                                g->ctr.as<Counters>()));
        }
        if (time_hops) FL_CUDA(cudaEventRecord(g->hop_ev[0], st));
        if (k <= 16 && g->sched.hop_group != 32)
            FL_TRY(launch_hop<16>(g, hop, list, n_list, pin, pout, used_slots, !dense));
        else
            FL_TRY(launch_hop<32>(g, hop, list, n_list, pin, pout, used_slots, !dense));
        if (time_hops) FL_CUDA(cudaEventRecord(g->hop_ev[1], st));
        regions.push_back({used_slots, slots});
        used_slots += slots;
        FL_TRY(read_counters(g));
        {
            float hop_ms = 0.f;
            if (time_hops) FL_CUDA(cudaEventElapsedTime(&hop_ms, g->hop_ev[0], g->hop_ev[1]));
            g->hop_scanned.push_back(census ? (int64_t)g->h_ctr->scanned : 0);
            g->hop_mask.push_back(census ? (int64_t)g->h_ctr->mask_scanned : 0);
            g->hop_changed.push_back((int64_t)g->h_ctr->frontier);
            g->hop_ms.push_back(hop_ms);
            g->hop_E.push_back(hop_merges);
            g->hop_A.push_back((int64_t)g->h_ctr->merging);
            g->hop_R.push_back((int64_t)g->h_ctr->cand_reads);
            g->hop_SD.push_back(hop_delta);
            g->hop_new.push_back((int64_t)g->h_ctr->new_entries);
        }
        n_front = (int64_t)g->h_ctr->frontier;
        next_merges = (int64_t)g->h_ctr->merges;
        next_delta = (int64_t)g->h_ctr->delta_next;
        // algorithmic bytes of this hop's merge: row offsets of each merging
        // vertex (8 B), frontier columns (4 B per edge-merge), neighbour delta
        // ranks read (8 B each), own sketch read + write (16k B per merging
        // vertex); the ADS entries (12 B each) are added after the last hop
        {
            const double A = (double)g->h_ctr->merging, SD = (double)g->h_ctr->cand_reads;
            g->prof.bytes[kProfSketchMerge] += 8.0 * A + 4.0 * (double)hop_merges + 8.0 * SD + 16.0 * k * A;
        }
        if (n_front == 0) break;
        // a small frontier makes the next hop sparse: collect its list
        fr_list_ready = false;
        if (n_front * g->sched.sparse_div < g->n_low + g->n_hubs) {
            FL_CUDA(cudaMemsetAsync(&g->ctr.as<Counters>()->aux0, 0, 8, st));
            if (n_list > 0)
                FL_LAUNCH(kProfSketchExpand, k_collect_frontier<<<grid_for(n_list, 256), 256, 0, st>>>(
                                                 list, n_list, g->Dcnt[pout].as<uint8_t>(),
                                                 g->frontier[pout].as<int32_t>(), &g->ctr.as<Counters>()->aux0));
            if (g->n_hubs > 0)
                FL_LAUNCH(kProfSketchExpand, k_collect_frontier<<<grid_for(g->n_hubs, 256), 256, 0, st>>>(
                                                 g->hub_list.as<int32_t>(), g->n_hubs, g->Dcnt[pout].as<uint8_t>(),
                                                 g->frontier[pout].as<int32_t>(), &g->ctr.as<Counters>()->aux0));
            FL_CUDA(cudaGetLastError());
            FL_TRY(read_counters(g));
            fr_list_ready = true;
        }
    }
    dfree_after(st, {&act});
    if (rc != FL_OK) return rc;
    g->hops = hop - 1;
    g->edge_merges = total_merges;

    // vertex-major ADS
    FL_TRY(dalloc(g->gofs, (size_t)(n + 1) * 8));
    FL_TRY(dalloc(g->eofs, (size_t)(n + 1) * 8));
    FL_TRY(scan_exclusive_i32_to_i64(g->vg.as<int32_t>(), g->gofs.as<int64_t>(), n, st, g->scratch));
    FL_TRY(scan_exclusive_i32_to_i64(g->ve.as<int32_t>(), g->eofs.as<int64_t>(), n, st, g->scratch));
    FL_TRY(scan_total(g->gofs.as<int64_t>(), g->vg.as<int32_t>(), n, st, &g->n_groups));
    FL_TRY(scan_total(g->eofs.as<int64_t>(), g->ve.as<int32_t>(), n, st, &g->n_entries));
    g->prof.bytes[kProfSketchMerge] += 12.0 * (double)(g->n_entries - n);
    FL_TRY(dalloc(g->ginfo, (size_t)std::max<int64_t>(g->n_groups, 1) * 4));
    FL_TRY(dalloc(g->gwt, (size_t)std::max<int64_t>(g->n_groups, 1) * 8));
    FL_TRY(dalloc(g->eid, (size_t)std::max<int64_t>(g->n_entries, 1) * 4));
    FL_CUDA(cudaMemcpyAsync(g->gofs.as<int64_t>() + n, &g->n_groups, 8, cudaMemcpyHostToDevice, st));
    FL_CUDA(cudaMemcpyAsync(g->eofs.as<int64_t>() + n, &g->n_entries, 8, cudaMemcpyHostToDevice, st));
    int log2_kp = 0;
    while ((1 << log2_kp) < k) ++log2_kp;
    for (const auto& r : regions)
        if (r.second > 0) {
            const bool hop0 = r.first == 0;
            const int lk = hop0 ? 0 : log2_kp;
            FL_LAUNCH(kProfSketchOther, k_ads_scatter<<<grid_for(r.second << lk, 256), 256, 0, st>>>(
                                            g->stg_grp.as<StgGroup>(), r.second, r.first, k, lk, hop0,
                                            g->stg_ent.as<int32_t>(), g->gofs.as<int64_t>(), g->eofs.as<int64_t>(),
                                            g->ginfo.as<uint32_t>(), g->gwt.as<double>(), g->eid.as<int32_t>()));
        }
    FL_CUDA(cudaGetLastError());
    FL_CUDA(cudaStreamSynchronize(st));
    FL_TRY(compute_ecc_bound(g));
    g->built = 1;
    return FL_OK;
}

// ------------------------------------------------------------------ eccentricity bound
// The minimum rank of a component (S[v][0] at the fixed point) names a root
// for every vertex of it; a multi-source BFS from the roots gives d(v, root)
// and ecc(root), and ecc(v) <= d(v, root) + ecc(root).

__global__ void k_roots(const uint64_t* __restrict__ S, int k, uint64_t seed, int64_t n,
                        IdMap ids, int32_t* __restrict__ roots, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        int64_t v = base + lane_id();
        bool is_root = false;
        if (v < n) is_root = (int64_t)rank_vertex(seed, S[v * k]) == rank_id(ids, v);
        long long at = warp_append(is_root, &ctr->aux0);
        if (at >= 0) roots[at] = (int32_t)v;
    }
}

__global__ void k_ecc_max(const int32_t* __restrict__ label, const int32_t* __restrict__ dist, int64_t n,
                          int32_t* __restrict__ eccr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (dist[v] > 0 && eccr[label[v]] < dist[v]) atomicMax(&eccr[label[v]], dist[v]);
}

__global__ void k_ecc_ub(const int32_t* __restrict__ label, const int32_t* __restrict__ dist,
                         const int32_t* __restrict__ eccr, int64_t n, int32_t* __restrict__ ub) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        ub[v] = dist[v] + eccr[label[v]];
}

int compute_ecc_bound(fl_graph* g) {
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    DBuf roots, label, dist, eccr, X, stampb, fr[2], frval;
    int rc = FL_OK;
    do {
        if ((rc = dalloc(roots, (size_t)n * 4))) break;
        if ((rc = dalloc(label, (size_t)n * 4))) break;
        if ((rc = dalloc(dist, (size_t)n * 4))) break;
        if ((rc = dalloc(eccr, (size_t)n * 4))) break;
        if ((rc = dalloc(g->ecc_ub, (size_t)n * 4))) break;
        cudaError_t e = cudaMemsetAsync(g->ctr.p, 0, sizeof(Counters), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(eccr.p, 0, (size_t)n * 4, st);
        if (e != cudaSuccess) { rc = status_of(e, "ecc init", __FILE__, __LINE__); break; }
        FL_LAUNCH(kProfSketchOther, k_roots<<<grid_for(n, 256), 256, 0, st>>>(
                                        g->S.as<uint64_t>(), g->k, g->seed, n,
                                        idmap_of(g), roots.as<int32_t>(),
                                        g->ctr.as<Counters>()));
        if ((rc = read_counters(g))) break;
        int64_t n_roots = (int64_t)g->h_ctr->aux0;
        if ((rc = msbfs(g, roots.as<int32_t>(), n_roots, label.as<int32_t>(), dist.as<int32_t>(), X, stampb,
                        fr, frval, kProfSketchOther)))
            break;
        FL_LAUNCH(kProfSketchOther, k_ecc_max<<<grid_for(n, 256), 256, 0, st>>>(label.as<int32_t>(),
                                                                                dist.as<int32_t>(), n,
                                                                                eccr.as<int32_t>()));
        FL_LAUNCH(kProfSketchOther, k_ecc_ub<<<grid_for(n, 256), 256, 0, st>>>(
                                        label.as<int32_t>(), dist.as<int32_t>(), eccr.as<int32_t>(), n,
                                        g->ecc_ub.as<int32_t>()));
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = status_of(e, "ecc bound", __FILE__, __LINE__); break; }
    } while (0);
    dfree_after(st, {&roots, &label, &dist, &eccr, &X, &stampb, &fr[0], &fr[1], &frval});
    return rc;
}

}  // namespace fl
