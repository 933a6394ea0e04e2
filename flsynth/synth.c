/*
 * flsynth: seeded synthetic inputs for the graph facility-location path.
 *
 * This module only makes inputs: graphs (Erdos-Renyi G(n,M) and R-MAT),
 * client/facility masks and opening costs.  It holds none of the method's
 * arithmetic (no ranks, sketches, estimators, radii, MIS or BFS); both the
 * CPU oracle and the CUDA path consume what it writes.
 *
 * Randomness: a counter-based hash (the 64-bit finaliser of MurmurHash3,
 * Appleby 2011) applied to (stream seed, counter).  Every value depends
 * only on its counter, so results do not depend on the thread count or on
 * the machine (x86-64 and aarch64 give the same graphs).
 *
 * Graph output format: symmetric CSR, rows sorted ascending, no self-loops,
 * no duplicate entries; row offsets int64 (n+1), column ids int32.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* Hash of (stream, counter): two finaliser rounds over a keyed counter. */
static inline uint64_t hash2(uint64_t stream, uint64_t ctr) {
    return fmix64(fmix64(stream ^ 0x5bd1e9955bd1e995ULL) + ctr * 0x9fb21c651e98df25ULL + 1);
}

/* Uniform integer in [0, m) by the multiply-high method. */
static inline uint64_t below(uint64_t h, uint64_t m) {
    return (uint64_t)(((__uint128_t)h * (__uint128_t)m) >> 64);
}

/* Uniform double in (0, 1) with 53 random bits. */
static inline double unit_open(uint64_t h) {
    return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* Edge list -> symmetric, deduplicated, sorted CSR.                   */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Sort a row in place: insertion sort for short rows, qsort otherwise. */
static void sort_row(int32_t* a, int64_t len) {
    if (len < 64) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t x = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
            a[j + 1] = x;
        }
        return;
    }
    qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
}

/*
 * Build a symmetric CSR from `m` directed pairs (src[i], dst[i]); both
 * directions are inserted, self-loops dropped, duplicates removed.
 * rowp: n+1 int64 (written); cols: capacity 2*m int32 (written, prefix
 * of length nnz).  Returns nnz, or -1 on allocation failure.
 */
static int64_t build_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         int64_t* rowp, int32_t* cols) {
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* cur = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t* tmp = (int32_t*)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
    if (!deg || !cur || !tmp) { free(deg); free(cur); free(tmp); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s == d) continue;
#pragma omp atomic
        deg[s + 1]++;
#pragma omp atomic
        deg[d + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) deg[v + 1] += deg[v];
    memcpy(cur, deg, ((size_t)n + 1) * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s == d) continue;
        int64_t p = __atomic_fetch_add(&cur[s], 1, __ATOMIC_RELAXED);
        tmp[p] = d;
        p = __atomic_fetch_add(&cur[d], 1, __ATOMIC_RELAXED);
        tmp[p] = s;
    }
    /* sort + dedupe each row in place; cur[v] becomes the deduped length */
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = deg[v], len = deg[v + 1] - deg[v];
        sort_row(tmp + b, len);
        int64_t w = 0;
        for (int64_t i = 0; i < len; ++i)
            if (w == 0 || tmp[b + i] != tmp[b + w - 1]) tmp[b + w++] = tmp[b + i];
        cur[v] = w;
    }
    /* row offsets of the deduplicated rows, then copy the rows out */
    rowp[0] = 0;
    for (int64_t v = 0; v < n; ++v) rowp[v + 1] = rowp[v] + cur[v];
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v)
        memcpy(cols + rowp[v], tmp + deg[v], (size_t)cur[v] * sizeof(int32_t));
    int64_t total = rowp[n];
    free(deg);
    free(cur);
    free(tmp);
    return total;
}

/* ------------------------------------------------------------------ */
/* Erdos-Renyi G(n, M): M distinct unordered pairs, uniform.           */
/* ------------------------------------------------------------------ */

/*
 * G(n, M) with exactly M distinct undirected edges and no self-loops
 * (requires M <= n(n-1)/2).  Candidate pairs are drawn from counter
 * stream `seed` in counter order; repeats are rejected.  Output CSR has
 * nnz = 2M.  Returns nnz or -1.
 */
int64_t syn_er(int64_t n, int64_t M, uint64_t seed, int64_t* rowp, int32_t* cols) {
    if (n < 2 || M < 0 || (double)M > 0.5 * (double)n * (double)(n - 1)) return -1;
    /* open-addressing set of accepted pairs, key = lo * n + hi + 1 */
    uint64_t cap = 16;
    while (cap < (uint64_t)M * 3 + 16) cap <<= 1;
    uint64_t* set = (uint64_t*)calloc(cap, sizeof(uint64_t));
    int32_t* s = (int32_t*)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    int32_t* d = (int32_t*)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    if (!set || !s || !d) { free(set); free(s); free(d); return -1; }
    int64_t got = 0;
    uint64_t ctr = 0;
    while (got < M) {
        uint64_t h1 = hash2(seed, 2 * ctr), h2 = hash2(seed, 2 * ctr + 1);
        ++ctr;
        int64_t a = (int64_t)below(h1, (uint64_t)n), b = (int64_t)below(h2, (uint64_t)n);
        if (a == b) continue;
        int64_t lo = a < b ? a : b, hi = a < b ? b : a;
        uint64_t key = (uint64_t)lo * (uint64_t)n + (uint64_t)hi + 1;
        uint64_t slot = fmix64(key) & (cap - 1);
        int dup = 0;
        while (set[slot]) {
            if (set[slot] == key) { dup = 1; break; }
            slot = (slot + 1) & (cap - 1);
        }
        if (dup) continue;
        set[slot] = key;
        s[got] = (int32_t)lo;
        d[got] = (int32_t)hi;
        ++got;
    }
    int64_t nnz = build_csr(n, M, s, d, rowp, cols);
    free(set); free(s); free(d);
    return nnz;
}

/* ------------------------------------------------------------------ */
/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004).                          */
/* ------------------------------------------------------------------ */

/* Keyed bijection on [0, 2^scale): odd multiplies and xor-shifts, all mod 2^scale. */
static inline uint64_t relabel(uint64_t x, int scale, uint64_t key) {
    uint64_t mask = (scale >= 64) ? ~0ULL : ((1ULL << scale) - 1);
    int sh = scale / 2 > 0 ? scale / 2 : 1;
    for (int r = 0; r < 3; ++r) {
        uint64_t k = fmix64(key + (uint64_t)r);
        x = (x * (k | 1ULL)) & mask;
        x = (x + (k >> 17)) & mask;
        x ^= x >> sh;
    }
    return x & mask;
}

/*
 * R-MAT graph with 2^scale vertices from `ndraws` directed draws.  Each
 * draw descends `scale` levels; at each level one 16-bit uniform u picks
 * quadrant (0,0) if u < ta, (0,1) if u < tb, (1,0) if u < tc, else (1,1),
 * where ta, tb, tc are the cumulative probabilities a, a+b, a+b+c scaled
 * to 2^16.  Vertex ids are then relabelled by a seeded bijection,
 * self-loops dropped, both directions inserted and duplicates removed.
 * cols must hold 2*ndraws entries.  Returns nnz or -1.
 */
int64_t syn_rmat(int scale, int64_t ndraws, uint32_t ta, uint32_t tb, uint32_t tc,
                 uint64_t seed, int64_t* rowp, int32_t* cols) {
    if (scale < 1 || scale > 30 || ndraws < 0) return -1;
    int64_t n = (int64_t)1 << scale;
    int32_t* s = (int32_t*)malloc((size_t)(ndraws > 0 ? ndraws : 1) * sizeof(int32_t));
    int32_t* d = (int32_t*)malloc((size_t)(ndraws > 0 ? ndraws : 1) * sizeof(int32_t));
    if (!s || !d) { free(s); free(d); return -1; }
    uint64_t relabel_key = fmix64(seed ^ 0x2545f4914f6cdd1dULL);
    int groups = (scale + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ndraws; ++i) {
        uint64_t u = 0, v = 0;
        int lvl = 0;
        for (int g = 0; g < groups; ++g) {
            uint64_t h = hash2(seed, (uint64_t)i * (uint64_t)groups + (uint64_t)g);
            for (int q = 0; q < 4 && lvl < scale; ++q, ++lvl) {
                uint32_t r = (uint32_t)(h >> (16 * q)) & 0xffffu;
                uint64_t bu, bv;
                if (r < ta) { bu = 0; bv = 0; }
                else if (r < tb) { bu = 0; bv = 1; }
                else if (r < tc) { bu = 1; bv = 0; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
        }
        s[i] = (int32_t)relabel(u, scale, relabel_key);
        d[i] = (int32_t)relabel(v, scale, relabel_key);
    }
    int64_t nnz = build_csr(n, ndraws, s, d, rowp, cols);
    free(s); free(d);
    return nnz;
}

/* ------------------------------------------------------------------ */
/* Per-vertex masks and costs.                                         */
/* ------------------------------------------------------------------ */

/* mask[v] = 1 with probability p_num / 2^32, from counter stream `seed`. */
void syn_bernoulli(int64_t n, uint64_t seed, uint32_t p_num, uint8_t* mask) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v)
        mask[v] = (uint8_t)((hash2(seed, (uint64_t)v) >> 32) < (uint64_t)p_num);
}

/*
 * Log-uniform costs in [lo, hi]: cost[v] = exp(ln lo + u (ln hi - ln lo)),
 * u uniform in (0,1).  Vertices with facility_mask[v] == 0 (when a mask is
 * given) get +infinity.
 */
void syn_loguniform(int64_t n, uint64_t seed, double lo, double hi,
                    const uint8_t* facility_mask, double* cost) {
    double a = log(lo), b = log(hi);
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        if (facility_mask && !facility_mask[v]) { cost[v] = INFINITY; continue; }
        cost[v] = exp(a + unit_open(hash2(seed, (uint64_t)v)) * (b - a));
    }
}

/* Uniform doubles in (lo, hi) from counter stream `seed`, one per counter. */
void syn_uniform(int64_t m, uint64_t seed, double lo, double hi, double* out) {
    for (int64_t i = 0; i < m; ++i) out[i] = lo + unit_open(hash2(seed, (uint64_t)i)) * (hi - lo);
}

/* Raw 64-bit hashes hash2(seed, i), i < m (for sampling and shuffles). */
void syn_hash(int64_t m, uint64_t seed, uint64_t* out) {
    for (int64_t i = 0; i < m; ++i) out[i] = hash2(seed, (uint64_t)i);
}
