/*
 * fl_oracle.c -- TEST INFRASTRUCTURE.  A plain, slow CPU oracle for the
 * data-parallel hot path of scalable graph facility location (Garimella,
 * De Francisci Morales, Gionis, Sozio: "Scalable Facility Location for
 * Massive Graphs on Pregel-like Systems").  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load or run this code; the
 * product path never does.  It shares no code with the CUDA library.
 *
 * Every routine follows the paper's definitions step by step, in the
 * paper's order, with no blocking or fusion.  Readings taken where the
 * paper is silent (all cited at the routine):
 *   - ranks r(u) are SplitMix64 outputs (Steele, Lea, Flood 2014);
 *   - within one hop, vertices at equal distance are presented to the
 *     bottom-k sketch in ascending rank (so hop-synchronous propagation and
 *     Algorithm 1 build the same ADS);
 *   - HIP weights condition on all ranks except the entry's own, with all
 *     vertices at one distance treated together (weight 2^64 / t, t the
 *     k-th smallest rank of the ball, counting the k-1 smallest only);
 *   - radius r_f is the root of the epsilon->0, all-unfrozen form of Eq. 1;
 *   - facility selection is the lexicographically-first MIS of the
 *     conflict graph under the key (r_f, pi_f).
 *
 * Floating point: every FP64 operation is a single IEEE-754 operation in
 * the order written (build with -ffp-contract=off, no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 3
#define ORC_ESTATE 2

/* ---------------------------------------------------------------------- */
/* Ranks: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).                    */
/* The paper only says r(u) is a hash of u (Section 3.3, Algorithm 1).     */
/* ---------------------------------------------------------------------- */

#define SM_GAMMA 0x9e3779b97f4a7c15ULL

/* One SplitMix64 step: advance the state by the golden-gamma increment
   and return the mixed state. */
uint64_t orc_splitmix64_next(uint64_t* state) {
    *state += SM_GAMMA;
    uint64_t z = *state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* r(v): the (v+1)-th output of SplitMix64 started from state `seed`. */
uint64_t orc_rank(uint64_t seed, int64_t v) {
    uint64_t state = seed + (uint64_t)v * SM_GAMMA;
    return orc_splitmix64_next(&state);
}

/* pi(f): MIS priority (Section 4.3 draws a random ID per facility).  The
   (f+1)-th output of a second SplitMix64 stream whose starting state is
   the first SplitMix64 output for `seed`.  Injective in f, like r. */
uint64_t orc_priority(uint64_t seed, int64_t f) {
    uint64_t s = seed;
    uint64_t stream = orc_splitmix64_next(&s);
    uint64_t state = stream + (uint64_t)f * SM_GAMMA;
    return orc_splitmix64_next(&state);
}

/* ---------------------------------------------------------------------- */
/* Graph handle                                                            */
/* ---------------------------------------------------------------------- */

typedef struct {
    int32_t hop;      /* distance d(v, u) of the entries */
    int32_t cnt;      /* entries in this group */
    int32_t counted;  /* leading entries that carry the weight */
    double wt;        /* HIP adjusted weight of each counted entry */
    int64_t first;    /* index of the first entry in the entry arrays */
} orc_group;

typedef struct {
    int64_t n;
    int64_t* rowp;
    int32_t* cols;
    /* sketch state */
    int k;
    uint64_t seed;
    int built;
    uint64_t* S;      /* n*k final bottom-k sketch (ascending ranks) */
    int32_t* Scnt;    /* n */
    int64_t hops;     /* last hop at which some sketch changed */
    int64_t edge_merges;
    /* ADS, vertex-major: groups of v are gofs[v]..gofs[v+1], entries of v
       are eofs[v]..eofs[v+1]; within v ordered by hop, then by rank */
    int64_t* gofs;
    int64_t* eofs;
    orc_group* grp;
    int32_t* ent_id;
    uint64_t* ent_rank;
    int64_t ngroups, nentries;
    int32_t* wts;     /* edge lengths per CSR entry (weighted graphs), or NULL */
} orc_graph;

static void orc_clear_ads(orc_graph* g) {
    free(g->S); free(g->Scnt); free(g->gofs); free(g->eofs);
    free(g->grp); free(g->ent_id); free(g->ent_rank);
    g->S = NULL; g->Scnt = NULL; g->gofs = NULL; g->eofs = NULL;
    g->grp = NULL; g->ent_id = NULL; g->ent_rank = NULL;
    g->built = 0;
}

orc_graph* orc_graph_create(int64_t n, const int64_t* rowp, const int32_t* cols) {
    if (n < 0 || !rowp) return NULL;
    orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
    if (!g) return NULL;
    g->n = n;
    int64_t nnz = rowp[n];
    g->rowp = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    g->cols = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!g->rowp || !g->cols) { free(g->rowp); free(g->cols); free(g); return NULL; }
    memcpy(g->rowp, rowp, ((size_t)n + 1) * sizeof(int64_t));
    if (nnz > 0) memcpy(g->cols, cols, (size_t)nnz * sizeof(int32_t));
    return g;
}

void orc_graph_destroy(orc_graph* g) {
    if (!g) return;
    orc_clear_ads(g);
    free(g->rowp); free(g->cols); free(g->wts);
    free(g);
}

/* ---------------------------------------------------------------------- */
/* Bottom-k insertion (Algorithm 1 / Algorithm 2 inner step).              */
/* ---------------------------------------------------------------------- */

/* Insert rank x into the ascending list L (length *len, capacity k) if the
   list has fewer than k entries or x is below its k-th entry, and x is not
   already present.  This is the reading of the test "r(u) < max_r(BKMH)"
   of Algorithms 1 and 2 for a list that is not yet full. */
static void bottomk_insert(uint64_t* L, int32_t* len, int k, uint64_t x) {
    int32_t m = *len;
    if (m == k && x >= L[k - 1]) return;
    int32_t pos = 0;
    while (pos < m && L[pos] < x) ++pos;
    if (pos < m && L[pos] == x) return;          /* already present */
    int32_t last = (m < k) ? m : k - 1;          /* drop the old k-th if full */
    for (int32_t i = last; i > pos; --i) L[i] = L[i - 1];
    L[pos] = x;
    if (m < k) *len = m + 1;
}

typedef struct { uint64_t rank; int32_t id; } rank_id;

static int rank_id_cmp(const void* a, const void* b) {
    uint64_t x = ((const rank_id*)a)->rank, y = ((const rank_id*)b)->rank;
    return (x > y) - (x < y);
}

/* ---------------------------------------------------------------------- */
/* HIP weight of the entries that join a sketch at one distance.           */
/* ---------------------------------------------------------------------- */

/* Given S_h(v) = bottom-k of the ball of radius h (length len), an entry w
   at distance h that is at position i of S_h(v) is counted by the HIP
   estimator iff len < k or i < k-1; its inclusion probability conditioned
   on all other ranks is then 1 (len < k) or t / 2^64 with t = S_h(v)[k-1]
   (the (k-1)-th smallest rank of the ball without w).  The adjusted weight
   is the inverse (Cohen 2014, HIP; cited in Section 3.3). */
static double hip_weight(const uint64_t* Sh, int32_t len, int k) {
    if (len < k) return 1.0;
    return 18446744073709551616.0 / (double)Sh[k - 1];
}

/* ---------------------------------------------------------------------- */
/* Phase (i): sketches and ADS by hop-synchronous propagation.             */
/* Section 3.3, Algorithm 2 (unweighted: no CleanUp is needed because one  */
/* superstep delivers exactly the vertices of one distance).               */
/* ---------------------------------------------------------------------- */

typedef struct { int32_t v; int32_t hop; int64_t at; int32_t cnt; } hop_rec;

/* Threads the OpenMP loops of this oracle use. */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Hop-synchronous build; stops after `max_hops` hops (a bounded sample of
   the build for timing) or at the fixed point, whichever comes first. */
int orc_build_sketches_hops(orc_graph* g, int k, uint64_t seed, int64_t max_hops) {
    if (!g || k < 2 || k > 64) return ORC_EINVAL;
    orc_clear_ads(g);
    const int64_t n = g->n;
    g->k = k;
    g->seed = seed;
    g->hops = 0;
    g->edge_merges = 0;

    uint64_t* S = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * k * sizeof(uint64_t));
    int32_t* Scnt = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    uint64_t* Dprev = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * k * sizeof(uint64_t));
    int32_t* Dprev_cnt = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    uint64_t* Dcur = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * k * sizeof(uint64_t));
    int32_t* Dcur_cnt = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    double* Dcur_wt = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int32_t* Dcur_counted = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    /* hop-major record of every (v, hop) group, appended in (hop, v) order */
    int64_t rec_cap = n + 16, rec_n = 0;
    hop_rec* rec = (hop_rec*)malloc((size_t)rec_cap * sizeof(hop_rec));
    double* rec_wt = (double*)malloc((size_t)rec_cap * sizeof(double));
    int32_t* rec_counted = (int32_t*)malloc((size_t)rec_cap * sizeof(int32_t));
    int64_t ent_cap = n + 16, ent_n = 0;
    uint64_t* ent = (uint64_t*)malloc((size_t)ent_cap * sizeof(uint64_t));
    if (!S || !Scnt || !Dprev || !Dprev_cnt || !Dcur || !Dcur_cnt || !Dcur_wt ||
        !Dcur_counted || !rec || !rec_wt || !rec_counted || !ent) {
        free(S); free(Scnt); free(Dprev); free(Dprev_cnt); free(Dcur); free(Dcur_cnt);
        free(Dcur_wt); free(Dcur_counted); free(rec); free(rec_wt); free(rec_counted); free(ent);
        return ORC_ENOMEM;
    }

    /* hop 0: every vertex knows itself (distance 0) */
    for (int64_t v = 0; v < n; ++v) {
        uint64_t r = orc_rank(seed, v);
        S[v * k] = r;
        Scnt[v] = 1;
        Dprev[v * k] = r;
        Dprev_cnt[v] = 1;
        rec[rec_n].v = (int32_t)v; rec[rec_n].hop = 0; rec[rec_n].at = ent_n; rec[rec_n].cnt = 1;
        rec_wt[rec_n] = hip_weight(&S[v * k], 1, k);
        rec_counted[rec_n] = 1;
        ++rec_n;
        ent[ent_n++] = r;
    }

    int64_t merges = 0;
    for (int64_t h = 1;; ++h) {
        int64_t changed = 0;
        /* every vertex merges the entries its neighbours added at hop h-1 */
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : changed, merges)
        for (int64_t v = 0; v < n; ++v) {
            uint64_t old[64];
            int32_t oldn = Scnt[v];
            memcpy(old, &S[v * k], (size_t)oldn * sizeof(uint64_t));
            uint64_t* L = &S[v * k];
            int32_t len = oldn;
            for (int64_t e = g->rowp[v]; e < g->rowp[v + 1]; ++e) {
                int32_t u = g->cols[e];
                if (Dprev_cnt[u] == 0) continue;
                ++merges;
                for (int32_t i = 0; i < Dprev_cnt[u]; ++i)
                    bottomk_insert(L, &len, k, Dprev[(int64_t)u * k + i]);
            }
            Scnt[v] = len;
            /* new entries: in the new sketch but not in the old one */
            int32_t dn = 0, counted = 0, oi = 0;
            for (int32_t i = 0; i < len; ++i) {
                while (oi < oldn && old[oi] < L[i]) ++oi;
                if (oi < oldn && old[oi] == L[i]) continue;
                Dcur[v * k + dn] = L[i];
                if (len < k || i < k - 1) ++counted;
                ++dn;
            }
            Dcur_cnt[v] = dn;
            Dcur_counted[v] = counted;
            Dcur_wt[v] = hip_weight(L, len, k);
            if (dn) ++changed;
        }
        if (!changed) { g->hops = h - 1; break; }
        if (h >= max_hops) { g->hops = h; }
        /* append this hop's groups in vertex order */
        for (int64_t v = 0; v < n; ++v) {
            if (!Dcur_cnt[v]) continue;
            if (rec_n == rec_cap) {
                rec_cap *= 2;
                rec = (hop_rec*)realloc(rec, (size_t)rec_cap * sizeof(hop_rec));
                rec_wt = (double*)realloc(rec_wt, (size_t)rec_cap * sizeof(double));
                rec_counted = (int32_t*)realloc(rec_counted, (size_t)rec_cap * sizeof(int32_t));
                if (!rec || !rec_wt || !rec_counted) return ORC_ENOMEM;
            }
            while (ent_n + Dcur_cnt[v] > ent_cap) {
                ent_cap *= 2;
                ent = (uint64_t*)realloc(ent, (size_t)ent_cap * sizeof(uint64_t));
                if (!ent) return ORC_ENOMEM;
            }
            rec[rec_n].v = (int32_t)v; rec[rec_n].hop = (int32_t)h;
            rec[rec_n].at = ent_n; rec[rec_n].cnt = Dcur_cnt[v];
            rec_wt[rec_n] = Dcur_wt[v];
            rec_counted[rec_n] = Dcur_counted[v];
            ++rec_n;
            memcpy(&ent[ent_n], &Dcur[v * k], (size_t)Dcur_cnt[v] * sizeof(uint64_t));
            ent_n += Dcur_cnt[v];
        }
        uint64_t* t = Dprev; Dprev = Dcur; Dcur = t;
        int32_t* tc = Dprev_cnt; Dprev_cnt = Dcur_cnt; Dcur_cnt = tc;
        if (h >= max_hops) break;
    }
    g->edge_merges = merges;

    /* vertex-major ADS: stable counting sort of the records by vertex */
    g->gofs = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->eofs = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->grp = (orc_group*)malloc((size_t)(rec_n > 0 ? rec_n : 1) * sizeof(orc_group));
    g->ent_id = (int32_t*)malloc((size_t)(ent_n > 0 ? ent_n : 1) * sizeof(int32_t));
    g->ent_rank = (uint64_t*)malloc((size_t)(ent_n > 0 ? ent_n : 1) * sizeof(uint64_t));
    int64_t* gcur = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    int64_t* ecur = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!g->gofs || !g->eofs || !g->grp || !g->ent_id || !g->ent_rank || !gcur || !ecur)
        return ORC_ENOMEM;
    for (int64_t i = 0; i < rec_n; ++i) {
        g->gofs[rec[i].v + 1] += 1;
        g->eofs[rec[i].v + 1] += rec[i].cnt;
    }
    for (int64_t v = 0; v < n; ++v) { g->gofs[v + 1] += g->gofs[v]; g->eofs[v + 1] += g->eofs[v]; }
    memcpy(gcur, g->gofs, ((size_t)n + 1) * sizeof(int64_t));
    memcpy(ecur, g->eofs, ((size_t)n + 1) * sizeof(int64_t));
    /* rank -> vertex id: ranks of distinct vertices are distinct (SplitMix64
       outputs of distinct counters), so a table sorted by rank maps each
       entry's rank back to its vertex */
    rank_id* tab = (rank_id*)malloc((size_t)(n > 0 ? n : 1) * sizeof(rank_id));
    if (!tab) return ORC_ENOMEM;
    for (int64_t v = 0; v < n; ++v) { tab[v].rank = orc_rank(seed, v); tab[v].id = (int32_t)v; }
    qsort(tab, (size_t)n, sizeof(rank_id), rank_id_cmp);
    for (int64_t i = 0; i < rec_n; ++i) {
        int64_t v = rec[i].v;
        int64_t gi = gcur[v]++;
        int64_t ei = ecur[v];
        ecur[v] += rec[i].cnt;
        g->grp[gi].hop = rec[i].hop;
        g->grp[gi].cnt = rec[i].cnt;
        g->grp[gi].counted = rec_counted[i];
        g->grp[gi].wt = rec_wt[i];
        g->grp[gi].first = ei;
        memcpy(&g->ent_rank[ei], &ent[rec[i].at], (size_t)rec[i].cnt * sizeof(uint64_t));
    }
#pragma omp parallel for schedule(static)
    for (int64_t e2 = 0; e2 < ent_n; ++e2) {
        uint64_t x = g->ent_rank[e2];
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (tab[mid].rank < x) lo = mid + 1; else hi = mid;
        }
        g->ent_id[e2] = tab[lo].id;
    }
    free(tab);
    free(gcur); free(ecur);
    g->ngroups = rec_n;
    g->nentries = ent_n;
    g->S = S;
    g->Scnt = Scnt;
    g->built = 1;
    free(Dprev); free(Dprev_cnt); free(Dcur); free(Dcur_cnt); free(Dcur_wt); free(Dcur_counted);
    free(rec); free(rec_wt); free(rec_counted); free(ent);
    return ORC_OK;
}

int orc_build_sketches(orc_graph* g, int k, uint64_t seed) {
    return orc_build_sketches_hops(g, k, seed, INT64_MAX);
}

int64_t orc_hops(const orc_graph* g) { return g && g->built ? g->hops : -1; }
int64_t orc_edge_merges(const orc_graph* g) { return g && g->built ? g->edge_merges : -1; }
int64_t orc_ads_groups(const orc_graph* g) { return g && g->built ? g->ngroups : -1; }
int64_t orc_ads_entries(const orc_graph* g) { return g && g->built ? g->nentries : -1; }

/* Final sketches: S[v*k + i] for i < cnt[v], UINT64_MAX padding after. */
int orc_export_sketch(const orc_graph* g, uint64_t* S, int32_t* cnt) {
    if (!g || !g->built) return ORC_ESTATE;
    for (int64_t v = 0; v < g->n; ++v) {
        cnt[v] = g->Scnt[v];
        for (int i = 0; i < g->k; ++i)
            S[v * g->k + i] = i < g->Scnt[v] ? g->S[v * g->k + i] : UINT64_MAX;
    }
    return ORC_OK;
}

/* ADS export, vertex-major.  gofs/eofs: n+1 offsets; per group: hop, cnt,
   counted, weight; per entry: vertex id and rank. */
int orc_export_ads(const orc_graph* g, int64_t* gofs, int64_t* eofs, int32_t* ghop,
                   int32_t* gcnt, int32_t* gcounted, double* gwt,
                   int32_t* eid, uint64_t* erank) {
    if (!g || !g->built) return ORC_ESTATE;
    memcpy(gofs, g->gofs, ((size_t)g->n + 1) * sizeof(int64_t));
    memcpy(eofs, g->eofs, ((size_t)g->n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < g->ngroups; ++i) {
        ghop[i] = g->grp[i].hop;
        gcnt[i] = g->grp[i].cnt;
        gcounted[i] = g->grp[i].counted;
        gwt[i] = g->grp[i].wt;
    }
    if (eid) memcpy(eid, g->ent_id, (size_t)g->nentries * sizeof(int32_t));
    if (erank) memcpy(erank, g->ent_rank, (size_t)g->nentries * sizeof(uint64_t));
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 for one vertex (sampled checks on large graphs).            */
/* ---------------------------------------------------------------------- */

/* Sequential ADS of vertex v (Algorithm 1): list vertices by increasing
   distance from v (equal distances in ascending rank), insert u when the
   bottom-k list has fewer than k entries or r(u) is below its k-th entry.
   Output arrays are sized by the caller: hop/id/rank capacity `cap`
   entries, group weight/counted capacity `cap`.  Returns the number of
   entries (or -1 when cap is too small / no memory).  Groups: per distance
   with at least one entry, gw[] = weight, gc[] = counted, gh[] = distance,
   gn[] = entry count; *ngroups set. */
int64_t orc_vertex_ads(const orc_graph* g, int k, uint64_t seed, int64_t v, int64_t cap,
                       int32_t* ids, uint64_t* ranks, int32_t* gh, int32_t* gn,
                       int32_t* gc, double* gw, int64_t* ngroups) {
    const int64_t n = g->n;
    int32_t* dist = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* q = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    rank_id* lvl = (rank_id*)malloc((size_t)n * sizeof(rank_id));
    if (!dist || !q || !lvl) { free(dist); free(q); free(lvl); return -1; }
    for (int64_t i = 0; i < n; ++i) dist[i] = -1;
    uint64_t B[64];
    int32_t blen = 0;
    int64_t ne = 0, ng = 0;
    int64_t qh = 0, qt = 0;
    dist[v] = 0;
    q[qt++] = (int32_t)v;
    int32_t d = 0;
    while (qh < qt) {
        /* one distance level: q[qh..level_end) */
        int64_t level_end = qt;
        int64_t m = 0;
        for (int64_t i = qh; i < level_end; ++i) { lvl[m].id = q[i]; lvl[m].rank = orc_rank(seed, q[i]); ++m; }
        qsort(lvl, (size_t)m, sizeof(rank_id), rank_id_cmp);   /* ascending rank */
        int64_t first = ne;
        for (int64_t i = 0; i < m; ++i) {
            uint64_t r = lvl[i].rank;
            if (blen < k || r < B[k - 1]) {
                if (ne >= cap) { free(dist); free(q); free(lvl); return -1; }
                ids[ne] = lvl[i].id;
                ranks[ne] = r;
                ++ne;
                bottomk_insert(B, &blen, k, r);
            }
        }
        if (ne > first) {
            /* weight from the finished level (the ball of radius d) */
            int32_t counted = 0;
            for (int64_t e = first; e < ne; ++e) {
                int32_t pos = 0;
                while (B[pos] != ranks[e]) ++pos;
                if (blen < k || pos < k - 1) ++counted;
            }
            gh[ng] = d; gn[ng] = (int32_t)(ne - first); gc[ng] = counted;
            gw[ng] = hip_weight(B, blen, k);
            ++ng;
        }
        /* expand the next level */
        for (int64_t i = qh; i < level_end; ++i) {
            int32_t x = q[i];
            for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                int32_t u = g->cols[e];
                if (dist[u] < 0) { dist[u] = d + 1; q[qt++] = u; }
            }
        }
        qh = level_end;
        ++d;
    }
    *ngroups = ng;
    free(dist); free(q); free(lvl);
    return ne;
}

/* ---------------------------------------------------------------------- */
/* Phase (ii): per-facility radius.                                        */
/* Eq. 1 (Section 4.1) with all clients unfrozen and alpha(c) = alpha, as in */
/* Section 4.2 before Eq. 2, taken at epsilon -> 0: the served-client      */
/* slack sum_c max{0, r - d(c,f)} equals the opening cost c(f).  Client    */
/* counts per distance come from predicated HIP queries on the ADS         */
/* (Section 4.5, "How to estimate the number of unfrozen clients?").       */
/* ---------------------------------------------------------------------- */

/* Radius from per-distance client estimates (hop ascending): ng groups at
   distances hop[0] < hop[1] < ..., W[i] = HIP-estimated clients at
   distance hop[i]; distances without a group have W = 0.  N_j = sum_{h<=j}
   W_h; G_0 = 0, G_{j+1} = G_j + N_j (so g(r) = G_j + N_j (r - j) on
   [j, j+1]).  L = hop of the last group.  r = j + (c - G_j)/N_j for the
   smallest j < L with G_{j+1} >= c; otherwise r = L + (c - G_L)/N_L if
   N_L > 0, else +inf. */
static double radius_walk(const int32_t* hop, const double* W, int64_t ng, double cost) {
    if (!(cost < INFINITY) || ng == 0) return INFINITY;
    int64_t L = hop[ng - 1];
    double N = 0.0, G = 0.0;
    int64_t gi = 0;
    for (int64_t j = 0; j <= L; ++j) {
        double w = 0.0;
        if (gi < ng && hop[gi] == j) { w = W[gi]; ++gi; }
        N = N + w;
        if (j < L) {
            double Gn = G + N;
            if (Gn >= cost) return (double)j + (cost - G) / N;
            G = Gn;
        }
    }
    if (N > 0.0) return (double)L + (cost - G) / N;
    return INFINITY;
}

/* Radius of one facility from its ADS groups: W_h = (number of counted
   entries of the hop-h group that are clients) x the group's weight. */
static double radius_one(const orc_graph* g, int64_t f, double cost, const uint8_t* client) {
    if (!(cost < INFINITY)) return INFINITY;
    int64_t g0 = g->gofs[f], g1 = g->gofs[f + 1];
    if (g1 == g0) return INFINITY;
    int64_t ng = g1 - g0;
    int32_t* hop = (int32_t*)malloc((size_t)ng * sizeof(int32_t));
    double* W = (double*)malloc((size_t)ng * sizeof(double));
    if (!hop || !W) { free(hop); free(W); return NAN; }
    for (int64_t i = 0; i < ng; ++i) {
        const orc_group* gr = &g->grp[g0 + i];
        int64_t clients = 0;
        for (int32_t e = 0; e < gr->counted; ++e)
            if (client[g->ent_id[gr->first + e]]) ++clients;
        hop[i] = gr->hop;
        W[i] = (double)clients * gr->wt;
    }
    double r = radius_walk(hop, W, ng, cost);
    free(hop); free(W);
    return r;
}

/* The same radius from one vertex's ADS given as arrays (the output of
   orc_vertex_ads or an exported ADS row): ng groups with distance ghop,
   entry count gcnt, counted prefix gcounted and weight gw; ids holds the
   entries of the groups one after another. */
double orc_radius_of_ads(int64_t ng, const int32_t* ghop, const int32_t* gcnt, const int32_t* gcounted,
                         const double* gw, const int32_t* ids, const uint8_t* client, double cost) {
    if (!(cost < INFINITY) || ng == 0) return INFINITY;
    double* W = (double*)malloc((size_t)ng * sizeof(double));
    if (!W) return NAN;
    int64_t first = 0;
    for (int64_t i = 0; i < ng; ++i) {
        int64_t clients = 0;
        for (int32_t e = 0; e < gcounted[i]; ++e)
            if (client[ids[first + e]]) ++clients;
        W[i] = (double)clients * gw[i];
        first += gcnt[i];
    }
    double r = radius_walk(ghop, W, ng, cost);
    free(W);
    return r;
}

/* Nearest open facility of v by definition (Section 3.1, d(c, S)): BFS
   from v level by level; at the first level holding an open facility the
   smallest such id and the level are returned; -1 / -1 when v's component
   has none. */
int orc_nearest_open(const orc_graph* g, const uint8_t* open, int64_t v, int32_t* assign, int32_t* dist) {
    if (!g || v < 0 || v >= g->n) return ORC_EINVAL;
    const int64_t n = g->n;
    int32_t* d = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* q = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!d || !q) { free(d); free(q); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) d[i] = -1;
    *assign = -1;
    *dist = -1;
    int64_t qh = 0, qt = 0;
    d[v] = 0;
    q[qt++] = (int32_t)v;
    int32_t level = 0;
    while (qh < qt) {
        int64_t level_end = qt;
        int32_t best = -1;
        for (int64_t i = qh; i < level_end; ++i)
            if (open[q[i]] && (best < 0 || q[i] < best)) best = q[i];
        if (best >= 0) { *assign = best; *dist = level; break; }
        for (int64_t i = qh; i < level_end; ++i) {
            int32_t x = q[i];
            for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                int32_t u = g->cols[e];
                if (d[u] < 0) { d[u] = level + 1; q[qt++] = u; }
            }
        }
        qh = level_end;
        ++level;
    }
    free(d); free(q);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Exact neighbourhood sizes: the ground truth of the ADS accuracy study   */
/* (Section 5.1, "Accuracy vs. k", Fig. 1), by breadth-first search.       */
/* ---------------------------------------------------------------------- */

/* BFS from v; cnt[h] (h = 0..D) receives the number of vertices w with
   d(v, w) = h exactly and pred[w] != 0 (pred NULL: every vertex); returns
   the eccentricity of v (the last distance holding a vertex), capped at D
   when the search stops there; D < 0 searches the whole component (cnt
   then needs n entries).  dist and q are n-long scratch arrays (dist all
   -1 on entry and on return). */
static int64_t bfs_levels(const orc_graph* g, int64_t v, int64_t D, const uint8_t* pred,
                          int64_t* cnt, int32_t* dist, int32_t* q) {
    int64_t qh = 0, qt = 0, ecc = 0;
    cnt[0] = 0;
    dist[v] = 0;
    q[qt++] = (int32_t)v;
    while (qh < qt) {
        int32_t x = q[qh++];
        int32_t dx = dist[x];
        while (ecc < dx) cnt[++ecc] = 0;  /* first vertex of a new distance */
        if (!pred || pred[x]) ++cnt[dx];
        if (dx == D) continue;
        for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
            int32_t u = g->cols[e];
            if (dist[u] < 0) { dist[u] = dx + 1; q[qt++] = u; }
        }
    }
    for (int64_t j = 0; j < qt; ++j) dist[q[j]] = -1;
    for (int64_t h = ecc + 1; h <= D; ++h) cnt[h] = 0;
    return ecc;
}

/* out[s*(D+1) + h] = |{w : d(src[s], w) <= h and pred[w] != 0}| for
   h = 0..D (cumulative sums of the per-distance counts). */
int orc_ball_sizes(const orc_graph* g, int64_t n_src, const int32_t* src, int64_t D, const uint8_t* pred,
                   int64_t* out) {
    if (!g || D < 0) return ORC_EINVAL;
    for (int64_t s = 0; s < n_src; ++s)
        if (src[s] < 0 || src[s] >= g->n) return ORC_EINVAL;
    int rc = ORC_OK;
#pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(int32_t));
        int32_t* q = (int32_t*)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(int32_t));
        int64_t* cnt = (int64_t*)malloc((size_t)(D + 1) * sizeof(int64_t));
        if (!dist || !q || !cnt) {
#pragma omp atomic write
            rc = ORC_ENOMEM;
        } else {
            for (int64_t v = 0; v < g->n; ++v) dist[v] = -1;
#pragma omp for schedule(dynamic, 1)
            for (int64_t s = 0; s < n_src; ++s) {
                bfs_levels(g, src[s], D, pred, cnt, dist, q);
                int64_t acc = 0;
                for (int64_t h = 0; h <= D; ++h) {
                    acc += cnt[h];
                    out[s * (D + 1) + h] = acc;
                }
            }
        }
        free(dist); free(q); free(cnt);
    }
    return rc;
}

/* Radius of facility f with exact client counts (the exact-radius mode of
   the accuracy study): W_h = number of clients at distance exactly h of f,
   for h = 0..L with L the eccentricity of f, fed to the same walk as the
   sketch radius (radius_walk: Eq. 1 at epsilon -> 0).  With every vertex
   in f's sketch (k >= component size) the HIP weights are all 1 and the
   two radii are the same numbers. */
static double exact_radius_one(const orc_graph* g, int64_t f, double cost, const uint8_t* client,
                               int32_t* dist, int32_t* q, int64_t* cnt, int32_t* hop, double* W) {
    if (!(cost < INFINITY)) return INFINITY;
    int64_t L = bfs_levels(g, f, -1, client, cnt, dist, q);
    for (int64_t h = 0; h <= L; ++h) { hop[h] = (int32_t)h; W[h] = (double)cnt[h]; }
    return radius_walk(hop, W, L + 1, cost);
}

static int exact_radii_range(const orc_graph* g, int64_t m, const int32_t* fac, const double* cost,
                             const uint8_t* client, double* r) {
    const int64_t n = g->n;
    int rc = ORC_OK;
#pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t* q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int64_t* cnt = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
        int32_t* hop = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
        double* W = (double*)malloc((size_t)(n + 1) * sizeof(double));
        if (!dist || !q || !cnt || !hop || !W) {
#pragma omp atomic write
            rc = ORC_ENOMEM;
        } else {
            for (int64_t v = 0; v < n; ++v) dist[v] = -1;
#pragma omp for schedule(dynamic, 1)
            for (int64_t i = 0; i < m; ++i) {
                int64_t f = fac ? fac[i] : i;
                r[i] = exact_radius_one(g, f, cost[f], client, dist, q, cnt, hop, W);
            }
        }
        free(dist); free(q); free(cnt); free(hop); free(W);
    }
    return rc;
}

/* r[f] for every vertex (+inf for non-facilities). */
int orc_exact_radii(const orc_graph* g, const double* cost, const uint8_t* client, double* r) {
    if (!g) return ORC_EINVAL;
    return exact_radii_range(g, g->n, NULL, cost, client, r);
}

/* r[i] = the exact radius of facility fac[i] (a sample of the facilities). */
int orc_exact_radii_of(const orc_graph* g, int64_t m, const int32_t* fac, const double* cost,
                       const uint8_t* client, double* r) {
    if (!g) return ORC_EINVAL;
    for (int64_t i = 0; i < m; ++i)
        if (fac[i] < 0 || fac[i] >= g->n) return ORC_EINVAL;
    return exact_radii_range(g, m, fac, cost, client, r);
}

/* ---------------------------------------------------------------------- */
/* Quality references (Section 5.2, Table 2: the method's cost against a   */
/* sequential local-search algorithm): the optimum by enumeration on tiny  */
/* instances and a local search.  Cost of an open set S (Section 3.1):     */
/* sum_{f in S} c(f) + sum_{c in C} d(c, S); clients that no facility can  */
/* reach are left out, and a set that leaves a reachable client unserved   */
/* is infeasible.                                                          */
/* ---------------------------------------------------------------------- */

/* Hop distances from every facility to every vertex: D[i * n + v] for the
   i-th facility fac[i] (-1 = unreachable).  Caller frees. */
static int32_t* facility_distances(const orc_graph* g, int64_t nf, const int32_t* fac) {
    const int64_t n = g->n;
    int32_t* D = (int32_t*)malloc((size_t)(nf > 0 ? nf : 1) * (size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!D) return NULL;
    int fail = 0;
#pragma omp parallel
    {
        int32_t* q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        if (!q) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t i = 0; i < nf; ++i) {
                int32_t* d = D + i * n;
                for (int64_t v = 0; v < n; ++v) d[v] = -1;
                int64_t qh = 0, qt = 0;
                d[fac[i]] = 0;
                q[qt++] = fac[i];
                while (qh < qt) {
                    int32_t x = q[qh++];
                    for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                        int32_t u = g->cols[e];
                        if (d[u] < 0) { d[u] = d[x] + 1; q[qt++] = u; }
                    }
                }
            }
        }
        free(q);
    }
    if (fail) { free(D); return NULL; }
    return D;
}

/* Cost of the open set given by flags sel[i] over the facilities; returns
   +inf when a client that some facility reaches is left unserved. */
static double set_cost(const int32_t* D, int64_t n, int64_t nf, const int32_t* fac, const double* cost,
                       const uint8_t* client, const uint8_t* sel) {
    double open_cost = 0.0;
    for (int64_t i = 0; i < nf; ++i)
        if (sel[i]) open_cost = open_cost + cost[fac[i]];
    int64_t ds = 0;
    for (int64_t c = 0; c < n; ++c) {
        if (!client[c]) continue;
        int32_t best = -1, reach = 0;
        for (int64_t i = 0; i < nf; ++i) {
            int32_t d = D[i * n + c];
            if (d < 0) continue;
            reach = 1;
            if (sel[i] && (best < 0 || d < best)) best = d;
        }
        if (!reach) continue;
        if (best < 0) return INFINITY;
        ds += best;
    }
    return open_cost + (double)ds;
}

/* Facilities: vertices with finite cost, ascending. */
static int64_t facility_list(int64_t n, const double* cost, int32_t* fac) {
    int64_t nf = 0;
    for (int64_t v = 0; v < n; ++v)
        if (cost[v] < INFINITY) fac[nf++] = (int32_t)v;
    return nf;
}

/* The optimum by enumerating every non-empty set of at most 24 facilities;
   open[] receives an optimal set (the first found in the enumeration
   order of the subsets' bit patterns); *obj its cost. */
int orc_fl_optimum(const orc_graph* g, const double* cost, const uint8_t* client, uint8_t* open, double* obj) {
    if (!g) return ORC_EINVAL;
    const int64_t n = g->n;
    int32_t* fac = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!fac) return ORC_ENOMEM;
    const int64_t nf = facility_list(n, cost, fac);
    if (nf > 24) { free(fac); return ORC_EINVAL; }
    int32_t* D = facility_distances(g, nf, fac);
    uint8_t* sel = (uint8_t*)calloc((size_t)(nf > 0 ? nf : 1), 1);
    if (!D || !sel) { free(fac); free(D); free(sel); return ORC_ENOMEM; }
    double best = INFINITY;
    uint64_t best_mask = 0;
    for (uint64_t mask = 1; nf > 0 && mask < (1ULL << nf); ++mask) {
        for (int64_t i = 0; i < nf; ++i) sel[i] = (uint8_t)((mask >> i) & 1ULL);
        double c = set_cost(D, n, nf, fac, cost, client, sel);
        if (c < best) { best = c; best_mask = mask; }
    }
    for (int64_t v = 0; v < n; ++v) open[v] = 0;
    for (int64_t i = 0; i < nf; ++i)
        if ((best_mask >> i) & 1ULL) open[fac[i]] = 1;
    *obj = nf > 0 ? best : 0.0;
    free(fac); free(D); free(sel);
    return ORC_OK;
}

/* Nearest and second-nearest open facility distance of every client
   (-1 = none; reachable[c] = some facility reaches c). */
static void nearest_two(const int32_t* D, int64_t n, int64_t nf, const uint8_t* sel, const uint8_t* client,
                        int32_t* d1, int32_t* a1, int32_t* d2) {
    for (int64_t c = 0; c < n; ++c) {
        d1[c] = d2[c] = a1[c] = -1;
        if (!client[c]) continue;
        for (int64_t i = 0; i < nf; ++i) {
            int32_t d = D[i * n + c];
            if (!sel[i] || d < 0) continue;
            if (d1[c] < 0 || d < d1[c]) { d2[c] = d1[c]; d1[c] = d; a1[c] = (int32_t)i; }
            else if (d2[c] < 0 || d < d2[c]) d2[c] = d;
        }
    }
}

/* Local search with add, drop and swap moves (Arya, Garg, Khandekar,
   Meyerson, Munagala, Pandit, SIAM J. Comput. 2004: a local optimum costs at
   most 3 x the optimum) from the open set in open[] (an empty start opens
   the facility of least cost first).  Each pass takes the first improving
   move (adds, then drops, then swaps, in ascending facility order) whose
   cost change, from the clients' nearest and second-nearest open
   facilities, is below -1e-9 x the current cost; the cost is then
   recomputed from scratch.  Stops at a local optimum or after max_moves
   moves; open[], *obj and *moves receive the result. */
int orc_fl_local_search(const orc_graph* g, const double* cost, const uint8_t* client, int64_t max_moves,
                        uint8_t* open, double* obj, int64_t* moves) {
    if (!g) return ORC_EINVAL;
    const int64_t n = g->n;
    int32_t* fac = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!fac) return ORC_ENOMEM;
    const int64_t nf = facility_list(n, cost, fac);
    int32_t* D = facility_distances(g, nf, fac);
    uint8_t* sel = (uint8_t*)calloc((size_t)(nf > 0 ? nf : 1), 1);
    uint8_t* reach = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t* d1 = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* a1 = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* d2 = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!D || !sel || !reach || !d1 || !a1 || !d2) {
        free(fac); free(D); free(sel); free(reach); free(d1); free(a1); free(d2);
        return ORC_ENOMEM;
    }
    for (int64_t c = 0; c < n; ++c)
        for (int64_t i = 0; i < nf && client[c] && !reach[c]; ++i)
            if (D[i * n + c] >= 0) reach[c] = 1;
    int any = 0;
    for (int64_t i = 0; i < nf; ++i) { sel[i] = open[fac[i]] ? 1 : 0; any |= sel[i]; }
    if (!any && nf > 0) {
        int64_t b = 0;
        for (int64_t i = 1; i < nf; ++i)
            if (cost[fac[i]] < cost[fac[b]]) b = i;
        sel[b] = 1;
    }
    double cur = set_cost(D, n, nf, fac, cost, client, sel);
    int64_t m = 0;
    while (m < max_moves && nf > 0) {
        nearest_two(D, n, nf, sel, client, d1, a1, d2);
        const double tol = -1e-9 * (cur < INFINITY ? cur : 1.0);
        int64_t mi = -1, mj = -1;  /* move: close mi (or none), open mj (or none) */
        /* adds: every client moves to the new facility when it is nearer.
           While some reachable client is unserved (cur = +inf), the first
           facility that reaches an unserved client is added. */
        for (int64_t j = 0; j < nf && mi < 0 && mj < 0; ++j) {
            if (sel[j]) continue;
            double delta = cost[fac[j]];
            int64_t newly = 0;
            for (int64_t c = 0; c < n; ++c) {
                if (!client[c] || !reach[c]) continue;
                int32_t d = D[j * n + c];
                if (d1[c] < 0) { if (d >= 0) ++newly; continue; }
                if (d >= 0 && d < d1[c]) delta += (double)(d - d1[c]);
            }
            if (cur == INFINITY ? newly > 0 : delta < tol) mj = j;
        }
        if (cur == INFINITY && mj < 0) break;  /* cannot happen: every reachable client has a facility */
        /* drops: clients of the dropped facility move to their second nearest */
        for (int64_t i = 0; i < nf && mi < 0 && mj < 0; ++i) {
            if (!sel[i]) continue;
            double delta = -cost[fac[i]];
            for (int64_t c = 0; c < n && delta < INFINITY; ++c) {
                if (!client[c] || a1[c] != i) continue;
                if (d2[c] < 0) delta = INFINITY; else delta += (double)(d2[c] - d1[c]);
            }
            if (delta < tol) mi = i;
        }
        /* swaps: close i, open j */
        for (int64_t i = 0; i < nf && mi < 0 && mj < 0; ++i) {
            if (!sel[i]) continue;
            for (int64_t j = 0; j < nf && mi < 0 && mj < 0; ++j) {
                if (sel[j]) continue;
                double delta = cost[fac[j]] - cost[fac[i]];
                for (int64_t c = 0; c < n && delta < INFINITY; ++c) {
                    if (!client[c] || d1[c] < 0) continue;
                    int32_t keep = a1[c] == i ? d2[c] : d1[c];
                    int32_t d = D[j * n + c];
                    int32_t nb = keep < 0 ? d : (d >= 0 && d < keep ? d : keep);
                    if (nb < 0) delta = INFINITY; else delta += (double)(nb - d1[c]);
                }
                if (delta < tol) { mi = i; mj = j; }
            }
        }
        if (mi < 0 && mj < 0) break;
        if (mi >= 0) sel[mi] = 0;
        if (mj >= 0) sel[mj] = 1;
        cur = set_cost(D, n, nf, fac, cost, client, sel);
        ++m;
    }
    for (int64_t v = 0; v < n; ++v) open[v] = 0;
    for (int64_t i = 0; i < nf; ++i)
        if (sel[i]) open[fac[i]] = 1;
    *obj = nf > 0 ? cur : 0.0;
    *moves = m;
    free(fac); free(D); free(sel); free(reach); free(d1); free(a1); free(d2);
    return ORC_OK;
}

/* Cost of an open set by the same rule (+inf if a reachable client is left
   unserved). */
double orc_fl_cost(const orc_graph* g, const double* cost, const uint8_t* client, const uint8_t* open) {
    if (!g) return NAN;
    const int64_t n = g->n;
    int32_t* fac = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!fac) return NAN;
    const int64_t nf = facility_list(n, cost, fac);
    int32_t* D = facility_distances(g, nf, fac);
    uint8_t* sel = (uint8_t*)calloc((size_t)(nf > 0 ? nf : 1), 1);
    if (!D || !sel) { free(fac); free(D); free(sel); return NAN; }
    for (int64_t i = 0; i < nf; ++i) sel[i] = open[fac[i]] ? 1 : 0;
    double c = nf > 0 ? set_cost(D, n, nf, fac, cost, client, sel) : 0.0;
    free(fac); free(D); free(sel);
    return c;
}

int orc_compute_radii(const orc_graph* g, const double* cost, const uint8_t* client, double* r) {
    if (!g || !g->built) return ORC_ESTATE;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t f = 0; f < g->n; ++f) r[f] = radius_one(g, f, cost[f], client);
    return ORC_OK;
}

/* HIP estimate of the number of clients within distance h of v (the
   predicated neighbourhood query of Section 3.3): sum of counted client
   weights over groups with hop <= h.  Summed group by group in hop order:
   each group adds (#counted clients) * weight. */
double orc_hip_estimate(const orc_graph* g, int64_t v, int64_t h, const uint8_t* client) {
    if (!g || !g->built) return NAN;
    double N = 0.0;
    for (int64_t gi = g->gofs[v]; gi < g->gofs[v + 1]; ++gi) {
        const orc_group* gr = &g->grp[gi];
        if (gr->hop > h) break;
        int64_t clients = 0;
        for (int32_t i = 0; i < gr->counted; ++i)
            if (!client || client[g->ent_id[gr->first + i]]) ++clients;
        N = N + (double)clients * gr->wt;
    }
    return N;
}

/* ---------------------------------------------------------------------- */
/* Phase (iii): facility selection = lexicographically-first MIS of H-bar. */
/* Section 4.3 (Algorithm 3 lines building H-bar; Algorithm 6; the greedy  */
/* MIS of Blelloch, Fineman, Shun returns the lexicographically-first MIS  */
/* for its priority order).  Candidate facilities: r_f finite.  Ball(f) =  */
/* clients c with d(c,f) <= floor(r_f).  f ~ g iff their balls share a     */
/* client.  Key(f) = (r_f, pi_f).                                          */
/* ---------------------------------------------------------------------- */

typedef struct { double r; uint64_t pi; int32_t f; } cand_t;

static int cand_cmp(const void* a, const void* b) {
    const cand_t* x = (const cand_t*)a;
    const cand_t* y = (const cand_t*)b;
    if (x->r < y->r) return -1;
    if (x->r > y->r) return 1;
    if (x->pi < y->pi) return -1;
    if (x->pi > y->pi) return 1;
    return 0;
}

/* Sequential greedy in key order: f joins S iff no client of Ball(f) is
   already claimed; then it claims all of Ball(f).  open[f] = 1 for S. */
int orc_open_facilities(const orc_graph* g, const double* r, const uint8_t* client,
                        uint64_t seed, uint8_t* open, int64_t* n_open) {
    if (!g) return ORC_EINVAL;
    const int64_t n = g->n;
    int64_t m = 0;
    for (int64_t f = 0; f < n; ++f) if (r[f] < INFINITY) ++m;
    cand_t* c = (cand_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(cand_t));
    uint8_t* claimed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t* dist = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* ball = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!c || !claimed || !dist || !q || !ball) {
        free(c); free(claimed); free(dist); free(q); free(ball);
        return ORC_ENOMEM;
    }
    m = 0;
    for (int64_t f = 0; f < n; ++f)
        if (r[f] < INFINITY) { c[m].r = r[f]; c[m].pi = orc_priority(seed, f); c[m].f = (int32_t)f; ++m; }
    qsort(c, (size_t)m, sizeof(cand_t), cand_cmp);
    for (int64_t v = 0; v < n; ++v) { dist[v] = -1; open[v] = 0; }
    int64_t opened = 0;
    for (int64_t i = 0; i < m; ++i) {
        int32_t f = c[i].f;
        double fl = floor(c[i].r);
        int64_t B = fl > 2147483647.0 ? 2147483647 : (int64_t)fl;
        /* BFS from f to depth B; a claimed client stops it as soon as it is
           reached (Ball(f) then meets a ball already in S) */
        int64_t qh = 0, qt = 0, nb = 0;
        int conflict = client[f] && claimed[f];
        dist[f] = 0;
        q[qt++] = f;
        if (client[f] && !conflict) ball[nb++] = f;
        while (qh < qt && !conflict) {
            int32_t x = q[qh++];
            if (dist[x] == B) continue;
            for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                int32_t u = g->cols[e];
                if (dist[u] >= 0) continue;
                if (client[u] && claimed[u]) { conflict = 1; break; }
                dist[u] = dist[x] + 1;
                q[qt++] = u;
                if (client[u]) ball[nb++] = u;
            }
        }
        for (int64_t j = 0; j < qt; ++j) dist[q[j]] = -1;
        if (conflict) continue;
        open[f] = 1;
        ++opened;
        for (int64_t j = 0; j < nb; ++j) claimed[ball[j]] = 1;
    }
    *n_open = opened;
    free(c); free(claimed); free(dist); free(q); free(ball);
    return ORC_OK;
}

/* Check that open[] is the lexicographically-first MIS of H-bar under the
   keys (r_f, pi_f), without running the sequential greedy.  A set S of
   candidates is that MIS iff (i) S is independent and (ii) every candidate
   outside S conflicts with a member of S of smaller key (induction over the
   key order: the smallest candidate must be in S, and every later one is in S
   exactly when no earlier member conflicts with it).  With S independent,
   every client of a member's ball has exactly one owner, so (ii) reads: the
   ball of f holds a client whose owner has a smaller key.  Both steps are
   independent per facility (parallel).  Returns 1 when open[] is that MIS,
   0 when not (*bad = a facility that witnesses it), < 0 on error. */
static int key_less(const double* r, uint64_t seed, int32_t a, int32_t b) {
    if (r[a] < r[b]) return 1;
    if (r[a] > r[b]) return 0;
    return orc_priority(seed, a) < orc_priority(seed, b);
}

static int64_t ball_depth(double rf) {
    double fl = floor(rf);
    return fl > 2147483647.0 ? 2147483647 : (int64_t)fl;
}

int orc_check_open_facilities(const orc_graph* g, const double* r, const uint8_t* client, uint64_t seed,
                              const uint8_t* open, int64_t* bad) {
    if (!g) return -ORC_EINVAL;
    const int64_t n = g->n;
    *bad = -1;
    for (int64_t f = 0; f < n; ++f)
        if (open[f] && !(r[f] < INFINITY)) { *bad = f; return 0; }
    int32_t* owner = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!owner) return -ORC_ENOMEM;
    for (int64_t v = 0; v < n; ++v) owner[v] = -1;
    int64_t witness = -1;
    int fail = 0;
    /* (i) members claim their balls; a client claimed twice breaks independence */
#pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t* q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        if (!dist || !q) {
#pragma omp atomic write
            fail = 1;
        } else {
            for (int64_t v = 0; v < n; ++v) dist[v] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t f = 0; f < n; ++f) {
                if (!open[f]) continue;
                const int64_t B = ball_depth(r[f]);
                int64_t qh = 0, qt = 0;
                dist[f] = 0;
                q[qt++] = (int32_t)f;
                while (qh < qt) {
                    int32_t x = q[qh++];
                    if (client[x]) {
                        int32_t prev = __sync_val_compare_and_swap(&owner[x], -1, (int32_t)f);
                        if (prev != -1 && prev != (int32_t)f) {
#pragma omp critical
                            { if (witness < 0) witness = f; }
                        }
                    }
                    if (dist[x] == B) continue;
                    for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                        int32_t u = g->cols[e];
                        if (dist[u] < 0) { dist[u] = dist[x] + 1; q[qt++] = u; }
                    }
                }
                for (int64_t j = 0; j < qt; ++j) dist[q[j]] = -1;
            }
        }
        free(dist); free(q);
    }
    if (fail) { free(owner); return -ORC_ENOMEM; }
    if (witness >= 0) { free(owner); *bad = witness; return 0; }
    /* (ii) every other candidate meets a client owned by an earlier member */
#pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t* q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        if (!dist || !q) {
#pragma omp atomic write
            fail = 1;
        } else {
            for (int64_t v = 0; v < n; ++v) dist[v] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t f = 0; f < n; ++f) {
                if (open[f] || !(r[f] < INFINITY)) continue;
                const int64_t B = ball_depth(r[f]);
                int64_t qh = 0, qt = 0;
                /* a client is tested when the search first reaches it */
                int dominated = client[f] && owner[f] >= 0 && key_less(r, seed, owner[f], (int32_t)f);
                dist[f] = 0;
                q[qt++] = (int32_t)f;
                while (qh < qt && !dominated) {
                    int32_t x = q[qh++];
                    if (dist[x] == B) continue;
                    for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                        int32_t u = g->cols[e];
                        if (dist[u] >= 0) continue;
                        dist[u] = dist[x] + 1;
                        q[qt++] = u;
                        if (client[u] && owner[u] >= 0 && key_less(r, seed, owner[u], (int32_t)f)) {
                            dominated = 1;
                            break;
                        }
                    }
                }
                for (int64_t j = 0; j < qt; ++j) dist[q[j]] = -1;
                if (!dominated) {
#pragma omp critical
                    { if (witness < 0) witness = f; }
                }
            }
        }
        free(dist); free(q);
    }
    free(owner);
    if (fail) return -ORC_ENOMEM;
    if (witness >= 0) { *bad = witness; return 0; }
    return 1;
}

/* ---------------------------------------------------------------------- */
/* Assignment: every vertex to its nearest open facility (ties: smallest  */
/* facility id); Section 3.1 objective d(c,S) = min_{f in S} d(c,f), and  */
/* Algorithm 3's fallback of connecting a client to its nearest facility. */
/* Level-synchronous multi-source BFS; unreachable vertices get -1.       */
/* ---------------------------------------------------------------------- */

int orc_assign(const orc_graph* g, const uint8_t* open, int32_t* assign, int32_t* dist) {
    if (!g) return ORC_EINVAL;
    const int64_t n = g->n;
    int32_t* cur = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* nxt = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!cur || !nxt) { free(cur); free(nxt); return ORC_ENOMEM; }
    int64_t nc = 0;
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = -1;
        assign[v] = -1;
        if (open[v]) { dist[v] = 0; assign[v] = (int32_t)v; cur[nc++] = (int32_t)v; }
    }
    int32_t L = 0;
    while (nc > 0) {
        int64_t nn = 0;
        for (int64_t i = 0; i < nc; ++i) {
            int32_t x = cur[i];
            for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                int32_t u = g->cols[e];
                if (dist[u] < 0) {
                    dist[u] = L + 1;
                    assign[u] = assign[x];
                    nxt[nn++] = u;
                } else if (dist[u] == L + 1 && assign[x] < assign[u]) {
                    assign[u] = assign[x];
                }
            }
        }
        int32_t* t = cur; cur = nxt; nxt = t;
        nc = nn;
        ++L;
    }
    free(cur); free(nxt);
    return ORC_OK;
}

/* Objective (Section 3.1): sum_{f in S} c(f) + sum_{c in C} d(c, S).
   Opening costs are added in ascending facility id; distances of served
   clients are summed exactly in int64 and added once; clients with no
   open facility in their component are counted in *n_unserved and left
   out of the sum. */
int orc_objective(int64_t n, const uint8_t* open, const double* cost, const uint8_t* client,
                  const int32_t* dist, double* obj, int64_t* dist_sum, int64_t* n_unserved) {
    double open_cost = 0.0;
    int64_t ds = 0, un = 0;
    for (int64_t v = 0; v < n; ++v)
        if (open[v]) open_cost = open_cost + cost[v];
    for (int64_t v = 0; v < n; ++v) {
        if (!client[v]) continue;
        if (dist[v] < 0) ++un; else ds += dist[v];
    }
    *obj = open_cost + (double)ds;
    *dist_sum = ds;
    *n_unserved = un;
    return ORC_OK;
}

/* ====================================================================== */
/* The opening phase with epsilon > 0 (Section 4.1, Algorithm 3;          */
/* Section 4.2, Algorithms 4 and 5 with Eq. 2/3; Section 4.3, Algorithm 6).*/
/*                                                                        */
/* Readings (where the paper is silent or at odds with itself):           */
/*  - the grid R: alpha_0 = (gamma * (1 + eps)) / (m * m), m = |F||C| as   */
/*    doubles, alpha_j = alpha_{j-1} * (1 + eps); iteration j = 1, 2, ...  */
/*    runs at alpha_j (Algorithm 4 grows the radius before anything else); */
/*  - gamma = max over clients c with a reachable facility of             */
/*    min_f (c(f) + d(c,f)), one FP64 addition per pair;                  */
/*  - a client at hop distance delta lies in the shell of the smallest    */
/*    grid value >= delta: the shells (d/(1+eps), d] of Eq. 2/3, the first */
/*    read as [0, alpha_0] so that a client at distance 0 is counted;     */
/*  - q(f): Eq. 2 in the first iteration and Eq. 3 in every later one add */
/*    up, per client, to [d_c <= alpha(c)] ((1+eps) alpha(c) - d_c), with */
/*    d_c the client's shell value and alpha(c) the current radius, or    */
/*    the radius at which c was frozen (the increments telescope).  The   */
/*    oracle evaluates that sum over f's ADS (HIP-weighted client entries, */
/*    in ADS order); mode 1 runs the literal incremental Eq. 2/3 instead  */
/*    (a pin of the closed form);                                         */
/*  - in an iteration, every unopened facility with q(f) >= c(f) opens    */
/*    (alpha(f) = alpha_j); then every unfrozen client with an open       */
/*    facility within (1 + eps) alpha_j freezes (alpha(c) = alpha_j): the */
/*    freezing rule of Algorithm 3, which is also condition (2) of H's    */
/*    edges;                                                              */
/*  - U holds only clients with a facility in their component (the others */
/*    can never freeze); the loop runs while some facility is unopened    */
/*    and U is not empty (Algorithms 3 and 4);                            */
/*  - clients still unfrozen when every facility is open take            */
/*    alpha(c) = min_f d(c,f) (Algorithm 4's final step, "argmin" read as */
/*    min); that is no grid value, so they have no edge in H;             */
/*  - H has an edge (c, f) iff f is open, alpha(c) = alpha(f) and         */
/*    d(c,f) <= (1 + eps) alpha(c) (Section 4.2); H-bar joins facilities  */
/*    sharing a client; S is the lexicographically-first MIS of H-bar     */
/*    under pi (Algorithm 6 run until no facility is active).            */
/* ====================================================================== */

#define EPS_MAX_GRID (1 << 22)

/* gamma (see above); -1 when no client reaches a facility. */
double orc_eps_gamma(const orc_graph* g, const double* cost, const uint8_t* client) {
    if (!g) return NAN;
    const int64_t n = g->n;
    double gamma = -1.0;
#pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t* q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        double local = -1.0;
        if (dist && q) {
            for (int64_t v = 0; v < n; ++v) dist[v] = -1;
#pragma omp for schedule(dynamic, 16)
            for (int64_t c = 0; c < n; ++c) {
                if (!client[c]) continue;
                double best = INFINITY;
                int64_t qh = 0, qt = 0;
                dist[c] = 0;
                q[qt++] = (int32_t)c;
                while (qh < qt) {
                    int32_t x = q[qh++];
                    if (cost[x] < INFINITY) {
                        double t = cost[x] + (double)dist[x];
                        if (t < best) best = t;
                    }
                    for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                        int32_t u = g->cols[e];
                        if (dist[u] < 0) { dist[u] = dist[x] + 1; q[qt++] = u; }
                    }
                }
                for (int64_t j = 0; j < qt; ++j) dist[q[j]] = -1;
                if (best < INFINITY && best > local) local = best;
            }
        }
#pragma omp critical
        { if (local > gamma) gamma = local; }
        free(dist); free(q);
    }
    return gamma;
}

/* The grid: grid[0] = alpha_0, grid[j] = grid[j-1] * (1 + eps), up to the
   first value >= bound.  Returns J (the last index) or -1. */
static int64_t eps_grid(double alpha0, double eps, double bound, double** out) {
    const double onepe = 1.0 + eps;
    int64_t cap = 1024, J = 0;
    double* grid = (double*)malloc((size_t)cap * sizeof(double));
    if (!grid) return -1;
    grid[0] = alpha0;
    while (grid[J] < bound) {
        if (J + 1 >= EPS_MAX_GRID) { free(grid); return -1; }
        if (J + 1 == cap) {
            cap *= 2;
            double* t = (double*)realloc(grid, (size_t)cap * sizeof(double));
            if (!t) { free(grid); return -1; }
            grid = t;
        }
        grid[J + 1] = grid[J] * onepe;
        ++J;
    }
    *out = grid;
    return J;
}

/* Index of the smallest grid value >= delta (J + 1 when none). */
static int64_t shell_index(const double* grid, int64_t J, int64_t delta) {
    int64_t lo = 0, hi = J + 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (grid[mid] >= (double)delta) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Multi-source BFS from the open facilities: dist[v] = hop distance to the
   nearest one, -1 when none is reachable. */
static void dist_to_open(const orc_graph* g, const int32_t* fac_iter, int32_t* dist, int32_t* q) {
    const int64_t n = g->n;
    int64_t qh = 0, qt = 0;
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = -1;
        if (fac_iter[v] >= 0) { dist[v] = 0; q[qt++] = (int32_t)v; }
    }
    while (qh < qt) {
        int32_t x = q[qh++];
        for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
            int32_t u = g->cols[e];
            if (dist[u] < 0) { dist[u] = dist[x] + 1; q[qt++] = u; }
        }
    }
}

/* Component label of every vertex (smallest id of the component). */
static void components(const orc_graph* g, int32_t* comp, int32_t* q) {
    const int64_t n = g->n;
    for (int64_t v = 0; v < n; ++v) comp[v] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (comp[s] >= 0) continue;
        int64_t qh = 0, qt = 0;
        comp[s] = (int32_t)s;
        q[qt++] = (int32_t)s;
        while (qh < qt) {
            int32_t x = q[qh++];
            for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                int32_t u = g->cols[e];
                if (comp[u] < 0) { comp[u] = (int32_t)s; q[qt++] = u; }
            }
        }
    }
}

/* q(f) at iteration j by the closed form (see above), summed over f's ADS
   groups in hop order and their counted client entries in rank order. */
static double eps_q(const orc_graph* g, int64_t f, int64_t j, const double* grid, double onepe,
                    const int64_t* shell_of_hop, int64_t nhop, const uint8_t* client, const int32_t* cli_iter) {
    double q = 0.0;
    for (int64_t gi = g->gofs[f]; gi < g->gofs[f + 1]; ++gi) {
        const orc_group* gr = &g->grp[gi];
        const int64_t sj = gr->hop < nhop ? shell_of_hop[gr->hop] : INT64_MAX;
        for (int32_t e = 0; e < gr->counted; ++e) {
            const int32_t w = g->ent_id[gr->first + e];
            if (!client[w]) continue;
            const int64_t jw = cli_iter[w] >= 0 ? cli_iter[w] : j;
            if (sj > jw) continue;                      /* d_c > alpha(c): not yet counted */
            const double a = grid[jw];
            q = q + gr->wt * (onepe * a - grid[sj]);
        }
    }
    return q;
}

/* The literal increment of iteration j (Eq. 2 when j == 1, Eq. 3 after):
   t = sum over shells d <= alpha_j of n-hat(f, d) times the bracket, with
   n-hat(f, d) the HIP-estimated clients unfrozen at the start of the
   iteration whose hop distance lies in shell d. */
static double eps_increment(const orc_graph* g, int64_t f, int64_t j, const double* grid, double onepe,
                            const int64_t* shell_of_hop, int64_t nhop, const uint8_t* client,
                            const int32_t* cli_iter) {
    double t = 0.0;
    const double alpha = grid[j];
    int64_t gi = g->gofs[f];
    const int64_t g1 = g->gofs[f + 1];
    while (gi < g1) {
        const int64_t sj = g->grp[gi].hop < nhop ? shell_of_hop[g->grp[gi].hop] : INT64_MAX;
        if (sj > j) break;
        /* n-hat of shell sj: every group whose hop falls in it */
        double nhat = 0.0;
        while (gi < g1 && (g->grp[gi].hop < nhop ? shell_of_hop[g->grp[gi].hop] : INT64_MAX) == sj) {
            const orc_group* gr = &g->grp[gi];
            int64_t cnt = 0;
            for (int32_t e = 0; e < gr->counted; ++e) {
                const int32_t w = g->ent_id[gr->first + e];
                if (client[w] && cli_iter[w] < 0) ++cnt;
            }
            nhat = nhat + (double)cnt * gr->wt;
            ++gi;
        }
        const double d = grid[sj];
        const double hi = onepe * alpha - d > 0.0 ? onepe * alpha - d : 0.0;
        const double lo = alpha - d > 0.0 ? alpha - d : 0.0;
        t = t + nhat * (j == 1 ? hi : hi - lo);
    }
    return t;
}

/* Algorithms 3-5 with epsilon > 0.  fac_iter[f] = iteration at which f
   opened, cli_iter[c] = iteration at which c froze (-1: never); q_out[f] =
   q(f) at its opening, or at the last iteration for facilities that stay
   closed.  mode 0: q by the closed form; mode 1: q accumulated by Eq. 2/3.
   Returns ORC_OK, or ORC_ESTATE when the grid would exceed its cap (eps too
   small). */
int orc_eps_open(const orc_graph* g, double eps, const double* cost, const uint8_t* client, int mode,
                 int32_t* fac_iter, int32_t* cli_iter, double* q_out, double* alpha0_out, double* gamma_out,
                 int64_t* iters_out) {
    if (!g || !g->built || !(eps > 0.0)) return ORC_EINVAL;
    const int64_t n = g->n;
    const double onepe = 1.0 + eps;
    int64_t nF = 0, nC = 0;
    double max_cost = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        fac_iter[v] = -1;
        cli_iter[v] = -1;
        q_out[v] = 0.0;
        if (cost[v] < INFINITY) { ++nF; if (cost[v] > max_cost) max_cost = cost[v]; }
        if (client[v]) ++nC;
    }
    *iters_out = 0;
    *alpha0_out = 0.0;
    *gamma_out = -1.0;
    if (nF == 0 || nC == 0) return ORC_OK;
    const double gamma = orc_eps_gamma(g, cost, client);
    *gamma_out = gamma;
    if (!(gamma >= 0.0)) return ORC_OK;        /* no client reaches a facility */
    const double m = (double)nF * (double)nC;
    const double alpha0 = (gamma * onepe) / (m * m);
    *alpha0_out = alpha0;
    double* grid = NULL;
    const int64_t J = eps_grid(alpha0, eps, 2.0 * (max_cost + (double)n + 1.0), &grid);
    if (J < 0) return ORC_ESTATE;
    int64_t nhop = 0;
    for (int64_t i = 0; i < g->ngroups; ++i) if (g->grp[i].hop + 1 > nhop) nhop = g->grp[i].hop + 1;
    int64_t* shell_of_hop = (int64_t*)malloc((size_t)(nhop > 0 ? nhop : 1) * sizeof(int64_t));
    int32_t* comp = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* q = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* dist = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    uint8_t* comp_has_fac = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* newly = (uint8_t*)calloc((size_t)n, 1);
    if (!shell_of_hop || !comp || !q || !dist || !comp_has_fac || !newly) {
        free(grid); free(shell_of_hop); free(comp); free(q); free(dist); free(comp_has_fac); free(newly);
        return ORC_ENOMEM;
    }
    for (int64_t h = 0; h < nhop; ++h) shell_of_hop[h] = shell_index(grid, J, h);
    components(g, comp, q);
    for (int64_t v = 0; v < n; ++v) if (cost[v] < INFINITY) comp_has_fac[comp[v]] = 1;
    int64_t unopened = nF, unfrozen = 0;
    for (int64_t v = 0; v < n; ++v) if (client[v] && comp_has_fac[comp[v]]) ++unfrozen;
    /* iterations beyond alpha_J change nothing: with alpha >= max cost + n + 1
       every facility that has an unfrozen client in its ADS has opened and
       every client that reaches an open facility has frozen (a sampled ADS
       may show a facility none of its component's clients, which then never
       opens) */
    int64_t j = 0;
    while (unopened > 0 && unfrozen > 0 && j < J) {
        ++j;
        /* OpenFacilities (Algorithm 5): every unopened facility at once */
        int64_t opened = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : opened)
        for (int64_t f = 0; f < n; ++f) {
            newly[f] = 0;
            if (!(cost[f] < INFINITY) || fac_iter[f] >= 0) continue;
            double qf;
            if (mode == 0)
                qf = eps_q(g, f, j, grid, onepe, shell_of_hop, nhop, client, cli_iter);
            else
                qf = q_out[f] + eps_increment(g, f, j, grid, onepe, shell_of_hop, nhop, client, cli_iter);
            q_out[f] = qf;
            if (qf >= cost[f]) { newly[f] = 1; ++opened; }
        }
        if (opened > 0) {
            for (int64_t f = 0; f < n; ++f) if (newly[f]) fac_iter[f] = (int32_t)j;
            unopened -= opened;
        }
        /* freeze every unfrozen client with an open facility within (1+eps) alpha_j */
        dist_to_open(g, fac_iter, dist, q);
        const double reach = onepe * grid[j];
        for (int64_t c = 0; c < n; ++c) {
            if (!client[c] || cli_iter[c] >= 0 || !comp_has_fac[comp[c]]) continue;
            if (dist[c] >= 0 && (double)dist[c] <= reach) { cli_iter[c] = (int32_t)j; --unfrozen; }
        }
    }
    *iters_out = j;
    free(grid); free(shell_of_hop); free(comp); free(q); free(dist); free(comp_has_fac); free(newly);
    return ORC_OK;
}

/* Algorithm 6 (Section 4.3): the lexicographically-first MIS under pi of
   H-bar, H's edges as read above.  Sequential greedy in pi order: an open
   facility f joins S iff no client c with alpha(c) = alpha(f) within
   floor((1+eps) alpha(f)) hops of f is claimed; then it claims them.
   Clients frozen at different iterations never meet, so this is the greedy
   of every iteration's facilities on their own. */
int orc_eps_select(const orc_graph* g, double eps, double alpha0, const int32_t* fac_iter,
                   const int32_t* cli_iter, uint64_t seed, uint8_t* open, int64_t* n_open) {
    if (!g || !(eps > 0.0)) return ORC_EINVAL;
    const int64_t n = g->n;
    const double onepe = 1.0 + eps;
    int64_t jmax = 0, m = 0;
    for (int64_t v = 0; v < n; ++v) {
        open[v] = 0;
        if (fac_iter[v] > jmax) jmax = fac_iter[v];
        if (fac_iter[v] >= 0) ++m;
    }
    *n_open = 0;
    if (m == 0) return ORC_OK;
    /* grid values up to jmax (the same products as the opening phase) */
    double* grid = (double*)malloc((size_t)(jmax + 1) * sizeof(double));
    cand_t* c = (cand_t*)malloc((size_t)m * sizeof(cand_t));
    uint8_t* claimed = (uint8_t*)calloc((size_t)n, 1);
    int32_t* dist = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* q = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* ball = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!grid || !c || !claimed || !dist || !q || !ball) {
        free(grid); free(c); free(claimed); free(dist); free(q); free(ball);
        return ORC_ENOMEM;
    }
    grid[0] = alpha0;
    for (int64_t j = 1; j <= jmax; ++j) grid[j] = grid[j - 1] * onepe;
    m = 0;
    for (int64_t f = 0; f < n; ++f)
        if (fac_iter[f] >= 0) { c[m].r = 0.0; c[m].pi = orc_priority(seed, f); c[m].f = (int32_t)f; ++m; }
    qsort(c, (size_t)m, sizeof(cand_t), cand_cmp);   /* all r equal: pi order */
    for (int64_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t opened = 0;
    for (int64_t i = 0; i < m; ++i) {
        const int32_t f = c[i].f;
        const int32_t jf = fac_iter[f];
        const int64_t B = ball_depth(onepe * grid[jf]);
        int64_t qh = 0, qt = 0, nb = 0;
        int conflict = cli_iter[f] == jf && claimed[f];
        dist[f] = 0;
        q[qt++] = f;
        if (cli_iter[f] == jf && !conflict) ball[nb++] = f;
        while (qh < qt && !conflict) {
            int32_t x = q[qh++];
            if (dist[x] == B) continue;
            for (int64_t e = g->rowp[x]; e < g->rowp[x + 1]; ++e) {
                int32_t u = g->cols[e];
                if (dist[u] >= 0) continue;
                if (cli_iter[u] == jf && claimed[u]) { conflict = 1; break; }
                dist[u] = dist[x] + 1;
                q[qt++] = u;
                if (cli_iter[u] == jf) ball[nb++] = u;
            }
        }
        for (int64_t k2 = 0; k2 < qt; ++k2) dist[q[k2]] = -1;
        if (conflict) continue;
        open[f] = 1;
        ++opened;
        for (int64_t k2 = 0; k2 < nb; ++k2) claimed[ball[k2]] = 1;
    }
    *n_open = opened;
    free(grid); free(c); free(claimed); free(dist); free(q); free(ball);
    return ORC_OK;
}

/* ====================================================================== */
/* Weighted graphs (NEXT f3).  Section 3.3, after Algorithm 2: the Giraph  */
/* algorithm handles weighted graphs too; vertices then reach an ADS in    */
/* BFS order rather than by distance, so an entry accepted early can stop  */
/* belonging to the ADS when a closer one arrives, and a CleanUp step      */
/* removes it.  Section 5 draws edge weights uniformly in [1, 100].        */
/* Readings: lengths are positive integers, equal in both directions of an */
/* edge (the graph is undirected), so distances are exact integers; equal  */
/* distances are presented in ascending rank, as in the unweighted build;  */
/* an ADS group is the set of entries at one distance, and its HIP weight  */
/* and counted prefix follow the unweighted build with "hop" read as       */
/* "distance".                                                             */
/* ====================================================================== */

/* Edge lengths, one per CSR entry: positive, equal for (u, v) and (v, u). */
int orc_graph_set_weights(orc_graph* g, const int32_t* w) {
    if (!g || !w) return ORC_EINVAL;
    const int64_t nnz = g->rowp[g->n];
    for (int64_t e = 0; e < nnz; ++e)
        if (w[e] < 1) return ORC_EINVAL;
    int32_t* c = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!c) return ORC_ENOMEM;
    if (nnz > 0) memcpy(c, w, (size_t)nnz * sizeof(int32_t));
    free(g->wts);
    g->wts = c;
    orc_clear_ads(g);
    return ORC_OK;
}

/* ---- binary min-heap of (key, tie, vertex), lexicographic ---- */
typedef struct { int64_t key; int64_t tie; int32_t v; } heap_item;

static int heap_less(const heap_item* a, const heap_item* b) {
    if (a->key != b->key) return a->key < b->key;
    if (a->tie != b->tie) return a->tie < b->tie;
    return a->v < b->v;
}

static void heap_push(heap_item* h, int64_t* n, heap_item x) {
    int64_t i = (*n)++;
    h[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_less(&h[i], &h[p])) break;
        heap_item t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item* h, int64_t* n) {
    heap_item top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *n && heap_less(&h[l], &h[m])) m = l;
        if (r < *n && heap_less(&h[r], &h[m])) m = r;
        if (m == i) break;
        heap_item t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return top;
}

/* Dijkstra from src: dist[x] = d(src, x), -1 when unreachable.  The heap
   holds at most one item per relaxed edge plus the source. */
static int dijkstra(const orc_graph* g, int32_t src, int64_t* dist, heap_item* heap) {
    const int64_t n = g->n;
    for (int64_t i = 0; i < n; ++i) dist[i] = -1;
    int64_t hn = 0;
    heap_item s0 = {0, 0, src};
    heap_push(heap, &hn, s0);
    while (hn > 0) {
        heap_item it = heap_pop(heap, &hn);
        if (dist[it.v] >= 0) continue;
        dist[it.v] = it.key;
        for (int64_t e = g->rowp[it.v]; e < g->rowp[it.v + 1]; ++e) {
            int32_t u = g->cols[e];
            if (dist[u] >= 0) continue;
            heap_item nx = {it.key + g->wts[e], 0, u};
            heap_push(heap, &hn, nx);
        }
    }
    return ORC_OK;
}

typedef struct { int64_t d; uint64_t rank; int32_t id; } dist_rank;

static int dist_rank_cmp(const void* a, const void* b) {
    const dist_rank* x = (const dist_rank*)a;
    const dist_rank* y = (const dist_rank*)b;
    if (x->d != y->d) return (x->d > y->d) - (x->d < y->d);
    return (x->rank > y->rank) - (x->rank < y->rank);
}

/* One vertex's ADS by Algorithm 1 in Dijkstra order (see the section
   comment); appends its groups and entries to the per-vertex buffers. */
typedef struct {
    int32_t ng, ne;
    orc_group* grp;   /* .first relative to this vertex's entries */
    int32_t* id;
    uint64_t* rank;
    uint64_t S[64];
    int32_t slen;
} wads_row;

static int wads_one(const orc_graph* g, int k, uint64_t seed, int32_t v, int64_t* dist, heap_item* heap,
                    dist_rank* order, wads_row* row) {
    const int64_t n = g->n;
    dijkstra(g, v, dist, heap);
    int64_t m = 0;
    for (int64_t x = 0; x < n; ++x)
        if (dist[x] >= 0) { order[m].d = dist[x]; order[m].rank = orc_rank(seed, x); order[m].id = (int32_t)x; ++m; }
    qsort(order, (size_t)m, sizeof(dist_rank), dist_rank_cmp);
    row->grp = (orc_group*)malloc((size_t)(m > 0 ? m : 1) * sizeof(orc_group));
    row->id = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    row->rank = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    if (!row->grp || !row->id || !row->rank) return ORC_ENOMEM;
    int32_t blen = 0, ne = 0, ng = 0;
    for (int64_t i = 0; i < m;) {
        int64_t j = i;
        while (j < m && order[j].d == order[i].d) ++j;
        if (order[i].d > 2147483647LL) return ORC_EINVAL;
        const int32_t first = ne;
        for (int64_t t = i; t < j; ++t) {
            uint64_t r = order[t].rank;
            if (blen < k || r < row->S[k - 1]) {
                row->id[ne] = order[t].id;
                row->rank[ne] = r;
                ++ne;
                bottomk_insert(row->S, &blen, k, r);
            }
        }
        if (ne > first) {
            int32_t counted = 0;
            for (int32_t e = first; e < ne; ++e) {
                int32_t pos = 0;
                while (row->S[pos] != row->rank[e]) ++pos;
                if (blen < k || pos < k - 1) ++counted;
            }
            row->grp[ng].hop = (int32_t)order[i].d;
            row->grp[ng].cnt = ne - first;
            row->grp[ng].counted = counted;
            row->grp[ng].wt = hip_weight(row->S, blen, k);
            row->grp[ng].first = first;
            ++ng;
        }
        i = j;
    }
    row->ng = ng;
    row->ne = ne;
    row->slen = blen;
    return ORC_OK;
}

/* Every vertex's ADS of a weighted graph by the definition (Algorithm 1 in
   Dijkstra order), stored like the unweighted build (group "hop" = the
   distance); the final sketch S is the bottom-k of each component.  hops =
   the largest distance of an entry; edge_merges = 0 (no propagation). */
int orc_build_sketches_weighted(orc_graph* g, int k, uint64_t seed) {
    if (!g || !g->wts || k < 2 || k > 64) return ORC_EINVAL;
    orc_clear_ads(g);
    const int64_t n = g->n;
    const int64_t nnz = g->rowp[n];
    wads_row* rows = (wads_row*)calloc((size_t)(n > 0 ? n : 1), sizeof(wads_row));
    if (!rows) return ORC_ENOMEM;
    int rc = ORC_OK;
#pragma omp parallel
    {
        int64_t* dist = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        heap_item* heap = (heap_item*)malloc((size_t)(nnz + 2) * sizeof(heap_item));
        dist_rank* order = (dist_rank*)malloc((size_t)(n > 0 ? n : 1) * sizeof(dist_rank));
        int lrc = (dist && heap && order) ? ORC_OK : ORC_ENOMEM;
#pragma omp for schedule(dynamic, 16)
        for (int64_t v = 0; v < n; ++v)
            if (lrc == ORC_OK) lrc = wads_one(g, k, seed, (int32_t)v, dist, heap, order, &rows[v]);
        if (lrc != ORC_OK) {
#pragma omp critical
            rc = lrc;
        }
        free(dist); free(heap); free(order);
    }
    if (rc == ORC_OK) {
        g->gofs = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
        g->eofs = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
        g->S = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * k * sizeof(uint64_t));
        g->Scnt = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        if (!g->gofs || !g->eofs || !g->S || !g->Scnt) rc = ORC_ENOMEM;
    }
    if (rc == ORC_OK) {
        for (int64_t v = 0; v < n; ++v) {
            g->gofs[v + 1] = g->gofs[v] + rows[v].ng;
            g->eofs[v + 1] = g->eofs[v] + rows[v].ne;
        }
        g->ngroups = g->gofs[n];
        g->nentries = g->eofs[n];
        g->grp = (orc_group*)malloc((size_t)(g->ngroups > 0 ? g->ngroups : 1) * sizeof(orc_group));
        g->ent_id = (int32_t*)malloc((size_t)(g->nentries > 0 ? g->nentries : 1) * sizeof(int32_t));
        g->ent_rank = (uint64_t*)malloc((size_t)(g->nentries > 0 ? g->nentries : 1) * sizeof(uint64_t));
        if (!g->grp || !g->ent_id || !g->ent_rank) rc = ORC_ENOMEM;
    }
    if (rc == ORC_OK) {
        int64_t maxd = 0;
        for (int64_t v = 0; v < n; ++v) {
            const wads_row* w = &rows[v];
            for (int32_t i = 0; i < w->ng; ++i) {
                orc_group gr = w->grp[i];
                gr.first += g->eofs[v];
                g->grp[g->gofs[v] + i] = gr;
                if (gr.hop > maxd) maxd = gr.hop;
            }
            if (w->ne > 0) {
                memcpy(&g->ent_id[g->eofs[v]], w->id, (size_t)w->ne * sizeof(int32_t));
                memcpy(&g->ent_rank[g->eofs[v]], w->rank, (size_t)w->ne * sizeof(uint64_t));
            }
            g->Scnt[v] = w->slen;
            for (int i = 0; i < k; ++i) g->S[v * k + i] = i < w->slen ? w->S[i] : UINT64_MAX;
        }
        g->k = k;
        g->seed = seed;
        g->hops = maxd;
        g->edge_merges = 0;
        g->built = 1;
    }
    for (int64_t v = 0; v < n; ++v) { free(rows[v].grp); free(rows[v].id); free(rows[v].rank); }
    free(rows);
    if (rc != ORC_OK) orc_clear_ads(g);
    return rc;
}

/* ---- the paper's Algorithm 2 with CleanUp (the second form) ---- */

typedef struct { uint64_t rank; int64_t d; int32_t id; int32_t fresh; } went;

static int dist_rank_cmp_went(const void* a, const void* b) {
    const went* x = (const went*)a;
    const went* y = (const went*)b;
    if (x->d != y->d) return (x->d > y->d) - (x->d < y->d);
    return (x->rank > y->rank) - (x->rank < y->rank);
}

/* Position of the first entry after (d, rank) in (distance, rank) order. */
static int32_t went_upper(const went* L, int32_t len, int64_t d, uint64_t rank) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        int32_t mid = (lo + hi) / 2;
        if (L[mid].d < d || (L[mid].d == d && L[mid].rank <= rank)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Receiver test of Algorithm 2 for a candidate (id, d): fewer than k
   entries of the list precede it in (distance, rank) order with a smaller
   rank.  Entries of the list sit at their current (upper-bound) distances. */
static int went_accepts(const went* L, int32_t len, int k, int64_t d, uint64_t rank) {
    int32_t smaller = 0;
    for (int32_t i = 0; i < len; ++i) {
        if (L[i].d > d || (L[i].d == d && L[i].rank >= rank)) break;
        if (L[i].rank < rank && ++smaller >= k) return 0;
    }
    return 1;
}

/* CleanUp: keep an entry iff fewer than k kept entries before it (in
   (distance, rank) order) have a smaller rank.  Returns entries removed. */
static int64_t went_cleanup(went* L, int32_t* len, int k) {
    uint64_t B[64];
    int32_t blen = 0, out = 0;
    int64_t removed = 0;
    for (int32_t i = 0; i < *len; ++i) {
        uint64_t r = L[i].rank;
        if (blen < k || r < B[k - 1]) {
            bottomk_insert(B, &blen, k, r);
            L[out++] = L[i];
        } else {
            ++removed;
        }
    }
    *len = out;
    return removed;
}

/* Supersteps: in each, every vertex sends the entries it accepted in the
   previous superstep (distance + edge length) to its neighbours; each
   receiver takes its candidates in (distance, rank) order, skips those whose
   vertex it already holds at a distance <= d, drops a farther entry of the
   same vertex, inserts the candidate when the receiver test passes, and then
   runs CleanUp.  Until no vertex accepts anything.  Output: per vertex its
   entries in (distance, rank) order (eofs n+1 offsets; eid, edist up to
   `cap` entries), the supersteps run and the entries CleanUp removed. */
int orc_wads_rounds(const orc_graph* g, int k, uint64_t seed, int64_t cap, int64_t* eofs, int32_t* eid,
                    int64_t* edist, int64_t* steps, int64_t* cleaned) {
    if (!g || !g->wts || k < 2 || k > 64) return ORC_EINVAL;
    const int64_t n = g->n;
    went** L = (went**)calloc((size_t)(n > 0 ? n : 1), sizeof(went*));
    int32_t* len = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    int32_t* capv = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    if (!L || !len || !capv) { free(L); free(len); free(capv); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (int64_t v = 0; v < n && rc == ORC_OK; ++v) {
        capv[v] = 8;
        L[v] = (went*)malloc(8 * sizeof(went));
        if (!L[v]) { rc = ORC_ENOMEM; break; }
        L[v][0].rank = orc_rank(seed, v); L[v][0].d = 0; L[v][0].id = (int32_t)v; L[v][0].fresh = 1;
        len[v] = 1;
    }
    int64_t step = 0, removed = 0;
    went* cand = NULL;
    int64_t cand_cap = 0;
    while (rc == ORC_OK) {
        /* snapshot of this superstep's messages: the fresh entries */
        int64_t nmsg = 0;
        for (int64_t v = 0; v < n; ++v)
            for (int32_t i = 0; i < len[v]; ++i) nmsg += L[v][i].fresh ? 1 : 0;
        if (nmsg == 0) break;
        ++step;
        went** msg = (went**)calloc((size_t)n, sizeof(went*));
        int32_t* mlen = (int32_t*)calloc((size_t)n, sizeof(int32_t));
        if (!msg || !mlen) { free(msg); free(mlen); rc = ORC_ENOMEM; break; }
        for (int64_t v = 0; v < n && rc == ORC_OK; ++v) {
            int32_t c = 0;
            for (int32_t i = 0; i < len[v]; ++i) c += L[v][i].fresh ? 1 : 0;
            msg[v] = (went*)malloc((size_t)(c > 0 ? c : 1) * sizeof(went));
            if (!msg[v]) { rc = ORC_ENOMEM; break; }
            c = 0;
            for (int32_t i = 0; i < len[v]; ++i)
                if (L[v][i].fresh) { msg[v][c++] = L[v][i]; L[v][i].fresh = 0; }
            mlen[v] = c;
        }
        for (int64_t v = 0; v < n && rc == ORC_OK; ++v) {
            /* candidates from every neighbour's messages */
            int64_t nc = 0;
            for (int64_t e = g->rowp[v]; e < g->rowp[v + 1]; ++e) nc += mlen[g->cols[e]];
            if (nc == 0) continue;
            if (nc > cand_cap) {
                cand_cap = nc * 2;
                went* t = (went*)realloc(cand, (size_t)cand_cap * sizeof(went));
                if (!t) { rc = ORC_ENOMEM; break; }
                cand = t;
            }
            nc = 0;
            for (int64_t e = g->rowp[v]; e < g->rowp[v + 1]; ++e) {
                int32_t u = g->cols[e];
                for (int32_t i = 0; i < mlen[u]; ++i) {
                    cand[nc] = msg[u][i];
                    cand[nc].d = msg[u][i].d + g->wts[e];
                    cand[nc].fresh = 1;
                    ++nc;
                }
            }
            qsort(cand, (size_t)nc, sizeof(went), dist_rank_cmp_went);
            for (int64_t c = 0; c < nc; ++c) {
                went x = cand[c];
                int32_t at = -1;
                for (int32_t i = 0; i < len[v]; ++i)
                    if (L[v][i].id == x.id) { at = i; break; }
                if (at >= 0 && L[v][at].d <= x.d) continue;
                if (!went_accepts(L[v], len[v], k, x.d, x.rank)) continue;
                if (at >= 0) {  /* the same vertex, farther: replaced */
                    memmove(&L[v][at], &L[v][at + 1], (size_t)(len[v] - at - 1) * sizeof(went));
                    --len[v];
                }
                if (len[v] == capv[v]) {
                    capv[v] *= 2;
                    went* t = (went*)realloc(L[v], (size_t)capv[v] * sizeof(went));
                    if (!t) { rc = ORC_ENOMEM; break; }
                    L[v] = t;
                }
                int32_t pos = went_upper(L[v], len[v], x.d, x.rank);
                memmove(&L[v][pos + 1], &L[v][pos], (size_t)(len[v] - pos) * sizeof(went));
                L[v][pos] = x;
                ++len[v];
            }
            removed += went_cleanup(L[v], &len[v], k);
        }
        for (int64_t v = 0; v < n; ++v) free(msg[v]);
        free(msg); free(mlen);
    }
    free(cand);
    if (rc == ORC_OK) {
        eofs[0] = 0;
        for (int64_t v = 0; v < n; ++v) eofs[v + 1] = eofs[v] + len[v];
        if (eofs[n] > cap) rc = ORC_EINVAL;
    }
    if (rc == ORC_OK) {
        for (int64_t v = 0; v < n; ++v)
            for (int32_t i = 0; i < len[v]; ++i) {
                eid[eofs[v] + i] = L[v][i].id;
                edist[eofs[v] + i] = L[v][i].d;
            }
        *steps = step;
        *cleaned = removed;
    }
    for (int64_t v = 0; v < n; ++v) free(L[v]);
    free(L); free(len); free(capv);
    return rc;
}

/* ---- phase (iii) and assignment on weighted distances ---- */

/* The lexicographically-first MIS of H-bar under (r_f, pi_f) with balls of
   weighted distance: Ball(f) = clients within distance floor(r_f) of f,
   found by Dijkstra from f, stopped at the first claimed client. */
int orc_open_facilities_weighted(const orc_graph* g, const double* r, const uint8_t* client, uint64_t seed,
                                 uint8_t* open, int64_t* n_open) {
    if (!g || !g->wts) return ORC_EINVAL;
    const int64_t n = g->n;
    const int64_t nnz = g->rowp[n];
    int64_t m = 0;
    for (int64_t f = 0; f < n; ++f) if (r[f] < INFINITY) ++m;
    cand_t* c = (cand_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(cand_t));
    uint8_t* claimed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t* dist = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int32_t* seen = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* ball = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    heap_item* heap = (heap_item*)malloc((size_t)(nnz + 2) * sizeof(heap_item));
    if (!c || !claimed || !dist || !seen || !ball || !heap) {
        free(c); free(claimed); free(dist); free(seen); free(ball); free(heap);
        return ORC_ENOMEM;
    }
    m = 0;
    for (int64_t f = 0; f < n; ++f)
        if (r[f] < INFINITY) { c[m].r = r[f]; c[m].pi = orc_priority(seed, f); c[m].f = (int32_t)f; ++m; }
    qsort(c, (size_t)m, sizeof(cand_t), cand_cmp);
    for (int64_t v = 0; v < n; ++v) { dist[v] = -1; open[v] = 0; }
    int64_t opened = 0;
    for (int64_t i = 0; i < m; ++i) {
        const int32_t f = c[i].f;
        const int64_t B = ball_depth(c[i].r);
        int64_t hn = 0, ns = 0, nb = 0;
        int conflict = 0;
        heap_item s0 = {0, 0, f};
        heap_push(heap, &hn, s0);
        while (hn > 0 && !conflict) {
            heap_item it = heap_pop(heap, &hn);
            if (dist[it.v] >= 0) continue;
            dist[it.v] = it.key;
            seen[ns++] = it.v;
            if (client[it.v]) {
                if (claimed[it.v]) { conflict = 1; break; }
                ball[nb++] = it.v;
            }
            for (int64_t e = g->rowp[it.v]; e < g->rowp[it.v + 1]; ++e) {
                int32_t u = g->cols[e];
                int64_t du = it.key + g->wts[e];
                if (dist[u] >= 0 || du > B) continue;
                heap_item nx = {du, 0, u};
                heap_push(heap, &hn, nx);
            }
        }
        for (int64_t j = 0; j < ns; ++j) dist[seen[j]] = -1;
        if (conflict) continue;
        open[f] = 1;
        ++opened;
        for (int64_t j = 0; j < nb; ++j) claimed[ball[j]] = 1;
    }
    *n_open = opened;
    free(c); free(claimed); free(dist); free(seen); free(ball); free(heap);
    return ORC_OK;
}

/* Nearest open facility by weighted distance (Section 3.1, d(c, S)): one
   Dijkstra from every open facility at once, ordered by (distance, facility
   id), so a vertex is settled with its smallest distance and, among the
   facilities at that distance, the smallest id.  -1 / -1 when none is
   reachable. */
int orc_assign_weighted(const orc_graph* g, const uint8_t* open, int32_t* assign, int32_t* dist) {
    if (!g || !g->wts) return ORC_EINVAL;
    const int64_t n = g->n;
    const int64_t nnz = g->rowp[n];
    heap_item* heap = (heap_item*)malloc((size_t)(nnz + n + 2) * sizeof(heap_item));
    if (!heap) return ORC_ENOMEM;
    int64_t hn = 0;
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = -1;
        assign[v] = -1;
        if (open[v]) { heap_item s0 = {0, v, (int32_t)v}; heap_push(heap, &hn, s0); }
    }
    int rc = ORC_OK;
    while (hn > 0) {
        heap_item it = heap_pop(heap, &hn);
        if (dist[it.v] >= 0) continue;
        if (it.key > 2147483647LL) { rc = ORC_EINVAL; break; }
        dist[it.v] = (int32_t)it.key;
        assign[it.v] = (int32_t)it.tie;
        for (int64_t e = g->rowp[it.v]; e < g->rowp[it.v + 1]; ++e) {
            int32_t u = g->cols[e];
            if (dist[u] >= 0) continue;
            heap_item nx = {it.key + g->wts[e], it.tie, u};
            heap_push(heap, &hn, nx);
        }
    }
    free(heap);
    return rc;
}
