/*
 * fl.h -- C ABI of the GB300 graph facility-location library (libflgpu.so).
 *
 * The library computes, on one GPU, the data-parallel hot path of the
 * facility-location method of Garimella, De Francisci Morales, Gionis and
 * Sozio ("Scalable Facility Location for Massive Graphs on Pregel-like
 * Systems"):
 *   (i)   bottom-k min-hash sketches and all-distances sketches (ADS) with HIP
 *         weights, by hop-synchronous propagation (Section 3.3, Alg. 1-2);
 *   (ii)  per-facility opening radii from predicated HIP estimates of client
 *         counts (Eq. 1 at epsilon -> 0, Sections 4.2 and 4.5);
 *   (iii) facility selection as the lexicographically-first maximal
 *         independent set of the conflict graph H-bar under key (r_f, pi_f)
 *         (Alg. 3 and Section 4.3, Alg. 6);
 *   then each client's nearest open facility and the objective (Section 3.1).
 *
 * Conventions for every entry point:
 *   - Return value: FL_OK (0) or one of the FL_E* codes below; no exception
 *     or signal crosses the ABI.  fl_last_error() gives the message of the
 *     most recent failure on the calling thread.
 *   - Pointers are host or device memory as the call's `mem_kind` says
 *     (FL_MEM_HOST or FL_MEM_DEVICE); device pointers must belong to the
 *     current CUDA device.  The caller keeps ownership of every array it
 *     passes; the library copies inputs before returning and writes outputs
 *     into caller arrays.  Handles own all device memory they allocate.
 *   - Work is issued on the stream given to fl_graph_create (NULL = legacy
 *     default stream).  Calls return after their results are complete
 *     (outputs are valid on return for both memory kinds).
 *   - Handles are thread-compatible: use one handle from one thread at a
 *     time.  A graph may serve many solves created from it, one at a time.
 *   - Vertex ids are int32 in [0, n); row offsets are int64 (graphs with
 *     more than 2^31 directed edges are supported).
 *   - The graph must be undirected: the CSR must be symmetric (u in N(v) iff
 *     v in N(u)), as in the paper's undirected setting (Section 3.1).
 */
#ifndef FL_H
#define FL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define FL_OK 0
#define FL_EINVAL 1   /* bad argument: null handle, bad CSR, unsupported k, bad cost */
#define FL_ESTATE 2   /* called out of order (e.g. radii before sketches) */
#define FL_ENOMEM 3   /* device or host allocation failed */
#define FL_ECUDA 4    /* a CUDA runtime call or kernel failed */
#define FL_ETIMEOUT 5 /* a bounded device-side loop hit its iteration limit */

/* Memory kinds of pointer arguments. */
#define FL_MEM_HOST 0
#define FL_MEM_DEVICE 1

typedef struct fl_graph fl_graph; /* device CSR + sketches + ADS of one graph */
typedef struct fl_solve fl_solve; /* one instance: costs, clients, radii, open set, assignment */

/*
 * fl_graph_create -- upload a graph (Section 3.1: G = (V, E), unweighted).
 *   n        number of vertices, 1 <= n <= 2^31 - 1.
 *   row_off  int64[n+1] CSR row offsets, row_off[0] = 0, non-decreasing,
 *            row_off[n] = nnz.
 *   cols     int32[nnz] neighbour ids in [0, n); must be symmetric.
 *   nnz      number of directed CSR entries (2 x undirected edges).
 *   mem_kind FL_MEM_HOST or FL_MEM_DEVICE for row_off and cols.
 *   stream   cudaStream_t on which all work of this graph and its solves runs.
 *   out      receives the new handle.
 * The CSR is validated on the device (offsets monotone, ids in range);
 * violations return FL_EINVAL.  Self-loops and duplicates are tolerated.
 */
int fl_graph_create(int64_t n, const int64_t* row_off, const int32_t* cols, int64_t nnz,
                    int mem_kind, void* stream, fl_graph** out);

/*
 * fl_graph_create_weighted -- upload a weighted graph (Section 3.3, after
 * Algorithm 2: the Giraph ADS algorithm also handles weighted graphs;
 * Section 5 draws weights uniformly in [1, 100]).  Arguments as
 * fl_graph_create, plus
 *   lengths  int32[nnz] edge length of each CSR entry, an integer in
 *            [1, 65535], equal for (u, v) and (v, u) (same mem_kind): the
 *            entries (u, v) and (v, u) of each length must be equally many
 *            (FL_EINVAL otherwise); nnz < 2^32.
 * fl_build_sketches then builds the ADS in Dijkstra order: one group per
 * distance (the group's "hop" is the distance, at most 65535, else
 * FL_EINVAL), with the HIP weights and counted prefixes of the unweighted
 * build, equal to the ADS that the paper's BFS-order supersteps reach after
 * CleanUp; fl_sketch_stats reports the largest distance as hops and 0
 * edge-merges.  fl_compute_radii solves Eq. 1 over these distances, and
 * fl_open_facilities / fl_assign_clients / fl_objective measure balls and
 * nearest facilities by the sum of lengths (Section 3.1's d(u, v)).  The
 * epsilon > 0 phase, exact ball sizes and batches are not built for weighted
 * graphs: those calls return FL_ESTATE.  The graph keeps the caller's vertex
 * numbering.
 */
int fl_graph_create_weighted(int64_t n, const int64_t* row_off, const int32_t* cols, const int32_t* lengths,
                             int64_t nnz, int mem_kind, void* stream, fl_graph** out);

/* fl_graph_destroy -- free the handle and all its device memory (NULL ok). */
int fl_graph_destroy(fl_graph* g);

/*
 * fl_build_sketches -- phase (i): per-vertex bottom-k sketches and the ADS.
 * Section 3.3 (Alg. 1 sequential, Alg. 2 vertex program): hop h merges into
 * each vertex the sketch entries its neighbours gained at hop h-1 and keeps
 * the k smallest ranks; it stops when no sketch changes.  Ranks are
 * r(v) = SplitMix64 output v+1 from state `seed`.  Every entry that joins
 * S_h(v) is an ADS entry (v, u, h); its HIP weight is 1 when S_h(v) holds
 * fewer than k ranks, else entries at positions < k-1 weigh
 * 2^64 / S_h(v)[k-1] and the entry at position k-1 weighs 0.
 *   k     sketch size, 2 <= k <= 32.
 *   seed  rank seed.
 * Returns FL_EINVAL if k is unsupported or a vertex's rank would equal
 * UINT64_MAX (the empty-slot sentinel; probability n / 2^64).
 * Rebuilding with other (k, seed) replaces the previous sketches and
 * invalidates solves created before (they return FL_ESTATE).
 */
int fl_build_sketches(fl_graph* g, int k, uint64_t seed);

/*
 * fl_sketch_stats -- counters of the last build (any pointer may be NULL).
 *   hops         last hop at which some sketch changed (H*).
 *   edge_merges  sum over processed hops h of the CSR entries (v, u) whose
 *                u gained entries at hop h-1 (the unit of work of Alg. 2).
 *   ads_entries  total ADS entries; ads_groups: total (vertex, hop) groups.
 */
int fl_sketch_stats(const fl_graph* g, int64_t* hops, int64_t* edge_merges,
                    int64_t* ads_entries, int64_t* ads_groups);

/*
 * fl_export_sketches -- copy the final sketches out.
 *   S    uint64[n*k]: S[v*k + i] = i-th smallest rank of v's component, or
 *        UINT64_MAX past cnt[v];  cnt int32[n] (either may be NULL).
 */
int fl_export_sketches(fl_graph* g, uint64_t* S, int32_t* cnt, int mem_kind);

/*
 * fl_export_ads -- copy the ADS out, vertex-major (groups of v ordered by hop,
 * entries of a group by ascending rank).  Sizes from fl_sketch_stats.
 *   gofs, eofs     int64[n+1] group / entry offsets per vertex.
 *   ghop, gcnt     int32[groups] distance and entry count of each group.
 *   gcounted       int32[groups] leading entries that carry the weight.
 *   gwt            double[groups] HIP weight of each counted entry.
 *   eid            int32[entries] vertex id of each entry.
 * Any pointer may be NULL (that array is skipped).
 */
int fl_export_ads(fl_graph* g, int64_t* gofs, int64_t* eofs, int32_t* ghop, int32_t* gcnt,
                  int32_t* gcounted, double* gwt, int32_t* eid, int mem_kind);

/* fl_solve_create / fl_solve_destroy -- one facility-location instance on a
   graph whose sketches are built (else FL_ESTATE). */
int fl_solve_create(fl_graph* g, fl_solve** out);
int fl_solve_destroy(fl_solve* s);

/*
 * fl_compute_radii -- phase (ii): opening radius of every facility.
 * Eq. 1 with all clients unfrozen and alpha(c) = r (Section 4.2), at
 * epsilon -> 0: r_f solves sum_h W_h max(0, r - h) = c(f), where W_h is the
 * HIP estimate of the clients at distance h of f, read off f's ADS with the
 * client predicate (Section 4.5).  In FP64 with a fixed operation order.
 *   open_cost   double[n]; +INFINITY = not a facility; facilities need a
 *               finite cost > 0 (else FL_EINVAL).
 *   client_mask uint8[n]; nonzero = client.
 *   mem_kind    memory kind of open_cost, client_mask and radii_out.
 *   radii_out   double[n] or NULL; +INFINITY for non-facilities and for
 *               facilities that reach no client.
 */
int fl_compute_radii(fl_solve* s, const double* open_cost, const uint8_t* client_mask,
                     int mem_kind, double* radii_out);

/*
 * fl_open_facilities -- phase (iii): the lexicographically-first maximal
 * independent set S of H-bar (Section 4.3, Alg. 6 with the greedy MIS of
 * Blelloch, Fineman and Shun).  Candidates: facilities with finite r_f.
 * Ball(f) = clients within floor(r_f) hops of f (distance: the sum of the
 * lengths on a weighted graph); f, g conflict iff their balls share a client.  Keys (r_f, pi_f), pi_f = SplitMix64 output f+1 from
 * the state given by the first output for the sketch seed.
 *   open_out  uint8[n] or NULL (1 = open).   n_open  receives |S| (or NULL).
 * Needs fl_compute_radii first (else FL_ESTATE).
 */
int fl_open_facilities(fl_solve* s, uint8_t* open_out, int64_t* n_open, int mem_kind);

/*
 * fl_open_facilities_eps -- the paper's opening phase with accuracy eps > 0
 * (Section 4.1, Algorithm 3; Section 4.2, Algorithms 4-5 and Eq. 2/3) and the
 * facility selection of Algorithm 6 (Section 4.3), in place of
 * fl_compute_radii + fl_open_facilities.  Radii grow on the grid alpha_j =
 * alpha_{j-1} (1 + eps) from alpha_0 = gamma (1 + eps) / m^2 (m = |F||C|,
 * gamma = max over clients reaching a facility of min_f c(f) + d(c, f)); in
 * iteration j every unopened facility with q(f) >= c(f) opens, then every
 * unfrozen client within (1 + eps) alpha_j of an open facility freezes.
 * q(f) is the sum Eq. 2 and Eq. 3 accumulate, over the HIP-weighted client
 * entries of f's ADS, each client counted at the smallest grid value >= its
 * hop distance (the first shell read as [0, alpha_0]).  Clients that reach
 * no facility never freeze; the phase ends when every facility is open or
 * every client that reaches one is frozen.  Selection: the lexicographically
 * first MIS under pi(f) of H-bar, where a client joins the facilities that
 * opened in the iteration it froze and lie within (1 + eps) alpha of it.
 *   eps            accuracy, 0 < eps <= 1e6 (FL_EINVAL otherwise; FL_EINVAL
 *                  too when the grid would need more than 2^22 radii).
 *   open_cost      double[n]: > 0 finite for facilities, +inf otherwise.
 *   client_mask    uint8[n]: nonzero = client.
 *   open_out       uint8[n] or NULL: the selected facilities.
 *   n_open         int64 or NULL: their number.
 *   fac_iter_out   int32[n] or NULL: iteration at which each vertex opened
 *                  as a facility (-1: never).
 *   cli_iter_out   int32[n] or NULL: iteration at which each client froze
 *                  (-1: never).
 * Arrays live in the memory mem_kind names; outputs are complete on return.
 * Afterwards fl_assign_clients and fl_objective serve the selected set.
 * Requires built sketches (FL_ESTATE).
 */
int fl_open_facilities_eps(fl_solve* s, double eps, const double* open_cost, const uint8_t* client_mask,
                           int mem_kind, uint8_t* open_out, int64_t* n_open, int32_t* fac_iter_out,
                           int32_t* cli_iter_out);

/* fl_eps_stats -- gamma, alpha_0, the last iteration run, the number of
   iterations with an opening or a freezing ("events", the ones the GPU
   evaluates), and of iterations whose facilities needed an MIS, for the
   last fl_open_facilities_eps of s (FL_ESTATE before one); pointers may be
   NULL. */
int fl_eps_stats(const fl_solve* s, double* gamma, double* alpha0, int64_t* iterations, int64_t* events,
                 int64_t* groups);

/*
 * fl_assign_clients -- nearest open facility of every vertex (Section 3.1,
 * d(c, S) = min over open f of d(c, f)); ties go to the smallest facility id.
 *   assign_out int32[n] or NULL (-1 = no open facility in the component).
 *   dist_out   int32[n] or NULL (hop distance, -1 when unassigned; on a
 *              weighted graph the sum of lengths, FL_EINVAL when one is
 *              above 2^31 - 1).
 */
int fl_assign_clients(fl_solve* s, int32_t* assign_out, int32_t* dist_out, int mem_kind);

/*
 * fl_objective -- sum_{f in S} c(f) + sum_{c in C} d(c, S) (Section 3.1).
 * Clients without an open facility in their component are left out of the
 * sum and counted in n_unserved.  obj is FP64; dist_sum is exact.
 */
int fl_objective(fl_solve* s, double* obj, int64_t* dist_sum, int64_t* n_unserved);

/* fl_solve_stats -- counters of the last MIS: rounds of the greedy MIS and
   the number of candidates (any pointer may be NULL). */
int fl_solve_stats(const fl_solve* s, int64_t* mis_rounds, int64_t* candidates);

/*
 * fl_mis_log -- the rounds of the last greedy MIS (fl_open_facilities), six
 * int64 per row: (greedy round, kind, step, frontier size at the start,
 * pulled (1) or pushed (0), host microseconds).  kind 0: a round of the cover
 * sweep (step = time t); 1: a round of the gather sweep (step = radius b);
 * 2: a bucket of the undecided facilities (step = ball radius, frontier =
 * its size); 3: the greedy round's total (step = its largest ball radius T,
 * frontier = undecided facilities at its start, pulled = those it decided);
 * 4: a round of the kill sweep that removes the facilities whose ball holds
 * a client claimed in that greedy round (step = distance, frontier = the
 * vertices it marked).  On a weighted graph each sweep (a time-stepped
 * propagation over the lengths) logs one row: kinds 0 (cover), 1 (gather) and 4
 * (kill) with step = the last time step run and frontier = the time steps
 * run, pulled 0; kind 3 as above.
 *   rows    int64[6 * cap] or NULL; the first min(cap, *n_rows) rows are written.
 *   n_rows  receives the number of rows of the last MIS.
 * Host-side timings include the launches and the synchronisation of a round.
 */
int fl_mis_log(const fl_solve* s, int64_t cap, int64_t* n_rows, int64_t* rows);

/*
 * Exact neighbourhood sizes and exact-count radii.  The paper checks the
 * ADS estimates against exact neighbourhood sizes on sampled vertices
 * (Section 5.1, "Accuracy vs. k", Fig. 1: relative error |S_E - S_ADS| / S_E
 * per distance, against k).  These calls give both sides of that comparison
 * on the GPU and an exact-radius mode of phase (ii).  The exact sizes come
 * from a bit-parallel breadth-first search (256 sources per sweep, 96 bytes
 * of device scratch per vertex, held by the graph), so their cost grows
 * with the number of sources times the balls' edges: meant for sampled
 * vertices and small or medium graphs.
 */

/*
 * fl_ball_sizes -- exact sizes: out[s * (max_dist + 1) + h] = the number of
 * vertices w with d(src[s], w) <= h and pred[w] != 0 (pred NULL: every
 * vertex), h = 0..max_dist.  Needs fl_graph_create only.
 *   src       int32[n_src], ids in [0, n) (else FL_EINVAL); repeats allowed.
 *   max_dist  >= 0 (else FL_EINVAL).
 *   pred      uint8[n] or NULL.
 *   out       int64[n_src * (max_dist + 1)], source-major.
 *   mem_kind  memory kind of src, pred and out.
 */
int fl_ball_sizes(fl_graph* g, int64_t n_src, const int32_t* src, int32_t max_dist, const uint8_t* pred,
                  int mem_kind, int64_t* out);

/*
 * fl_ball_estimates -- the HIP estimates of the same sizes read off the ADS
 * (Section 3.3's neighbourhood queries; with a predicate, the estimator of
 * Section 4.5): out[s * (max_dist + 1) + h] = the sum over src[s]'s ADS
 * groups at distance <= h, in distance order, of (entries of the group's
 * weighted prefix with pred != 0) x the group's HIP weight, one FP64 add and
 * multiply per group.  Needs fl_build_sketches (else FL_ESTATE).  Arguments
 * as for fl_ball_sizes; out is double[n_src * (max_dist + 1)].
 */
int fl_ball_estimates(fl_graph* g, int64_t n_src, const int32_t* src, int32_t max_dist, const uint8_t* pred,
                      int mem_kind, double* out);

/*
 * fl_compute_radii_exact -- phase (ii) with exact client counts: Eq. 1 at
 * epsilon -> 0 as in fl_compute_radii, with W_h = the number of clients at
 * distance exactly h of f (from breadth-first search) for h = 0..L, L the
 * eccentricity of f.  r_f = j + (c - G_j) / N_j at the first j < L with
 * G_{j+1} >= c, else L + (c - G_L) / N_L, +inf when N_L = 0 (N_j, G_j exact
 * integers; three IEEE FP64 operations).  With k at least the component
 * size every HIP weight is 1 and fl_compute_radii gives the same numbers.
 * Arguments, state and errors as for fl_compute_radii; the later phases
 * (fl_open_facilities ...) then run on these radii.
 */
int fl_compute_radii_exact(fl_solve* s, const double* open_cost, const uint8_t* client_mask, int mem_kind,
                           double* radii_out);

/*
 * Profiling (launch accounting and kernel timing of a graph and its solves).
 * The paper reports per-phase running times (Section 5); these calls give the
 * same split on the GPU.  Every kernel launch is counted per class; when
 * timing is on, each launch is bracketed by CUDA events on the graph's stream
 * and the elapsed times are summed when the API call that issued it returns.
 * Classes: FL_PROF_SKETCH_MERGE (the hop merge kernel), FL_PROF_SKETCH_EXPAND
 * (frontier expansion), FL_PROF_SKETCH_OTHER (rank init, ADS compaction,
 * eccentricity bound), FL_PROF_RADIUS, FL_PROF_KEYS (candidate sort),
 * FL_PROF_MIS, FL_PROF_BFS (assignment), FL_PROF_OTHER, FL_PROF_EXACT
 * (exact sizes, their estimates, exact-count radii); -1 = all classes.
 * alg_bytes is filled for FL_PROF_SKETCH_MERGE: per hop, 8 B per merging
 * vertex (row offsets) + 4 B per edge-merge (column) + 8 B per neighbour
 * delta rank read + 16k B per merging vertex (own sketch read and write) +
 * 12 B per new ADS entry; and for FL_PROF_EXACT: per search level, 68 B per
 * vertex (list id, visited words read, next words written) + 16 B per
 * scanned row (offsets) + 36 B per scanned entry (column and the
 * neighbour's frontier words).
 */
#define FL_PROF_SKETCH_MERGE 0
#define FL_PROF_SKETCH_EXPAND 1
#define FL_PROF_SKETCH_OTHER 2
#define FL_PROF_RADIUS 3
#define FL_PROF_KEYS 4
#define FL_PROF_MIS 5
#define FL_PROF_BFS 6
#define FL_PROF_OTHER 7
#define FL_PROF_EXACT 8

/* fl_profile_enable -- CUDA-event timing of launches off (0), on (1), or on
   with the per-hop census of the sketch build (2: extra kernels that count
   the scanned and mask-merged CSR entries of each hop, fl_hop_stats). */
int fl_profile_enable(fl_graph* g, int on);
/* fl_profile_reset -- zero all counters and times (synchronises the stream). */
int fl_profile_reset(fl_graph* g);
/* fl_profile_query -- launches, summed kernel milliseconds and algorithmic
   bytes of one class (or all, kernel_class = -1); any pointer may be NULL. */
int fl_profile_query(const fl_graph* g, int kernel_class, int64_t* launches, double* ms, double* alg_bytes);

/*
 * fl_hop_stats -- per-hop counters of the last build (Alg. 2): the hops
 * 1..H* that changed some sketch and the final hop H*+1 that changed none.
 *   n_hops        set to the number of processed hops, H* + 1 (entries
 *                 written: min(n_hops, cap)).
 *   changed[h-1]  vertices whose sketch changed at hop h.
 * With the census on (fl_profile_enable level 2) during the build, also:
 *   scanned[h-1]  CSR entries read at hop h (neighbours of the processed
 *                 vertices, hub segments included), else 0;
 *   mask[h-1]     of those, entries read by the mask merge of saturated
 *                 sketches (full sketches whose k-th rank is among the 1024
 *                 smallest ranks of the graph), else 0;
 * and with profiling on (level 1 or 2):
 *   ms[h-1]       kernel milliseconds of hop h, else 0.
 * Host arrays of cap entries; any of them may be NULL.
 */
int fl_hop_stats(const fl_graph* g, int64_t cap, int64_t* n_hops, int64_t* scanned, int64_t* mask,
                 int64_t* changed, double* ms);

/*
 * Schedules: how the kernels lay out work, never what they compute.
 *   hop_group   lanes per vertex in the sketch hop when k <= 16: 16 or 32
 *               (0 = 16); k > 16 always uses 32.
 *   sparse_div  a hop runs sparse (only the neighbours of the previous
 *               hop's frontier) when frontier * sparse_div < the listed
 *               vertices (default 16).
 *   dense_div   a relaxation round (MIS sweeps, BFS levels) pulls when its
 *               frontier * dense_div >= the listed vertices (default 8) ...
 *   edge_div    ... or when its frontier's edges * edge_div >= nnz
 *               (default 16); otherwise it pushes.
 *   graph_bfs   1: the assignment BFS runs as one CUDA graph whose
 *               conditional WHILE node repeats one pull level on the device
 *               (no host round trip per level; capped at n + 2 levels,
 *               FL_ETIMEOUT beyond); 0 (default): push/pull levels driven by
 *               the host.
 *   level_cap   BFS levels at most (both forms; 0 = n + 2, never reached by
 *               a BFS); a BFS that would need more returns FL_ETIMEOUT.
 * Divisors lie in [1, 1024], graph_bfs in {0, 1}, level_cap >= 0 (FL_EINVAL
 * otherwise).
 */
typedef struct fl_schedule {
    int32_t hop_group;
    int32_t sparse_div;
    int32_t dense_div;
    int32_t edge_div;
    int32_t graph_bfs;
    int32_t level_cap;
} fl_schedule;

/* fl_get_schedule / fl_set_schedule -- the graph's schedule (the default
   until set or tuned); it applies to every later build and solve. */
int fl_get_schedule(const fl_graph* g, fl_schedule* out);
int fl_set_schedule(fl_graph* g, const fl_schedule* sched);

/*
 * fl_autotune -- pick g's schedule for k: times the whole path (sketches
 * with `seed`, radii, keys and MIS, assignment) on g with the given costs and
 * clients (memory per mem_kind) under candidate schedules, by coordinate
 * descent from the default over at most max_trials timed configurations
 * (each the best of two passes), keeps the fastest (a change needs a 1 %
 * gain) and sets it on g; g's sketches are left built with (k, seed).  The
 * choice is cached for the process per graph signature (vertices, CSR
 * entries, hub / small / medium vertex counts) and k: a later call on a
 * graph of the same signature sets the cached schedule without timing.
 * chosen, ms_default, ms_tuned (per pass) may be NULL.
 */
int fl_autotune(fl_graph* g, int k, uint64_t seed, const double* open_cost, const uint8_t* client_mask, int mem_kind,
                int max_trials, fl_schedule* chosen, double* ms_default, double* ms_tuned);
/* fl_autotune_forget -- empty the autotuner's cache. */
int fl_autotune_forget(void);

/*
 * fl_hop_model -- per-hop terms of the algorithmic-bytes model of the sketch
 * hop (Alg. 2; one hop of the last build is one round of messages), filled
 * by every build whether or not profiling is on.  For hop h = 1..n_hops:
 *   edge_merges[h-1]  E_h: CSR entries (v, u) whose u gained entries at hop
 *                     h-1 (every entry at hop 1);
 *   merging[h-1]      A_h: vertices with at least one such entry;
 *   delta_read[h-1]   neighbour-delta ranks the merge kernels read (filtering
 *                     loads of the list merge; 4 words per neighbour and
 *                     256-bit slice in the mask merge; 0 at hop 1, which
 *                     recomputes its neighbours' ranks);
 *   delta_sum[h-1]    the sum of |D_{h-1}(u)| over the E_h edge-merges (the
 *                     ranks the paper's messages carry; = E_1 at hop 1);
 *   new_entries[h-1]  |D_h|: ADS entries gained at hop h.
 * The model's bytes of hop h are 8 A_h + 4 E_h + 8 delta_sum + 16 k A_h +
 * 12 |D_h| (row offsets, columns, neighbour delta ranks, own sketch read and
 * write, ADS id and weight).  Host arrays of cap entries; any may be NULL.
 */
int fl_hop_model(const fl_graph* g, int64_t cap, int64_t* n_hops, int64_t* edge_merges, int64_t* merging,
                 int64_t* delta_read, int64_t* delta_sum, int64_t* new_entries);

/*
 * fl_assign_nearest_noalloc -- nearest open facility of every vertex without
 * any device allocation.  (The paper has no counterpart: this is a deployment
 * variant of fl_assign_clients for callers that cannot let a library call
 * cudaMalloc -- applications that reserve the whole device for their own
 * memory pool, and latency-critical loops that cannot take an allocation's
 * implicit synchronisation.)
 *   n, row_off, cols, nnz   CSR as for fl_graph_create, in DEVICE memory;
 *                           1 <= n <= 1048576 (the fixed scratch), else
 *                           FL_EINVAL; the CSR is validated (FL_EINVAL).
 *   open                    uint8[n] device memory, nonzero = open facility.
 *   assign_out, dist_out    int32[n] device memory (either may be NULL):
 *                           smallest-id nearest open facility and its hop
 *                           distance, -1 where none is reachable.
 *   stream                  cudaStream_t for all work; returns after it ends.
 * Scratch (about 28 MB) is one fixed device array of the library, held by
 * every GPU that loads it until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture on the device.  Every call
 * synchronises `stream` several times: after validating the CSR and once per
 * BFS level, to read the next frontier's size into host memory, so no call
 * can be captured into a CUDA graph.  All calls
 * share the array and each clears what must start at zero; calls that
 * overlap on the GPU race.
 */
int fl_assign_nearest_noalloc(int64_t n, const int64_t* row_off, const int32_t* cols, int64_t nnz,
                              const uint8_t* open, int32_t* assign_out, int32_t* dist_out, void* stream);

/*
 * Batches: many instances solved in one pass (one set of launches and
 * synchronisations for all of them).  Each instance is a connected part of
 * one device graph; ranks r(v) and priorities pi(f) use the instance's own
 * vertex ids, and the instances share no vertex or edge, so every result is
 * the one the plain fl_* sequence gives for that instance alone (Sections 3.1, 4.1:
 * the objective and the conflict graph H-bar of Alg. 3 decompose over
 * components).
 *
 * fl_batch_create_union -- a batch of independent graphs (one instance
 * each).  Graph i: n_of[i] >= 1 vertices, nnz_of[i] CSR entries, row
 * offsets row_off[i] (int64[n_of[i]+1], from 0 to nnz_of[i]) and columns
 * cols[i] (int32, in [0, n_of[i])), all in the memory mem_kind names.  The
 * union (at most 2^31-1 vertices) is copied and kept on the device; instance
 * i occupies vertices [off_i, off_i + n_of[i]), off_i = n_of[0]+..+n_of[i-1].
 * FL_EINVAL on a bad CSR or a column outside its graph.
 */
typedef struct fl_batch fl_batch;
int fl_batch_create_union(int n_graphs, const int64_t* n_of, const int64_t* nnz_of, const int64_t* const* row_off,
                          const int32_t* const* cols, int mem_kind, void* cuda_stream, fl_batch** out);

/*
 * fl_batch_create_replicas -- up to n_inst instances (each with its own
 * costs and client set) on the resident graph g, whose sketches are built and
 * shared: one kernel reads every instance's radius off g's ADS; keys, MIS and
 * assignment run on device copies of g's CSR (n_inst * n at most 2^31-1
 * vertices).  Instance i occupies vertices [i*n, (i+1)*n).  The batch's work
 * runs on cuda_stream (NULL: g's stream), so batches on different streams
 * overlap on the device; they only read g.  g must outlive the batch;
 * rebuilding g's sketches is allowed between solves (the solve checks k and
 * seed against the build).
 */
int fl_batch_create_replicas(fl_graph* g, int n_inst, void* cuda_stream, fl_batch** out);

/*
 * fl_batch_solve -- solve the first n_active instances (all of them for a
 * union batch; 1..n_inst for a replica batch, whose cost of a solve then
 * scales with n_active): sketches (union batches build them here with k and
 * seed; replica batches require g's build to have used the same k and seed,
 * else FL_ESTATE), radii (Eq. 1), keys, MIS (Alg. 6 reading), assignment and
 * objective, as fl_compute_radii ... fl_objective.
 *   cost, client     float64 / uint8 [N] (N = the vertex count of the first
 *                    n_active instances, instance-major as placed by the
 *                    create call), memory as mem_kind says; cost > 0 finite
 *                    for facilities, +inf otherwise (FL_EINVAL).
 *   open_out         uint8[N] or NULL.
 *   assign_out       int32[N] or NULL: nearest open facility as an id of the
 *                    vertex's own instance, -1 if none is reachable.
 *   dist_out         int32[N] or NULL.
 *   n_open, objective, dist_sum, n_unserved   per instance, HOST arrays of
 *                    n_active entries (any may be NULL), as
 *                    fl_open_facilities and fl_objective give them.
 */
int fl_batch_solve(fl_batch* b, int n_active, int k, uint64_t seed, const double* cost, const uint8_t* client,
                   uint8_t* open_out, int32_t* assign_out, int32_t* dist_out, int64_t* n_open, double* objective,
                   int64_t* dist_sum, int64_t* n_unserved, int mem_kind);

/* fl_batch_info -- number of instances and total vertices N of a batch. */
int fl_batch_info(const fl_batch* b, int64_t* n_inst, int64_t* n_total);

/* fl_batch_destroy -- free the batch (not the graph of a replica batch). */
/* fl_batch_set_schedule -- the schedule of the batch's union graph (see
   fl_set_schedule). */
int fl_batch_set_schedule(fl_batch* b, const fl_schedule* sched);
int fl_batch_destroy(fl_batch* b);

/* fl_status_str -- static text for a status code. */
const char* fl_status_str(int status);

/* fl_last_error -- copy the calling thread's last error message into buf
   (NUL-terminated, truncated to len); returns the last status code. */
int fl_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* FL_H */
