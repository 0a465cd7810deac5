/*
 * ch.h - C ABI of the GB300 contraction-hierarchy library (libch.so).
 *
 * Round-synchronous contraction-hierarchy (CH) construction and batched CH
 * s-t distance queries, after "Parallel Contraction Hierarchies Can Be
 * Efficient and Scalable" (arXiv 2412.18008). Every step runs in CUDA
 * kernels for sm_103a on one GPU; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *   - Return value: CH_OK (0) or a negative CH_E* code. On error nothing is
 *     written to output handles, and ch_last_error() describes the failure
 *     (a thread-local string owned by the library, valid until the calling
 *     thread's next call into it).
 *   - Vertex ids are uint32 in [0, n). Weights are uint32 in
 *     [1, 0xFFFFFFFE]. CH_INF (0xFFFFFFFF) means "unreachable". Distances
 *     are exact sums; a distance >= 2^32 - 1 is reported as CH_INF.
 *   - The caller owns every input and output buffer it passes; the library
 *     owns ch_t and all device memory behind it until ch_free().
 *   - Everything is deterministic: the same graph and parameters give a
 *     bitwise-identical hierarchy and identical query answers.
 *   - A handle keeps one set of query work buffers: query batches on one
 *     ch_t must not overlap in time (issue them on one stream, or wait
 *     between streams). Separate handles are independent. No call may race
 *     with ch_free() of the same handle.
 */
#ifndef GB300_CH_H
#define GB300_CH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CH_OK 0
#define CH_EINVAL (-1)    /* bad argument, id out of range, weight 0 or 0xFFFFFFFF */
#define CH_ENOMEM (-2)    /* device or host allocation failed */
#define CH_ECUDA (-3)     /* a CUDA call failed (message in ch_last_error) */
#define CH_ETIMEOUT (-4)  /* a bounded device-side wait expired */
#define CH_ERANGE (-5)    /* a size limit of this library was exceeded */
#define CH_EAGAIN (-6)    /* no room right now (query server): retry after polling */

#define CH_INF 0xFFFFFFFFu

/* Tie-break label of the selection key (Alg. 5 breaks ties "by the label of
 * each vertex"): CH_TIE_HASHED uses the MurmurHash3 32-bit finaliser of
 * (id XOR tie_seed), a bijection; CH_TIE_ID uses the id itself. */
#define CH_TIE_HASHED 0u
#define CH_TIE_ID 1u

/* Vertex score: CH_PRIO_EDGE_DIFF is the edge difference of Alg. 4.
 * CH_PRIO_LEARNED (no counterpart in the paper) replaces it by
 * round(1024 * MLP(features)), an MLP 12 -> 64 -> 64 -> 1 over the integer
 * features of the rescored vertex (see ch_export_trace), BF16 weights on the
 * tensor cores with FP32 accumulation. The edge difference is still computed
 * (it is a feature). Any priority yields a hierarchy with exact distances. */
#define CH_PRIO_EDGE_DIFF 0u
#define CH_PRIO_LEARNED 1u
/* CH_PRIO_COMPOSITE: the combination Sec. 3.2 names (edge difference,
 * vertex degree, hop distance, hierarchy depth; no weights given), read as
 * 4 * ED + (|N_in| + |N_out|) + 8 * depth, clamped to +-2^30, where depth is
 * 1 + the largest depth among contracted neighbours (0 if none). Hop counts
 * per overlay edge are not kept, so the hop-distance term is left out. */
#define CH_PRIO_COMPOSITE 2u

/* MLP parameters, FP32, in this order: W1[12][64] (input-major), b1[64],
 * W2[64][64] (input-major), b2[64], W3[64], b3. */
#define CH_MLP_NPARAM 5057u
#define CH_NFEAT 12u

/* Input graph, a directed out-CSR (Sec. 4.1: "our input graph is given in
 * the CSR format"). offsets[n+1] (offsets[0] = 0, non-decreasing,
 * offsets[n] = m), targets[m], weights[m]. Self-loops are dropped and
 * parallel edges merged by minimum weight. Pointers are host memory when
 * on_device = 0 and device memory of the current device when on_device = 1.
 * The library only reads them, and only during ch_build. */
typedef struct {
    uint32_t n;
    uint64_t m;
    const uint64_t *offsets;
    const uint32_t *targets;
    const uint32_t *weights;
    int32_t on_device;
} ch_graph_t;

/* Construction parameters. Fill with ch_default_params() first.
 *   hop_limit  H of the witness test: a candidate shortcut (v1, u, v2) is kept
 *              iff w(v1,u) + w(u,v2) <= d_H(v1, v2), the least weight of a
 *              walk with at most H edges in the current overlay graph
 *              (Alg. 3, 4, 6 with a hop bound in place of the unstated
 *              settled-vertex bound). Any H >= 0 yields exact distances;
 *              default 5.
 *   priority   CH_PRIO_EDGE_DIFF (default), CH_PRIO_LEARNED or CH_PRIO_COMPOSITE.
 *   tie_break  CH_TIE_HASHED (default) or CH_TIE_ID; tie_seed feeds the hash.
 *   max_candidates_per_vertex  Cmax: a rescored vertex u with
 *              |N_in(u)| * |N_out(u)| > Cmax is not eligible (not scored,
 *              never selected) until a later rescoring finds it within the
 *              bound. When a round finds no eligible vertex, the live
 *              vertices form the core: they get that round's index as their
 *              level (and score INT32_MAX - 1), their overlay edges become
 *              E_up and E_down, and construction stops. Queries then also
 *              search the core, so distances stay exact. UINT64_MAX (the
 *              default) contracts every vertex.
 *   stream     cudaStream_t the build runs on (NULL: the legacy stream).
 *              ch_build returns after the work on it has finished.
 *   mlp_weights  host pointer to CH_MLP_NPARAM floats (CH_PRIO_LEARNED only;
 *              read during ch_build).
 *   trace      nonzero: record one row per rescoring (its features) and the
 *              priority each rescoring produced, for ch_export_trace.
 *   witness_route_deg  a witness source whose middles' out-degrees sum above
 *              this runs on a block (8 warps) instead of one warp; 0 = 64.
 *              Performance only: the hierarchy does not depend on it.
 *   witness_ball_limit  θ, the settled-vertex cap of Alg. 3 read per hop
 *              level: a witness search keeps only labels below its source's
 *              heaviest candidate weight and stops after the first hop level
 *              at which more than θ vertices (the source included) hold one;
 *              the distances of that level replace d_H. Still upper bounds
 *              on real walks, so distances stay exact (only more shortcuts
 *              may be kept). 0 = no bound (the default).
 *   witness_memo_limit  nonzero: witness distances are memoised across
 *              phases and rounds (Alg. 3's dist map, Sec. 4.2). A source
 *              searches only for targets whose pair has no recorded
 *              distance, keeping labels below its new targets' heaviest
 *              candidate weight; a source with none is not searched. The
 *              value recorded is the label the search held, else INF.
 *              Decisions read the map. The map is cleared after any round
 *              that leaves more than this many pairs in it. Every recorded
 *              value is the weight of a real walk (or INF), so distances
 *              stay exact. The map takes 12 bytes per slot; it keeps at
 *              least twice (its pairs + 8 per input edge) slots, growing
 *              between rounds, and a round that overfills it fails with
 *              CH_ENOMEM.
 *              0 = off (the default).
 *   witness_level_work  W, a bound on a hop-limited witness search's work
 *              (not in the paper; for power-law graphs): a hop level from
 *              the second on whose frontier (the vertices whose label
 *              dropped in the level before) has more than W out-edges in
 *              total is not run, and the labels of the level before are the
 *              result. Still upper bounds on real walks, so distances stay
 *              exact. 0 = no bound (the default). A bound of 0 itself would
 *              leave only the first hop level, which is the search of
 *              hop_limit = 1: pass that instead.
 *   witness_prune  nonzero: after each round's rescoring searches, every
 *              overlay edge (s, v) heavier than the distance recorded for a
 *              pair (s, v) of those searches is deleted (Alg. 3's last step),
 *              and the scores are taken on the pruned overlay. The searches'
 *              label bound then also covers the direct edges (s, v) to their
 *              new targets (without a ball bound). A pruned edge lies on no
 *              shortest path, so distances stay exact. Uses the distance map
 *              of witness_memo_limit (held for one phase when that is 0).
 *   witness_settle_cap  θ > 0: the witness search is Alg. 3's own, a
 *              Dijkstra from the source that stops once its targets or θ
 *              vertices (the source included) are settled, equal labels
 *              settled in id order; an unsettled target's distance is INF.
 *              hop_limit and witness_level_work do not apply, and a ball
 *              bound is an error (CH_EINVAL). 0 = the hop-limited search. */
typedef struct {
    uint32_t hop_limit;
    uint32_t priority;
    uint32_t tie_break;
    uint32_t tie_seed;
    uint64_t max_candidates_per_vertex;
    void *stream;
    const float *mlp_weights;
    int32_t trace;
    uint32_t witness_route_deg;
    uint32_t witness_ball_limit;
    uint32_t witness_memo_limit;
    uint32_t witness_level_work;
    uint32_t witness_prune;
    uint32_t witness_settle_cap;
    uint32_t reserved;  /* 0 */
} ch_params_t;

/* Training parameters of ch_mlp_train (Adam, mean squared error). */
typedef struct {
    uint32_t epochs;   /* passes over the samples; 0 = compute the gradient of the first batch only */
    uint32_t batch;    /* samples per step */
    float lr, beta1, beta2, eps;
} ch_train_params_t;

typedef struct ch_s ch_t;

/* Summary of a built hierarchy. */
typedef struct {
    uint32_t n;             /* vertices */
    uint64_t m_input;       /* edges after normalisation */
    uint32_t rounds;        /* contraction rounds (= levels) */
    uint64_t shortcuts;     /* shortcuts inserted over all rounds */
    uint64_t up_edges;      /* |E_up|: out-edges of each vertex at its contraction */
    uint64_t down_edges;    /* |E_down|: in-edges of each vertex at its contraction */
    double build_ms;        /* device time of ch_build, ms (CUDA events) */
    uint64_t witness_sources;   /* witness searches run, score + contract */
    uint64_t witness_fallback;  /* of which outgrew a warp's shared-memory tables */
    /* Device time per phase, ms, summed over rounds (CUDA events on the
     * build stream): input normalisation, rescoring (steps 1-2), selection,
     * contraction bookkeeping, contraction witness searches, overlay update,
     * ranking and CSR construction. */
    double normalise_ms, score_ms, select_ms, prep_ms, contract_ms, update_ms, postprocess_ms;
    /* The witness-search kernels alone (both phases): device time, launch
     * count, and algorithmic bytes read: 4 per search (source id), 12 per
     * vertex whose out-list is read (offset + degree), 8 per adjacency entry
     * read (id + weight). */
    double witness_ms;
    uint64_t witness_launches;
    uint64_t witness_bytes;
    uint64_t witness_dense;     /* of which outgrew a block's tables too (global-memory path) */
    uint64_t trace_rows;        /* rescorings recorded (params.trace or CH_PRIO_LEARNED) */
    uint64_t core_vertices;     /* vertices left uncontracted (finite max_candidates_per_vertex) */
} ch_stats_t;

/* Number of per-round statistics fields written by ch_get_round_stats, in
 * this order: affected |A_r|, score sources |N_in(A_r)|, selected |V_F|,
 * contract sources |N_in(V_F)|, candidates (in x out pairs of V_F, v1 != v2),
 * kept (pass the witness test), merged (distinct (v1, v2) among kept),
 * inserted (shortcuts written), live vertices after, live edges after. */
#define CH_NSTAT 10u

void ch_default_params(ch_params_t *p);

/* Build a contraction hierarchy of `g` (Alg. 2: rounds of LocalSearch,
 * Score, Select, Contract until the overlay is empty; then Postprocess,
 * which ranks vertices by (level, score, id)). On success *out receives a
 * new handle. Errors: CH_EINVAL for a malformed graph or parameter,
 * CH_ENOMEM, CH_ECUDA, CH_ERANGE (more than 2^32 - 1 hierarchy edges). */
int ch_build(const ch_graph_t *g, const ch_params_t *params, ch_t **out);

/* Batched s-t distances (Sec. 5): for i < k, dist_out[i] = length of a
 * shortest path src[i] -> dst[i] in the input graph, via the upward search
 * from src[i] over E_up and from dst[i] over reversed E_down, minimised over
 * the vertices both reach. src, dst, dist_out (uint32[k]) and settled_out
 * (uint32[k] or NULL: number of vertices the two searches reached, the
 * paper's "query iterations") are DEVICE pointers; the work is enqueued on
 * `stream` (a cudaStream_t, NULL = legacy stream) and the call returns
 * without waiting. Ids >= n give CH_EINVAL for the whole batch (checked on
 * the device; the status is returned by the next synchronising call on the
 * handle, or by ch_query_status). k = 0 is a no-op. */
int ch_query_batch(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k,
                   uint32_t *dist_out, uint32_t *settled_out, void *stream);

/* Same as ch_query_batch with HOST pointers: copies the batch to the device,
 * runs it, copies the answers back, and returns when they are in dist_out. */
int ch_query_batch_host(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k,
                        uint32_t *dist_out, uint32_t *settled_out);

/* Largest batch ch_query_batch_static accepts. */
#define CH_STATIC_QUERY_MAX (1u << 18)

/* The same batched s-t distances as ch_query_batch (device pointers, async on
 * `stream`, no search-space sizes), for callers that must not allocate
 * device memory: a serving thread that may not block on the device-wide
 * synchronisation an allocation can imply, or a process whose device memory
 * is entirely reserved by another allocator. The paper has no counterpart;
 * this is plumbing of this library.
 *
 * The call allocates nothing: its per-call scratch (work counters and the
 * list of queries that outgrow the shared-memory search) is a file-scope
 * device array of about 1 MiB, which every GPU that loads the library holds
 * until the process exits. The first call on a device resolves that array's
 * device address (cudaGetSymbolAddress) with the device current, so make
 * the first call on each device before any stream capture. All calls on a
 * device share the array, which keeps the last call's contents (the call
 * clears the counters it needs): calls whose work overlaps on the GPU race
 * on it, so serialise them (one stream, or events), across handles too.
 * The hierarchy's device must be the current device (the scratch address is
 * resolved per current device). Errors: CH_ERANGE when
 * k > CH_STATIC_QUERY_MAX; CH_EINVAL when another device is current; ids >= n
 * are reported by ch_query_status as for ch_query_batch. */
int ch_query_batch_static(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k,
                          uint32_t *dist_out, void *stream);

/* Waits for `stream` and reports (then clears) a device-side error recorded
 * by earlier ch_query_batch calls on this handle. */
int ch_query_status(ch_t *ch, void *stream);

/* One-to-many distances from s to each of k targets (Sec. 5's query for
 * every pair (s, dst[i])): dst and dist_out are device pointers, the call
 * is asynchronous on `stream` like ch_query_batch and follows its no-overlap
 * rule. CH_EINVAL if s >= n; target ids >= n are reported by
 * ch_query_status. */
int ch_query_one_to_many(ch_t *ch, uint32_t s, const uint32_t *dst, uint64_t k,
                         uint32_t *dist_out, void *stream);

/* One-to-all distances (the PHAST scheme the paper cites for single-source
 * distances on a CH, Sec. 5): for each of the k sources src[i],
 * dist_out[i * n + v] = length of a shortest path src[i] -> v in the input
 * graph, for every vertex v (0xFFFFFFFF if unreachable). src (uint32[k]) and
 * dist_out (uint32[k * n], row-major, caller-owned) are DEVICE pointers; the
 * work is enqueued on `stream`. The sweeps run over the rank order, 16
 * sources at a time, in library-owned scratch of 64 bytes per vertex, so
 * calls on one handle must not overlap on the GPU. A hierarchy with a core
 * iterates the core on the host's command, so the call then waits for
 * `stream` once per core pass. Ids >= n are reported by ch_query_status as
 * for ch_query_batch (that source's row is left all 0xFFFFFFFF). k = 0 is a
 * no-op. */
int ch_one_to_all(ch_t *ch, const uint32_t *src, uint64_t k, uint32_t *dist_out, void *stream);

/* Saves a built hierarchy to `path` (binary, little-endian; everything
 * ch_query_batch, ch_export and ch_get_stats use, not learned-priority
 * traces) and loads one back onto the current device. CH_EINVAL on I/O
 * errors, a file that is not a saved hierarchy, or a truncated or
 * inconsistent one; on error nothing is written to *out. */
int ch_save(const ch_t *ch, const char *path);
int ch_load(const char *path, ch_t **out);

/* ---- Query kernel configuration and autotuning (performance only) ----
 *
 * One block runs one query at a time (Sec. 5's two upward searches, level
 * by level), its labels in a shared-memory hash table. The layout says how a
 * level's out-edges are spread over the block: CH_QUERY_BLOCK_FLAT over all
 * its threads (block-wide scan, two barriers per tile of frontier entries),
 * CH_QUERY_WARP_FLAT per warp (entries dealt to warps round-robin, a warp
 * spreads its entries' edges over its lanes; one barrier per level).
 * threads is 128 or 256. small_first = 1 runs a first pass on 2048-slot
 * tables, which fit twice as many blocks per SM, and redoes only the
 * queries that overflow them on 4096-slot tables; 0 uses 4096-slot tables
 * only. Queries that overflow those go to a kernel with per-vertex label
 * arrays. stall = 1 (warp layout only) skips expanding a vertex whose label
 * a reached higher neighbour already beats through one edge ("stall on
 * demand"; it applies to pruned searches, not to those that report search-
 * space sizes). delta > 0 (with stall = 1 only, so for pruned searches)
 * orders each search's levels like delta-stepping: a level expands only the
 * queued vertices whose label is at most the least queued label of their
 * direction plus delta, and keeps the others queued, so fewer vertices are
 * expanded again after a later improvement; delta = 0 expands every queued
 * vertex. A built or loaded hierarchy starts with the warp layout, 256
 * threads, small_first 1, stall 1 and delta = 128 x its weight scale (the
 * median weight of 1024 evenly spaced E_up edges; delta = 0 when it has a
 * core, whose searches outgrow the shared tables anyway). Every
 * configuration gives the same answers and search-space sizes. */
#define CH_QUERY_BLOCK_FLAT 0u
#define CH_QUERY_WARP_FLAT 1u
typedef struct {
    uint32_t layout;
    uint32_t threads;
    uint32_t small_first;
    uint32_t stall;
    uint32_t delta;
} ch_query_config_t;

int ch_set_query_config(ch_t *ch, const ch_query_config_t *cfg);  /* CH_EINVAL on other values */
int ch_get_query_config(const ch_t *ch, ch_query_config_t *cfg);

/* Times each configuration on `sample` seeded uniform random queries (a
 * warm-up run, then one run timed with CUDA events on `stream`) and keeps
 * the fastest for the handle. ms_out (or NULL) receives the
 * CH_QUERY_AUTOTUNE_CONFIGS times: index 4 * small_first +
 * 2 * (layout == WARP_FLAT) + (threads == 256) without stalling or delta;
 * then 8 + 2 * small_first + (threads == 256) for the warp layout with
 * stalling and no delta; then 12, 13, 14 for the warp layout, 256 threads,
 * small_first 1, stalling, and delta = 64, 128, 256 x the weight scale.
 * chosen (or NULL) receives the configuration kept. Waits for `stream`. */
#define CH_QUERY_AUTOTUNE_CONFIGS 15
int ch_query_autotune(ch_t *ch, uint64_t sample, uint32_t seed, void *stream,
                      ch_query_config_t *chosen, double *ms_out);

/* ---- Build autotuning ----
 *
 * Builds `graph` once per (hop limit, witness_route_deg) pair of the two
 * lists, other parameters as in `params` (NULL: defaults), and times each
 * build (ch_stats_t.build_ms) and a batch of `sample` seeded uniform random
 * queries on it (a warm-up run, then one run timed with CUDA events on
 * params->stream). A candidate's cost is
 *     build_ms + query_ms * queries_per_build / sample;
 * the cheapest hierarchy is returned in *out and the others are freed.
 * results (or NULL) receives one row per candidate, hop limits outer, and
 * *chosen (or NULL) the index of the kept one. The hop limit changes the
 * hierarchy (every hop limit gives exact distances); the routing threshold
 * does not. */
typedef struct {
    uint32_t hop_limit;
    uint32_t witness_route_deg;
    double build_ms;
    double query_ms;
    double cost;
    uint64_t shortcuts;
    uint64_t core_vertices;
} ch_tune_row_t;

int ch_build_autotune(const ch_graph_t *graph, const ch_params_t *params,
                      const uint32_t *hop_limits, uint32_t n_hop,
                      const uint32_t *route_degs, uint32_t n_route, uint64_t sample,
                      double queries_per_build, ch_t **out, ch_tune_row_t *results,
                      uint32_t *chosen);

/* Work of the query searches since the previous call (then cleared), summed
 * over the handle's batches: out[0] = queued entries expanded (a stalled
 * entry counts: its stall test read it), out[1] = adjacency entries scanned,
 * the stall tests' included. Waits for `stream`. */
int ch_query_work(ch_t *ch, void *stream, uint64_t out[2]);

/* ---- Query batches as CUDA graphs ----
 *
 * ch_query_graph_create captures one ch_query_batch call on fixed device
 * buffers (k queries from src/dst to dist_out) into an executable CUDA graph,
 * in the handle's current query configuration; ch_query_graph_launch replays
 * it on `stream` (one graph launch in place of the batch's API calls) and
 * answers whatever src/dst hold when it runs. Replays use the handle's query
 * work buffers, so they follow ch_query_batch's no-overlap rule. The graph
 * must be freed before the handle. */
typedef struct ch_query_graph_s ch_query_graph_t;
int ch_query_graph_create(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k,
                          uint32_t *dist_out, ch_query_graph_t **out);
int ch_query_graph_launch(ch_query_graph_t *g, void *stream);
void ch_query_graph_free(ch_query_graph_t *g);

int ch_get_stats(const ch_t *ch, ch_stats_t *out);

/* Copies min(rounds, max_rounds) rows of CH_NSTAT uint64 values to `out`. */
int ch_get_round_stats(const ch_t *ch, uint64_t *out, uint32_t max_rounds);

/* Per-round device time (ms, CUDA events on the build stream), CH_NTIME
 * doubles per round in this order: rescoring (steps 1-2), selection,
 * contraction bookkeeping, contraction witness searches, overlay update,
 * witness-search kernels alone (both phases). The per-round breakdown of
 * the paper's Sec. 6 experiments. */
#define CH_NTIME 6u
int ch_get_round_times(const ch_t *ch, double *out, uint32_t max_rounds);

/* Core distance table (the partial hierarchy of Sec. 3: a candidate bound
 * max_candidates_per_vertex leaves a core; its queries are the paper's
 * core-aware queries). Computes, for every pair of core vertices, the
 * shortest-path distance between them (one search per core vertex inside
 * the core, on the device) and keeps it with the hierarchy: core_size^2
 * uint32 in device memory. From then on ch_query_batch and
 * ch_query_batch_static stop both upward searches at the core's vertices
 * and join them through the table, min over core entries c1 of s's search
 * and c2 of t's of d_s(c1) + table(c1, c2) + d_t(c2), besides the meetings
 * below the core; answers are unchanged, search spaces smaller (a query
 * with more than one tile of core entries in either direction falls back
 * to the search inside the core). Synchronous on `stream`. Errors:
 * CH_ERANGE when core_size^2 * 4 > max_bytes (nothing is kept); a handle
 * without a core keeps no table. The table is not saved by ch_save. */
int ch_core_table(ch_t *ch, uint64_t max_bytes, void *stream);

/* Copies the hierarchy to HOST buffers; any pointer may be NULL to skip it.
 *   level[n]    round in which each vertex was contracted
 *   priority[n] its score (int32) when it was contracted
 *   rank[n]     its position in the (level, score, id) order
 *   shortcuts   5 x uint32 per shortcut: (round, v1, v2, w, via), sorted by
 *               (round, v1, v2); ch_stats_t.shortcuts rows
 *   up          3 x uint32 per upward edge (u, x, w), sorted by (u, x);
 *               ch_stats_t.up_edges rows
 *   down        3 x uint32 per downward edge (x, u, w), sorted by (u, x);
 *               ch_stats_t.down_edges rows */
int ch_export(const ch_t *ch, uint32_t *level, int32_t *priority, uint32_t *rank,
              uint32_t *shortcuts, uint32_t *up, uint32_t *down);

/* Learned-priority data of a build made with params.trace (or the learned
 * priority), to HOST buffers; any pointer may be NULL.
 *   rows     14 int64 per rescoring, in rescoring order within each round:
 *            round, vertex, then its 12 features on the overlay of that
 *            round: kept pairs S, |N_in|, |N_out|, distinct neighbours, edge
 *            difference S - |N_in| - |N_out|, incident edges removed by
 *            earlier contractions, hierarchy depth (1 + the largest depth
 *            among contracted neighbours, 0 if none), round,
 *            |N_in| * |N_out|, degree in the normalised input, times
 *            rescored before, mean incident weight (integer division).
 *            Rows of one round are sorted by vertex.
 *   prio     per row, the int32 priority the rescoring produced.
 *   labels   per vertex (n), the training label: its edge difference at its
 *            last rescoring plus its depth, both at its contraction.
 * ch_stats_t.trace_rows rows. */
int ch_export_trace(const ch_t *ch, int64_t *rows, int32_t *prio, int32_t *labels);

/* Trains the priority MLP on DEVICE data: rows (n x 14 int64 as exported by
 * ch_export_trace), labels (n floats), weights_io (CH_MLP_NPARAM floats, the
 * start point on entry, the trained weights on return). loss_out (host,
 * `epochs` floats, or NULL) receives each epoch's mean squared error; with
 * epochs = 0 nothing is trained and grad_out (device, CH_MLP_NPARAM floats,
 * or NULL) receives the gradient of the mean squared error over the first
 * `batch` rows. Forward passes round as the tensor-core inference does; the
 * sums run in a fixed order, so training is deterministic. Synchronous on
 * `stream`. */
int ch_mlp_train(const int64_t *rows, const float *labels, uint64_t n,
                 const ch_train_params_t *tp, float *weights_io, float *loss_out,
                 float *grad_out, void *stream);

/* Training targets of trace rows on the device (not in the paper; the
 * learned priority's label): y_out[r] = sign(x) * log2(1 + |x|) with
 * x = edge difference + 2 * hierarchy depth of row r (its features 4 and 6),
 * the same transform the features get. The network learns this score; the
 * transform is monotone, so the priority it gives orders vertices as the
 * score does. rows (n x 14 int64) and y_out (n floats) are DEVICE pointers;
 * asynchronous on `stream`. */
int ch_mlp_targets(const int64_t *rows, uint64_t n, float *y_out, void *stream);

/* MLP outputs for trace rows on the device (the inference the learned
 * priority runs, before scaling by 1024): rows (n x 14 int64, device),
 * weights (host, CH_MLP_NPARAM floats), y_out (device, n floats). */
int ch_mlp_forward(const float *weights, const int64_t *rows, uint64_t n, float *y_out,
                   void *stream);

/* ---- Query server: continuous batching (no counterpart in the paper) ----
 *
 * A persistent kernel on its own stream serves requests published by the
 * host: a source and 1..k targets (k = 1 is an s-t query, k > 1
 * one-to-many). The unit of work is one (source, target) pair; its blocks
 * take pairs in publication order, so the targets of a large request are
 * spread over all free blocks and requests that arrive while others are on
 * the device start as blocks free up, overlapping with them. Admission is
 * by memory: targets and answers live in a pool of `pool` entries and the
 * ring holds `ring` requests; ch_server_submit returns CH_EAGAIN when
 * either is full (poll completed requests, then retry). Each answer equals
 * what ch_query_batch returns for the same pair. The kernel's idle wait is
 * bounded by idle_ms: after that long without a published request it ends
 * (its blocks take only published work, so nothing is lost), and the next
 * submit, poll or replay launches it again. Calls that synchronise the
 * whole device (cudaFree, cudaDeviceSynchronize, ch_free of any hierarchy,
 * ...) wait for the running loop, so in the same process they return only
 * after it has ended at the idle limit; keep them out of serving windows or
 * choose a short idle_ms. The handle `ch` must outlive the server. */
typedef struct {
    uint32_t blocks;   /* blocks of the device loop; 0 = as many as are resident at once */
    uint32_t ring;     /* requests in flight at most */
    uint64_t pool;     /* target/answer entries at most */
    uint32_t idle_ms;  /* idle limit of the device loop */
    uint32_t reserved;
} ch_server_params_t;

typedef struct ch_server_s ch_server_t;

int ch_server_start(ch_t *ch, const ch_server_params_t *params, ch_server_t **out);

/* Number of blocks the device loop runs (after the default is resolved). */
uint32_t ch_server_blocks(const ch_server_t *sv);

/* 1 while the device loop's kernel runs, 0 when it has ended at the idle
 * limit (or the server was stopped); the next submit, poll or replay
 * launches it again. CH_ECUDA (with the loop's state in ch_last_error) if
 * it ended on a failed check. */
int ch_server_running(ch_server_t *sv);

/* Copies the k targets (host memory) and publishes the request; *ticket
 * identifies it for ch_server_poll. */
int ch_server_submit(ch_server_t *sv, uint32_t s, const uint32_t *targets, uint32_t k,
                     uint64_t *ticket);

/* *done = 1 and the k answers in dist_out (host) once the request has been
 * served, else *done = 0. device_ns (or NULL) receives its service time on
 * the device. A served ticket is retired by this call. */
int ch_server_poll(ch_server_t *sv, uint64_t ticket, uint32_t *dist_out, int32_t *done,
                   uint64_t *device_ns);

/* Replays a request schedule (host arrays): request i = (src[i], its k[i]
 * targets at targets[toff[i]..]), due at arrival_ns[i] after the call
 * starts. Answers go to answers[toff[i]..]; latency_ns[i] = time from the
 * scheduled arrival to the moment its answers were seen on the host;
 * service_ns[i] (or NULL) = time on the device. Fails with CH_ETIMEOUT
 * after limit_s seconds. */
int ch_server_replay(ch_server_t *sv, uint64_t nreq, const uint32_t *src, const uint32_t *k,
                     const uint64_t *toff, const uint32_t *targets, const uint64_t *arrival_ns,
                     uint32_t *answers, uint64_t *latency_ns, uint64_t *service_ns,
                     double limit_s);

/* Stops the device loop once every published request is served (a bounded
 * wait) and frees the server. Returns CH_ECUDA if an index or capacity
 * check failed in the device loop during the server's life, or a published
 * entry never matched its request. */
int ch_server_stop(ch_server_t *sv);

/* Frees the hierarchy. Waits for the device first (no work that reads the
 * hierarchy may still be in flight; a running server of another hierarchy
 * delays it until that loop ends at its idle limit). The memory goes back
 * to the library's device-memory cache. */
void ch_free(ch_t *ch);

/* Device memory: the library keeps the blocks of freed buffers (hierarchies,
 * build and query temporaries) in a per-device cache and reuses them, so
 * repeated builds allocate nothing from CUDA. ch_trim_memory waits for the
 * current device and returns that device's cached blocks to CUDA; it
 * returns the bytes released. */
size_t ch_trim_memory(void);

/* Failure injection for tests of the error paths (not part of the method).
 * After ch_debug_fail_alloc(k) with k >= 0, the library's device
 * allocations succeed k more times; the next one fails as if the device were
 * out of memory (the call in progress returns CH_ENOMEM and releases what it
 * had allocated), and later allocations succeed again. A negative k turns
 * the injection off. Returns the previous setting (-1 when it was off).
 * Process-wide; makes no CUDA call. */
int64_t ch_debug_fail_alloc(int64_t after);

const char *ch_last_error(void);

/* Library version string, e.g. "gb300-ch 0.1 sm_103a". */
const char *ch_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles, all threads). Instrumentation for benchmarks. */
uint64_t ch_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_CH_H */
