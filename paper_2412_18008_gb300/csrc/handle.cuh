// The library-owned hierarchy handle (ch_t) and the entry points shared by
// the build, query and API translation units.
#pragma once

#include <array>
#include <vector>

#include "common.cuh"

struct ch_server_s;
struct ch_query_graph_s;

struct ch_s {
    uint32_t n = 0;
    uint64_t m_input = 0;
    uint32_t hop_limit = 0;
    int device = 0;

    // Hierarchy in rank order (Sec. 5 layout): vertex i of these arrays is the
    // vertex of rank i; targets are ranks too. up_* hold E_up (out-edges of a
    // vertex at its contraction, all to higher ranks), dn_* hold E_down stored
    // at the lower endpoint (in-edges at contraction, reversed for the
    // backward search).
    gbch::DevBuf<uint32_t> rank;     // [n] id -> rank
    gbch::DevBuf<uint32_t> perm;     // [n] rank -> id
    gbch::DevBuf<uint32_t> up_off;   // [n+1]
    gbch::DevBuf<uint32_t> dn_off;   // [n+1]
    gbch::DevBuf<uint2> up_adj;      // (target rank, weight)
    gbch::DevBuf<uint2> dn_adj;

    // Build products kept for export.
    gbch::DevBuf<uint32_t> level;    // [n]
    gbch::DevBuf<int32_t> prio;      // [n]
    gbch::DevBuf<uint4> sc;          // shortcut log (v1, v2, w, via)
    gbch::DevBuf<uint32_t> sc_round; // round of each log entry
    uint64_t n_shortcuts = 0;
    uint64_t n_up = 0, n_down = 0;

    // learned-priority trace (params.trace): rows, priorities, labels
    gbch::DevBuf<long long> trace;
    gbch::DevBuf<int32_t> trace_prio;
    gbch::DevBuf<int32_t> labels;
    uint64_t trace_rows = 0;   // row slots of the trace (rows of ineligible rescorings marked)
    uint64_t trace_valid = 0;  // rows of eligible rescorings
    uint64_t core_size = 0;

    std::vector<std::array<uint64_t, CH_NSTAT>> round_stats;
    std::vector<std::array<double, CH_NTIME>> round_times;
    ch_stats_t stats{};

    // Per-phase device time of the build (ms) and the witness kernels'
    // algorithmic traffic, for the roofline report.
    double t_score_ms = 0, t_select_ms = 0, t_prep_ms = 0, t_contract_ms = 0,
           t_update_ms = 0, t_norm_ms = 0, t_post_ms = 0;
    double t_witness_ms = 0;
    uint64_t witness_bytes = 0;
    uint64_t witness_launches = 0;

    // Query state.
    gbch::DevBuf<uint32_t> qerr;            // device error word of query batches
    gbch::DevBuf<uint32_t> qwork;           // work counters
    gbch::DevBuf<uint32_t> q_ovf_list;      // overflowed queries
    gbch::DevBuf<uint32_t> q_dense;         // fallback slots
    gbch::DevBuf<unsigned long long> q_stats;  // [0] expansions, [1] edges scanned
    uint32_t q_layout = CH_QUERY_WARP_FLAT;  // query block configuration (performance only)
    uint32_t q_threads = 256;
    uint32_t q_small_first = 1;  // first pass on 2^11-slot tables
    uint32_t q_stall = 1;        // stall on demand (warp layout, pruned searches)
    uint32_t q_delta = 0;        // delta-stepping bucket width (warp layout; 0: off)
    uint32_t q_wscale = 1;       // weight scale: median of sampled E_up weights
    uint32_t q_slots = 0;
    uint64_t q_ovf_cap = 0;
    gbch::DevBuf<uint32_t> q_src_fill;  // repeated source of one-to-many queries

    // One-to-all scratch: interleaved labels of a batch of sources, level
    // boundaries, the core pass's change flag.
    gbch::DevBuf<uint32_t> phast_d;
    gbch::DevBuf<uint32_t> phast_lv;
    gbch::DevBuf<uint32_t> phast_flag;

    // Core distance table (ch_core_table): core_n x core_n shortest-path
    // distances between the core vertices, which are the ranks
    // [core_lo, n); empty when none was built (core_lo = n).
    gbch::DevBuf<uint32_t> core_tab;
    uint32_t core_lo = 0, core_n = 0;
};

namespace gbch {

// Build a hierarchy into `h` (h->n etc. are set by the callee).
void build_hierarchy(ch_s *h, const ch_graph_t *g, const ch_params_t *p);

// Enqueue a query batch on `st` (device pointers).
void query_batch(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                 uint32_t *dist_out, uint32_t *settled_out, cudaStream_t st);

// Prepare query scratch after a build.
void query_init(ch_s *h);

// Enqueue a query batch whose per-call scratch is a static device array.
void query_batch_static(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                        uint32_t *dist_out, cudaStream_t st);

// Query configuration, autotuning, work counters, graphs (query.cu).
void query_set_config(ch_s *h, uint32_t layout, uint32_t threads, uint32_t small_first, uint32_t stall,
                      uint32_t delta);
void query_autotune(ch_s *h, uint64_t sample, uint32_t seed, cudaStream_t st, ch_query_config_t *chosen,
                    double *ms_out);
void query_work(ch_s *h, cudaStream_t st, uint64_t out[2]);
// Device time (ms) of a batch of `sample` seeded random queries (after one warm-up batch).
double query_time_sample(ch_s *h, uint64_t sample, uint32_t seed, cudaStream_t st);
ch_query_graph_s *query_graph_create(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                                     uint32_t *dist_out);
void query_graph_launch(ch_query_graph_s *g, cudaStream_t st);
void query_graph_free(ch_query_graph_s *g);

// Saving and loading, one-to-many queries (io.cu).
void save_hierarchy(const ch_s *h, const char *path);
ch_s *load_hierarchy(const char *path);
void query_one_to_many(ch_s *h, uint32_t s, const uint32_t *dst, uint64_t k, uint32_t *dist_out,
                       cudaStream_t st);

// Core distance table (core.cu); CH_ERANGE when it would exceed max_bytes.
void core_table(ch_s *h, uint64_t max_bytes, cudaStream_t st);

// One-to-all distances for k sources (phast.cu).
void one_to_all(ch_s *h, const uint32_t *src, uint64_t k, uint32_t *dist_out, cudaStream_t st);

// Query server (serve.cu).
ch_server_s *server_new();
void server_delete(ch_server_s *sv);
void server_start(ch_server_s *sv, ch_s *h, const ch_server_params_t *p);
int server_submit(ch_server_s *sv, uint32_t s, const uint32_t *targets, uint32_t k, uint64_t *ticket);
bool server_poll(ch_server_s *sv, uint64_t ticket, uint32_t *out, uint64_t *dev_ns);
int server_stop(ch_server_s *sv, uint32_t *status);
void server_free(ch_server_s *sv);
uint32_t server_blocks(const ch_server_s *sv);
std::string server_state(ch_server_s *sv);
int server_running(ch_server_s *sv);
void server_replay(ch_server_s *sv, uint64_t nreq, const uint32_t *src, const uint32_t *k,
                   const uint64_t *toff, const uint32_t *targets, const uint64_t *arrival_ns,
                   uint32_t *answers, uint64_t *latency_ns, uint64_t *service_ns, double limit_s);

}  // namespace gbch
