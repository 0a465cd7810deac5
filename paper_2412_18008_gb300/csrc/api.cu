// C ABI of libch.so: argument checks, error translation, host-side export.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <numeric>
#include <tuple>

#include "handle.cuh"
#include "mlp.cuh"

namespace gbch {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
// Allocations left before the injected failure; negative = off.
std::atomic<int64_t> g_alloc_countdown{-1};
}

bool inject_alloc_failure() {
    if (g_alloc_countdown.load(std::memory_order_relaxed) < 0) return false;
    // the allocation that takes the count from 0 to -1 fails; later ones do not
    return g_alloc_countdown.fetch_sub(1, std::memory_order_relaxed) == 0;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void kernel_launch_add(int64_t d) { g_launches.fetch_add((uint64_t)d, std::memory_order_relaxed); }

void set_last_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 152;
    if (dev >= 0 && dev < 64) cached[dev] = sms;
    return sms;
}

template <class F>
int guarded(F &&f) {
    try {
        f();
        return CH_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return CH_ENOMEM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return CH_ECUDA;
    }
}

}  // namespace gbch

using namespace gbch;

extern "C" {

const char *ch_last_error(void) { return g_last_error.c_str(); }

const char *ch_version(void) { return "gb300-ch 0.1 sm_103a"; }

uint64_t ch_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t ch_debug_fail_alloc(int64_t after) {
    return g_alloc_countdown.exchange(after < 0 ? -1 : after, std::memory_order_relaxed);
}

void ch_default_params(ch_params_t *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->hop_limit = 5;
    p->priority = CH_PRIO_EDGE_DIFF;
    p->tie_break = CH_TIE_HASHED;
    p->tie_seed = 0;
    p->max_candidates_per_vertex = UINT64_MAX;
    p->stream = nullptr;
    p->mlp_weights = nullptr;
    p->trace = 0;
    p->witness_route_deg = 0;
    p->witness_ball_limit = 0;
    p->witness_memo_limit = 0;
    p->witness_level_work = 0;
    p->witness_prune = 0;
    p->witness_settle_cap = 0;
    p->reserved = 0;
}

int ch_build(const ch_graph_t *g, const ch_params_t *params, ch_t **out) {
    if (!g || !out) {
        g_last_error = "null graph or output handle";
        return CH_EINVAL;
    }
    ch_params_t p;
    if (params) p = *params;
    else ch_default_params(&p);
    if (p.priority != CH_PRIO_EDGE_DIFF && p.priority != CH_PRIO_LEARNED &&
        p.priority != CH_PRIO_COMPOSITE) {
        g_last_error = "unsupported priority mode";
        return CH_EINVAL;
    }
    if (p.priority == CH_PRIO_LEARNED && !p.mlp_weights) {
        g_last_error = "CH_PRIO_LEARNED needs mlp_weights";
        return CH_EINVAL;
    }
    if (p.tie_break > CH_TIE_ID) {
        g_last_error = "unknown tie_break";
        return CH_EINVAL;
    }
    if (p.witness_settle_cap && p.witness_ball_limit) {
        g_last_error = "the settled-vertex cap replaces the hop-limited search and its ball bound";
        return CH_EINVAL;
    }
    if (g->n == 0xFFFFFFFFu) {
        g_last_error = "n must be below 2^32 - 1";
        return CH_ERANGE;
    }
    if (g->n > 0 && (!g->offsets || (g->m > 0 && (!g->targets || !g->weights)))) {
        g_last_error = "null CSR array";
        return CH_EINVAL;
    }
    ch_s *h = new (std::nothrow) ch_s();
    if (!h) {
        g_last_error = "host allocation failed";
        return CH_ENOMEM;
    }
    int rc = guarded([&] {
        CH_CUDA_TRY(cudaGetDevice(&h->device));
        build_hierarchy(h, g, &p);
        query_init(h);
        h->stats.n = h->n;
        h->stats.m_input = h->m_input;
        h->stats.rounds = (uint32_t)h->round_stats.size();
        h->stats.shortcuts = h->n_shortcuts;
        h->stats.up_edges = h->n_up;
        h->stats.down_edges = h->n_down;
        h->stats.normalise_ms = h->t_norm_ms;
        h->stats.score_ms = h->t_score_ms;
        h->stats.select_ms = h->t_select_ms;
        h->stats.prep_ms = h->t_prep_ms;
        h->stats.contract_ms = h->t_contract_ms;
        h->stats.update_ms = h->t_update_ms;
        h->stats.postprocess_ms = h->t_post_ms;
        h->stats.witness_ms = h->t_witness_ms;
        h->stats.witness_launches = h->witness_launches;
        h->stats.witness_bytes = h->witness_bytes;
        h->stats.trace_rows = h->trace_valid;
        h->stats.core_vertices = h->core_size;
    });
    if (rc != CH_OK) {
        delete h;
        cudaGetLastError();
        return rc;
    }
    *out = h;
    return CH_OK;
}

int ch_query_batch(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k,
                   uint32_t *dist_out, uint32_t *settled_out, void *stream) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    if (k == 0) return CH_OK;
    if (!src || !dst || !dist_out) {
        g_last_error = "null query array";
        return CH_EINVAL;
    }
    return guarded([&] {
        query_batch(ch, src, dst, k, dist_out, settled_out, (cudaStream_t)stream);
    });
}

int ch_query_batch_static(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k,
                          uint32_t *dist_out, void *stream) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    if (k > CH_STATIC_QUERY_MAX) {
        g_last_error = "batch larger than CH_STATIC_QUERY_MAX queries";
        return CH_ERANGE;
    }
    if (k == 0) return CH_OK;
    if (!src || !dst || !dist_out) {
        g_last_error = "null query array";
        return CH_EINVAL;
    }
    return guarded([&] {
        query_batch_static(ch, src, dst, k, dist_out, (cudaStream_t)stream);
    });
}

int ch_build_autotune(const ch_graph_t *graph, const ch_params_t *params, const uint32_t *hop_limits,
                      uint32_t n_hop, const uint32_t *route_degs, uint32_t n_route, uint64_t sample,
                      double queries_per_build, ch_t **out, ch_tune_row_t *results, uint32_t *chosen) {
    if (!graph || !out || !hop_limits || !route_degs || n_hop == 0 || n_route == 0 || sample == 0 ||
        !(queries_per_build >= 0)) {
        g_last_error = "bad autotune arguments";
        return CH_EINVAL;
    }
    ch_params_t base;
    if (params) base = *params;
    else ch_default_params(&base);
    ch_t *best = nullptr;
    double best_cost = 0;
    uint32_t best_i = 0;
    for (uint32_t i = 0; i < n_hop; ++i)
        for (uint32_t j = 0; j < n_route; ++j) {
            ch_params_t p = base;
            p.hop_limit = hop_limits[i];
            p.witness_route_deg = route_degs[j];
            ch_t *h = nullptr;
            int rc = ch_build(graph, &p, &h);
            if (rc != CH_OK) {
                if (best) ch_free(best);
                return rc;
            }
            double qms = 0;
            rc = guarded([&] { qms = query_time_sample(h, sample, 1234u + i, (cudaStream_t)p.stream); });
            if (rc != CH_OK) {
                ch_free(h);
                if (best) ch_free(best);
                return rc;
            }
            const double cost = h->stats.build_ms + qms * queries_per_build / (double)sample;
            const uint32_t k = i * n_route + j;
            if (results) {
                results[k].hop_limit = p.hop_limit;
                results[k].witness_route_deg = p.witness_route_deg;
                results[k].build_ms = h->stats.build_ms;
                results[k].query_ms = qms;
                results[k].cost = cost;
                results[k].shortcuts = h->stats.shortcuts;
                results[k].core_vertices = h->stats.core_vertices;
            }
            if (!best || cost < best_cost) {
                if (best) ch_free(best);
                best = h;
                best_cost = cost;
                best_i = k;
            } else {
                ch_free(h);
            }
        }
    *out = best;
    if (chosen) *chosen = best_i;
    return CH_OK;
}

int ch_query_one_to_many(ch_t *ch, uint32_t s, const uint32_t *dst, uint64_t k, uint32_t *dist_out,
                         void *stream) {
    if (!ch || (k && (!dst || !dist_out))) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    if (k && s >= ch->n) {
        g_last_error = "source id out of range";
        return CH_EINVAL;
    }
    return guarded([&] { query_one_to_many(ch, s, dst, k, dist_out, static_cast<cudaStream_t>(stream)); });
}

int ch_one_to_all(ch_t *ch, const uint32_t *src, uint64_t k, uint32_t *dist_out, void *stream) {
    if (!ch || (k && (!src || !dist_out))) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    return guarded([&] { one_to_all(ch, src, k, dist_out, static_cast<cudaStream_t>(stream)); });
}

int ch_save(const ch_t *ch, const char *path) {
    if (!ch || !path) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    return guarded([&] { save_hierarchy(ch, path); });
}

int ch_load(const char *path, ch_t **out) {
    if (!path || !out) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    ch_s *h = nullptr;
    const int rc = guarded([&] { h = load_hierarchy(path); });
    if (rc == CH_OK) *out = h;
    return rc;
}

int ch_set_query_config(ch_t *ch, const ch_query_config_t *cfg) {
    if (!ch || !cfg) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    return guarded([&] { query_set_config(ch, cfg->layout, cfg->threads, cfg->small_first, cfg->stall, cfg->delta); });
}

int ch_get_query_config(const ch_t *ch, ch_query_config_t *cfg) {
    if (!ch || !cfg) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    cfg->layout = ch->q_layout;
    cfg->threads = ch->q_threads;
    cfg->small_first = ch->q_small_first;
    cfg->stall = ch->q_stall;
    cfg->delta = ch->q_delta;
    return CH_OK;
}

int ch_query_autotune(ch_t *ch, uint64_t sample, uint32_t seed, void *stream, ch_query_config_t *chosen,
                      double *ms_out) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    return guarded([&] { query_autotune(ch, sample, seed, static_cast<cudaStream_t>(stream), chosen, ms_out); });
}

int ch_query_work(ch_t *ch, void *stream, uint64_t out[2]) {
    if (!ch || !out) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    return guarded([&] { query_work(ch, static_cast<cudaStream_t>(stream), out); });
}

int ch_query_graph_create(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k, uint32_t *dist_out,
                          ch_query_graph_t **out) {
    if (!ch || !out || (k && (!src || !dst || !dist_out))) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    ch_query_graph_s *g = nullptr;
    const int rc = guarded([&] { g = query_graph_create(ch, src, dst, k, dist_out); });
    if (rc == CH_OK) *out = g;
    return rc;
}

int ch_query_graph_launch(ch_query_graph_t *g, void *stream) {
    if (!g) {
        g_last_error = "null graph";
        return CH_EINVAL;
    }
    return guarded([&] { query_graph_launch(g, static_cast<cudaStream_t>(stream)); });
}

void ch_query_graph_free(ch_query_graph_t *g) {
    if (g) query_graph_free(g);
}

int ch_query_status(ch_t *ch, void *stream) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    uint32_t err = 0;
    int rc = guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        CH_CUDA_TRY(cudaMemcpyAsync(&err, ch->qerr.ptr, 4, cudaMemcpyDeviceToHost, st));
        CH_CUDA_TRY(cudaStreamSynchronize(st));
        if (err) CH_CUDA_TRY(cudaMemsetAsync(ch->qerr.ptr, 0, 4, st));
        CH_CUDA_TRY(cudaStreamSynchronize(st));
    });
    if (rc != CH_OK) return rc;
    if (err & 2u) {
        g_last_error = "internal index check failed in a query kernel";
        return CH_ECUDA;
    }
    if (err) {
        g_last_error = "query vertex id out of range";
        return CH_EINVAL;
    }
    return CH_OK;
}

int ch_query_batch_host(ch_t *ch, const uint32_t *src, const uint32_t *dst, uint64_t k,
                        uint32_t *dist_out, uint32_t *settled_out) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    if (k == 0) return CH_OK;
    if (!src || !dst || !dist_out) {
        g_last_error = "null query array";
        return CH_EINVAL;
    }
    int rc = guarded([&] {
        DevBuf<uint32_t> buf;
        buf.alloc(k * (settled_out ? 4 : 3));
        uint32_t *ds = buf.ptr, *dt = buf.ptr + k, *dd = buf.ptr + 2 * k;
        uint32_t *dset = settled_out ? buf.ptr + 3 * k : nullptr;
        cudaStream_t st = nullptr;
        CH_CUDA_TRY(cudaMemcpyAsync(ds, src, k * 4, cudaMemcpyHostToDevice, st));
        CH_CUDA_TRY(cudaMemcpyAsync(dt, dst, k * 4, cudaMemcpyHostToDevice, st));
        query_batch(ch, ds, dt, k, dd, dset, st);
        CH_CUDA_TRY(cudaMemcpyAsync(dist_out, dd, k * 4, cudaMemcpyDeviceToHost, st));
        if (dset)
            CH_CUDA_TRY(cudaMemcpyAsync(settled_out, dset, k * 4, cudaMemcpyDeviceToHost, st));
        CH_CUDA_TRY(cudaStreamSynchronize(st));
    });
    if (rc != CH_OK) return rc;
    return ch_query_status(ch, nullptr);
}

int ch_get_stats(const ch_t *ch, ch_stats_t *out) {
    if (!ch || !out) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    *out = ch->stats;
    return CH_OK;
}

int ch_get_round_stats(const ch_t *ch, uint64_t *out, uint32_t max_rounds) {
    if (!ch || (!out && max_rounds)) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    const uint32_t r = std::min<uint32_t>(max_rounds, (uint32_t)ch->round_stats.size());
    for (uint32_t i = 0; i < r; ++i)
        for (uint32_t f = 0; f < CH_NSTAT; ++f) out[(size_t)i * CH_NSTAT + f] = ch->round_stats[i][f];
    return CH_OK;
}

int ch_get_round_times(const ch_t *ch, double *out, uint32_t max_rounds) {
    if (!ch || (!out && max_rounds)) {
        g_last_error = "null argument";
        return CH_EINVAL;
    }
    const uint32_t r = std::min<uint32_t>(max_rounds, (uint32_t)ch->round_times.size());
    for (uint32_t i = 0; i < r; ++i)
        for (uint32_t f = 0; f < CH_NTIME; ++f) out[(size_t)i * CH_NTIME + f] = ch->round_times[i][f];
    return CH_OK;
}

int ch_export(const ch_t *ch, uint32_t *level, int32_t *priority, uint32_t *rank,
              uint32_t *shortcuts, uint32_t *up, uint32_t *down) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    return guarded([&] {
        const uint32_t n = ch->n;
        if (level && n) CH_CUDA_TRY(cudaMemcpy(level, ch->level.ptr, n * 4ull, cudaMemcpyDeviceToHost));
        if (priority && n) CH_CUDA_TRY(cudaMemcpy(priority, ch->prio.ptr, n * 4ull, cudaMemcpyDeviceToHost));
        if (rank && n) CH_CUDA_TRY(cudaMemcpy(rank, ch->rank.ptr, n * 4ull, cudaMemcpyDeviceToHost));
        if (shortcuts && ch->n_shortcuts) {
            const uint64_t k = ch->n_shortcuts;
            std::vector<uint4> sc(k);
            std::vector<uint32_t> rr(k);
            CH_CUDA_TRY(cudaMemcpy(sc.data(), ch->sc.ptr, k * sizeof(uint4), cudaMemcpyDeviceToHost));
            CH_CUDA_TRY(cudaMemcpy(rr.data(), ch->sc_round.ptr, k * 4, cudaMemcpyDeviceToHost));
            std::vector<uint64_t> idx(k);
            std::iota(idx.begin(), idx.end(), 0);
            std::sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t b) {
                return std::make_tuple(rr[a], sc[a].x, sc[a].y) < std::make_tuple(rr[b], sc[b].x, sc[b].y);
            });
            for (uint64_t i = 0; i < k; ++i) {
                const uint4 &c = sc[idx[i]];
                uint32_t *o = shortcuts + 5 * i;
                o[0] = rr[idx[i]];
                o[1] = c.x;
                o[2] = c.y;
                o[3] = c.z;
                o[4] = c.w;
            }
        }
        for (int dir = 0; dir < 2; ++dir) {
            uint32_t *dst = dir == 0 ? up : down;
            const uint64_t cnt = dir == 0 ? ch->n_up : ch->n_down;
            if (!dst || !cnt) continue;
            std::vector<uint32_t> off(n + 1), perm(n);
            std::vector<uint2> adj(cnt);
            CH_CUDA_TRY(cudaMemcpy(off.data(), (dir == 0 ? ch->up_off : ch->dn_off).ptr, (n + 1ull) * 4,
                                   cudaMemcpyDeviceToHost));
            CH_CUDA_TRY(cudaMemcpy(adj.data(), (dir == 0 ? ch->up_adj : ch->dn_adj).ptr,
                                   cnt * sizeof(uint2), cudaMemcpyDeviceToHost));
            CH_CUDA_TRY(cudaMemcpy(perm.data(), ch->perm.ptr, n * 4ull, cudaMemcpyDeviceToHost));
            // rows (lower endpoint u, other endpoint x, w), sorted by (u, x)
            std::vector<std::array<uint32_t, 3>> rows;
            rows.reserve(cnt);
            for (uint32_t i = 0; i < n; ++i)
                for (uint32_t j = off[i]; j < off[i + 1]; ++j)
                    rows.push_back({perm[i], perm[adj[j].x], adj[j].y});
            std::sort(rows.begin(), rows.end());
            for (uint64_t i = 0; i < cnt; ++i) {
                uint32_t *o = dst + 3 * i;
                if (dir == 0) {
                    o[0] = rows[i][0];
                    o[1] = rows[i][1];
                } else {
                    o[0] = rows[i][1];
                    o[1] = rows[i][0];
                }
                o[2] = rows[i][2];
            }
        }
    });
}

int ch_export_trace(const ch_t *ch, int64_t *rows, int32_t *prio, int32_t *labels) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    return guarded([&] {
        const uint64_t k = ch->trace_rows;
        if (labels && ch->n) {
            if (ch->labels.count < ch->n) throw Error{CH_EINVAL, "no labels recorded"};
            CH_CUDA_TRY(cudaMemcpy(labels, ch->labels.ptr, ch->n * 4ull, cudaMemcpyDeviceToHost));
        }
        if (!k || (!rows && !prio)) return;
        std::vector<long long> r(k * 14);
        std::vector<int32_t> pr(k);
        CH_CUDA_TRY(cudaMemcpy(r.data(), ch->trace.ptr, k * 14 * sizeof(long long), cudaMemcpyDeviceToHost));
        CH_CUDA_TRY(cudaMemcpy(pr.data(), ch->trace_prio.ptr, k * 4, cudaMemcpyDeviceToHost));
        // rows of rescorings that were not eligible are marked with round -1
        std::vector<uint64_t> idx;
        idx.reserve(ch->trace_valid);
        for (uint64_t i = 0; i < k; ++i)
            if (r[i * 14] >= 0) idx.push_back(i);
        if (idx.size() != ch->trace_valid) throw Error{CH_ECUDA, "internal: trace row count"};
        std::sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t b) {
            return std::make_pair(r[a * 14], r[a * 14 + 1]) < std::make_pair(r[b * 14], r[b * 14 + 1]);
        });
        for (uint64_t i = 0; i < idx.size(); ++i) {
            if (rows)
                for (int c = 0; c < 14; ++c) rows[i * 14 + c] = r[idx[i] * 14 + c];
            if (prio) prio[i] = pr[idx[i]];
        }
    });
}

int ch_mlp_train(const int64_t *rows, const float *labels, uint64_t n, const ch_train_params_t *tp,
                 float *weights_io, float *loss_out, float *grad_out, void *stream) {
    if (!rows || !labels || !tp || !weights_io || n == 0 || tp->batch == 0) {
        g_last_error = "bad training arguments";
        return CH_EINVAL;
    }
    return guarded([&] {
        mlp_train(reinterpret_cast<const long long *>(rows), labels, n, tp, weights_io, loss_out,
                  grad_out, (cudaStream_t)stream);
    });
}

int ch_core_table(ch_t *ch, uint64_t max_bytes, void *stream) {
    if (!ch) {
        g_last_error = "null handle";
        return CH_EINVAL;
    }
    return guarded([&] { core_table(ch, max_bytes, (cudaStream_t)stream); });
}

int ch_mlp_targets(const int64_t *rows, uint64_t n, float *y_out, void *stream) {
    if (n && (!rows || !y_out)) {
        g_last_error = "bad target arguments";
        return CH_EINVAL;
    }
    return guarded([&] {
        mlp_targets(reinterpret_cast<const long long *>(rows), n, y_out, (cudaStream_t)stream);
    });
}

int ch_mlp_forward(const float *weights, const int64_t *rows, uint64_t n, float *y_out,
                   void *stream) {
    if (!weights || (n && (!rows || !y_out))) {
        g_last_error = "bad inference arguments";
        return CH_EINVAL;
    }
    return guarded([&] {
        cudaStream_t st = (cudaStream_t)stream;
        MlpDevice m;
        m.load(weights, st);
        DevBuf<float> x;
        x.alloc(n * 16);
        rows_to_features(reinterpret_cast<const long long *>(rows), n, x.ptr, st);
        m.infer(x.ptr, n, y_out, st);
        CH_CUDA_TRY(cudaStreamSynchronize(st));
    });
}

int ch_server_start(ch_t *ch, const ch_server_params_t *params, ch_server_t **out) {
    if (!ch || !params || !out || params->ring == 0 || params->pool == 0) {
        g_last_error = "bad server arguments";
        return CH_EINVAL;
    }
    ch_server_s *sv = server_new();
    if (!sv) {
        g_last_error = "host allocation failed";
        return CH_ENOMEM;
    }
    const int rc = guarded([&] { server_start(sv, ch, params); });
    if (rc != CH_OK) {
        guarded([&] { server_free(sv); });
        server_delete(sv);
        return rc;
    }
    *out = sv;
    return CH_OK;
}

uint32_t ch_server_blocks(const ch_server_t *sv) { return sv ? server_blocks(sv) : 0; }

int ch_server_running(ch_server_t *sv) {
    if (!sv) {
        g_last_error = "no server";
        return CH_EINVAL;
    }
    int r = 0;
    const int rc = guarded([&] { r = server_running(sv); });
    return rc != CH_OK ? rc : r;
}

int ch_server_submit(ch_server_t *sv, uint32_t s, const uint32_t *targets, uint32_t k,
                     uint64_t *ticket) {
    if (!sv || !targets || !ticket || k == 0) {
        g_last_error = "bad submit arguments";
        return CH_EINVAL;
    }
    int rc = CH_OK;
    const int g = guarded([&] { rc = server_submit(sv, s, targets, k, ticket); });
    if (g != CH_OK) return g;
    if (rc == CH_EAGAIN) g_last_error = "server full";
    return rc;
}

int ch_server_poll(ch_server_t *sv, uint64_t ticket, uint32_t *dist_out, int32_t *done,
                   uint64_t *device_ns) {
    if (!sv || !done) {
        g_last_error = "bad poll arguments";
        return CH_EINVAL;
    }
    return guarded([&] { *done = server_poll(sv, ticket, dist_out, device_ns) ? 1 : 0; });
}

int ch_server_replay(ch_server_t *sv, uint64_t nreq, const uint32_t *src, const uint32_t *k,
                     const uint64_t *toff, const uint32_t *targets, const uint64_t *arrival_ns,
                     uint32_t *answers, uint64_t *latency_ns, uint64_t *service_ns,
                     double limit_s) {
    if (!sv || (nreq && (!src || !k || !toff || !targets || !arrival_ns || !answers || !latency_ns))) {
        g_last_error = "bad replay arguments";
        return CH_EINVAL;
    }
    return guarded([&] {
        server_replay(sv, nreq, src, k, toff, targets, arrival_ns, answers, latency_ns, service_ns,
                      limit_s);
    });
}

int ch_server_stop(ch_server_t *sv) {
    if (!sv) return CH_OK;
    uint32_t status = 0;
    int rc = guarded([&] {
        const int r = server_stop(sv, &status);
        if (r != CH_OK) throw Error{r, "server kernel did not finish within its bounded wait"};
    });
    guarded([&] { server_free(sv); });
    server_delete(sv);
    if (rc != CH_OK) return rc;
    if (status & 2u) {
        g_last_error = "index or capacity check failed in the server loop";
        return CH_ECUDA;
    }
    if (status & 4u) {
        g_last_error = "a published pool entry never matched its request in the server loop";
        return CH_ECUDA;
    }
    return CH_OK;
}

void ch_free(ch_t *ch) {
    if (!ch) return;
    // the hierarchy's memory goes back to the library's cache: no work that
    // reads it may still be in flight
    cudaDeviceSynchronize();
    cudaGetLastError();
    delete ch;
}

size_t ch_trim_memory(void) {
    size_t b = 0;
    guarded([&] { b = dev_trim(); });
    return b;
}

}  // extern "C"
