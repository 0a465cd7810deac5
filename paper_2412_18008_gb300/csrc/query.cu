// Batched CH s-t queries (Sec. 5 of arXiv 2412.18008): an upward search
// from s over E_up and an upward search from t over reversed E_down; the
// answer is the least d_s(v) + d_t(v) over the vertices both searches reach.
//
// The hierarchy is stored in rank order, so both searches run on a DAG whose
// edges all point to higher ranks. Each search is label-correcting: a
// frontier of improved vertices is expanded until no label changes, which
// gives exact shortest distances on any graph with positive weights, and
// the result cannot depend on the order of the relaxations.
//
// One block serves one query at a time and pulls the next index from a
// counter (persistent grid, three blocks per SM). Its labels live in a
// shared-memory hash table whose entries carry both directions' distances,
// so the meeting minimum is one pass over the table. A query whose search
// spaces do not fit is redone by a second kernel that keeps labels in dense
// per-vertex arrays in global memory (one block per array slot).

#include <algorithm>
#include <mutex>
#include <vector>

#include "handle.cuh"
#include "qsearch.cuh"

namespace gbch {
namespace {

constexpr uint64_t Q_CHUNK = 1u << 22;  // queries per launch pair

// (The stalling variants are held to six resident blocks per SM, about 40
// registers a thread, so that six 2^11-slot blocks fit an SM.)
template <bool PRUNE, bool WARP, int TB, bool STALL, bool DELTA = false>
__global__ void __launch_bounds__(QB_THREADS, (STALL || DELTA) ? 6 : 1) k_query_block(QArgs a) {
    extern __shared__ __align__(16) unsigned char qb_raw[];
    QBSmem<TB> &q = *reinterpret_cast<QBSmem<TB> *>(qb_raw);
    const uint32_t tid = threadIdx.x;
    QStat stat;
    qb_clear(q);
    const uint64_t nitems = a.in_list ? a.work[a.in_cnt] : a.k;
    while (true) {
        __syncthreads();
        if (tid == 0) q.item = atomicAdd(&a.work[a.ctr], 1u);
        __syncthreads();
        const uint32_t j = q.item;
        if (j >= nitems) break;
        const uint32_t i = a.in_list ? a.in_list[j] : j;
        if (i >= a.k) {
            if (tid == 0) atomicOr(a.err, QERR_BOUND);
            continue;
        }
        const uint32_t s = a.src[i], t = a.dst[i];
        if (s >= a.n || t >= a.n) {
            if (tid == 0) {
                atomicOr(a.err, QERR_RANGE);
                a.out[i] = INF;
                if (a.settled) a.settled[i] = 0;
            }
            continue;
        }
        const uint32_t rs = a.rank[s], rt = a.rank[t];
        if (rs >= a.n || rt >= a.n) {
            if (tid == 0) {
                atomicOr(a.err, QERR_BOUND);
                a.out[i] = INF;
            }
            continue;
        }
        uint32_t mu, cnt;
        if (!block_query<PRUNE, WARP, TB, STALL, DELTA>(q, a, rs, rt, mu, cnt, stat)) {
            if (tid == 0) a.ovf[atomicAdd(&a.work[a.ovf_cnt], 1u)] = i;
            continue;
        }
        if (tid == 0) {
            a.out[i] = mu;
            if (a.settled) a.settled[i] = cnt;
        }
    }
    qb_flush_stat(stat, a.stats);
}

// Dense fallback: one block per slot; labels in per-vertex arrays.
struct QDense {
    uint32_t *df, *db, *fst, *fa, *fb, *touched;
    uint32_t nslots;
};

__device__ void dense_search(uint32_t root, uint32_t *dist, uint32_t *fst, uint32_t *fa,
                             uint32_t *fb, uint32_t *touched, uint32_t *s_nt, uint32_t *s_nf,
                             const uint32_t *off, const uint2 *adj, uint32_t n,
                             uint32_t n_edges, uint32_t *err, uint32_t &stamp) {
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        dist[root] = 0;
        touched[(*s_nt)++] = root;
        fa[0] = root;
        s_nf[0] = 1;
    }
    __syncthreads();
    uint32_t *cur = fa, *nx = fb;
    uint32_t c = 0;
    while (true) {
        const uint32_t nf = s_nf[c];
        if (nf == 0) break;
        ++stamp;
        __syncthreads();
        if (tid == 0) s_nf[c ^ 1] = 0;
        __syncthreads();
        for (uint32_t f = tid; f < nf; f += blockDim.x) {
            const uint32_t x = cur[f];
            if (x >= n) {
                atomicOr(err, QERR_BOUND);
                continue;
            }
            const uint32_t dx = dist[x];
            const uint32_t jb = off[x], je = off[x + 1];
            if (jb > je || je > n_edges) {
                atomicOr(err, QERR_BOUND);
                continue;
            }
            for (uint32_t j = jb; j < je; ++j) {
                const uint2 e = adj[j];
                const uint32_t nd = sat_add(dx, e.y);
                if (nd == INF) continue;
                if (e.x >= n) {
                    atomicOr(err, QERR_BOUND);
                    continue;
                }
                const uint32_t old = atomicMin(&dist[e.x], nd);
                if (nd < old) {
                    if (old == INF) touched[atomicAdd(s_nt, 1u)] = e.x;
                    if (atomicExch(&fst[e.x], stamp) != stamp) nx[atomicAdd(&s_nf[c ^ 1], 1u)] = e.x;
                }
            }
        }
        __syncthreads();
        uint32_t *t = cur;
        cur = nx;
        nx = t;
        c ^= 1u;
    }
}

__global__ void __launch_bounds__(256) k_query_dense(QArgs a, QDense dn) {
    const size_t base = (size_t)blockIdx.x * a.n;
    uint32_t *df = dn.df + base, *db = dn.db + base, *fst = dn.fst + base;
    uint32_t *fa = dn.fa + base, *fb = dn.fb + base, *touched = dn.touched + 2 * base;
    __shared__ uint32_t s_item, s_nt, s_nf[2], s_mu;
    const uint32_t tid = threadIdx.x;
    const uint32_t novf = a.work[a.ovf_cnt];
    uint32_t stamp = 0;
    while (true) {
        __syncthreads();
        if (tid == 0) {
            s_item = atomicAdd(&a.work[1], 1u);
            s_nt = 0;
            s_mu = INF;
        }
        __syncthreads();
        if (s_item >= novf) break;
        const uint32_t i = a.ovf[s_item];
        const uint32_t rs = a.rank[a.src[i]], rt = a.rank[a.dst[i]];
        if (rs >= a.n || rt >= a.n) {
            if (tid == 0) atomicOr(a.err, QERR_BOUND);
            continue;
        }
        // forward labels live in df, backward in db; touched lists both
        dense_search(rs, df, fst, fa, fb, touched, &s_nt, s_nf, a.up_off, a.up_adj, a.n, a.n_up,
                     a.err, stamp);
        __syncthreads();
        const uint32_t nt_f = s_nt;
        dense_search(rt, db, fst, fa, fb, touched, &s_nt, s_nf, a.dn_off, a.dn_adj, a.n, a.n_dn,
                     a.err, stamp);
        __syncthreads();
        const uint32_t nt = s_nt;
        // The touched list holds each vertex reached forward once (first nt_f
        // entries), then each vertex reached backward once; every meeting
        // vertex is in the forward part.
        uint32_t mu = INF;
        for (uint32_t p = tid; p < nt_f; p += blockDim.x) {
            const uint32_t v = touched[p];
            mu = min(mu, sat_add(df[v], db[v]));
        }
        atomicMin(&s_mu, mu);
        __syncthreads();
        if (tid == 0) {
            a.out[i] = s_mu;
            if (a.settled) a.settled[i] = nt;
        }
        __syncthreads();
        for (uint32_t p = tid; p < nt; p += blockDim.x) {
            const uint32_t v = touched[p];
            df[v] = INF;
            db[v] = INF;
            fst[v] = 0;
        }
    }
}

// Resident blocks per SM of each block-kernel configuration
// [table bits == 11][block-flat, warp-flat, warp-flat with stalling,
// the same with delta-stepping levels][threads == 256], resolved once.
int g_qb_bps[2][4][2] = {{{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}}, {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}}};

template <int TB>
void qb_resolve(int s) {
    const int smem = (int)sizeof(QBSmem<TB>);
    CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<true, true, TB, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<true, false, TB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<false, false, TB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<true, true, TB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<false, true, TB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<true, true, TB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    for (int l = 0; l < 4; ++l)
        for (int t = 0; t < 2; ++t) {
            int b = 0;
            const int threads = t ? 256 : 128;
            if (l == 3) CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_query_block<true, true, TB, true, true>, threads, smem));
            else if (l == 2) CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_query_block<true, true, TB, true>, threads, smem));
            else if (l == 1) CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_query_block<true, true, TB, false>, threads, smem));
            else CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_query_block<true, false, TB, false>, threads, smem));
            g_qb_bps[s][l][t] = std::max(1, b);
        }
}

void qb_resolve_occupancy() {
    if (g_qb_bps[0][0][0] >= 0) return;
    qb_resolve<12>(0);
    qb_resolve<11>(1);
}

template <int TB>
void launch_tb(const QArgs &a, bool prune, bool warp, bool stall, bool delta, int blocks, int threads,
               cudaStream_t st) {
    const size_t smem = sizeof(QBSmem<TB>);
    if (warp) {
        if (prune && stall && delta) k_query_block<true, true, TB, true, true><<<blocks, threads, smem, st>>>(a);
        else if (prune && stall) k_query_block<true, true, TB, true><<<blocks, threads, smem, st>>>(a);
        else if (prune) k_query_block<true, true, TB, false><<<blocks, threads, smem, st>>>(a);
        else k_query_block<false, true, TB, false><<<blocks, threads, smem, st>>>(a);
    } else {
        if (prune) k_query_block<true, false, TB, false><<<blocks, threads, smem, st>>>(a);
        else k_query_block<false, false, TB, false><<<blocks, threads, smem, st>>>(a);
    }
    CH_CHECK_LAUNCH();
}

// Launches one block-kernel pass in the handle's layout and block size: a
// persistent grid of as many blocks as are resident at once (no more than
// the items), with 2^11-slot tables when small is set, else 2^12. Stall on
// demand applies to pruned searches in the warp layout only, and
// delta-stepping levels to those with stalling.
void launch_query_block(const ch_s *h, const QArgs &a, bool prune, bool small, uint64_t items,
                        cudaStream_t st) {
    const bool warp = h->q_layout == CH_QUERY_WARP_FLAT;
    const bool stall = warp && prune && h->q_stall;
    const bool delta = stall && h->q_delta != 0;
    const int l = delta ? 3 : (stall ? 2 : (warp ? 1 : 0));
    const int t = h->q_threads == 256 ? 1 : 0;
    const int threads = t ? 256 : 128;
    const int blocks = (int)std::max<uint64_t>(
        1, std::min<uint64_t>(items, (uint64_t)device_sm_count() * g_qb_bps[small ? 1 : 0][l][t]));
    if (small) launch_tb<11>(a, prune, warp, stall, delta, blocks, threads, st);
    else launch_tb<12>(a, prune, warp, stall, delta, blocks, threads, st);
}

// Weights of `cnt` evenly spaced entries of an adjacency array.
__global__ void k_sample_weights(const uint2 *adj, uint64_t m, uint32_t *out, uint32_t cnt) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) out[i] = adj[(uint64_t)i * m / cnt].y;
}

constexpr uint32_t WSCALE_SAMPLE = 1024;
constexpr uint32_t DELTA_DEFAULT_MULT = 128;         // default delta, in weight scales
constexpr uint32_t DELTA_TUNE_MULT[3] = {64, 128, 256};  // autotuner candidates 12-14

// mult x the weight scale, at least 1 and below INF.
uint32_t delta_of(const ch_s *h, uint32_t mult) {
    const uint64_t d = (uint64_t)mult * h->q_wscale;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(d, INF - 1));
}

}  // namespace

void query_init(ch_s *h) {
    const uint32_t n = h->n;
    h->qerr.alloc(1);
    h->qerr.zero(0);
    h->qwork.alloc(8);
    h->q_ovf_cap = Q_CHUNK;
    h->q_ovf_list.alloc(2 * Q_CHUNK);  // overflow lists of the two block-kernel passes
    // per slot: df, db, fst, two frontiers (n each) and the touched list
    // of both directions (2n)
    const uint64_t per_slot = (uint64_t)std::max<uint32_t>(n, 1) * 7 * 4;
    h->q_slots = (uint32_t)std::max<uint64_t>(2, std::min<uint64_t>(64, (1024ull << 20) / per_slot));
    h->q_dense.alloc((size_t)h->q_slots * std::max<uint32_t>(n, 1) * 7);
    const size_t sn = (size_t)h->q_slots * std::max<uint32_t>(n, 1);
    // df, db: INF; fst: 0; the rest need no initial value
    CH_CUDA_TRY(cudaMemset(h->q_dense.ptr, 0xFF, sn * 2 * 4));
    CH_CUDA_TRY(cudaMemset(h->q_dense.ptr + 2 * sn, 0, sn * 4));
    h->q_stats.alloc(2);
    h->q_stats.zero(0);
    qb_resolve_occupancy();
    // weight scale of the hierarchy (the median of sampled E_up weights) and
    // the default delta
    h->q_wscale = 1;
    if (h->n_up > 0) {
        DevBuf<uint32_t> wb;
        wb.alloc(WSCALE_SAMPLE);
        k_sample_weights<<<(WSCALE_SAMPLE + 255) / 256, 256>>>(h->up_adj.ptr, h->n_up, wb.ptr, WSCALE_SAMPLE);
        CH_CHECK_LAUNCH();
        std::vector<uint32_t> w(WSCALE_SAMPLE);
        CH_CUDA_TRY(cudaMemcpy(w.data(), wb.ptr, WSCALE_SAMPLE * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        std::nth_element(w.begin(), w.begin() + WSCALE_SAMPLE / 2, w.end());
        h->q_wscale = std::max<uint32_t>(1, w[WSCALE_SAMPLE / 2]);
    }
    // Without delta when the hierarchy has a core: its queries search the
    // core, outgrow the shared tables and are redone on the dense kernel;
    // delta-stepping levels only delay that overflow.
    h->q_delta = h->core_size ? 0 : delta_of(h, DELTA_DEFAULT_MULT);
    CH_CUDA_TRY(cudaDeviceSynchronize());
}

void query_batch(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                 uint32_t *dist_out, uint32_t *settled_out, cudaStream_t st) {
    if (k == 0) return;
    const size_t sn = (size_t)h->q_slots * std::max<uint32_t>(h->n, 1);
    QDense dn;
    dn.df = h->q_dense.ptr;
    dn.db = dn.df + sn;
    dn.fst = dn.df + 2 * sn;
    dn.fa = dn.df + 3 * sn;
    dn.fb = dn.df + 4 * sn;
    dn.touched = dn.df + 5 * sn;  // 2 * sn entries
    dn.nslots = h->q_slots;
    for (uint64_t c0 = 0; c0 < k; c0 += Q_CHUNK) {
        const uint64_t kc = std::min<uint64_t>(Q_CHUNK, k - c0);
        QArgs a;
        a.n = h->n;
        a.n_up = (uint32_t)h->n_up;
        a.n_dn = (uint32_t)h->n_down;
        a.rank = h->rank.ptr;
        a.up_off = h->up_off.ptr;
        a.dn_off = h->dn_off.ptr;
        a.up_adj = h->up_adj.ptr;
        a.dn_adj = h->dn_adj.ptr;
        a.src = src + c0;
        a.dst = dst + c0;
        a.out = dist_out + c0;
        a.settled = settled_out ? settled_out + c0 : nullptr;
        a.k = kc;
        a.work = h->qwork.ptr;
        a.err = h->qerr.ptr;
        a.stats = h->q_stats.ptr;
        a.in_list = nullptr;
        a.in_cnt = 0;
        a.core_tab = h->core_n ? h->core_tab.ptr : nullptr;
        a.core_lo = h->core_lo;
        a.core_n = h->core_n;
        a.delta = h->q_delta ? h->q_delta : INF;
        CH_CUDA_TRY(cudaMemsetAsync(h->qwork.ptr, 0, 8 * sizeof(uint32_t), st));
        // Pruned searches unless the caller asked for search-space sizes,
        // which are defined by the exhaustive upward searches.
        const bool prune = settled_out == nullptr;
        if (h->q_small_first) {
            // pass 1 on small tables (twice the resident queries); the
            // queries that overflow them are redone on the large tables
            a.ctr = 0;
            a.ovf = h->q_ovf_list.ptr + Q_CHUNK;
            a.ovf_cnt = 4;
            launch_query_block(h, a, prune, true, kc, st);
            a.ctr = 3;
            a.in_list = h->q_ovf_list.ptr + Q_CHUNK;
            a.in_cnt = 4;
        }
        a.ctr = a.in_list ? 3 : 0;
        a.ovf = h->q_ovf_list.ptr;
        a.ovf_cnt = 2;
        launch_query_block(h, a, prune, false, kc, st);
        k_query_dense<<<h->q_slots, 256, 0, st>>>(a, dn);
        CH_CHECK_LAUNCH();
    }
}

// ---------------------------------------------------------------------------
// Configuration, autotuning, work counters, CUDA graphs
// ---------------------------------------------------------------------------

namespace {

// Seeded uniform pairs for the autotuner's sample (MurmurHash3 finaliser of
// a counter, reduced modulo n).
__global__ void k_sample_pairs(uint32_t *s, uint32_t *t, uint64_t k, uint32_t n, uint32_t seed) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < k;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = murmur_fmix32((uint32_t)(2 * i) ^ murmur_fmix32(seed));
        const uint32_t b = murmur_fmix32((uint32_t)(2 * i + 1) ^ murmur_fmix32(seed + 0x9e3779b9u));
        s[i] = a % n;
        t[i] = b % n;
    }
}

}  // namespace

void query_set_config(ch_s *h, uint32_t layout, uint32_t threads, uint32_t small_first, uint32_t stall,
                      uint32_t delta) {
    if ((layout != CH_QUERY_BLOCK_FLAT && layout != CH_QUERY_WARP_FLAT) || (threads != 128 && threads != 256) ||
        small_first > 1 || stall > 1 || (stall && layout != CH_QUERY_WARP_FLAT) || (delta && !stall) ||
        delta == INF)
        throw Error{CH_EINVAL, "query configuration: layout BLOCK_FLAT or WARP_FLAT, threads 128 or 256, "
                               "small_first 0 or 1, stall 0 or 1 (WARP_FLAT only), delta below 2^32 - 1 "
                               "(with stall 1 only when not 0)"};
    h->q_layout = layout;
    h->q_threads = threads;
    h->q_small_first = small_first;
    h->q_stall = stall;
    h->q_delta = delta;
}

void query_autotune(ch_s *h, uint64_t sample, uint32_t seed, cudaStream_t st, ch_query_config_t *chosen,
                    double *ms_out) {
    if (sample == 0 || h->n == 0) throw Error{CH_EINVAL, "autotune needs a sample and a non-empty graph"};
    DevBuf<uint32_t> buf;
    buf.alloc(3 * sample);
    uint32_t *s = buf.ptr, *t = buf.ptr + sample, *out = buf.ptr + 2 * sample;
    k_sample_pairs<<<grid_for(sample, 256, device_sm_count() * 4), 256, 0, st>>>(s, t, sample, h->n, seed);
    CH_CHECK_LAUNCH();
    const uint32_t keep_l = h->q_layout, keep_t = h->q_threads, keep_s = h->q_small_first,
                   keep_st = h->q_stall, keep_d = h->q_delta;
    cudaEvent_t e0, e1;
    CH_CUDA_TRY(cudaEventCreate(&e0));
    CH_CUDA_TRY(cudaEventCreate(&e1));
    // candidates 0-7: 4 * small_first + 2 * warp layout + (threads == 256);
    // 8-11: warp layout with stalling, 8 + 2 * small_first + (threads == 256);
    // 12-14: warp layout, 256 threads, small tables first, stalling, delta
    // at three multiples of the weight scale
    auto apply = [&](int i) {
        if (i < 8)
            query_set_config(h, (i & 2) ? CH_QUERY_WARP_FLAT : CH_QUERY_BLOCK_FLAT, (i & 1) ? 256 : 128,
                             (i & 4) ? 1 : 0, 0, 0);
        else if (i < 12)
            query_set_config(h, CH_QUERY_WARP_FLAT, (i & 1) ? 256 : 128, (i & 2) ? 1 : 0, 1, 0);
        else
            query_set_config(h, CH_QUERY_WARP_FLAT, 256, 1, 1, delta_of(h, DELTA_TUNE_MULT[i - 12]));
    };
    double best = 0;
    int best_i = -1;
    try {
        for (int i = 0; i < CH_QUERY_AUTOTUNE_CONFIGS; ++i) {
            apply(i);
            query_batch(h, s, t, sample, out, nullptr, st);  // warm-up
            CH_CUDA_TRY(cudaEventRecord(e0, st));
            query_batch(h, s, t, sample, out, nullptr, st);
            CH_CUDA_TRY(cudaEventRecord(e1, st));
            CH_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0;
            CH_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (ms_out) ms_out[i] = ms;
            if (best_i < 0 || ms < best) {
                best = ms;
                best_i = i;
            }
        }
    } catch (...) {
        h->q_layout = keep_l;
        h->q_threads = keep_t;
        h->q_small_first = keep_s;
        h->q_stall = keep_st;
        h->q_delta = keep_d;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply(best_i);
    if (chosen) {
        chosen->layout = h->q_layout;
        chosen->threads = h->q_threads;
        chosen->small_first = h->q_small_first;
        chosen->stall = h->q_stall;
        chosen->delta = h->q_delta;
    }
    // the sample's work is not the caller's: clear the counters
    CH_CUDA_TRY(cudaMemsetAsync(h->q_stats.ptr, 0, 2 * sizeof(unsigned long long), st));
    CH_CUDA_TRY(cudaStreamSynchronize(st));
}

double query_time_sample(ch_s *h, uint64_t sample, uint32_t seed, cudaStream_t st) {
    if (sample == 0 || h->n == 0) return 0.0;
    DevBuf<uint32_t> buf;
    buf.alloc(3 * sample);
    uint32_t *s = buf.ptr, *t = buf.ptr + sample, *out = buf.ptr + 2 * sample;
    k_sample_pairs<<<grid_for(sample, 256, device_sm_count() * 4), 256, 0, st>>>(s, t, sample, h->n, seed);
    CH_CHECK_LAUNCH();
    cudaEvent_t e0, e1;
    CH_CUDA_TRY(cudaEventCreate(&e0));
    CH_CUDA_TRY(cudaEventCreate(&e1));
    float ms = 0;
    cudaError_t e = cudaSuccess;
    try {
        query_batch(h, s, t, sample, out, nullptr, st);  // warm-up
        CH_CUDA_TRY(cudaEventRecord(e0, st));
        query_batch(h, s, t, sample, out, nullptr, st);
        CH_CUDA_TRY(cudaEventRecord(e1, st));
        CH_CUDA_TRY(cudaEventSynchronize(e1));
        e = cudaEventElapsedTime(&ms, e0, e1);
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) throw Error{CH_ECUDA, cudaGetErrorString(e)};
    CH_CUDA_TRY(cudaMemsetAsync(h->q_stats.ptr, 0, 2 * sizeof(unsigned long long), st));
    CH_CUDA_TRY(cudaStreamSynchronize(st));
    return ms;
}

void query_work(ch_s *h, cudaStream_t st, uint64_t out[2]) {
    unsigned long long v[2] = {0, 0};
    CH_CUDA_TRY(cudaMemcpyAsync(v, h->q_stats.ptr, sizeof(v), cudaMemcpyDeviceToHost, st));
    CH_CUDA_TRY(cudaMemsetAsync(h->q_stats.ptr, 0, sizeof(v), st));
    CH_CUDA_TRY(cudaStreamSynchronize(st));
    out[0] = v[0];
    out[1] = v[1];
}

}  // namespace gbch

struct ch_query_graph_s {
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;  // kernel launches one replay makes
};

namespace gbch {

ch_query_graph_s *query_graph_create(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                                     uint32_t *dist_out) {
    cudaStream_t st = nullptr;
    CH_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    try {
        CH_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            query_batch(h, src, dst, k, dist_out, nullptr, st);
        } catch (...) {
            cudaStreamEndCapture(st, &graph);
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            throw;
        }
        CH_CUDA_TRY(cudaStreamEndCapture(st, &graph));
    } catch (...) {
        cudaStreamDestroy(st);
        throw;
    }
    cudaStreamDestroy(st);
    auto *g = new ch_query_graph_s();
    cudaError_t e = cudaSuccess;
    if (graph) {
        // the launches were counted at capture; count them when replays run them
        size_t nn = 0;
        e = cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
        for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
            cudaGraphNodeType ty;
            e = cudaGraphNodeGetType(nodes[i], &ty);
            if (e == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++g->kernels;
        }
        kernel_launch_add(-(int64_t)g->kernels);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
    }
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        delete g;
        cudaGetLastError();
        throw Error{CH_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e)};
    }
    return g;
}

void query_graph_launch(ch_query_graph_s *g, cudaStream_t st) {
    if (!g->exec) return;  // k = 0: nothing was captured
    CH_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    kernel_launch_add((int64_t)g->kernels);
}

void query_graph_free(ch_query_graph_s *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
}

// ---------------------------------------------------------------------------
// Query batches that allocate nothing (ch_query_batch_static)
// ---------------------------------------------------------------------------
//
// Same kernels as query_batch; the only difference is where the per-call
// scratch lives (the work counters and the list of queries handed to the
// dense kernel). Here it is one file-scope device array, so a call needs no
// allocation at all; every GPU that loads the library holds the array
// (about 1 MiB) until the process exits. The array is shared by all calls
// and all handles on a device: calls whose work overlaps on the GPU race on
// it and must be serialised by the caller (one stream, or events).

namespace {

constexpr uint32_t kStaticScratchHead = 4;  // [0] block counter, [1] dense counter, [2] overflow count
__device__ __align__(256) uint32_t g_static_query_scratch[kStaticScratchHead + CH_STATIC_QUERY_MAX];

std::mutex g_static_mu;
uint32_t *g_static_ptr[64] = {nullptr};

// Device address of the scratch array for the current device. The first call
// on a device resolves it (cudaGetSymbolAddress) with that device current;
// later calls reuse it.
uint32_t *static_scratch() {
    int dev = 0;
    CH_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{CH_ERANGE, "device ordinal above 63"};
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        CH_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_query_scratch));
        g_static_ptr[dev] = static_cast<uint32_t *>(p);
    }
    return g_static_ptr[dev];
}

}  // namespace

void query_batch_static(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                        uint32_t *dist_out, cudaStream_t st) {
    if (k > CH_STATIC_QUERY_MAX)
        throw Error{CH_ERANGE, "batch larger than CH_STATIC_QUERY_MAX queries"};
    if (k == 0) return;
    int dev = 0;
    CH_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != h->device)
        throw Error{CH_EINVAL, "the current device is not the hierarchy's device"};
    uint32_t *scratch = static_scratch();
    const size_t sn = (size_t)h->q_slots * std::max<uint32_t>(h->n, 1);
    QDense dn;
    dn.df = h->q_dense.ptr;
    dn.db = dn.df + sn;
    dn.fst = dn.df + 2 * sn;
    dn.fa = dn.df + 3 * sn;
    dn.fb = dn.df + 4 * sn;
    dn.touched = dn.df + 5 * sn;
    dn.nslots = h->q_slots;
    QArgs a;
    a.n = h->n;
    a.n_up = (uint32_t)h->n_up;
    a.n_dn = (uint32_t)h->n_down;
    a.rank = h->rank.ptr;
    a.up_off = h->up_off.ptr;
    a.dn_off = h->dn_off.ptr;
    a.up_adj = h->up_adj.ptr;
    a.dn_adj = h->dn_adj.ptr;
    a.src = src;
    a.dst = dst;
    a.out = dist_out;
    a.settled = nullptr;
    a.k = k;
    a.work = scratch;
    a.in_list = nullptr;
    a.in_cnt = 0;
    a.ctr = 0;
    a.ovf = scratch + kStaticScratchHead;
    a.ovf_cnt = 2;
    a.err = h->qerr.ptr;
    a.stats = h->q_stats.ptr;
    a.core_tab = h->core_n ? h->core_tab.ptr : nullptr;
    a.core_lo = h->core_lo;
    a.core_n = h->core_n;
    a.delta = h->q_delta ? h->q_delta : INF;
    // the counters keep the previous call's values: clear them
    CH_CUDA_TRY(cudaMemsetAsync(scratch, 0, kStaticScratchHead * sizeof(uint32_t), st));
    // one block-kernel pass (large tables): the scratch holds one list
    launch_query_block(h, a, true, false, k, st);
    k_query_dense<<<h->q_slots, 256, 0, st>>>(a, dn);
    CH_CHECK_LAUNCH();
}

}  // namespace gbch
