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

#include "handle.cuh"

namespace gbch {
namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr uint32_t QERR_RANGE = 1u;
constexpr uint32_t QERR_BOUND = 2u;  // an index check failed; the access was skipped

constexpr int QB_THREADS = 256;        // threads per query block
constexpr int QB_TBITS = 12;           // 4096 vertices per query table
constexpr int QB_T = 1 << QB_TBITS;
constexpr int QB_FC = 2048;            // frontier capacity
constexpr uint64_t Q_CHUNK = 1u << 22;  // queries per launch pair

// Shared state of one query block (about 70 KB, three blocks per SM): a
// hash table of reached vertices whose entries carry both directions'
// labels, claim bitmaps that keep a slot from being queued twice in one
// level and direction (one bitmap per level parity, the idle one cleared
// during the level), a double-buffered frontier holding both directions'
// entries (slot | dir<<31) and a triple-buffered frontier counter, so that
// one barrier per level suffices (see block_search).
constexpr int QB_CW = QB_T / 32;  // claim-bitmap words per direction
struct QBSmem {
    uint32_t key[QB_T];
    uint32_t df[QB_T];
    uint32_t db[QB_T];
    uint32_t claim[2][2][QB_CW];  // [level parity][direction][word]
    uint32_t front[2][QB_FC];
    // one tile of frontier entries, flattened block-wide: exclusive prefix of
    // their out-degrees, first edge index, label, slot | dir << 31
    uint32_t t_excl[QB_THREADS];
    uint32_t t_beg[QB_THREADS];
    uint32_t t_dx[QB_THREADS];
    uint32_t t_ent[QB_THREADS];
    uint32_t wtot[QB_THREADS / 32 + 1];
    uint32_t cnt3[3];
    uint32_t item, ovf, mu, cnt, ss, st;
};

struct QArgs {
    uint32_t n;
    uint32_t n_up, n_dn;  // edge counts of the two CSRs, for index checks
    const uint32_t *rank;
    const uint32_t *up_off, *dn_off;
    const uint2 *up_adj, *dn_adj;
    const uint32_t *src, *dst;
    uint32_t *out, *settled;
    uint64_t k;
    uint32_t *work;      // [0]: block path counter, [1]: fallback counter, [2]: overflow count
    uint32_t *ovf;
    uint32_t *err;
};

__device__ __forceinline__ uint32_t qb_hash(uint32_t v) {
    return (v * 2654435761u) >> (32 - QB_TBITS);
}

__device__ __forceinline__ uint32_t qb_insert(uint32_t *keys, uint32_t v) {
    uint32_t h = qb_hash(v);
    for (uint32_t probe = 0; probe < (uint32_t)QB_T; ++probe) {
        uint32_t k = keys[h];
        if (k == v) return h;
        if (k == EMPTY) {
            uint32_t old = atomicCAS(&keys[h], EMPTY, v);
            if (old == EMPTY || old == v) return h;
        }
        h = (h + 1) & (QB_T - 1);
    }
    return EMPTY;
}

// Marks `slot` as queued in direction `dir` for the next level (bitmap of
// the level's parity); true if it was not queued yet.
__device__ __forceinline__ bool qb_claim(QBSmem &q, uint32_t slot, uint32_t dir, uint32_t lvl) {
    const uint32_t bit = 1u << (slot & 31u);
    return !(atomicOr(&q.claim[lvl & 1u][dir][slot >> 5], bit) & bit);
}

// Both upward searches at once, label-correcting over the rank DAG: the
// frontier holds forward (E_up) and backward (reversed E_down) entries,
// each level relaxes the out-edges of every queued vertex with its current
// label, and the search ends when no label changed. With PRUNE, a relaxation
// whose new label is not below the best meeting sum found so far is skipped
// (it cannot improve the answer); the answer is always recomputed at the
// end as the least df + db over the table, so it is exact either way.
//
// Barrier discipline: the only barrier of a level is at its top. The
// frontier counter of level k lives in cnt3[k % 3]; thread 0 clears the
// counter of level k + 2 during level k, when no thread reads it any more.
template <bool PRUNE>
__device__ bool block_search(QBSmem &q, const QArgs &a) {
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    for (uint32_t lvl = 1;; ++lvl) {
        __syncthreads();
        const uint32_t cur = (lvl - 1) & 1u;
        const uint32_t nfront = q.cnt3[(lvl - 1) % 3];
        const uint32_t ovf = q.ovf;
        if (ovf) return false;
        if (nfront == 0) return true;
        if (lvl >= 0xFFFFu) {  // a label-correcting search on a DAG never gets here
            if (tid == 0) atomicOr(a.err, QERR_BOUND);
            return false;
        }
        if (tid == 0) q.cnt3[(lvl + 1) % 3] = 0;
        // the bitmap of the other parity was last used two levels ago and is
        // next used one level from now
        for (uint32_t j = tid; j < 2u * QB_CW; j += blockDim.x) (&q.claim[(lvl + 1) & 1u][0][0])[j] = 0;
        const uint32_t nxt_cnt = lvl % 3;
        // Tiles of blockDim frontier entries; the out-edges of a tile are
        // spread evenly over all threads of the block.
        for (uint32_t t0 = 0; t0 < nfront; t0 += blockDim.x) {
            const uint32_t fi = t0 + tid;
            const bool fv = fi < nfront && fi < (uint32_t)QB_FC;
            const uint32_t ent = fv ? q.front[cur][fi] : 0;
            const uint32_t dir = ent >> 31;
            const uint32_t slot = ent & 0x7FFFFFFFu;
            const bool sok = fv && slot < (uint32_t)QB_T;
            if (fv && !sok) atomicOr(a.err, QERR_BOUND);
            const uint32_t x = sok ? q.key[slot] : 0;
            const bool xok = sok && x < a.n;
            if (sok && !xok) atomicOr(a.err, QERR_BOUND);
            const uint32_t *off = dir ? a.dn_off : a.up_off;
            const uint32_t n_edges = dir ? a.n_dn : a.n_up;
            const uint32_t b = xok ? off[x] : 0;
            const uint32_t e_end = xok ? off[x + 1] : 0;
            uint32_t cnt = 0;
            if (xok && b <= e_end && e_end <= n_edges) cnt = e_end - b;
            else if (xok) atomicOr(a.err, QERR_BOUND);
            const uint32_t dx = cnt ? (dir ? q.db[slot] : q.df[slot]) : INF;
            // block-wide exclusive scan of cnt
            const uint32_t incl = warp_incl_scan(cnt);
            if (lane == 31) q.wtot[warp] = incl;
            q.t_beg[tid] = b;
            q.t_dx[tid] = dx;
            q.t_ent[tid] = ent;
            __syncthreads();
            uint32_t wbase = 0, total = 0;
            for (uint32_t w2 = 0; w2 < nwarps; ++w2) {
                const uint32_t wt = q.wtot[w2];
                if (w2 < warp) wbase += wt;
                total += wt;
            }
            q.t_excl[tid] = wbase + incl - cnt;
            __syncthreads();
            for (uint32_t e0 = tid; e0 < total; e0 += blockDim.x) {
                // owner entry: the largest k with t_excl[k] <= e0
                uint32_t lo = 0, hi = blockDim.x;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (q.t_excl[mid] <= e0) lo = mid;
                    else hi = mid;
                }
                const uint32_t oent = q.t_ent[lo];
                const uint32_t odir = oent >> 31;
                const uint2 e = (odir ? a.dn_adj : a.up_adj)[q.t_beg[lo] + (e0 - q.t_excl[lo])];
                const uint32_t nd = sat_add(q.t_dx[lo], e.y);
                if (e.x >= a.n) {
                    atomicOr(a.err, QERR_BOUND);
                    continue;
                }
                if (nd == INF) continue;
                if (PRUNE && nd >= q.mu) continue;
                const uint32_t ys = qb_insert(q.key, e.x);
                if (ys == EMPTY) {
                    q.ovf = 1;
                    continue;
                }
                uint32_t *dist = odir ? q.db : q.df;
                const uint32_t old = atomicMin(&dist[ys], nd);
                if (nd >= old) continue;
                if (PRUNE) {
                    const uint32_t other = odir ? q.df[ys] : q.db[ys];
                    if (other != INF) atomicMin(&q.mu, sat_add(nd, other));
                }
                if (qb_claim(q, ys, odir, lvl)) {
                    const uint32_t p = atomicAdd(&q.cnt3[nxt_cnt], 1u);
                    if (p < (uint32_t)QB_FC) q.front[cur ^ 1u][p] = ys | (odir << 31);
                    else q.ovf = 1;
                }
            }
            __syncthreads();
        }
    }
}

template <bool PRUNE>
__global__ void __launch_bounds__(QB_THREADS) k_query_block(QArgs a) {
    extern __shared__ __align__(16) unsigned char qb_raw[];
    QBSmem &q = *reinterpret_cast<QBSmem *>(qb_raw);
    const uint32_t tid = threadIdx.x;
    while (true) {
        __syncthreads();
        if (tid == 0) q.item = atomicAdd(&a.work[0], 1u);
        __syncthreads();
        const uint32_t i = q.item;
        if (i >= a.k) break;
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
        for (uint32_t j = tid; j < (uint32_t)QB_T; j += blockDim.x) {
            q.key[j] = EMPTY;
            q.df[j] = INF;
            q.db[j] = INF;
        }
        for (uint32_t j = tid; j < 4u * QB_CW; j += blockDim.x) (&q.claim[0][0][0])[j] = 0;
        __syncthreads();
        if (tid == 0) {
            const uint32_t ss = qb_insert(q.key, rs);
            q.df[ss] = 0;
            const uint32_t st = qb_insert(q.key, rt);
            q.db[st] = 0;
            q.ovf = 0;
            q.mu = ss == st ? 0u : INF;
            q.cnt = 0;
            q.front[0][0] = ss;
            q.front[0][1] = st | 0x80000000u;
            q.cnt3[0] = 2;
            q.cnt3[1] = 0;
            q.cnt3[2] = 0;
        }
        const bool ok = block_search<PRUNE>(q, a);
        if (!ok) {
            if (tid == 0) a.ovf[atomicAdd(&a.work[2], 1u)] = i;
            continue;
        }
        // q.mu only steered pruning; the answer is the least meeting sum.
        __syncthreads();
        if (tid == 0) q.mu = INF;
        __syncthreads();
        uint32_t mu = INF, cnt = 0;
        for (uint32_t j = tid; j < (uint32_t)QB_T; j += blockDim.x) {
            const uint32_t f = q.df[j], g = q.db[j];
            mu = min(mu, sat_add(f, g));
            cnt += (f != INF) + (g != INF);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mu = min(mu, __shfl_xor_sync(FULL, mu, o));
            cnt += __shfl_xor_sync(FULL, cnt, o);
        }
        if (lane_id() == 0) {
            atomicMin(&q.mu, mu);
            atomicAdd(&q.cnt, cnt);
        }
        __syncthreads();
        if (tid == 0) {
            a.out[i] = q.mu;
            if (a.settled) a.settled[i] = q.cnt;
        }
    }
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
    const uint32_t novf = a.work[2];
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

int g_qb_blocks_per_sm = -1;

}  // namespace

void query_init(ch_s *h) {
    const uint32_t n = h->n;
    h->qerr.alloc(1);
    h->qerr.zero(0);
    h->qwork.alloc(4);
    h->q_ovf_cap = Q_CHUNK;
    h->q_ovf_list.alloc(Q_CHUNK);
    // per slot: df, db, fst, two frontiers (n each) and the touched list
    // of both directions (2n)
    const uint64_t per_slot = (uint64_t)std::max<uint32_t>(n, 1) * 7 * 4;
    h->q_slots = (uint32_t)std::max<uint64_t>(2, std::min<uint64_t>(64, (1024ull << 20) / per_slot));
    h->q_dense.alloc((size_t)h->q_slots * std::max<uint32_t>(n, 1) * 7);
    const size_t sn = (size_t)h->q_slots * std::max<uint32_t>(n, 1);
    // df, db: INF; fst: 0; the rest need no initial value
    CH_CUDA_TRY(cudaMemset(h->q_dense.ptr, 0xFF, sn * 2 * 4));
    CH_CUDA_TRY(cudaMemset(h->q_dense.ptr + 2 * sn, 0, sn * 4));
    if (g_qb_blocks_per_sm < 0) {
        const size_t smem = sizeof(QBSmem);
        CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CH_CUDA_TRY(cudaFuncSetAttribute(k_query_block<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_query_block<true>,
                                                                  QB_THREADS, smem));
        g_qb_blocks_per_sm = std::max(1, b);
    }
    CH_CUDA_TRY(cudaDeviceSynchronize());
}

void query_batch(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                 uint32_t *dist_out, uint32_t *settled_out, cudaStream_t st) {
    if (k == 0) return;
    const size_t smem = sizeof(QBSmem);
    const int sms = device_sm_count();
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
        a.ovf = h->q_ovf_list.ptr;
        a.err = h->qerr.ptr;
        CH_CUDA_TRY(cudaMemsetAsync(h->qwork.ptr, 0, 4 * sizeof(uint32_t), st));
        const int blocks = (int)std::min<uint64_t>(kc, (uint64_t)sms * g_qb_blocks_per_sm);
        // Pruned searches unless the caller asked for search-space sizes,
        // which are defined by the exhaustive upward searches.
        if (settled_out) k_query_block<false><<<blocks, QB_THREADS, smem, st>>>(a);
        else k_query_block<true><<<blocks, QB_THREADS, smem, st>>>(a);
        CH_CHECK_LAUNCH();
        k_query_dense<<<h->q_slots, 256, 0, st>>>(a, dn);
        CH_CHECK_LAUNCH();
    }
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
    uint32_t *scratch = static_scratch();
    const size_t smem = sizeof(QBSmem);
    const int sms = device_sm_count();
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
    a.ovf = scratch + kStaticScratchHead;
    a.err = h->qerr.ptr;
    // the counters keep the previous call's values: clear them
    CH_CUDA_TRY(cudaMemsetAsync(scratch, 0, kStaticScratchHead * sizeof(uint32_t), st));
    const int blocks = (int)std::min<uint64_t>(k, (uint64_t)sms * g_qb_blocks_per_sm);
    k_query_block<true><<<blocks, QB_THREADS, smem, st>>>(a);
    CH_CHECK_LAUNCH();
    k_query_dense<<<h->q_slots, 256, 0, st>>>(a, dn);
    CH_CHECK_LAUNCH();
}

}  // namespace gbch
