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
// One warp serves one query at a time and pulls the next index from a
// counter (persistent grid). Its labels live in a shared-memory hash table
// whose entries carry both directions' distances, so the meeting minimum is
// one pass over the table. A query whose search spaces do not fit is
// redone by a second kernel that keeps labels in dense per-vertex arrays in
// global memory (one block per array slot).

#include <algorithm>

#include "handle.cuh"

namespace gbch {
namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr uint32_t QERR_RANGE = 1u;

constexpr int Q_WARPS = 4;            // warps per block
constexpr int Q_TBITS = 10;           // 1024 vertices per query table
constexpr int Q_T = 1 << Q_TBITS;
constexpr int Q_FC = 512;             // frontier capacity
constexpr uint64_t Q_CHUNK = 1u << 22;  // queries per launch pair

struct QSmem {
    uint32_t key[Q_T];
    uint32_t df[Q_T];
    uint32_t db[Q_T];
    uint32_t fst[Q_T];
    uint32_t front[2][Q_FC];
    uint32_t nf[2];
    uint32_t flag;
};

struct QArgs {
    uint32_t n;
    const uint32_t *rank;
    const uint32_t *up_off, *dn_off;
    const uint2 *up_adj, *dn_adj;
    const uint32_t *src, *dst;
    uint32_t *out, *settled;
    uint64_t k;
    uint32_t *work;      // [0]: warp path counter, [1]: fallback counter, [2]: overflow count
    uint32_t *ovf;
    uint32_t *err;
};

__device__ __forceinline__ uint32_t q_hash(uint32_t v) {
    return (v * 2654435761u) >> (32 - Q_TBITS);
}

__device__ __forceinline__ uint32_t q_insert(uint32_t *keys, uint32_t v) {
    uint32_t h = q_hash(v);
    for (uint32_t probe = 0; probe < (uint32_t)Q_T; ++probe) {
        uint32_t k = keys[h];
        if (k == v) return h;
        if (k == EMPTY) {
            uint32_t old = atomicCAS(&keys[h], EMPTY, v);
            if (old == EMPTY || old == v) return h;
        }
        h = (h + 1) & (Q_T - 1);
    }
    return EMPTY;
}

// Label-correcting upward search of one direction inside the warp's table.
// Returns false on table or frontier overflow.
__device__ bool warp_search(QSmem &q, uint32_t root_slot, uint32_t *dist,
                            const uint32_t *off, const uint2 *adj, uint32_t &stamp) {
    const uint32_t lane = lane_id();
    if (lane == 0) {
        q.front[0][0] = root_slot;
        q.nf[0] = 1;
    }
    __syncwarp();
    uint32_t cur = 0;
    while (true) {
        const uint32_t nfront = q.nf[cur];
        if (nfront == 0) break;
        const uint32_t nxt = cur ^ 1u;
        ++stamp;
        __syncwarp();
        if (lane == 0) q.nf[nxt] = 0;
        __syncwarp();
        for (uint32_t f0 = 0; f0 < nfront; f0 += 32) {
            const uint32_t fi = f0 + lane;
            const bool fv = fi < nfront;
            const uint32_t slot = fv ? q.front[cur][fi] : 0;
            const uint32_t x = fv ? q.key[slot] : 0;
            const uint32_t b = fv ? off[x] : 0;
            const uint32_t cnt = fv ? off[x + 1] - b : 0;
            const uint32_t incl = warp_incl_scan(cnt);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const uint32_t excl = incl - cnt;
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t idx = base + lane;
                const uint32_t o = warp_owner(excl, idx);
                const uint32_t b_o = __shfl_sync(FULL, b, o);
                const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                const uint32_t slot_o = __shfl_sync(FULL, slot, o);
                if (idx < total) {
                    const uint2 e = adj[b_o + (idx - ex_o)];
                    const uint32_t nd = sat_add(dist[slot_o], e.y);
                    if (nd != INF) {
                        const uint32_t ys = q_insert(q.key, e.x);
                        if (ys == EMPTY) {
                            q.flag = 1;
                        } else {
                            const uint32_t old = atomicMin(&dist[ys], nd);
                            if (nd < old && atomicExch(&q.fst[ys], stamp) != stamp) {
                                const uint32_t p = atomicAdd(&q.nf[nxt], 1u);
                                if (p < (uint32_t)Q_FC) q.front[nxt][p] = ys;
                                else q.flag = 1;
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (q.flag) return false;
        cur = nxt;
    }
    return true;
}

__global__ void __launch_bounds__(Q_WARPS * 32) k_query_warp(QArgs a) {
    extern __shared__ __align__(16) unsigned char q_raw[];
    QSmem &q = reinterpret_cast<QSmem *>(q_raw)[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    while (true) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(&a.work[0], 1u);
        i = __shfl_sync(FULL, i, 0);
        if (i >= a.k) break;
        const uint32_t s = a.src[i], t = a.dst[i];
        if (s >= a.n || t >= a.n) {
            if (lane == 0) {
                atomicOr(a.err, QERR_RANGE);
                a.out[i] = INF;
                if (a.settled) a.settled[i] = 0;
            }
            continue;
        }
        const uint32_t rs = a.rank[s], rt = a.rank[t];
        for (uint32_t j = lane; j < (uint32_t)Q_T; j += 32) {
            q.key[j] = EMPTY;
            q.df[j] = INF;
            q.db[j] = INF;
            q.fst[j] = 0;
        }
        __syncwarp();
        if (lane == 0) q.flag = 0;
        uint32_t ss = 0, st = 0;
        if (lane == 0) {
            ss = q_insert(q.key, rs);
            q.df[ss] = 0;
            st = q_insert(q.key, rt);
            q.db[st] = 0;
        }
        ss = __shfl_sync(FULL, ss, 0);
        st = __shfl_sync(FULL, st, 0);
        __syncwarp();
        uint32_t stamp = 0;
        bool ok = warp_search(q, ss, q.df, a.up_off, a.up_adj, stamp);
        if (ok) ok = warp_search(q, st, q.db, a.dn_off, a.dn_adj, stamp);
        if (!ok) {
            if (lane == 0) a.ovf[atomicAdd(&a.work[2], 1u)] = i;
            __syncwarp();
            continue;
        }
        uint32_t mu = INF, cnt = 0;
        for (uint32_t j = lane; j < (uint32_t)Q_T; j += 32) {
            const uint32_t f = q.df[j], g = q.db[j];
            mu = min(mu, sat_add(f, g));
            cnt += (f != INF) + (g != INF);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mu = min(mu, __shfl_xor_sync(FULL, mu, o));
            cnt += __shfl_xor_sync(FULL, cnt, o);
        }
        if (lane == 0) {
            a.out[i] = mu;
            if (a.settled) a.settled[i] = cnt;
        }
        __syncwarp();
    }
}

// Dense fallback: one block per slot; labels in per-vertex arrays.
struct QDense {
    uint32_t *df, *db, *fst, *fa, *fb, *touched;
    uint32_t nslots;
};

__device__ void dense_search(uint32_t root, uint32_t *dist, uint32_t *fst, uint32_t *fa,
                             uint32_t *fb, uint32_t *touched, uint32_t *s_nt, uint32_t *s_nf,
                             const uint32_t *off, const uint2 *adj, uint32_t &stamp) {
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
            const uint32_t dx = dist[x];
            for (uint32_t j = off[x]; j < off[x + 1]; ++j) {
                const uint2 e = adj[j];
                const uint32_t nd = sat_add(dx, e.y);
                if (nd == INF) continue;
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
        // forward labels live in df, backward in db; touched lists both
        dense_search(rs, df, fst, fa, fb, touched, &s_nt, s_nf, a.up_off, a.up_adj, stamp);
        __syncthreads();
        const uint32_t nt_f = s_nt;
        dense_search(rt, db, fst, fa, fb, touched, &s_nt, s_nf, a.dn_off, a.dn_adj, stamp);
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

int g_q_blocks_per_sm = -1;

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
    h->q_slots = (uint32_t)std::max<uint64_t>(2, std::min<uint64_t>(64, (1ull << 30) / per_slot));
    h->q_dense.alloc((size_t)h->q_slots * std::max<uint32_t>(n, 1) * 7);
    const size_t sn = (size_t)h->q_slots * std::max<uint32_t>(n, 1);
    // df, db: INF; fst: 0; the rest need no initial value
    CH_CUDA_TRY(cudaMemset(h->q_dense.ptr, 0xFF, sn * 2 * 4));
    CH_CUDA_TRY(cudaMemset(h->q_dense.ptr + 2 * sn, 0, sn * 4));
    if (g_q_blocks_per_sm < 0) {
        const size_t smem = sizeof(QSmem) * Q_WARPS;
        CH_CUDA_TRY(cudaFuncSetAttribute(k_query_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        int b = 0;
        CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_query_warp,
                                                                  Q_WARPS * 32, smem));
        g_q_blocks_per_sm = std::max(1, b);
    }
    CH_CUDA_TRY(cudaDeviceSynchronize());
}

void query_batch(ch_s *h, const uint32_t *src, const uint32_t *dst, uint64_t k,
                 uint32_t *dist_out, uint32_t *settled_out, cudaStream_t st) {
    if (k == 0) return;
    const size_t smem = sizeof(QSmem) * Q_WARPS;
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
        const uint64_t want = (kc + Q_WARPS - 1) / Q_WARPS;
        const int blocks = (int)std::min<uint64_t>(want, (uint64_t)sms * g_q_blocks_per_sm);
        k_query_warp<<<blocks, Q_WARPS * 32, smem, st>>>(a);
        CH_CHECK_LAUNCH();
        k_query_dense<<<h->q_slots, 256, 0, st>>>(a, dn);
        CH_CHECK_LAUNCH();
    }
}

}  // namespace gbch
