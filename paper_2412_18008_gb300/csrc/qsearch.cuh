// Shared-memory bidirectional upward search of one CH s-t query by one
// block (Sec. 5 of arXiv 2412.18008), used by the batch query kernel and by
// the query server. Everything here has internal linkage.
#pragma once

#include "common.cuh"

namespace gbch {
namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr uint32_t QERR_RANGE = 1u;
constexpr uint32_t QERR_BOUND = 2u;  // an index check failed; the access was skipped

constexpr int QB_THREADS = 256;        // threads per query block
constexpr int QB_TBITS = 12;           // 4096 vertices per query table
constexpr int QB_T = 1 << QB_TBITS;
constexpr int QB_FC = 2048;            // frontier capacity

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

// One s-t query (rank ids rs, rt < n) by the whole block, on the shared
// table: clears it, seeds both roots, searches and reduces the answer.
// Returns false, in every thread, when the search spaces overflowed the
// table or the frontier (the caller redoes the query elsewhere); otherwise
// mu and cnt hold, in every thread, the least meeting sum and the number of
// labels set. Every thread of the block must call it.
template <bool PRUNE>
__device__ bool block_query(QBSmem &q, const QArgs &a, uint32_t rs, uint32_t rt, uint32_t &mu_out,
                            uint32_t &cnt_out) {
    const uint32_t tid = threadIdx.x;
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
    if (!block_search<PRUNE>(q, a)) return false;
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
    mu_out = q.mu;
    cnt_out = q.cnt;
    return true;
}

}  // namespace
}  // namespace gbch
