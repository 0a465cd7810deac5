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

constexpr int QB_THREADS = 256;  // threads per query block, at most

// Shared state of one query block, for a table of 2^TB vertices (TB = 12:
// about 69 KB, three blocks per SM; TB = 11: about 35 KB, six): a hash table
// of reached vertices whose entries carry both directions' labels, claim
// bitmaps that keep a slot from being queued twice in one level and
// direction (one bitmap per level parity, the idle one cleared during the
// level), a double-buffered frontier holding both directions' entries
// (slot | dir<<31), and a triple-buffered frontier counter and pair of
// least queued labels (see block_search).
template <int TB>
struct QBSmem {
    static constexpr uint32_t T = 1u << TB;   // table slots
    // frontier capacity (the small table's is trimmed so that six blocks fit
    // an SM's 228 KB of shared memory)
    static constexpr uint32_t FC = TB >= 12 ? T / 2 : 3 * T / 8;
    static constexpr uint32_t CW = T / 32;    // claim-bitmap words per direction
    uint32_t key[T];
    uint32_t df[T];
    uint32_t db[T];
    uint32_t claim[2][2][CW];  // [level parity][direction][word]
    uint32_t front[2][FC];
    // one tile of frontier entries, flattened block-wide: exclusive prefix of
    // their out-degrees, first edge index, label, slot | dir << 31
    uint32_t t_excl[QB_THREADS];
    uint32_t t_beg[QB_THREADS];
    uint32_t t_dx[QB_THREADS];
    uint32_t t_ent[QB_THREADS];
    uint32_t wtot[QB_THREADS / 32 + 1];
    uint32_t cnt3[3];
    uint32_t lmin3[3][2];  // least label queued per level (mod 3) and direction
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
    // Work items and counters. A block kernel takes items from work[ctr]:
    // query j for j < k, or, with in_list, query in_list[j] for
    // j < work[in_cnt]. A query whose search overflows is appended to ovf,
    // counted in work[ovf_cnt]. The dense kernel takes ovf entries from
    // work[1].
    uint32_t *work;
    const uint32_t *in_list;
    uint32_t in_cnt, ctr, ovf_cnt;
    uint32_t *ovf;
    uint32_t *err;
    unsigned long long *stats;  // [0] expansions, [1] edges scanned (or null)
    // Core distance table (or null): the searches do not expand the core's
    // vertices (ranks >= core_lo) and join through core_tab (core_n x
    // core_n distances) instead.
    const uint32_t *core_tab = nullptr;
    uint32_t core_lo = 0, core_n = 0;
    // Bucket width of delta-stepping levels (the DELTA kernels): a level
    // expands only the entries whose label is at most the least queued
    // label of their direction plus delta and keeps the rest queued.
    uint32_t delta = INF;
};

template <int TB>
__device__ __forceinline__ uint32_t qb_insert(uint32_t *keys, uint32_t v) {
    constexpr uint32_t T = 1u << TB;
    uint32_t h = (v * 2654435761u) >> (32 - TB);
    for (uint32_t probe = 0; probe < T; ++probe) {
        uint32_t k = keys[h];
        if (k == v) return h;
        if (k == EMPTY) {
            uint32_t old = atomicCAS(&keys[h], EMPTY, v);
            if (old == EMPTY || old == v) return h;
        }
        h = (h + 1) & (T - 1);
    }
    return EMPTY;
}

// Slot of v, or EMPTY if v is not in the table (read-only probe; an insert
// racing with it may be missed, which only makes a stall test weaker).
template <int TB>
__device__ __forceinline__ uint32_t qb_find(const uint32_t *keys, uint32_t v) {
    constexpr uint32_t T = 1u << TB;
    uint32_t h = (v * 2654435761u) >> (32 - TB);
    for (uint32_t probe = 0; probe < T; ++probe) {
        const uint32_t k = keys[h];
        if (k == v) return h;
        if (k == EMPTY) return EMPTY;
        h = (h + 1) & (T - 1);
    }
    return EMPTY;
}

// Bits lo..hi-1 of a lane mask (0 <= lo <= hi <= 32).
__device__ __forceinline__ uint32_t qb_lane_range(uint32_t lo, uint32_t hi) {
    const uint32_t h = hi >= 32 ? FULL : ((1u << hi) - 1u);
    return h & ~((1u << lo) - 1u);
}

// Marks `slot` as queued in direction `dir` for the next level (bitmap of
// the level's parity); true if it was not queued yet.
template <int TB>
__device__ __forceinline__ bool qb_claim(QBSmem<TB> &q, uint32_t slot, uint32_t dir, uint32_t lvl) {
    const uint32_t bit = 1u << (slot & 31u);
    return !(atomicOr(&q.claim[lvl & 1u][dir][slot >> 5], bit) & bit);
}

// Per-thread work counters of the searches (queued entries expanded, edges
// scanned), summed once per thread when a kernel ends.
struct QStat {
    unsigned long long exp = 0, edges = 0;
};

// Relaxes one edge e = (y, w) of a vertex labelled dx in direction dir.
// Returns nothing; records an overflow in q.ovf, an index error in a.err.
// With TRACK, lmf / lmb keep the least new forward / backward label this
// thread has set in the level (every vertex whose label drops is queued for
// the next level).
template <bool PRUNE, int TB, bool TRACK = false>
__device__ __forceinline__ void qb_relax(QBSmem<TB> &q, const QArgs &a, uint32_t dir, uint2 e, uint32_t dx,
                                         uint32_t lvl, uint32_t nxt_cnt, uint32_t *next_front, uint32_t &lmf,
                                         uint32_t &lmb) {
    const uint32_t nd = sat_add(dx, e.y);
    if (e.x >= a.n) {
        atomicOr(a.err, QERR_BOUND);
        return;
    }
    if (nd == INF) return;
    if (PRUNE && nd >= q.mu) return;
    const uint32_t ys = qb_insert<TB>(q.key, e.x);
    if (ys == EMPTY) {
        q.ovf = 1;
        return;
    }
    uint32_t *dist = dir ? q.db : q.df;
    const uint32_t old = atomicMin(&dist[ys], nd);
    if (nd >= old) return;
    if (TRACK) {
        if (dir) lmb = min(lmb, nd);
        else lmf = min(lmf, nd);
    }
    if (PRUNE) {
        const uint32_t other = dir ? q.df[ys] : q.db[ys];
        if (other != INF) atomicMin(&q.mu, sat_add(nd, other));
    }
    if (qb_claim(q, ys, dir, lvl)) {
        const uint32_t p = atomicAdd(&q.cnt3[nxt_cnt], 1u);
        if (p < QBSmem<TB>::FC) next_front[p] = ys | (dir << 31);
        else q.ovf = 1;
    }
}

// Loads what expanding one frontier entry needs: its vertex's edge range in
// the direction's CSR and its label. cnt = 0 for an invalid entry.
template <int TB>
__device__ __forceinline__ void qb_entry(const QBSmem<TB> &q, const QArgs &a, bool fv, uint32_t ent,
                                         uint32_t &b, uint32_t &cnt, uint32_t &dx) {
    const uint32_t dir = ent >> 31;
    const uint32_t slot = ent & 0x7FFFFFFFu;
    const bool sok = fv && slot < QBSmem<TB>::T;
    if (fv && !sok) atomicOr(a.err, QERR_BOUND);
    const uint32_t x = sok ? q.key[slot] : 0;
    const bool xok = sok && x < a.n;
    if (sok && !xok) atomicOr(a.err, QERR_BOUND);
    const uint32_t *off = dir ? a.dn_off : a.up_off;
    const uint32_t n_edges = dir ? a.n_dn : a.n_up;
    b = xok ? off[x] : 0;
    const uint32_t e_end = xok ? off[x + 1] : 0;
    cnt = 0;
    if (xok && b <= e_end && e_end <= n_edges) cnt = e_end - b;
    else if (xok) atomicOr(a.err, QERR_BOUND);
    if (a.core_tab && x >= a.core_lo) cnt = 0;  // a core vertex: joined through the table
    dx = cnt ? (dir ? q.db[slot] : q.df[slot]) : INF;
}

// qb_entry plus the stall test's edge range: the offsets of the entry's
// vertex in both CSRs, loaded together before any check, so that they cost
// one round trip to L2 instead of two. sb / se: the other CSR's range
// (0, 0 when cnt = 0).
template <int TB>
__device__ __forceinline__ void qb_entry_both(const QBSmem<TB> &q, const QArgs &a, bool fv, uint32_t ent,
                                              uint32_t &b, uint32_t &cnt, uint32_t &dx, uint32_t &sb,
                                              uint32_t &se) {
    const uint32_t dir = ent >> 31;
    const uint32_t slot = ent & 0x7FFFFFFFu;
    const bool sok = fv && slot < QBSmem<TB>::T;
    const uint32_t x = sok ? q.key[slot] : 0;
    const bool xok = sok && x < a.n;
    const uint32_t *off = dir ? a.dn_off : a.up_off;
    const uint32_t *soff = dir ? a.up_off : a.dn_off;
    uint32_t e_end = 0;
    b = sb = se = 0;
    if (xok) {
        b = off[x];
        e_end = off[x + 1];
        sb = soff[x];
        se = soff[x + 1];
    }
    if (fv && !sok) atomicOr(a.err, QERR_BOUND);
    if (sok && !xok) atomicOr(a.err, QERR_BOUND);
    const uint32_t n_edges = dir ? a.n_dn : a.n_up;
    cnt = 0;
    if (xok && b <= e_end && e_end <= n_edges) cnt = e_end - b;
    else if (xok) atomicOr(a.err, QERR_BOUND);
    if (a.core_tab && x >= a.core_lo) cnt = 0;  // a core vertex: joined through the table
    dx = cnt ? (dir ? q.db[slot] : q.df[slot]) : INF;
    if (!cnt) sb = se = 0;
}

// Both upward searches at once, label-correcting over the rank DAG: the
// frontier holds forward (E_up) and backward (reversed E_down) entries,
// each level relaxes the out-edges of every queued vertex with its current
// label, and the search ends when no label changed. With PRUNE, a relaxation
// whose new label is not below the best meeting sum found so far is skipped
// (it cannot improve the answer); the answer is always recomputed at the
// end as the least df + db over the table, so it is exact either way.
//
// Two ways to spread a level over the block (same result, different cost):
//  - block-flattened (WARP = false): tiles of blockDim frontier entries; the
//    out-edges of a tile are spread evenly over all threads (block-wide
//    scan, owner found by binary search); two barriers per tile.
//  - warp-flattened (WARP = true): frontier entries are dealt to warps
//    round-robin, each warp spreads the out-edges of its (up to 32) entries
//    over its lanes (warp scan, owner found by shuffles); no barrier inside
//    a level.
//
// DELTA (warp-flattened, pruned searches) orders the levels like
// delta-stepping: a level expands only the entries within a.delta of their
// direction's least queued label and keeps the others queued, so fewer
// vertices are expanded again after a later improvement; an entry whose
// label is not below the best meeting sum is dropped (every relaxation from
// it would be skipped). The least queued label of each direction is
// expanded every level and new labels exceed it, so the least label grows
// every level and the search ends.
//
// Barrier discipline: the frontier counter of level k lives in cnt3[k % 3],
// and (DELTA) the least labels queued for it in lmin3[k % 3]; thread 0
// clears both for level k + 2 during level k, when no thread reads them any
// more. Each level reads its frontier size and the overflow
// flag right after a barrier that follows every write to them: the barrier
// at the top of the level (warp-flattened; block-flattened at level 1) or
// the barrier that ends the previous level's last tile (block-flattened).
template <bool PRUNE, bool WARP, int TB, bool STALL, bool DELTA = false>
__device__ bool block_search(QBSmem<TB> &q, const QArgs &a, QStat &stat) {
    static_assert(!DELTA || (PRUNE && WARP), "delta-stepping levels: pruned warp-flattened searches");
    constexpr uint32_t FC = QBSmem<TB>::FC, CW = QBSmem<TB>::CW;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    for (uint32_t lvl = 1;; ++lvl) {
        if (WARP || lvl == 1) __syncthreads();
        const uint32_t cur = (lvl - 1) & 1u;
        const uint32_t nfront = q.cnt3[(lvl - 1) % 3];
        const uint32_t ovf = q.ovf;
        if (ovf) return false;
        if (nfront == 0) return true;
        if (lvl >= 0xFFFFu) {  // a label-correcting search on a DAG never gets here
            if (tid == 0) atomicOr(a.err, QERR_BOUND);
            return false;
        }
        uint32_t thr_f = INF, thr_b = INF;  // DELTA: this level's label thresholds
        if (DELTA) {
            thr_f = sat_add(q.lmin3[(lvl - 1) % 3][0], a.delta);
            thr_b = sat_add(q.lmin3[(lvl - 1) % 3][1], a.delta);
        }
        if (tid == 0) {
            q.cnt3[(lvl + 1) % 3] = 0;
            if (DELTA) q.lmin3[(lvl + 1) % 3][0] = q.lmin3[(lvl + 1) % 3][1] = INF;
        }
        // the bitmap of the other parity was last used two levels ago and is
        // next used one level from now
        for (uint32_t j = tid; j < 2u * CW; j += blockDim.x) (&q.claim[(lvl + 1) & 1u][0][0])[j] = 0;
        const uint32_t nxt_cnt = lvl % 3;
        uint32_t *next_front = q.front[cur ^ 1u];
        uint32_t lmf = INF, lmb = INF;  // DELTA: least labels this thread queues
        if (WARP) {
            const uint32_t stride = blockDim.x;
            for (uint32_t p0 = 0; p0 < nfront; p0 += stride) {
                const uint32_t fi = p0 + warp + nwarps * lane;
                bool fv = fi < nfront && fi < FC;
                const uint32_t ent = fv ? q.front[cur][fi] : 0;
                if (DELTA) {
                    // keep an entry above its direction's threshold queued
                    // (warp-aggregated push); drop one that cannot improve
                    // the meeting sum
                    const uint32_t edir = ent >> 31, eslot = ent & 0x7FFFFFFFu;
                    const bool sok = fv && eslot < QBSmem<TB>::T;
                    const uint32_t lab = sok ? (edir ? q.db[eslot] : q.df[eslot]) : INF;
                    const bool drop = sok && lab >= q.mu;
                    const bool keep = sok && !drop && lab > (edir ? thr_b : thr_f);
                    const bool won = keep && qb_claim(q, eslot, edir, lvl);
                    const uint32_t m = __ballot_sync(FULL, won);
                    if (m) {
                        const uint32_t leader = __ffs(m) - 1;
                        uint32_t p = 0;
                        if (lane == leader) p = atomicAdd(&q.cnt3[nxt_cnt], (uint32_t)__popc(m));
                        p = __shfl_sync(FULL, p, leader) + __popc(m & ((1u << lane) - 1u));
                        if (won) {
                            if (p < FC) next_front[p] = ent;
                            else q.ovf = 1;
                            if (edir) lmb = min(lmb, lab);
                            else lmf = min(lmf, lab);
                        }
                    }
                    if (keep || drop) fv = false;
                }
                uint32_t b, cnt, dx, psb = 0, pse = 0;
                if (DELTA) qb_entry_both(q, a, fv, ent, b, cnt, dx, psb, pse);
                else qb_entry(q, a, fv, ent, b, cnt, dx);
                stat.exp += cnt ? 1u : 0u;
                if (STALL) {
                    // Stall on demand: the entry's vertex x is not expanded
                    // when a reached higher neighbour y gives a shorter path
                    // to it (forward: an E_down edge y -> x with
                    // df[y] + w < df[x]; backward: an E_up edge x -> y with
                    // w + db[y] < db[x]). Its label then exceeds the true
                    // distance, so x with that label lies on no shortest
                    // up-path; a vertex whose label is exact is never stalled,
                    // and a later improvement queues x again.
                    const uint32_t dir = ent >> 31;
                    const uint32_t slot = ent & 0x7FFFFFFFu;
                    const uint32_t x = (cnt && !DELTA) ? q.key[slot] : 0;
                    const uint32_t *soff = dir ? a.up_off : a.dn_off;
                    const uint32_t s_edges = dir ? a.n_up : a.n_dn;
                    const uint32_t sb = DELTA ? psb : (cnt ? soff[x] : 0);
                    const uint32_t se = DELTA ? pse : (cnt ? soff[x + 1] : 0);
                    uint32_t scnt = 0;
                    if (cnt && sb <= se && se <= s_edges) scnt = se - sb;
                    else if (cnt) atomicOr(a.err, QERR_BOUND);
                    const uint32_t sincl = warp_incl_scan(scnt);
                    const uint32_t stotal = __shfl_sync(FULL, sincl, 31);
                    const uint32_t sexcl = sincl - scnt;
                    bool stalled = false;
                    for (uint32_t base = 0; base < stotal; base += 32) {
                        const uint32_t e0 = base + lane;
                        const uint32_t o = warp_owner(sexcl, e0);
                        const uint32_t osb = __shfl_sync(FULL, sb, o);
                        const uint32_t oex = __shfl_sync(FULL, sexcl, o);
                        const uint32_t odx = __shfl_sync(FULL, dx, o);
                        const uint32_t odir = __shfl_sync(FULL, ent, o) >> 31;
                        bool st = false;
                        if (e0 < stotal) {
                            ++stat.edges;
                            const uint2 e = (odir ? a.up_adj : a.dn_adj)[osb + (e0 - oex)];
                            const uint32_t ys = e.x < a.n ? qb_find<TB>(q.key, e.x) : EMPTY;
                            if (ys != EMPTY) st = sat_add(odir ? q.db[ys] : q.df[ys], e.y) < odx;
                        }
                        const uint32_t B = __ballot_sync(FULL, st);
                        const uint32_t lo = max(sexcl, base), hi = min(sexcl + scnt, base + 32);
                        if (hi > lo && (B & qb_lane_range(lo - base, hi - base))) stalled = true;
                    }
                    if (stalled) cnt = 0;
                }
                const uint32_t incl = warp_incl_scan(cnt);
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                const uint32_t excl = incl - cnt;
                for (uint32_t base = 0; base < total; base += 32) {
                    const uint32_t e0 = base + lane;
                    const uint32_t o = warp_owner(excl, e0);
                    const uint32_t ob = __shfl_sync(FULL, b, o);
                    const uint32_t oex = __shfl_sync(FULL, excl, o);
                    const uint32_t odx = __shfl_sync(FULL, dx, o);
                    const uint32_t odir = __shfl_sync(FULL, ent, o) >> 31;
                    if (e0 < total) {
                        ++stat.edges;
                        const uint2 e = (odir ? a.dn_adj : a.up_adj)[ob + (e0 - oex)];
                        qb_relax<PRUNE, TB, DELTA>(q, a, odir, e, odx, lvl, nxt_cnt, next_front, lmf, lmb);
                    }
                }
            }
            if (DELTA) {
                // the least labels queued for the next level, one atomic per
                // warp and direction
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lmf = min(lmf, __shfl_xor_sync(FULL, lmf, o));
                    lmb = min(lmb, __shfl_xor_sync(FULL, lmb, o));
                }
                if (lane == 0) {
                    if (lmf != INF) atomicMin(&q.lmin3[nxt_cnt][0], lmf);
                    if (lmb != INF) atomicMin(&q.lmin3[nxt_cnt][1], lmb);
                }
            }
        } else {
            for (uint32_t t0 = 0; t0 < nfront; t0 += blockDim.x) {
                const uint32_t fi = t0 + tid;
                const bool fv = fi < nfront && fi < FC;
                const uint32_t ent = fv ? q.front[cur][fi] : 0;
                uint32_t b, cnt, dx;
                qb_entry(q, a, fv, ent, b, cnt, dx);
                stat.exp += cnt ? 1u : 0u;
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
                    ++stat.edges;
                    const uint32_t odir = q.t_ent[lo] >> 31;
                    const uint2 e = (odir ? a.dn_adj : a.up_adj)[q.t_beg[lo] + (e0 - q.t_excl[lo])];
                    qb_relax<PRUNE, TB>(q, a, odir, e, q.t_dx[lo], lvl, nxt_cnt, next_front, lmf, lmb);
                }
                __syncthreads();
            }
        }
    }
}

// Empties the block's table and claim bitmaps (at kernel start; every query
// leaves them empty again).
template <int TB>
__device__ __forceinline__ void qb_clear(QBSmem<TB> &q) {
    for (uint32_t j = threadIdx.x; j < QBSmem<TB>::T; j += blockDim.x) {
        q.key[j] = EMPTY;
        q.df[j] = INF;
        q.db[j] = INF;
    }
    for (uint32_t j = threadIdx.x; j < 4u * QBSmem<TB>::CW; j += blockDim.x) (&q.claim[0][0][0])[j] = 0;
}

// One s-t query (rank ids rs, rt < n) by the whole block, on the shared
// table, which must be empty on entry and is empty again on return: seeds
// both roots, searches, then reduces the answer in the same pass that
// empties the table. Returns false, in every thread, when the search spaces
// overflowed the table or the frontier (the caller redoes the query
// elsewhere); otherwise mu and cnt hold, in every thread, the least meeting
// sum and the number of labels set. Every thread of the block must call it.
template <bool PRUNE, bool WARP, int TB, bool STALL = false, bool DELTA = false>
__device__ bool block_query(QBSmem<TB> &q, const QArgs &a, uint32_t rs, uint32_t rt, uint32_t &mu_out,
                            uint32_t &cnt_out, QStat &stat) {
    const uint32_t tid = threadIdx.x;
    __syncthreads();
    if (tid == 0) {
        const uint32_t ss = qb_insert<TB>(q.key, rs);
        q.df[ss] = 0;
        const uint32_t st = qb_insert<TB>(q.key, rt);
        q.db[st] = 0;
        q.ovf = 0;
        q.mu = ss == st ? 0u : INF;
        q.cnt = 0;
        q.front[0][0] = ss;
        q.front[0][1] = st | 0x80000000u;
        q.cnt3[0] = 2;
        q.cnt3[1] = 0;
        q.cnt3[2] = 0;
        if (DELTA) {
            q.lmin3[0][0] = q.lmin3[0][1] = 0;  // the two roots
            q.lmin3[1][0] = q.lmin3[1][1] = INF;
        }
    }
    bool ok = block_search<PRUNE, WARP, TB, STALL, DELTA>(q, a, stat);
    // q.mu only steered pruning; the answer is the least meeting sum.
    __syncthreads();
    if (tid == 0) {
        q.mu = INF;
        q.cnt3[0] = 0;
        q.cnt3[1] = 0;
    }
    __syncthreads();
    uint32_t mu = INF, cnt = 0;
    if (a.core_tab && ok) {
        // Core entries of the two searches (their slots, in the two
        // frontier arrays, free now), then the least
        // d_s(c1) + table(c1, c2) + d_t(c2) over every pair.
        constexpr uint32_t FC = QBSmem<TB>::FC;
        for (uint32_t j = tid; j < QBSmem<TB>::T; j += blockDim.x) {
            const uint32_t k = q.key[j];
            if (k == EMPTY || k < a.core_lo || k >= a.n) continue;
            if (q.df[j] != INF) {
                const uint32_t p = atomicAdd(&q.cnt3[0], 1u);
                if (p < FC) q.front[0][p] = j;
            }
            if (q.db[j] != INF) {
                const uint32_t p = atomicAdd(&q.cnt3[1], 1u);
                if (p < FC) q.front[1][p] = j;
            }
        }
        __syncthreads();
        const uint32_t nf = q.cnt3[0], nb = q.cnt3[1];
        if (nf > FC || nb > FC) {
            ok = false;  // too many core entries: redone by the full search
        } else {
            const uint64_t pairs = (uint64_t)nf * nb;
            for (uint64_t p = tid; p < pairs; p += blockDim.x) {
                const uint32_t sf = q.front[0][p / nb], sb = q.front[1][p % nb];
                const uint32_t cf = q.key[sf] - a.core_lo, cb = q.key[sb] - a.core_lo;
                const uint32_t dcc = a.core_tab[(uint64_t)cf * a.core_n + cb];
                mu = min(mu, sat_add(sat_add(q.df[sf], dcc), q.db[sb]));
            }
        }
        __syncthreads();
    }
    for (uint32_t j = tid; j < QBSmem<TB>::T; j += blockDim.x) {
        const uint32_t f = q.df[j], g = q.db[j];
        mu = min(mu, sat_add(f, g));
        cnt += (f != INF) + (g != INF);
        q.key[j] = EMPTY;
        q.df[j] = INF;
        q.db[j] = INF;
    }
    for (uint32_t j = tid; j < 4u * QBSmem<TB>::CW; j += blockDim.x) (&q.claim[0][0][0])[j] = 0;
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
    return ok;
}

// Adds the block's counters to stats[0] (expansions) and stats[1] (edges).
__device__ __forceinline__ void qb_flush_stat(const QStat &stat, unsigned long long *stats) {
    if (!stats) return;
    unsigned long long e = stat.exp, g = stat.edges;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(FULL, e, o);
        g += __shfl_xor_sync(FULL, g, o);
    }
    if (lane_id() == 0) {
        atomicAdd(&stats[0], e);
        atomicAdd(&stats[1], g);
    }
}

}  // namespace
}  // namespace gbch
