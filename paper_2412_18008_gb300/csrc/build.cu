// Round-synchronous contraction-hierarchy construction on one GPU.
//
// Paper: "Parallel Contraction Hierarchies Can Be Efficient and Scalable"
// (arXiv 2412.18008), Alg. 2 (round loop), Alg. 3 (LocalSearch, batched per
// source), Alg. 4 (Score = edge difference), Alg. 5 (Select = strict local
// minimum of the score, ties by label), Alg. 6 (Contract), Sec. 4 (overlay in
// CSR form, duplicate shortcuts keep the minimum weight) and the
// Postprocessing of Sec. 3.5 (vertices ranked by level, then score).
//
// GPU design (one round = the steps below, one host synchronisation):
//   1 score_prep     A_r: P[u] = -(|N_in|+|N_out|); sources N_in(A_r) listed
//   2 witness SCORE  one warp per source s: hop-limited Bellman-Ford from s
//                    in shared memory, then every pair (s, u, v2) with u in
//                    A_r adds 1 to P[u] when w(s,u)+w(u,v2) <= d_H(s, v2)
//   3 select         V_F = strict local minima of key(u) = (P[u], tie(u))
//   4 contract_prep  sources N_in(V_F), next affected set N(V_F), bounds
//   -- host reads the round's counters once and grows buffers if needed --
//   5 witness PRUNE  same search; kept candidates merged per (s, v2) in
//                    shared memory (min weight, then min via) and checked
//                    against the existing overlay edge
//   6 emit_ch        out/in lists of V_F become E_up / E_down
//   7 compact_lists  neighbour lists of N(V_F) drop the contracted vertices
//   8 reserve        lists short of slack are moved by a prefix sum over
//                    their new capacities
//   9 insert         shortcuts appended into the slack (or weights lowered)
//  10 compact VO     stable compaction of the live-vertex list
//
// The witness distance is d_H(a, b), the least weight of a walk a -> b with
// at most H edges in the round's overlay (INF if none); a candidate
// (v1, u, v2), v1 != v2, is kept iff w(v1,u) + w(u,v2) <= d_H(v1, v2). Each
// search keeps only partial walks lighter than the heaviest candidate
// weight of its source, which leaves every decision unchanged: a walk at
// least that heavy can only show d_H >= the candidate's weight.
//
// Everything the kernels compute is a function of the overlay's edge *sets*
// (searches take minima, selection compares keys, merges take minima), so
// results do not depend on the order in which atomics append to lists.

#include <algorithm>
#include <chrono>
#include <cstring>

#include "handle.cuh"
#include "mlp.cuh"
#include "prims.cuh"

namespace gbch {
namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr uint32_t ERR_INPUT = 1u;
constexpr uint32_t ERR_REC_OVERFLOW = 2u;
constexpr uint32_t ERR_CH_OVERFLOW = 4u;
constexpr uint32_t ERR_BOUND = 8u;  // an index check failed; the access was skipped
constexpr uint32_t ERR_MAP_FULL = 16u;  // the memoised-distance map has no free slot

constexpr int MODE_SCORE = 0;
constexpr int MODE_PRUNE = 1;

// Optional witness-search features, instantiated separately so that the
// plain kernels stay as they are: memoised distances across rounds, and the
// bound on a hop level's frontier out-edges.
constexpr int F_XM = 1;
constexpr int F_LW = 2;
// Pruning of overlay edges heavier than their pair's witness distance: the
// searches' label bound also covers the direct edges (s, v) to new targets
// (without a ball bound), so the recorded value decides the deletion. Needs
// F_XM (the recorded values live in the memoised-distance map).
constexpr int F_PR = 4;
// Alg. 3's search itself: a Dijkstra from the source that stops once its new
// targets or theta vertices are settled, equal labels settled in id order.
// Replaces the hop-limited search; the block tier is skipped (its sources go
// to the global-memory tier).
constexpr int F_TH = 8;

// Weight of the overlay edge (s, v) from s's out-list, INF if none.
__device__ __forceinline__ uint32_t direct_weight(const uint2 *out_adj, uint64_t sb, uint32_t sd, uint32_t v) {
    for (uint32_t j = 0; j < sd; ++j) {
        const uint2 e = out_adj[sb + j];
        if (e.x == v) return e.y;
    }
    return INF;
}

// Shared-memory search state of one warp.
constexpr int WIT_WARPS = 4;       // warps per block
constexpr int WIT_TBITS = 8;       // hash table of 2^8 vertices
constexpr int WIT_T = 1 << WIT_TBITS;
constexpr int WIT_FC = 128;        // frontier capacity per level
constexpr int WIT_MC = 128;        // distinct targets merged per source

struct Ctl {
    uint32_t nVO, nVO2, nS, nS2, nF, nAnext, nOvf, nRec;
    uint32_t err, work, work2, work3, nOvf2, pad;
    unsigned long long candBound, degFout, degFin, degAnext;
    unsigned long long cand, kept, merged, inserted, newEdges;
    unsigned long long out_tail, in_tail, ch_up_tail, ch_dn_tail;
    unsigned long long relocOut, relocIn;
    unsigned long long wit_sources, wit_fallback, wit_vertices, wit_edges, wit_middles,
        wit_midedges, wit_block;
    unsigned long long trace_valid;  // trace rows of eligible rescorings
    unsigned long long dm_count;     // keys in the memoised-distance map since its last clear
    unsigned long long pruned;       // overlay edges pruned this round
    uint32_t nDirty;                 // vertices whose lists hold pruned entries
    uint32_t longRows;               // rank-ordered CSR rows left for the radix sort
    // shortcut log entries so far (device-side, so that k_insert needs no
    // host value), and the contraction counters of the last finished round,
    // copied by k_round_end for the host's next read
    unsigned long long log_tail;
    unsigned long long s_cand, s_kept, s_merged, s_inserted, s_newEdges, s_nRec, s_dm_count;
};

struct Dev {
    uint32_t n;
    uint32_t H;
    uint32_t tie_mode, tie_seed;
    uint64_t *out_beg, *in_beg;
    uint32_t *out_deg, *in_deg, *out_cap, *in_cap;
    uint2 *out_adj, *in_adj;
    uint32_t *level;
    int32_t *P;
    uint32_t *amark, *smark;
    uint32_t *new_out, *new_in;
    Ctl *ctl;
    uint64_t out_arena, in_arena;  // arena capacities (entries), for index checks
    // learned-priority bookkeeping (see k_features)
    uint32_t *cn, *depth, *rescore, *orig_deg;
    int32_t *ed_last, *label;
    // candidate bound: a rescored vertex with |N_in| * |N_out| > cmax is not
    // eligible (not scored, never selected) until rescored within the bound
    uint64_t cmax;
    uint8_t *inel;
    // witness ball bound: a search stops after the first hop level at which
    // more than `ball` vertices (the source included) hold a label
    uint32_t ball;
    // In-round memo of the score phase's decisions (only without a ball
    // bound, where both phases decide every candidate the same way):
    // emask[p] for the overlay edge (s, u) at arena position p holds bit j
    // set iff the candidate (s, u, j-th out-neighbour of u) was kept; valid
    // when kround[u] == round + 1 (u rescored this round, at most 64
    // out-edges).
    unsigned long long *emask;
    uint32_t *kround;
    bool memo;
};

constexpr uint32_t MEMO_MAX_OUT = 64;

constexpr int32_t P_INELIGIBLE = 2147483646;  // INT32_MAX - 1
constexpr uint32_t AMARK_NONE = 0xFFFFFFFFu;   // never a round index

// Memoised witness distances across phases and rounds (Alg. 3's dist map):
// open addressing on 64-bit keys (s << 32 | v) with linear probing, the
// distance in a parallel array. Only the source s touches keys (s, .), and it
// inserts them only after all of its decisions of the phase are made, so a
// key a search finds was written, with its value, by an earlier launch. Keys
// are never removed between two clears, so a probe that reaches an empty
// slot before its key proves the key absent.
constexpr unsigned long long DMAP_EMPTY = ~0ull;
// An insertion never places a key further than this from its home slot (it
// reports the map full instead), so a lookup may stop there too.
constexpr unsigned long long DMAP_MAXPROBE = 4096;

struct DMap {
    unsigned long long *keys;
    uint32_t *vals;
    unsigned long long mask;  // capacity - 1; the capacity is a power of two
    unsigned long long *count;
};

__device__ __forceinline__ unsigned long long dmap_key(uint32_t s, uint32_t v) {
    return ((unsigned long long)s << 32) | v;
}

// SplitMix64's output finaliser (Steele, Lea and Flood, OOPSLA 2014) spreads
// the keys over the slots.
__device__ __forceinline__ unsigned long long dmap_hash(unsigned long long x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ bool dmap_get(const DMap &m, unsigned long long key, uint32_t *val) {
    unsigned long long i = dmap_hash(key) & m.mask;
    for (unsigned long long p = 0; p < DMAP_MAXPROBE && p <= m.mask; ++p) {
        const unsigned long long k = m.keys[i];
        if (k == key) {
            *val = m.vals[i];
            return true;
        }
        if (k == DMAP_EMPTY) return false;
        i = (i + 1) & m.mask;
    }
    return false;
}

// Records key -> val unless the key is present: 1 = inserted, 0 = present,
// -1 = no free slot.
__device__ __forceinline__ int dmap_put(const DMap &m, unsigned long long key, uint32_t val) {
    unsigned long long i = dmap_hash(key) & m.mask;
    for (unsigned long long p = 0; p < DMAP_MAXPROBE && p <= m.mask; ++p) {
        unsigned long long k = m.keys[i];
        if (k == key) return 0;
        if (k == DMAP_EMPTY) {
            k = atomicCAS(&m.keys[i], DMAP_EMPTY, key);
            if (k == DMAP_EMPTY) {
                m.vals[i] = val;
                return 1;
            }
            if (k == key) return 0;
        }
        i = (i + 1) & m.mask;
    }
    return -1;
}

// Moves every key of `from` into the larger map `to` (the count is unchanged).
__global__ void k_dmap_rehash(DMap from, DMap to, Ctl *ctl) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i <= from.mask;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long k = from.keys[i];
        if (k != DMAP_EMPTY && dmap_put(to, k, from.vals[i]) < 0) atomicOr(&ctl->err, ERR_MAP_FULL);
    }
}

struct WArgs {
    Dev d;
    DMap dm;                 // memoised distances (witness kernels instantiated with XM)
    const uint32_t *S;       // source list
    const uint32_t *nS;      // its length (device)
    uint32_t *work;          // dynamic work counter
    uint32_t round;
    uint32_t *ovf;           // sources the warp tier could not hold (for the block tier)
    uint32_t *ovf2;          // sources the block tier could not hold (for the dense tier)
    uint4 *rec;              // PRUNE: shortcut records (v1, v2, w, via)
    uint8_t *rec_flag;       // PRUNE: 1 = lowers an existing edge
    uint64_t rec_cap;
    // Routing to the block tier without a warp attempt: every source when
    // the phase has at most route_all sources (16 times the block tier's
    // grid: with that few sources per-source latency decides, and a block
    // finishes a source sooner than a warp), and any source whose middles'
    // out-degrees sum above route_deg (its ball would overflow).
    uint32_t route_all, route_deg;
    // F_LW: a hop level from the second on whose frontier has more
    // out-edges than this is not run
    unsigned long long level_work;
    uint32_t theta;  // F_TH: settled-vertex cap
};

struct Dense {
    uint32_t *dist, *fst, *fa, *fb, *fda, *fdb, *touched, *mt;
    uint32_t *direct;  // weight of the edge (s, v) of the current source s, INF if none
    unsigned long long *merge;
    uint32_t nslots;
};

// Sources with more out-edges than this skip the shared-memory tiers (their
// balls and existing-edge checks belong to the global-memory tier).
constexpr uint32_t DENSE_SD = 1024;

__device__ __forceinline__ uint64_t select_key(const Dev &d, uint32_t v) {
    uint32_t hi = (uint32_t)d.P[v] ^ 0x80000000u;
    uint32_t lo = d.tie_mode == CH_TIE_ID ? v : murmur_fmix32(v ^ d.tie_seed);
    return ((uint64_t)hi << 32) | lo;
}

template <int MODE>
__device__ __forceinline__ bool is_middle(const Dev &d, uint32_t u, uint32_t r) {
    if (MODE == MODE_SCORE) return d.amark[u] == r;
    return d.level[u] == r;
}

// Index checks: a list must lie inside its arena and hold ids below n. A
// failed check sets ERR_BOUND (reported as an error by the host) and the
// caller skips the access instead of faulting.
__device__ __forceinline__ bool out_list_ok(const Dev &d, uint64_t beg, uint32_t deg) {
    if (beg + deg <= d.out_arena) return true;
    atomicOr(&d.ctl->err, ERR_BOUND);
    return false;
}
__device__ __forceinline__ bool in_list_ok(const Dev &d, uint64_t beg, uint32_t deg) {
    if (beg + deg <= d.in_arena) return true;
    atomicOr(&d.ctl->err, ERR_BOUND);
    return false;
}
__device__ __forceinline__ bool id_ok(const Dev &d, uint32_t v) {
    if (v < d.n) return true;
    atomicOr(&d.ctl->err, ERR_BOUND);
    return false;
}

__device__ __forceinline__ uint32_t lane_bits(uint32_t lo, uint32_t hi) {
    uint32_t h = hi >= 32 ? FULL : ((1u << hi) - 1u);
    return h & ~((1u << lo) - 1u);
}

// --------------------------------------------------------------------------
// Normalisation (drop self-loops, merge parallel edges by minimum weight)
// --------------------------------------------------------------------------

__global__ void k_validate_offsets(const uint64_t *off, uint32_t n, uint64_t m, Ctl *ctl) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        bool bad = off[i] > off[i + 1];
        if (i == 0 && off[0] != 0) bad = true;
        if (i == n - 1 && off[n] != m) bad = true;
        if (bad) atomicOr(&ctl->err, ERR_INPUT);
    }
}

__global__ void k_edge_keys(const uint64_t *off, const uint32_t *tgt, const uint32_t *w,
                            uint32_t n, uint64_t m, uint64_t *keys, uint32_t *vals, Ctl *ctl) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = n;  // largest u with off[u] <= e
        while (hi - lo > 1) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (off[mid] <= e) lo = mid; else hi = mid;
        }
        uint32_t v = tgt[e], ww = w[e];
        if (v >= n || ww == 0 || ww == INF) atomicOr(&ctl->err, ERR_INPUT);
        keys[e] = ((uint64_t)lo << 32) | (v < n ? v : 0);
        vals[e] = ww;
    }
}

__global__ void k_norm_flags(const uint64_t *keys, uint64_t m, uint32_t *flag) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[e];
        bool head = e == 0 || keys[e - 1] != k;
        flag[e] = head && (uint32_t)(k >> 32) != (uint32_t)k ? 1u : 0u;
    }
}

__global__ void k_norm_scatter(const uint64_t *keys, const uint32_t *vals, uint64_t m,
                               const uint32_t *pos, uint64_t *okeys, uint32_t *ovals) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[e];
        bool head = e == 0 || keys[e - 1] != k;
        if (!head || (uint32_t)(k >> 32) == (uint32_t)k) continue;
        uint32_t ww = vals[e];
        for (uint64_t f = e + 1; f < m && keys[f] == k; ++f) ww = min(ww, vals[f]);
        okeys[pos[e]] = k;
        ovals[pos[e]] = ww;
    }
}

__global__ void k_swap_key_halves(uint64_t *keys, uint64_t m) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[e];
        keys[e] = (k << 32) | (k >> 32);
    }
}

// Degrees and segment starts of a (u, v)-sorted edge list keyed by u.
__global__ void k_seg_heads(const uint64_t *keys, uint64_t m, uint64_t *first) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = (uint32_t)(keys[e] >> 32);
        if (e == 0 || (uint32_t)(keys[e - 1] >> 32) != u) first[u] = e;
    }
}

__global__ void k_seg_deg(const uint64_t *keys, uint64_t m, const uint64_t *first,
                          uint32_t *deg) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = (uint32_t)(keys[e] >> 32);
        if (e + 1 == m || (uint32_t)(keys[e + 1] >> 32) != u) deg[u] = (uint32_t)(e + 1 - first[u]);
    }
}

__host__ __device__ __forceinline__ uint32_t initial_cap(uint32_t deg) {
    return deg < 2 ? deg + 2 : 2 * deg;
}

__global__ void k_caps(const uint32_t *deg, uint32_t n, uint32_t *cap, uint64_t *cap64) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t c = initial_cap(deg[v]);
        cap[v] = c;
        cap64[v] = c;
    }
}

__global__ void k_fill_adj(const uint64_t *keys, const uint32_t *vals, uint64_t m,
                           const uint64_t *first, const uint64_t *beg, uint2 *adj) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = (uint32_t)(keys[e] >> 32);
        adj[beg[u] + (e - first[u])] = make_uint2((uint32_t)keys[e], vals[e]);
    }
}

__global__ void k_iota(uint32_t *a, uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        a[v] = v;
}

// --------------------------------------------------------------------------
// Step 1: rescoring set and witness sources
// --------------------------------------------------------------------------

// One warp per rescored vertex u: its score starts at the edge term, and its
// in-neighbours become witness sources (each once per round).
__global__ void k_score_prep(Dev d, const uint32_t *A, uint32_t nA, uint32_t stamp,
                             uint32_t *S, uint32_t r) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nA; i += nwarps) {
        const uint32_t u = A[i];
        if (!id_ok(d, u)) continue;
        const uint32_t od = d.out_deg[u], id = d.in_deg[u];
        if ((uint64_t)od * id > d.cmax) {
            // not eligible: no score, and not a middle of this round's
            // score searches
            if (lane == 0) {
                d.inel[u] = 1;
                d.P[u] = P_INELIGIBLE;
                d.amark[u] = AMARK_NONE;
            }
            continue;
        }
        if (lane == 0) {
            d.inel[u] = 0;
            d.P[u] = -(int32_t)(od + id);
            d.kround[u] = (d.memo && od <= MEMO_MAX_OUT) ? r + 1 : 0;
        }
        const uint64_t ib = d.in_beg[u];
        if (!in_list_ok(d, ib, id)) continue;
        for (uint32_t j0 = 0; j0 < id; j0 += 32) {
            const uint32_t j = j0 + lane;
            bool add = false;
            uint32_t v1 = 0;
            if (j < id) {
                v1 = d.in_adj[ib + j].x;
                add = id_ok(d, v1) && atomicExch(&d.smark[v1], stamp) != stamp;
            }
            const uint32_t pos = warp_append(add, &d.ctl->nS);
            if (add) S[pos] = v1;
        }
    }
}

// --------------------------------------------------------------------------
// Steps 2 and 5: witness searches, one warp per source
// --------------------------------------------------------------------------

struct __align__(16) WarpSmem {
    uint32_t key[WIT_T];
    uint32_t val[WIT_T];
    uint32_t fst[WIT_T];
    uint2 front[2][WIT_FC];
    uint32_t mkey[WIT_MC];
    unsigned long long mval[WIT_MC];
    uint32_t cnt[32];
    uint32_t nf[2];
};

__device__ __forceinline__ uint32_t ht_hash(uint32_t v, int bits) {
    return (v * 2654435761u) >> (32 - bits);
}

// Slot of v in an open-addressing table (inserting it if absent), or EMPTY
// when the table is full.
__device__ __forceinline__ uint32_t ht_insert(uint32_t *keys, int bits, uint32_t v, bool *created = nullptr) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t h = ht_hash(v, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint32_t k = keys[h];
        if (k == v) return h;
        if (k == EMPTY) {
            uint32_t old = atomicCAS(&keys[h], EMPTY, v);
            if (old == EMPTY) {
                if (created) *created = true;
                return h;
            }
            if (old == v) return h;
        }
        h = (h + 1) & mask;
    }
    return EMPTY;
}

__device__ __forceinline__ uint32_t ht_find(const uint32_t *keys, int bits, uint32_t v) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t h = ht_hash(v, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint32_t k = keys[h];
        if (k == v) return h;
        if (k == EMPTY) return EMPTY;
        h = (h + 1) & mask;
    }
    return EMPTY;
}

template <int MODE, int FEAT>
__global__ void __launch_bounds__(WIT_WARPS * 32) k_witness(WArgs a) {
    constexpr bool XM = (FEAT & F_XM) != 0, LW = (FEAT & F_LW) != 0, PR = (FEAT & F_PR) != 0;
    constexpr bool TH = (FEAT & F_TH) != 0;
    __shared__ WarpSmem smem[WIT_WARPS];
    WarpSmem &w = smem[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const Dev d = a.d;
    Ctl *ctl = d.ctl;
    const uint32_t nS = *a.nS;
    const uint32_t r = a.round;
    const bool route_all = nS <= a.route_all;
    unsigned long long c_src = 0, c_vert = 0, c_edge = 0, c_mid = 0, c_midedge = 0;
    unsigned long long c_cand = 0, c_kept = 0, c_merged = 0, c_ins = 0, c_new = 0;
    unsigned long long c_dm = 0;  // keys added to the memoised-distance map

    while (true) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(a.work, 1u);
        i = __shfl_sync(FULL, i, 0);
        if (i >= nS) break;
        const uint32_t s = a.S[i];
        if (s >= d.n) {
            if (lane == 0) atomicOr(&ctl->err, ERR_BOUND);
            continue;
        }
        // where a source this tier cannot hold goes next (the settled-vertex
        // cap has no block tier)
        auto hand_on = [&]() {
            if (lane == 0) {
                if constexpr (TH) a.ovf2[atomicAdd(&ctl->nOvf2, 1u)] = s;
                else a.ovf[atomicAdd(&ctl->nOvf, 1u)] = s;
            }
        };
        if (route_all) {
            hand_on();
            continue;
        }
        const uint64_t sb = d.out_beg[s];
        const uint32_t sd = d.out_deg[s];
        if (sb + sd > d.out_arena) {
            if (lane == 0) atomicOr(&ctl->err, ERR_BOUND);
            continue;
        }
        if (sd > DENSE_SD) {  // a hub: straight to the global-memory tier
            if (lane == 0) a.ovf2[atomicAdd(&ctl->nOvf2, 1u)] = s;
            continue;
        }
        // Algorithmic-traffic counters of this source, added to the totals
        // only if this tier completes it (an overflowed source is redone,
        // and counted, by the next tier).
        unsigned long long l_vert = 0, l_edge = 0, l_mid = 0, l_midedge = 0;

        // Phase 0: heaviest candidate weight of this source, and whether every
        // contracted middle has its score-phase decisions memoised.
        uint32_t bound = 0;
        bool memo_all = MODE == MODE_PRUNE && d.memo;
        bool any = false;  // XM: a candidate exists (the bound covers new targets only)
        uint32_t direct = 0;  // PR: heaviest overlay edge (s, v) to a new target v
        for (uint32_t c0 = 0; c0 < sd; c0 += 32) {
            const uint32_t j = c0 + lane;
            const bool valid = j < sd;
            const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
            const bool mid = valid && id_ok(d, e.x) && is_middle<MODE>(d, e.x, r);
            uint32_t cnt = mid ? d.out_deg[e.x] : 0;
            const uint64_t ub = mid ? d.out_beg[e.x] : 0;
            if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
            if (MODE == MODE_PRUNE) memo_all = __all_sync(FULL, memo_all && (!mid || d.kround[e.x] == r + 1));
            l_mid += mid;
            l_midedge += cnt;
            const uint32_t incl = warp_incl_scan(cnt);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const uint32_t excl = incl - cnt;
            for (uint32_t b = 0; b < total; b += 32) {
                const uint32_t idx = b + lane;
                const uint32_t o = warp_owner(excl, idx);
                const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                const uint32_t w1 = __shfl_sync(FULL, e.y, o);
                const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                if (idx < total) {
                    const uint2 e2 = d.out_adj[ub_o + (idx - ex_o)];
                    if (e2.x != s) {
                        uint32_t known;
                        if constexpr (XM) any = true;
                        if (!(XM && dmap_get(a.dm, dmap_key(s, e2.x), &known))) {
                            bound = max(bound, sat_add(w1, e2.y));
                            if constexpr (PR) {
                                const uint32_t dw = direct_weight(d.out_adj, sb, sd, e2.x);
                                if (dw != INF) direct = max(direct, dw);
                            }
                        }
                    }
                }
            }
        }
        bound = warp_max(bound);
        // the search's label bound (PR without a ball bound: the direct
        // edges to new targets too)
        uint32_t sbound = bound;
        if constexpr (PR)
            if (d.ball == 0xFFFFFFFFu) sbound = max(bound, warp_max(direct));
        if (warp_sum((uint32_t)l_midedge) > a.route_deg) {
            hand_on();
            continue;
        }
        bool no_cand;
        if constexpr (XM) no_cand = !__any_sync(FULL, any);
        else no_cand = bound == 0;
        if (no_cand) {  // no candidate pair from this source
            c_src += (lane == 0);
            c_mid += l_mid;
            c_midedge += l_midedge;
            continue;
        }

        // Phase 1 with the settled-vertex cap: the new targets are flagged
        // in the table (bit 1 of fst), then each step settles the unsettled
        // vertex of least (label, id) (bit 0) and relaxes its out-edges,
        // until every new target or theta vertices are settled.
        if constexpr (TH) {
            if (!(XM && bound == 0)) {
                for (uint32_t t = lane; t < WIT_T; t += 32) {
                    w.key[t] = EMPTY;
                    w.val[t] = INF;
                    w.fst[t] = 0;
                }
                __syncwarp();
                if (lane == 0) w.val[ht_insert(w.key, WIT_TBITS, s)] = 0;
                __syncwarp();
                bool t_ovf = false;
                uint32_t l_targets = 0;
                for (uint32_t c0 = 0; c0 < sd; c0 += 32) {
                    const uint32_t j = c0 + lane;
                    const bool valid = j < sd;
                    const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
                    const bool mid = valid && id_ok(d, e.x) && is_middle<MODE>(d, e.x, r);
                    uint32_t cnt = mid ? d.out_deg[e.x] : 0;
                    const uint64_t ub = mid ? d.out_beg[e.x] : 0;
                    if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
                    const uint32_t incl = warp_incl_scan(cnt);
                    const uint32_t total = __shfl_sync(FULL, incl, 31);
                    const uint32_t excl = incl - cnt;
                    for (uint32_t b = 0; b < total; b += 32) {
                        const uint32_t idx = b + lane;
                        const uint32_t o = warp_owner(excl, idx);
                        const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                        const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                        if (idx >= total) continue;
                        const uint32_t v2 = d.out_adj[ub_o + (idx - ex_o)].x;
                        uint32_t known;
                        if (v2 == s || !id_ok(d, v2) || (XM && dmap_get(a.dm, dmap_key(s, v2), &known)))
                            continue;
                        const uint32_t slot = ht_insert(w.key, WIT_TBITS, v2);
                        if (slot == EMPTY) t_ovf = true;
                        else if ((atomicOr(&w.fst[slot], 2u) & 2u) == 0) ++l_targets;
                    }
                }
                uint32_t remaining = warp_sum(l_targets);
                t_ovf = __any_sync(FULL, t_ovf);
                uint32_t settled = 0;
                while (!t_ovf && remaining > 0 && settled < a.theta) {
                    __syncwarp();
                    unsigned long long best = ~0ull;
                    uint32_t bslot = 0;
                    for (uint32_t t = lane; t < WIT_T; t += 32) {
                        const uint32_t k = w.key[t];
                        if (k == EMPTY || (w.fst[t] & 1u) || w.val[t] == INF) continue;
                        const unsigned long long c = ((unsigned long long)w.val[t] << 32) | k;
                        if (c < best) {
                            best = c;
                            bslot = t;
                        }
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long ob = __shfl_xor_sync(FULL, best, o);
                        const uint32_t os = __shfl_xor_sync(FULL, bslot, o);
                        if (ob < best) {
                            best = ob;
                            bslot = os;
                        }
                    }
                    if (best == ~0ull) break;  // nothing reachable left
                    const uint32_t x = (uint32_t)best, dx = (uint32_t)(best >> 32);
                    ++settled;
                    remaining -= (w.fst[bslot] & 2u) ? 1u : 0u;
                    __syncwarp();
                    if (lane == 0) w.fst[bslot] |= 1u;
                    if (remaining == 0 || settled >= a.theta) break;
                    const uint64_t xb = d.out_beg[x];
                    uint32_t xd = d.out_deg[x];
                    if (!out_list_ok(d, xb, xd)) xd = 0;
                    l_vert += (lane == 0);
                    l_edge += (lane == 0) ? xd : 0;
                    bool ovf_here = false;
                    for (uint32_t j = lane; j < xd; j += 32) {
                        const uint2 e = d.out_adj[xb + j];
                        if (!id_ok(d, e.x)) continue;
                        const uint32_t nd = sat_add(dx, e.y);
                        if (nd == INF) continue;
                        const uint32_t slot = ht_insert(w.key, WIT_TBITS, e.x);
                        if (slot == EMPTY) {
                            ovf_here = true;
                            continue;
                        }
                        if (!(w.fst[slot] & 1u)) atomicMin(&w.val[slot], nd);
                    }
                    t_ovf = __any_sync(FULL, ovf_here);
                }
                __syncwarp();
                if (t_ovf) {
                    hand_on();
                    continue;
                }
            }
        } else {
        // Phase 1: hop-limited Bellman-Ford from s, levels 1..H, each level
        // relaxing from the previous level's values (frontier snapshots);
        // skipped when the decisions are memoised.
        if (!memo_all && !(XM && bound == 0)) {
        {
            uint4 *k4 = reinterpret_cast<uint4 *>(w.key), *v4 = reinterpret_cast<uint4 *>(w.val),
                  *f4 = reinterpret_cast<uint4 *>(w.fst);
            for (uint32_t t = lane; t < WIT_T / 4; t += 32) {
                k4[t] = make_uint4(EMPTY, EMPTY, EMPTY, EMPTY);
                v4[t] = make_uint4(INF, INF, INF, INF);
                f4[t] = make_uint4(0, 0, 0, 0);
            }
        }
        __syncwarp();
        if (lane == 0) {
            const uint32_t h = ht_hash(s, WIT_TBITS);
            w.key[h] = s;
            w.val[h] = 0;
            w.front[0][0] = make_uint2(h, 0);
        }
        // Control values (frontier size, overflow) stay in registers and are
        // made warp-uniform by __shfl_sync / __any_sync, never by polling
        // shared memory.
        uint32_t nfront = 1;
        uint32_t nkeys = 1;  // vertices holding a label (the ball), warp-uniform
        bool overflowed = false;
        uint32_t cur = 0;
        for (uint32_t lvl = 1; lvl <= d.H && nfront > 0 && nkeys <= d.ball; ++lvl) {
            if constexpr (LW) {
                if (lvl >= 2) {
                    unsigned long long wk = 0;
                    for (uint32_t f = lane; f < nfront; f += 32) wk += d.out_deg[w.key[w.front[cur][f].x]];
                    for (int o = 16; o > 0; o >>= 1) wk += __shfl_xor_sync(FULL, wk, o);
                    if (wk > a.level_work) break;
                }
            }
            const uint32_t nxt = cur ^ 1u;
            if (lane == 0) w.nf[nxt] = 0;
            __syncwarp();
            bool ovf = false;
            uint32_t l_created = 0;
            for (uint32_t f0 = 0; f0 < nfront; f0 += 32) {
                const uint32_t fi = f0 + lane;
                const bool fv = fi < nfront;
                const uint2 fe = fv ? w.front[cur][fi] : make_uint2(0, 0);
                const uint32_t x = fv ? w.key[fe.x] : 0;
                uint32_t cnt = fv ? d.out_deg[x] : 0;
                const uint64_t xb = fv ? d.out_beg[x] : 0;
                if (fv && !out_list_ok(d, xb, cnt)) cnt = 0;
                l_vert += fv;
                l_edge += cnt;
                const uint32_t incl = warp_incl_scan(cnt);
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                const uint32_t excl = incl - cnt;
                for (uint32_t b = 0; b < total; b += 32) {
                    const uint32_t idx = b + lane;
                    const uint32_t o = warp_owner(excl, idx);
                    const uint64_t xb_o = __shfl_sync(FULL, xb, o);
                    const uint32_t dx_o = __shfl_sync(FULL, fe.y, o);
                    const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                    if (idx < total) {
                        const uint2 e = d.out_adj[xb_o + (idx - ex_o)];
                        const uint32_t nd = sat_add(dx_o, e.y);
                        if (nd < sbound && id_ok(d, e.x)) {
                            bool created = false;
                            const uint32_t slot = ht_insert(w.key, WIT_TBITS, e.x, &created);
                            l_created += created;
                            if (slot == EMPTY) {
                                ovf = true;
                            } else {
                                const uint32_t old = atomicMin(&w.val[slot], nd);
                                if (nd < old && atomicExch(&w.fst[slot], lvl) != lvl) {
                                    const uint32_t p = atomicAdd(&w.nf[nxt], 1u);
                                    if (p < WIT_FC) w.front[nxt][p] = make_uint2(slot, 0);
                                    else ovf = true;
                                }
                            }
                        }
                    }
                }
            }
            __syncwarp();
            if (__any_sync(FULL, ovf)) {
                overflowed = true;
                break;
            }
            nkeys += warp_sum(l_created);
            uint32_t nn = 0;
            if (lane == 0) nn = w.nf[nxt];
            nn = __shfl_sync(FULL, nn, 0);
            for (uint32_t p = lane; p < nn; p += 32) w.front[nxt][p].y = w.val[w.front[nxt][p].x];
            __syncwarp();
            cur = nxt;
            nfront = nn;
        }
        __syncwarp();
        if (overflowed) {
            if (lane == 0) a.ovf[atomicAdd(&ctl->nOvf, 1u)] = s;
            continue;
        }
        }  // Phase 1
        }  // hop-limited search

        // Phase 2: decisions for every candidate (s, u, v2).
        if (MODE == MODE_PRUNE) {
            for (uint32_t t = lane; t < WIT_MC; t += 32) {
                w.mkey[t] = EMPTY;
                w.mval[t] = ~0ull;
            }
        }
        __syncwarp();
        uint32_t l_cand = 0, l_kept = 0;
        bool mover = false;
        for (uint32_t c0 = 0; c0 < sd; c0 += 32) {
            const uint32_t j = c0 + lane;
            const bool valid = j < sd;
            const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
            const bool mid = valid && id_ok(d, e.x) && is_middle<MODE>(d, e.x, r);
            uint32_t cnt = mid ? d.out_deg[e.x] : 0;
            const uint64_t ub = mid ? d.out_beg[e.x] : 0;
            if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
            const uint32_t incl = warp_incl_scan(cnt);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const uint32_t excl = incl - cnt;
            if (MODE == MODE_SCORE) w.cnt[lane] = 0;
            // memo of this edge (s, u): recorded in the score phase, read in
            // the contraction phase
            const bool mk = mid && d.memo && d.kround[e.x] == r + 1;
            if (MODE == MODE_SCORE && mk) d.emask[sb + j] = 0;
            const unsigned long long mword = (MODE == MODE_PRUNE && memo_all && mid) ? d.emask[sb + j] : 0;
            __syncwarp();
            for (uint32_t b = 0; b < total; b += 32) {
                const uint32_t idx = b + lane;
                const uint32_t o = warp_owner(excl, idx);
                const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                const uint32_t w1 = __shfl_sync(FULL, e.y, o);
                const uint32_t u_o = __shfl_sync(FULL, e.x, o);
                const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                const bool mk_o = __shfl_sync(FULL, mk, o);
                const unsigned long long mw_o = __shfl_sync(FULL, mword, o);
                if (idx < total) {
                    const uint32_t kj = idx - ex_o;  // index of v2 in u's out-list
                    const uint2 e2 = d.out_adj[ub_o + kj];
                    if (e2.x != s) {
                        const uint32_t via = sat_add(w1, e2.y);
                        bool keepit;
                        if (MODE == MODE_PRUNE && memo_all) {
                            keepit = (mw_o >> kj) & 1ull;
                        } else {
                            uint32_t dh;
                            if (!(XM && dmap_get(a.dm, dmap_key(s, e2.x), &dh))) {
                                const uint32_t slot = ht_find(w.key, WIT_TBITS, e2.x);
                                dh = slot == EMPTY ? INF : w.val[slot];
                                if constexpr (TH)  // an unsettled target counts as INF
                                    if (slot != EMPTY && !(w.fst[slot] & 1u)) dh = INF;
                            }
                            keepit = via != INF && via <= dh;
                        }
                        if (MODE == MODE_SCORE && keepit && mk_o)
                            atomicOr(&d.emask[sb + c0 + o], 1ull << kj);
                        ++l_cand;
                        if (keepit) {
                            ++l_kept;
                            if (MODE == MODE_SCORE) {
                                atomicAdd(&w.cnt[o], 1u);
                            } else {
                                const uint32_t ms = ht_insert(w.mkey, 7, e2.x);
                                if (ms == EMPTY) mover = true;
                                else atomicMin(&w.mval[ms], ((unsigned long long)via << 32) | u_o);
                            }
                        }
                    }
                }
            }
            __syncwarp();
            if (MODE == MODE_SCORE && mid && w.cnt[lane]) atomicAdd(&d.P[e.x], (int32_t)w.cnt[lane]);
            __syncwarp();
        }
        if (MODE == MODE_PRUNE) {
            __syncwarp();
            if (__any_sync(FULL, mover)) {
                hand_on();
                continue;
            }
            c_cand += l_cand;
            c_kept += l_kept;
            uint32_t l_new = 0;
            for (uint32_t t0 = 0; t0 < WIT_MC; t0 += 32) {
                const uint32_t t = t0 + lane;
                const uint32_t v2 = w.mkey[t];
                const bool have = v2 != EMPTY;
                const unsigned long long mv = w.mval[t];
                const uint32_t ws = (uint32_t)(mv >> 32), via = (uint32_t)mv;
                bool found = false;
                uint32_t ew = INF;
                if (have) {
                    for (uint32_t j = 0; j < sd; ++j) {
                        const uint2 e = d.out_adj[sb + j];
                        if (e.x == v2) {
                            found = true;
                            ew = e.y;
                            break;
                        }
                    }
                }
                const bool emit = have && (!found || ws < ew);
                c_merged += have;
                const uint32_t pos = warp_append(emit, &ctl->nRec);
                if (emit) {
                    if (pos < a.rec_cap) {
                        a.rec[pos] = make_uint4(s, v2, ws, via);
                        a.rec_flag[pos] = found ? 1 : 0;
                    } else {
                        atomicOr(&ctl->err, ERR_REC_OVERFLOW);
                    }
                    if (!found) atomicAdd(&d.new_in[v2], 1u);
                    ++c_ins;
                    if (!found) ++l_new;
                }
            }
            const uint32_t tot_new = warp_sum(l_new);
            c_new += l_new;
            if (lane == 0) d.new_out[s] = tot_new;
            __syncwarp();
        }
        // Phase 3 (memoised distances): the targets this search found new
        // get their labels (INF when none), now that all of the source's
        // decisions are made.
        if constexpr (XM) {
            if (bound != 0) {
                bool full = false;
                for (uint32_t c0 = 0; c0 < sd; c0 += 32) {
                    const uint32_t j = c0 + lane;
                    const bool valid = j < sd;
                    const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
                    const bool mid = valid && id_ok(d, e.x) && is_middle<MODE>(d, e.x, r);
                    uint32_t cnt = mid ? d.out_deg[e.x] : 0;
                    const uint64_t ub = mid ? d.out_beg[e.x] : 0;
                    if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
                    const uint32_t incl = warp_incl_scan(cnt);
                    const uint32_t total = __shfl_sync(FULL, incl, 31);
                    const uint32_t excl = incl - cnt;
                    for (uint32_t b = 0; b < total; b += 32) {
                        const uint32_t idx = b + lane;
                        const uint32_t o = warp_owner(excl, idx);
                        const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                        const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                        if (idx < total) {
                            const uint2 e2 = d.out_adj[ub_o + (idx - ex_o)];
                            if (e2.x != s) {
                                const uint32_t slot = ht_find(w.key, WIT_TBITS, e2.x);
                                uint32_t dv = slot == EMPTY ? INF : w.val[slot];
                                if constexpr (TH)
                                    if (slot != EMPTY && !(w.fst[slot] & 1u)) dv = INF;
                                const int put = dmap_put(a.dm, dmap_key(s, e2.x), dv);
                                full |= put < 0;
                                c_dm += put > 0;
                            }
                        }
                    }
                }
                if (full) atomicOr(&ctl->err, ERR_MAP_FULL);
            }
        }
        c_src += (lane == 0);
        c_vert += l_vert;
        c_edge += l_edge;
        c_mid += l_mid;
        c_midedge += l_midedge;
    }
    // Counters (lane-local sums folded per warp).
    c_src = warp_sum((uint32_t)c_src);
#define FOLD64(x)                                                               \
    {                                                                           \
        unsigned long long v_ = x;                                              \
        for (int o_ = 16; o_ > 0; o_ >>= 1) v_ += __shfl_xor_sync(FULL, v_, o_); \
        x = v_;                                                                 \
    }
    FOLD64(c_vert) FOLD64(c_edge) FOLD64(c_mid) FOLD64(c_midedge) FOLD64(c_cand)
    FOLD64(c_kept) FOLD64(c_merged) FOLD64(c_ins) FOLD64(c_new)
    if constexpr (XM) FOLD64(c_dm)
#undef FOLD64
    if (lane == 0) {
        if constexpr (XM) atomicAdd(a.dm.count, c_dm);
        atomicAdd(&ctl->wit_sources, c_src);
        atomicAdd(&ctl->wit_vertices, c_vert);
        atomicAdd(&ctl->wit_edges, c_edge);
        atomicAdd(&ctl->wit_middles, c_mid);
        atomicAdd(&ctl->wit_midedges, c_midedge);
        if (MODE == MODE_PRUNE) {
            atomicAdd(&ctl->cand, c_cand);
            atomicAdd(&ctl->kept, c_kept);
            atomicAdd(&ctl->merged, c_merged);
            atomicAdd(&ctl->inserted, c_ins);
            atomicAdd(&ctl->newEdges, c_new);
        }
    }
}

// Block tier: the same search for sources whose ball outgrew a warp's
// tables, run by a whole block with tables 16 times larger in shared memory
// (about 105 KB, two blocks per SM). Sources that outgrow these too go on to
// the dense tier. Control values (frontier size, overflow flag, bound) are
// read by all threads between two barriers and written only after the
// second.
constexpr int WB_THREADS = 256;
constexpr int WB_TBITS = 12;
constexpr int WB_T = 1 << WB_TBITS;
constexpr int WB_FC = 2048;
constexpr int WB_MBITS = 11;
constexpr int WB_M = 1 << WB_MBITS;

struct __align__(16) BlkSmem {
    uint32_t key[WB_T];
    uint32_t val[WB_T];
    uint32_t fst[WB_T];
    uint2 front[2][WB_FC];
    uint32_t mkey[WB_M];
    unsigned long long mval[WB_M];
    uint32_t cntw[WB_THREADS / 32][32];
    uint32_t nf[2];
    uint32_t item, ovf, bound, nnew, nkeys, memo_ok;
    uint32_t any;  // memoised-distance mode: the source has a candidate
    unsigned long long lwork;  // F_LW: out-edges of the next level's frontier
    uint32_t direct;           // F_PR: heaviest overlay edge (s, v) to a new target v
};

template <int MODE, int FEAT>
__global__ void __launch_bounds__(WB_THREADS) k_witness_block(WArgs a) {
    constexpr bool XM = (FEAT & F_XM) != 0, LW = (FEAT & F_LW) != 0, PR = (FEAT & F_PR) != 0;
    extern __shared__ __align__(16) unsigned char wb_raw[];
    BlkSmem &b = *reinterpret_cast<BlkSmem *>(wb_raw);
    const Dev d = a.d;
    Ctl *ctl = d.ctl;
    const uint32_t r = a.round;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t nIn = ctl->nOvf;
    unsigned long long c_src = 0, c_vert = 0, c_edge = 0, c_mid = 0, c_midedge = 0;
    unsigned long long c_cand = 0, c_kept = 0, c_merged = 0, c_ins = 0, c_new = 0;
    unsigned long long c_dm = 0;  // keys added to the memoised-distance map
    while (true) {
        __syncthreads();
        if (tid == 0) b.item = atomicAdd(&ctl->work3, 1u);
        __syncthreads();
        const uint32_t i = b.item;
        if (i >= nIn) break;
        const uint32_t s = a.ovf[i];
        if (s >= d.n) {
            if (tid == 0) atomicOr(&ctl->err, ERR_BOUND);
            continue;
        }
        const uint64_t sb = d.out_beg[s];
        const uint32_t sd = d.out_deg[s];
        if (sb + sd > d.out_arena) {
            if (tid == 0) atomicOr(&ctl->err, ERR_BOUND);
            continue;
        }
        if (sd > DENSE_SD) {  // a hub: straight to the global-memory tier
            if (tid == 0) a.ovf2[atomicAdd(&ctl->nOvf2, 1u)] = s;
            continue;
        }
        unsigned long long l_vert = 0, l_edge = 0, l_mid = 0, l_midedge = 0, l_cand = 0, l_kept = 0;
        if (tid == 0) {
            b.bound = 0;
            b.ovf = 0;
            b.nnew = 0;
            b.memo_ok = MODE == MODE_PRUNE && d.memo;
            if constexpr (XM) b.any = 0;
            if constexpr (PR) b.direct = 0;
        }
        __syncthreads();
        // Phase 0: heaviest candidate weight of the source, and whether every
        // contracted middle has its score-phase decisions memoised. Each warp
        // takes 32 of the source's out-edges and spreads their middles'
        // out-lists over its lanes.
        uint32_t lb = 0;
        for (uint32_t c0 = warp * 32; c0 < sd; c0 += nwarps * 32) {
            const uint32_t j = c0 + lane;
            const bool valid = j < sd;
            const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
            const bool mid = valid && id_ok(d, e.x) && is_middle<MODE>(d, e.x, r);
            if (MODE == MODE_PRUNE && mid && d.kround[e.x] != r + 1) b.memo_ok = 0;
            uint32_t cnt = mid ? d.out_deg[e.x] : 0;
            const uint64_t ub = mid ? d.out_beg[e.x] : 0;
            if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
            l_mid += mid;
            l_midedge += cnt;
            const uint32_t incl = warp_incl_scan(cnt);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const uint32_t excl = incl - cnt;
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t idx = base + lane;
                const uint32_t o = warp_owner(excl, idx);
                const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                const uint32_t w1 = __shfl_sync(FULL, e.y, o);
                const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                if (idx >= total) continue;
                const uint2 e2 = d.out_adj[ub_o + (idx - ex_o)];
                if (e2.x == s) continue;
                uint32_t known;
                if constexpr (XM) b.any = 1;
                if (!(XM && dmap_get(a.dm, dmap_key(s, e2.x), &known))) {
                    lb = max(lb, sat_add(w1, e2.y));
                    if constexpr (PR) {
                        const uint32_t dw = direct_weight(d.out_adj, sb, sd, e2.x);
                        if (dw != INF) atomicMax(&b.direct, dw);
                    }
                }
            }
        }
        if (lb) atomicMax(&b.bound, lb);
        __syncthreads();
        const uint32_t bound = b.bound;
        uint32_t sbound = bound;  // the search's label bound
        if constexpr (PR)
            if (d.ball == 0xFFFFFFFFu) sbound = max(bound, b.direct);
        const bool memo_all = b.memo_ok != 0;
        bool no_cand;
        if constexpr (XM) no_cand = b.any == 0;
        else no_cand = bound == 0;
        if (no_cand) {
            c_src += (tid == 0);
            c_mid += l_mid;
            c_midedge += l_midedge;
            continue;
        }
        // Empty the tables this source uses (16-byte stores): the search's
        // only when it runs, the merge table in the contraction phase.
        const bool searches = !memo_all && !(XM && bound == 0);
        if (searches) {
            uint4 *k4 = reinterpret_cast<uint4 *>(b.key), *v4 = reinterpret_cast<uint4 *>(b.val),
                  *f4 = reinterpret_cast<uint4 *>(b.fst);
            for (uint32_t t = tid; t < (uint32_t)WB_T / 4; t += blockDim.x) {
                k4[t] = make_uint4(EMPTY, EMPTY, EMPTY, EMPTY);
                v4[t] = make_uint4(INF, INF, INF, INF);
                f4[t] = make_uint4(0, 0, 0, 0);
            }
        }
        if (MODE == MODE_PRUNE) {
            uint4 *m4 = reinterpret_cast<uint4 *>(b.mkey);
            ulonglong2 *mv2 = reinterpret_cast<ulonglong2 *>(b.mval);
            for (uint32_t t = tid; t < (uint32_t)WB_M / 4; t += blockDim.x)
                m4[t] = make_uint4(EMPTY, EMPTY, EMPTY, EMPTY);
            for (uint32_t t = tid; t < (uint32_t)WB_M / 2; t += blockDim.x) mv2[t] = make_ulonglong2(~0ull, ~0ull);
        }
        __syncthreads();
        if (tid == 0 && !memo_all) {
            const uint32_t h = ht_insert(b.key, WB_TBITS, s);
            b.val[h] = 0;
            b.front[0][0] = make_uint2(h, 0);
            b.nf[0] = 1;
            b.nf[1] = 0;
            b.nkeys = 1;
        }
        // Phase 1: hop-limited Bellman-Ford, one level per iteration, each
        // level relaxing from the previous level's values (snapshots);
        // skipped when the decisions are memoised.
        uint32_t cur = 0;
        for (uint32_t lvl = 1; lvl <= d.H && !memo_all && !(XM && bound == 0); ++lvl) {
            __syncthreads();
            const uint32_t nfront = b.nf[cur];
            const uint32_t ovf = b.ovf;
            const uint32_t nkeys = b.nkeys;
            unsigned long long lwork = 0;
            if constexpr (LW) lwork = b.lwork;
            __syncthreads();
            if (ovf || nfront == 0 || nkeys > d.ball) break;
            if constexpr (LW)
                if (lvl >= 2 && lwork > a.level_work) break;
            const uint32_t nxt = cur ^ 1u;
            if (tid == 0) {
                b.nf[nxt] = 0;
                if constexpr (LW) b.lwork = 0;
            }
            __syncthreads();
            for (uint32_t f0 = warp * 32; f0 < nfront; f0 += nwarps * 32) {
                const uint32_t fi = f0 + lane;
                const bool fv = fi < nfront && fi < (uint32_t)WB_FC;
                const uint2 fe = fv ? b.front[cur][fi] : make_uint2(0, 0);
                const bool fok = fv && fe.x < (uint32_t)WB_T;
                if (fv && !fok) atomicOr(&ctl->err, ERR_BOUND);
                const uint32_t x = fok ? b.key[fe.x] : 0;
                const bool xok = fok && id_ok(d, x);
                uint32_t cnt = xok ? d.out_deg[x] : 0;
                const uint64_t xb = xok ? d.out_beg[x] : 0;
                if (xok && !out_list_ok(d, xb, cnt)) cnt = 0;
                l_vert += xok;
                l_edge += cnt;
                const uint32_t incl = warp_incl_scan(cnt);
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                const uint32_t excl = incl - cnt;
                for (uint32_t base = 0; base < total; base += 32) {
                    const uint32_t idx = base + lane;
                    const uint32_t o = warp_owner(excl, idx);
                    const uint64_t xb_o = __shfl_sync(FULL, xb, o);
                    const uint32_t dx_o = __shfl_sync(FULL, fe.y, o);
                    const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                    if (idx >= total) continue;
                    const uint2 e = d.out_adj[xb_o + (idx - ex_o)];
                    const uint32_t nd = sat_add(dx_o, e.y);
                    if (nd >= sbound || !id_ok(d, e.x)) continue;
                    bool created = false;
                    const uint32_t slot = ht_insert(b.key, WB_TBITS, e.x, &created);
                    if (created) atomicAdd(&b.nkeys, 1u);
                    if (slot == EMPTY) {
                        b.ovf = 1;
                        continue;
                    }
                    const uint32_t old = atomicMin(&b.val[slot], nd);
                    if (nd < old && atomicExch(&b.fst[slot], lvl) != lvl) {
                        const uint32_t p = atomicAdd(&b.nf[nxt], 1u);
                        if (p < (uint32_t)WB_FC) b.front[nxt][p] = make_uint2(slot, 0);
                        else b.ovf = 1;
                    }
                }
            }
            __syncthreads();
            const uint32_t nn = min(b.nf[nxt], (uint32_t)WB_FC);
            unsigned long long lw = 0;
            for (uint32_t p = tid; p < nn; p += blockDim.x) {
                b.front[nxt][p].y = b.val[b.front[nxt][p].x];
                if constexpr (LW) lw += d.out_deg[b.key[b.front[nxt][p].x]];
            }
            if constexpr (LW)
                if (lw) atomicAdd(&b.lwork, lw);
            cur = nxt;
        }
        __syncthreads();
        const uint32_t ovf1 = b.ovf;
        __syncthreads();
        if (ovf1) {
            if (tid == 0) a.ovf2[atomicAdd(&ctl->nOvf2, 1u)] = s;
            continue;
        }
        // Phase 2: decisions, each warp taking 32 of the source's out-edges.
        for (uint32_t c0 = warp * 32; c0 < sd; c0 += nwarps * 32) {
            const uint32_t j = c0 + lane;
            const bool valid = j < sd;
            const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
            const bool mid = valid && id_ok(d, e.x) && is_middle<MODE>(d, e.x, r);
            uint32_t cnt = mid ? d.out_deg[e.x] : 0;
            const uint64_t ub = mid ? d.out_beg[e.x] : 0;
            if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
            const uint32_t incl = warp_incl_scan(cnt);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const uint32_t excl = incl - cnt;
            if (MODE == MODE_SCORE) b.cntw[warp][lane] = 0;
            const bool mk = mid && d.memo && d.kround[e.x] == r + 1;
            if (MODE == MODE_SCORE && mk) d.emask[sb + j] = 0;
            const unsigned long long mword = (MODE == MODE_PRUNE && memo_all && mid) ? d.emask[sb + j] : 0;
            __syncwarp();
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t idx = base + lane;
                const uint32_t o = warp_owner(excl, idx);
                const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                const uint32_t w1 = __shfl_sync(FULL, e.y, o);
                const uint32_t u_o = __shfl_sync(FULL, e.x, o);
                const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                const bool mk_o = __shfl_sync(FULL, mk, o);
                const unsigned long long mw_o = __shfl_sync(FULL, mword, o);
                if (idx >= total) continue;
                const uint32_t kj = idx - ex_o;  // index of v2 in u's out-list
                const uint2 e2 = d.out_adj[ub_o + kj];
                if (e2.x == s) continue;
                const uint32_t via = sat_add(w1, e2.y);
                bool keepit;
                if (MODE == MODE_PRUNE && memo_all) {
                    keepit = (mw_o >> kj) & 1ull;
                } else {
                    uint32_t dh;
                    if (!(XM && dmap_get(a.dm, dmap_key(s, e2.x), &dh))) {
                        const uint32_t slot = ht_find(b.key, WB_TBITS, e2.x);
                        dh = slot == EMPTY ? INF : b.val[slot];
                    }
                    keepit = via != INF && via <= dh;
                }
                if (MODE == MODE_SCORE && keepit && mk_o) atomicOr(&d.emask[sb + c0 + o], 1ull << kj);
                ++l_cand;
                if (!keepit) continue;
                ++l_kept;
                if (MODE == MODE_SCORE) {
                    atomicAdd(&b.cntw[warp][o], 1u);
                } else {
                    const uint32_t ms = ht_insert(b.mkey, WB_MBITS, e2.x);
                    if (ms == EMPTY) b.ovf = 1;
                    else atomicMin(&b.mval[ms], ((unsigned long long)via << 32) | u_o);
                }
            }
            __syncwarp();
            if (MODE == MODE_SCORE && mid && b.cntw[warp][lane])
                atomicAdd(&d.P[e.x], (int32_t)b.cntw[warp][lane]);
            __syncwarp();
        }
        __syncthreads();
        if (MODE == MODE_PRUNE) {
            const uint32_t ovf2 = b.ovf;
            __syncthreads();
            if (ovf2) {
                if (tid == 0) a.ovf2[atomicAdd(&ctl->nOvf2, 1u)] = s;
                continue;
            }
            uint32_t l_new = 0;
            for (uint32_t t = tid; t < (uint32_t)WB_M; t += blockDim.x) {
                const uint32_t v2 = b.mkey[t];
                if (v2 == EMPTY) continue;
                const unsigned long long mv = b.mval[t];
                const uint32_t ws = (uint32_t)(mv >> 32), via = (uint32_t)mv;
                bool found = false;
                uint32_t ew = INF;
                for (uint32_t j = 0; j < sd; ++j) {
                    const uint2 e = d.out_adj[sb + j];
                    if (e.x == v2) {
                        found = true;
                        ew = e.y;
                        break;
                    }
                }
                ++c_merged;
                if (found && !(ws < ew)) continue;
                const uint32_t pos = atomicAdd(&ctl->nRec, 1u);
                if (pos < a.rec_cap) {
                    a.rec[pos] = make_uint4(s, v2, ws, via);
                    a.rec_flag[pos] = found ? 1 : 0;
                } else {
                    atomicOr(&ctl->err, ERR_REC_OVERFLOW);
                }
                ++c_ins;
                if (!found) {
                    ++l_new;
                    atomicAdd(&d.new_in[v2], 1u);
                }
            }
            if (l_new) atomicAdd(&b.nnew, l_new);
            __syncthreads();
            if (tid == 0) d.new_out[s] = b.nnew;
            c_cand += l_cand;
            c_kept += l_kept;
            c_new += l_new;
        }
        // Phase 3 (memoised distances): the targets this search found new
        // get their labels (INF when none), now that all of the source's
        // decisions are made. The next source's table reset waits for the
        // barrier at the top of the loop.
        if constexpr (XM) {
            if (bound != 0) {
                bool full = false;
                for (uint32_t c0 = warp * 32; c0 < sd; c0 += nwarps * 32) {
                    const uint32_t j = c0 + lane;
                    const bool valid = j < sd;
                    const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
                    const bool mid = valid && id_ok(d, e.x) && is_middle<MODE>(d, e.x, r);
                    uint32_t cnt = mid ? d.out_deg[e.x] : 0;
                    const uint64_t ub = mid ? d.out_beg[e.x] : 0;
                    if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
                    const uint32_t incl = warp_incl_scan(cnt);
                    const uint32_t total = __shfl_sync(FULL, incl, 31);
                    const uint32_t excl = incl - cnt;
                    for (uint32_t base = 0; base < total; base += 32) {
                        const uint32_t idx = base + lane;
                        const uint32_t o = warp_owner(excl, idx);
                        const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                        const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                        if (idx >= total) continue;
                        const uint2 e2 = d.out_adj[ub_o + (idx - ex_o)];
                        if (e2.x == s) continue;
                        const uint32_t slot = ht_find(b.key, WB_TBITS, e2.x);
                        const int put = dmap_put(a.dm, dmap_key(s, e2.x), slot == EMPTY ? INF : b.val[slot]);
                        full |= put < 0;
                        c_dm += put > 0;
                    }
                }
                if (full) atomicOr(&ctl->err, ERR_MAP_FULL);
            }
        }
        c_src += (tid == 0);
        c_vert += l_vert;
        c_edge += l_edge;
        c_mid += l_mid;
        c_midedge += l_midedge;
    }
#define FOLD64(x)                                                               \
    {                                                                           \
        unsigned long long v_ = x;                                              \
        for (int o_ = 16; o_ > 0; o_ >>= 1) v_ += __shfl_xor_sync(FULL, v_, o_); \
        x = v_;                                                                 \
    }
    FOLD64(c_src) FOLD64(c_vert) FOLD64(c_edge) FOLD64(c_mid) FOLD64(c_midedge) FOLD64(c_cand)
    FOLD64(c_kept) FOLD64(c_merged) FOLD64(c_ins) FOLD64(c_new)
    if constexpr (XM) FOLD64(c_dm)
#undef FOLD64
    if (lane == 0) {
        if constexpr (XM) atomicAdd(a.dm.count, c_dm);
        atomicAdd(&ctl->wit_block, c_src);
        atomicAdd(&ctl->wit_vertices, c_vert);
        atomicAdd(&ctl->wit_edges, c_edge);
        atomicAdd(&ctl->wit_middles, c_mid);
        atomicAdd(&ctl->wit_midedges, c_midedge);
        if (MODE == MODE_PRUNE) {
            atomicAdd(&ctl->cand, c_cand);
            atomicAdd(&ctl->kept, c_kept);
            atomicAdd(&ctl->merged, c_merged);
            atomicAdd(&ctl->inserted, c_ins);
            atomicAdd(&ctl->newEdges, c_new);
        }
    }
}

// Same search for the sources whose ball overflowed shared memory: one block
// per slot of dense per-vertex arrays in global memory (no capacity limit).
template <int MODE, int FEAT>
__global__ void __launch_bounds__(256) k_witness_dense(WArgs a, Dense dn) {
    constexpr bool XM = (FEAT & F_XM) != 0, LW = (FEAT & F_LW) != 0, PR = (FEAT & F_PR) != 0;
    constexpr bool TH = (FEAT & F_TH) != 0;
    const Dev d = a.d;
    Ctl *ctl = d.ctl;
    const uint32_t n = d.n;
    const uint32_t r = a.round;
    const size_t base = (size_t)blockIdx.x * n;
    uint32_t *dist = dn.dist + base, *fst = dn.fst + base, *touched = dn.touched + base;
    uint32_t *fa = dn.fa + base, *fb = dn.fb + base, *fda = dn.fda + base, *fdb = dn.fdb + base;
    uint32_t *mt = dn.mt + base, *direct = dn.direct + base;
    unsigned long long *merge = dn.merge + base;
    __shared__ uint32_t s_item, s_bound, s_nt, s_nm, s_nf[2], s_memo;
    __shared__ unsigned long long s_lw;  // F_LW: out-edges of the next level's frontier
    __shared__ uint32_t s_direct;        // F_PR: heaviest overlay edge (s, v) to a new target v
    __shared__ uint32_t s_rem, s_settled;  // F_TH: new targets not yet settled, vertices settled
    __shared__ unsigned long long s_best;  // F_TH: least (label, id) of an unsettled vertex
    __shared__ unsigned long long s_cnt[5];
    const uint32_t tid = threadIdx.x;
    const uint32_t nOvf = ctl->nOvf2;
    while (true) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(&ctl->work2, 1u);
        if (tid < 5) s_cnt[tid] = 0;
        __syncthreads();
        const uint32_t i = s_item;
        if (i >= nOvf) break;
        const uint32_t s = a.ovf2[i];
        const uint64_t sb = s < n ? d.out_beg[s] : 0;
        const uint32_t sd = (s < n && out_list_ok(d, sb, d.out_deg[s])) ? d.out_deg[s] : 0;
        if (s >= n) {
            if (tid == 0) atomicOr(&ctl->err, ERR_BOUND);
            continue;
        }
        if (tid == 0) {
            s_bound = 0;
            s_nt = 1;
            s_nm = 0;
            s_nf[0] = 1;
            s_nf[1] = 0;
            s_memo = MODE == MODE_PRUNE && d.memo;
            dist[s] = 0;
            touched[0] = s;
            fa[0] = s;
            fda[0] = 0;
            atomicAdd(&ctl->wit_fallback, 1ull);
            if constexpr (PR) s_direct = 0;
        }
        if constexpr (PR) {
            // the source's direct edges, for the widened label bound
            for (uint32_t j = tid; j < sd; j += blockDim.x) {
                const uint2 e = d.out_adj[sb + j];
                if (e.x < n) direct[e.x] = e.y;
            }
        }
        __syncthreads();
        for (uint32_t j = tid; j < sd; j += blockDim.x) {
            const uint2 e = d.out_adj[sb + j];
            if (!id_ok(d, e.x) || !is_middle<MODE>(d, e.x, r)) continue;
            if (MODE == MODE_PRUNE && d.kround[e.x] != r + 1) s_memo = 0;
            const uint64_t ub = d.out_beg[e.x];
            const uint32_t ud = out_list_ok(d, ub, d.out_deg[e.x]) ? d.out_deg[e.x] : 0;
            uint32_t bmax = 0;
            for (uint32_t jj = 0; jj < ud; ++jj) {
                const uint2 e2 = d.out_adj[ub + jj];
                uint32_t known;
                if (e2.x != s && !(XM && dmap_get(a.dm, dmap_key(s, e2.x), &known))) {
                    bmax = max(bmax, sat_add(e.y, e2.y));
                    if constexpr (PR)
                        if (e2.x < n && direct[e2.x] != INF) atomicMax(&s_direct, direct[e2.x]);
                }
            }
            atomicMax(&s_bound, bmax);
        }
        __syncthreads();
        const uint32_t bound = s_bound;
        uint32_t sbound = bound;  // the search's label bound
        if constexpr (PR)
            if (d.ball == 0xFFFFFFFFu) sbound = max(bound, s_direct);
        const bool memo_all = s_memo != 0;  // decisions memoised: no search
        uint32_t *cur = fa, *curd = fda, *nx = fb, *nxd = fdb;
        const uint32_t lane = lane_id(), warp = tid >> 5, nwarps = blockDim.x >> 5;
        // Alg. 3's search with the settled-vertex cap: bit 1 of fst flags a
        // new target, bit 0 a settled vertex; each step settles the
        // unsettled vertex of least (label, id) among those reached.
        if constexpr (TH) {
            if (bound > 0) {
                if (tid == 0) {
                    s_rem = 0;
                    s_settled = 0;
                }
                __syncthreads();
                for (uint32_t j = tid; j < sd; j += blockDim.x) {
                    const uint2 e = d.out_adj[sb + j];
                    if (!id_ok(d, e.x) || !is_middle<MODE>(d, e.x, r)) continue;
                    const uint64_t ub = d.out_beg[e.x];
                    const uint32_t ud = out_list_ok(d, ub, d.out_deg[e.x]) ? d.out_deg[e.x] : 0;
                    for (uint32_t jj = 0; jj < ud; ++jj) {
                        const uint32_t v2 = d.out_adj[ub + jj].x;
                        uint32_t known;
                        if (v2 == s || !id_ok(d, v2) || (XM && dmap_get(a.dm, dmap_key(s, v2), &known)))
                            continue;
                        if ((atomicOr(&fst[v2], 2u) & 2u) == 0) atomicAdd(&s_rem, 1u);
                    }
                }
                while (true) {
                    __syncthreads();
                    if (tid == 0) s_best = ~0ull;
                    __syncthreads();
                    if (s_rem == 0 || s_settled >= a.theta) break;  // read by all between barriers
                    const uint32_t nt = s_nt;
                    unsigned long long best = ~0ull;
                    for (uint32_t p = tid; p < nt; p += blockDim.x) {
                        const uint32_t v = touched[p];
                        if ((fst[v] & 1u) || dist[v] == INF) continue;
                        best = min(best, ((unsigned long long)dist[v] << 32) | v);
                    }
                    if (best != ~0ull) atomicMin(&s_best, best);
                    __syncthreads();
                    const unsigned long long b = s_best;
                    if (b == ~0ull) break;  // nothing reachable left
                    const uint32_t x = (uint32_t)b, dx = (uint32_t)(b >> 32);
                    __syncthreads();
                    if (tid == 0) {
                        fst[x] |= 1u;
                        ++s_settled;
                        if (fst[x] & 2u) --s_rem;
                    }
                    __syncthreads();
                    if (s_rem == 0 || s_settled >= a.theta) break;
                    const uint64_t xb = d.out_beg[x];
                    const uint32_t xd = out_list_ok(d, xb, d.out_deg[x]) ? d.out_deg[x] : 0;
                    for (uint32_t j = tid; j < xd; j += blockDim.x) {
                        const uint2 e = d.out_adj[xb + j];
                        if (!id_ok(d, e.x) || (fst[e.x] & 1u)) continue;
                        const uint32_t nd = sat_add(dx, e.y);
                        if (nd == INF) continue;
                        const uint32_t old = atomicMin(&dist[e.x], nd);
                        if (old == INF && nd < INF) touched[atomicAdd(&s_nt, 1u)] = e.x;
                    }
                }
                __syncthreads();
            }
        } else {
        for (uint32_t lvl = 1; lvl <= d.H && bound > 0 && !memo_all; ++lvl) {
            const uint32_t nf = s_nf[(lvl - 1) & 1];
            __syncthreads();
            if (tid == 0) {
                s_nf[lvl & 1] = 0;
                if constexpr (LW) s_lw = 0;
            }
            __syncthreads();
            // each warp takes 32 frontier entries and spreads their out-edges
            // over its lanes
            for (uint32_t f0 = warp * 32; f0 < nf; f0 += nwarps * 32) {
                const uint32_t f = f0 + lane;
                const bool fv = f < nf;
                const uint32_t x = fv ? cur[f] : 0, dx = fv ? curd[f] : 0;
                const uint64_t xb = fv ? d.out_beg[x] : 0;
                const uint32_t xd = (fv && out_list_ok(d, xb, d.out_deg[x])) ? d.out_deg[x] : 0;
                const uint32_t incl = warp_incl_scan(xd);
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                const uint32_t excl = incl - xd;
                for (uint32_t b0 = 0; b0 < total; b0 += 32) {
                    const uint32_t idx = b0 + lane;
                    const uint32_t o = warp_owner(excl, idx);
                    const uint64_t xb_o = __shfl_sync(FULL, xb, o);
                    const uint32_t dx_o = __shfl_sync(FULL, dx, o);
                    const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                    if (idx >= total) continue;
                    const uint2 e = d.out_adj[xb_o + (idx - ex_o)];
                    const uint32_t nd = sat_add(dx_o, e.y);
                    if (nd >= sbound || !id_ok(d, e.x)) continue;
                    const uint32_t old = atomicMin(&dist[e.x], nd);
                    if (nd < old) {
                        if (old == INF) touched[atomicAdd(&s_nt, 1u)] = e.x;
                        if (atomicExch(&fst[e.x], lvl) != lvl) nx[atomicAdd(&s_nf[lvl & 1], 1u)] = e.x;
                    }
                }
            }
            __syncthreads();
            const uint32_t nn = s_nf[lvl & 1];
            unsigned long long lw = 0;
            for (uint32_t p = tid; p < nn; p += blockDim.x) {
                nxd[p] = dist[nx[p]];
                if constexpr (LW) lw += d.out_deg[nx[p]];
            }
            if constexpr (LW)
                if (lw) atomicAdd(&s_lw, lw);
            __syncthreads();
            uint32_t *t1 = cur, *t2 = curd;
            cur = nx;
            curd = nxd;
            nx = t1;
            nxd = t2;
            if (nn == 0 || s_nt > d.ball) break;  // s_nt: vertices holding a label
            // the next level (the second or later) would expand too much
            if constexpr (LW)
                if (s_lw > a.level_work) break;
        }
        }  // hop-limited search
        // the source's direct edges, for the existing-edge test
        if (MODE == MODE_PRUNE) {
            for (uint32_t j = tid; j < sd; j += blockDim.x) {
                const uint2 e = d.out_adj[sb + j];
                if (e.x < n) direct[e.x] = e.y;
            }
            __syncthreads();
        }
        // decisions
        unsigned long long l_cand = 0, l_kept = 0;
        for (uint32_t j = tid; j < sd; j += blockDim.x) {
            const uint2 e = d.out_adj[sb + j];
            if (!id_ok(d, e.x) || !is_middle<MODE>(d, e.x, r)) continue;
            const uint64_t ub = d.out_beg[e.x];
            const uint32_t ud = out_list_ok(d, ub, d.out_deg[e.x]) ? d.out_deg[e.x] : 0;
            const bool mk = d.memo && d.kround[e.x] == r + 1;
            const unsigned long long mword = (MODE == MODE_PRUNE && memo_all) ? d.emask[sb + j] : 0;
            unsigned long long rec_mask = 0;
            int32_t kept_u = 0;
            for (uint32_t jj = 0; jj < ud; ++jj) {
                const uint2 e2 = d.out_adj[ub + jj];
                if (e2.x == s || !id_ok(d, e2.x)) continue;
                const uint32_t via = sat_add(e.y, e2.y);
                bool keepit;
                if (MODE == MODE_PRUNE && memo_all) {
                    keepit = (mword >> jj) & 1ull;
                } else {
                    uint32_t dh;
                    if (!(XM && dmap_get(a.dm, dmap_key(s, e2.x), &dh))) {
                        dh = dist[e2.x];
                        if constexpr (TH)  // an unsettled target counts as INF
                            if (!(fst[e2.x] & 1u)) dh = INF;
                    }
                    keepit = via != INF && via <= dh;
                }
                if (MODE == MODE_SCORE && keepit && mk) rec_mask |= 1ull << jj;
                ++l_cand;
                if (keepit) {
                    ++l_kept;
                    ++kept_u;
                    if (MODE == MODE_PRUNE) {
                        const unsigned long long old =
                            atomicMin(&merge[e2.x], ((unsigned long long)via << 32) | e.x);
                        if (old == ~0ull) mt[atomicAdd(&s_nm, 1u)] = e2.x;
                    }
                }
            }
            if (MODE == MODE_SCORE && kept_u) atomicAdd(&d.P[e.x], kept_u);
            if (MODE == MODE_SCORE && mk) d.emask[sb + j] = rec_mask;
        }
        __syncthreads();
        if (MODE == MODE_PRUNE) {
            atomicAdd(&s_cnt[0], l_cand);
            atomicAdd(&s_cnt[1], l_kept);
            const uint32_t nm = s_nm;
            unsigned long long l_ins = 0, l_new = 0;
            for (uint32_t p = tid; p < nm; p += blockDim.x) {
                const uint32_t v2 = mt[p];
                const unsigned long long mv = merge[v2];
                merge[v2] = ~0ull;
                const uint32_t ws = (uint32_t)(mv >> 32), via = (uint32_t)mv;
                const uint32_t ew = direct[v2];
                const bool found = ew != INF;
                if (found && !(ws < ew)) continue;
                const uint32_t pos = atomicAdd(&ctl->nRec, 1u);
                if (pos < a.rec_cap) {
                    a.rec[pos] = make_uint4(s, v2, ws, via);
                    a.rec_flag[pos] = found ? 1 : 0;
                } else {
                    atomicOr(&ctl->err, ERR_REC_OVERFLOW);
                }
                ++l_ins;
                if (!found) {
                    ++l_new;
                    atomicAdd(&d.new_in[v2], 1u);
                }
            }
            atomicAdd(&s_cnt[2], l_ins);
            atomicAdd(&s_cnt[3], l_new);
            __syncthreads();
            if (tid == 0) {
                atomicAdd(&ctl->cand, s_cnt[0]);
                atomicAdd(&ctl->kept, s_cnt[1]);
                atomicAdd(&ctl->merged, (unsigned long long)nm);
                atomicAdd(&ctl->inserted, s_cnt[2]);
                atomicAdd(&ctl->newEdges, s_cnt[3]);
                d.new_out[s] = (uint32_t)s_cnt[3];
            }
        }
        // Phase 3 (memoised distances): the targets this search found new
        // get their labels (INF when none), before the labels are reset.
        if constexpr (XM) {
            if (bound != 0) {
                unsigned long long l_dm = 0;
                bool full = false;
                for (uint32_t j = tid; j < sd; j += blockDim.x) {
                    const uint2 e = d.out_adj[sb + j];
                    if (!id_ok(d, e.x) || !is_middle<MODE>(d, e.x, r)) continue;
                    const uint64_t ub = d.out_beg[e.x];
                    const uint32_t ud = out_list_ok(d, ub, d.out_deg[e.x]) ? d.out_deg[e.x] : 0;
                    for (uint32_t jj = 0; jj < ud; ++jj) {
                        const uint2 e2 = d.out_adj[ub + jj];
                        if (e2.x == s || !id_ok(d, e2.x)) continue;
                        uint32_t dv = dist[e2.x];
                        if constexpr (TH)
                            if (!(fst[e2.x] & 1u)) dv = INF;
                        const int put = dmap_put(a.dm, dmap_key(s, e2.x), dv);
                        full |= put < 0;
                        l_dm += put > 0;
                    }
                }
                if (full) atomicOr(&ctl->err, ERR_MAP_FULL);
                if (l_dm) atomicAdd(a.dm.count, l_dm);
            }
        }
        __syncthreads();
        const uint32_t nt = s_nt;
        for (uint32_t p = tid; p < nt; p += blockDim.x) {
            const uint32_t v = touched[p];
            dist[v] = INF;
            fst[v] = 0;
        }
        if (MODE == MODE_PRUNE || PR)
            for (uint32_t j = tid; j < sd; j += blockDim.x) {
                const uint2 e = d.out_adj[sb + j];
                if (e.x < n) direct[e.x] = INF;
            }
        if constexpr (TH) {
            // targets never reached are not in the touched list: clear their flags
            for (uint32_t j = tid; j < sd; j += blockDim.x) {
                const uint2 e = d.out_adj[sb + j];
                if (!id_ok(d, e.x) || !is_middle<MODE>(d, e.x, r)) continue;
                const uint64_t ub = d.out_beg[e.x];
                const uint32_t ud = out_list_ok(d, ub, d.out_deg[e.x]) ? d.out_deg[e.x] : 0;
                for (uint32_t jj = 0; jj < ud; ++jj) {
                    const uint32_t v2 = d.out_adj[ub + jj].x;
                    if (v2 < n) fst[v2] = 0;
                }
            }
        }
    }
}

// --------------------------------------------------------------------------
// Learned priority: features of the rescored vertices
// --------------------------------------------------------------------------

// For u in A_r, right after its edge difference was computed (P[u]): its 12
// integer features (see ch_export_trace) as a trace row (round, u, f[12])
// and as transformed floats for the MLP; then ed_last[u] = P[u] and one more
// rescoring is counted.
__global__ void k_features(Dev d, const uint32_t *A, uint32_t nA, uint32_t r, long long *rows,
                           float *x) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nA;
         i += gridDim.x * blockDim.x) {
        const uint32_t u = A[i];
        if (!id_ok(d, u)) continue;
        if (d.inel[u]) {  // not scored: a row marked with round -1 (dropped on export)
            if (rows) rows[(uint64_t)i * 14] = -1;
            continue;
        }
        if (rows) atomicAdd(&d.ctl->trace_valid, 1ull);
        const uint64_t ob = d.out_beg[u], ib = d.in_beg[u];
        const uint32_t od = out_list_ok(d, ob, d.out_deg[u]) ? d.out_deg[u] : 0;
        const uint32_t id = in_list_ok(d, ib, d.in_deg[u]) ? d.in_deg[u] : 0;
        long long common = 0;
        unsigned long long wsum = 0;
        for (uint32_t j = 0; j < id; ++j) {
            const uint2 e = d.in_adj[ib + j];
            wsum += e.y;
            for (uint32_t k = 0; k < od; ++k)
                if (d.out_adj[ob + k].x == e.x) {
                    ++common;
                    break;
                }
        }
        for (uint32_t k = 0; k < od; ++k) wsum += d.out_adj[ob + k].y;
        const int32_t ed = d.P[u];
        long long f[MLP_NIN];
        f[0] = (long long)ed + id + od;
        f[1] = id;
        f[2] = od;
        f[3] = (long long)id + od - common;
        f[4] = ed;
        f[5] = d.cn[u];
        f[6] = d.depth[u];
        f[7] = r;
        f[8] = (long long)id * od;
        f[9] = d.orig_deg[u];
        f[10] = d.rescore[u];
        f[11] = (id + od) ? (long long)(wsum / (unsigned long long)(id + od)) : 0;
        if (rows) {
            long long *row = rows + (uint64_t)i * 14;
            row[0] = r;
            row[1] = u;
            for (int k = 0; k < MLP_NIN; ++k) row[2 + k] = f[k];
        }
        if (x) {
            float *xr = x + (uint64_t)i * 16;
            for (int k = 0; k < 16; ++k) xr[k] = k < MLP_NIN ? feature_transform(f[k]) : 0.f;
        }
        d.ed_last[u] = ed;
        d.rescore[u] += 1;
    }
}

// P[u] = round(1024 * y) (ties to even), clamped to +-2^30; log the priority.
__global__ void k_apply_learned(Dev d, const uint32_t *A, uint32_t nA, const float *y, int32_t *log) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nA;
         i += gridDim.x * blockDim.x) {
        const uint32_t u = A[i];
        if (!id_ok(d, u)) continue;
        if (d.inel[u]) {
            if (log) log[i] = P_INELIGIBLE;
            continue;
        }
        float v = y[i] * 1024.f;
        if (!(v == v)) v = 0.f;  // NaN
        v = fminf(fmaxf(v, -1073741824.f), 1073741824.f);
        const int32_t p = __float2int_rn(v);
        d.P[u] = p;
        if (log) log[i] = p;
    }
}

// CH_PRIO_COMPOSITE: P[u] = 4 * ED + (|N_in| + |N_out|) + 8 * depth,
// clamped to +-2^30, for the eligible rescored vertices (P holds the edge
// difference on entry).
__global__ void k_composite(Dev d, const uint32_t *A, uint32_t nA) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nA;
         i += gridDim.x * blockDim.x) {
        const uint32_t u = A[i];
        if (!id_ok(d, u) || d.inel[u]) continue;
        long long p = 4ll * d.P[u] + (long long)d.in_deg[u] + (long long)d.out_deg[u] + 8ll * d.depth[u];
        p = p < -(1ll << 30) ? -(1ll << 30) : (p > (1ll << 30) ? (1ll << 30) : p);
        d.P[u] = (int32_t)p;
    }
}

__global__ void k_log_priority(const Dev d, const uint32_t *A, uint32_t nA, int32_t *log) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nA;
         i += gridDim.x * blockDim.x) {
        const uint32_t u = A[i];
        log[i] = u < d.n ? d.P[u] : 0;
    }
}

__global__ void k_orig_deg(Dev d) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.n; v += gridDim.x * blockDim.x)
        d.orig_deg[v] = d.out_deg[v] + d.in_deg[v];
}

// --------------------------------------------------------------------------
// Step 3: select strict local minima of the key
// --------------------------------------------------------------------------

__global__ void k_select(Dev d, const uint32_t *VO, uint32_t nVO, uint32_t r, uint32_t *F) {
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t base = warp * 32; base < nVO; base += nwarps * 32) {
        const uint32_t i = base + lane;
        const bool valid = i < nVO;
        const uint32_t u = valid ? VO[i] : 0;
        const bool uok = valid && id_ok(d, u);
        const uint64_t ku = uok ? select_key(d, u) : 0;
        const uint64_t ob = uok ? d.out_beg[u] : 0;
        const uint64_t ib = uok ? d.in_beg[u] : 0;
        const uint32_t od = (uok && out_list_ok(d, ob, d.out_deg[u])) ? d.out_deg[u] : 0;
        const uint32_t id = (uok && in_list_ok(d, ib, d.in_deg[u])) ? d.in_deg[u] : 0;
        const uint32_t c = od + id;
        const uint32_t incl = warp_incl_scan(c);
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        const uint32_t excl = incl - c;
        bool beaten = false;
        for (uint32_t b = 0; b < total; b += 32) {
            const uint32_t idx = b + lane;
            const uint32_t o = warp_owner(excl, idx);
            const uint32_t ex_o = __shfl_sync(FULL, excl, o);
            const uint32_t od_o = __shfl_sync(FULL, od, o);
            const uint64_t ob_o = __shfl_sync(FULL, ob, o);
            const uint64_t ib_o = __shfl_sync(FULL, ib, o);
            const uint64_t ku_o = __shfl_sync(FULL, ku, o);
            bool bt = false;
            if (idx < total) {
                const uint32_t jj = idx - ex_o;
                const uint32_t nb = jj < od_o ? d.out_adj[ob_o + jj].x : d.in_adj[ib_o + (jj - od_o)].x;
                bt = id_ok(d, nb) && select_key(d, nb) < ku_o;
            }
            const uint32_t B = __ballot_sync(FULL, bt);
            const uint32_t lo = max(excl, b), hi = min(excl + c, b + 32);
            if (hi > lo && (B & lane_bits(lo - b, hi - b))) beaten = true;
        }
        const bool sel = uok && !beaten && !d.inel[u];
        if (sel) d.level[u] = r;
        const uint32_t pos = warp_append(sel, &d.ctl->nF);
        if (sel) F[pos] = u;
    }
}

// --------------------------------------------------------------------------
// Step 4: contraction bookkeeping for V_F
// --------------------------------------------------------------------------

// One warp per selected vertex u: counts its candidates and edges, and
// marks its neighbours as next round's affected set and its in-neighbours as
// the contraction phase's witness sources (each once).
__global__ void k_contract_prep(Dev d, const uint32_t *F, uint32_t src_stamp, uint32_t next_r,
                                uint32_t *S2, uint32_t *Anext) {
    const uint32_t nF = d.ctl->nF;
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    // the warp's sums over its vertices, added to the totals once at the end
    unsigned long long w_cand = 0, w_out = 0, w_in = 0, w_aff = 0;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nF; i += nwarps) {
        const uint32_t u = F[i];
        if (!id_ok(d, u)) continue;
        const uint64_t ob = d.out_beg[u], ib = d.in_beg[u];
        const uint32_t od = out_list_ok(d, ob, d.out_deg[u]) ? d.out_deg[u] : 0;
        const uint32_t id = in_list_ok(d, ib, d.in_deg[u]) ? d.in_deg[u] : 0;
        w_cand += (unsigned long long)od * id;
        w_out += od;
        w_in += id;
        unsigned long long deg_sum = 0;
        for (uint32_t j0 = 0; j0 < id + od; j0 += 32) {
            const uint32_t j = j0 + lane;
            bool src = false, aff = false;
            uint32_t x = 0;
            if (j < id + od) {
                x = j < id ? d.in_adj[ib + j].x : d.out_adj[ob + (j - id)].x;
                if (id_ok(d, x)) {
                    src = j < id && atomicExch(&d.smark[x], src_stamp) != src_stamp;
                    aff = atomicExch(&d.amark[x], next_r) != next_r;
                    if (aff) deg_sum += d.out_deg[x] + d.in_deg[x];
                }
            }
            const uint32_t ps = warp_append(src, &d.ctl->nS2);
            if (src) S2[ps] = x;
            const uint32_t pa = warp_append(aff, &d.ctl->nAnext);
            if (aff) Anext[pa] = x;
        }
        w_aff += deg_sum;  // lane-local; folded over the warp at the end
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w_aff += __shfl_xor_sync(FULL, w_aff, o);
    if (lane == 0) {
        if (w_aff) atomicAdd(&d.ctl->degAnext, w_aff);
        if (w_out + w_in) {
            atomicAdd(&d.ctl->candBound, w_cand);
            atomicAdd(&d.ctl->degFout, w_out);
            atomicAdd(&d.ctl->degFin, w_in);
        }
    }
}

// --------------------------------------------------------------------------
// Steps 6-9: CH edges, list maintenance, insertion
// --------------------------------------------------------------------------

// One warp per selected vertex u: its out-edges become E_up, its in-edges
// E_down. With core set, F is the live list of a round that found no
// eligible vertex: every live vertex gets level r and its overlay edges, and
// no neighbour bookkeeping is done (the build ends).
__global__ void k_emit_ch(Dev d, const uint32_t *F, uint32_t nF, uint2 *ch_up, uint2 *ch_dn,
                          uint64_t *up_beg, uint32_t *up_deg, uint64_t *dn_beg,
                          uint32_t *dn_deg, uint64_t up_cap, uint64_t dn_cap, bool core, uint32_t r) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nF; i += nwarps) {
        const uint32_t u = F[i];
        if (!id_ok(d, u)) continue;
        const uint64_t ob = d.out_beg[u], ib = d.in_beg[u];
        const uint32_t od = out_list_ok(d, ob, d.out_deg[u]) ? d.out_deg[u] : 0;
        const uint32_t id = in_list_ok(d, ib, d.in_deg[u]) ? d.in_deg[u] : 0;
        unsigned long long pu = 0, pd = 0;
        if (lane == 0) {
            pu = atomicAdd(&d.ctl->ch_up_tail, (unsigned long long)od);
            pd = atomicAdd(&d.ctl->ch_dn_tail, (unsigned long long)id);
        }
        pu = __shfl_sync(FULL, pu, 0);
        pd = __shfl_sync(FULL, pd, 0);
        if (pu + od > up_cap || pd + id > dn_cap) {
            if (lane == 0) atomicOr(&d.ctl->err, ERR_CH_OVERFLOW);
            continue;
        }
        for (uint32_t j = lane; j < od; j += 32) ch_up[pu + j] = d.out_adj[ob + j];
        for (uint32_t j = lane; j < id; j += 32) ch_dn[pd + j] = d.in_adj[ib + j];
        const uint32_t du = d.depth[u];
        if (lane == 0) {
            up_beg[u] = pu;
            up_deg[u] = od;
            dn_beg[u] = pd;
            dn_deg[u] = id;
            if (core) d.level[u] = r;
            d.label[u] = d.ed_last[u] + (int32_t)du;
        }
        if (core) continue;
        // learned-priority bookkeeping: neighbours inherit depth and count
        // the removed edges (V_F is independent, so no neighbour is being
        // contracted and depth[u] is stable here)
        for (uint32_t j = lane; j < od + id; j += 32) {
            const uint32_t x = j < od ? d.out_adj[ob + j].x : d.in_adj[ib + (j - od)].x;
            if (!id_ok(d, x)) continue;
            atomicAdd(&d.cn[x], 1u);
            atomicMax(&d.depth[x], du + 1);
        }
    }
}

constexpr uint32_t TOMB = 0xFFFFFFFFu;  // a pruned adjacency entry (never a vertex id)

// Stable in-place removal, by one warp, of this round's contracted vertices
// and of pruned entries (tombstones) from a list (32 entries per step;
// writes never pass the reads).
__device__ __forceinline__ uint32_t warp_compact_list(const Dev &d, uint2 *adj, uint64_t b, uint32_t dg,
                                                      uint32_t r) {
    const uint32_t lane = lane_id();
    uint32_t k = 0;
    for (uint32_t j0 = 0; j0 < dg; j0 += 32) {
        const uint32_t j = j0 + lane;
        uint2 e = make_uint2(0, 0);
        bool keep = false;
        if (j < dg) {
            e = adj[b + j];
            keep = e.x != TOMB && id_ok(d, e.x) && d.level[e.x] != r;
        }
        const uint32_t m = __ballot_sync(FULL, keep);
        if (keep) adj[b + k + __popc(m & ((1u << lane) - 1u))] = e;
        k += __popc(m);
        __syncwarp();
    }
    return k;
}

// --------------------------------------------------------------------------
// Pruning of overlay edges (Alg. 3's last step), after the rescoring searches
// --------------------------------------------------------------------------

// One warp per rescoring source s: every pair (s, v) of the step (v in
// N_out(u), u an affected out-neighbour of s, v != s) whose overlay edge
// weighs more than the distance recorded for (s, v) has that edge's weight
// set to 0 (weights are at least 1). Only ids are read while the pairs are
// enumerated, so marking changes no other warp's enumeration; a pair reached
// through several middles is marked once.
__global__ void k_prune_find(Dev d, DMap dm, const uint32_t *S, const uint32_t *nS_dev, uint32_t r) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nS = *nS_dev;
    Ctl *ctl = d.ctl;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nS; i += nwarps) {
        const uint32_t s = S[i];
        if (!id_ok(d, s)) continue;
        const uint64_t sb = d.out_beg[s];
        const uint32_t sd = d.out_deg[s];
        if (!out_list_ok(d, sb, sd)) continue;
        bool miss = false;
        for (uint32_t c0 = 0; c0 < sd; c0 += 32) {
            const uint32_t j = c0 + lane;
            const bool valid = j < sd;
            const uint2 e = valid ? d.out_adj[sb + j] : make_uint2(0, 0);
            const bool mid = valid && id_ok(d, e.x) && is_middle<MODE_SCORE>(d, e.x, r);
            uint32_t cnt = mid ? d.out_deg[e.x] : 0;
            const uint64_t ub = mid ? d.out_beg[e.x] : 0;
            if (mid && !out_list_ok(d, ub, cnt)) cnt = 0;
            const uint32_t incl = warp_incl_scan(cnt);
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const uint32_t excl = incl - cnt;
            for (uint32_t b = 0; b < total; b += 32) {
                const uint32_t idx = b + lane;
                const uint32_t o = warp_owner(excl, idx);
                const uint64_t ub_o = __shfl_sync(FULL, ub, o);
                const uint32_t ex_o = __shfl_sync(FULL, excl, o);
                if (idx >= total) continue;
                const uint32_t v = d.out_adj[ub_o + (idx - ex_o)].x;
                if (v == s || !id_ok(d, v)) continue;
                uint32_t dv;
                if (!dmap_get(dm, dmap_key(s, v), &dv)) {
                    miss = true;  // every pair of the step was recorded
                    continue;
                }
                for (uint32_t jj = 0; jj < sd; ++jj) {
                    const uint2 se = d.out_adj[sb + jj];
                    if (se.x != v) continue;
                    if (se.y > dv) atomicCAS(&d.out_adj[sb + jj].y, se.y, 0u);
                    break;
                }
            }
        }
        if (__any_sync(FULL, miss) && lane == 0) atomicOr(&ctl->err, ERR_BOUND);
    }
}

// One warp per rescoring source s: each out-entry marked by k_prune_find
// and its in-entry twin become tombstones; s and the edge's head are listed
// (once each) for compaction.
__global__ void k_prune_apply(Dev d, const uint32_t *S, const uint32_t *nS_dev, uint32_t *dirty,
                              uint32_t *pmark, uint32_t stamp) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nS = *nS_dev;
    Ctl *ctl = d.ctl;
    unsigned long long l_pruned = 0;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nS; i += nwarps) {
        const uint32_t s = S[i];
        if (!id_ok(d, s)) continue;
        const uint64_t sb = d.out_beg[s];
        const uint32_t sd = d.out_deg[s];
        if (!out_list_ok(d, sb, sd)) continue;
        bool any = false;
        for (uint32_t j = lane; j < sd; j += 32) {
            const uint2 e = d.out_adj[sb + j];
            if (e.y != 0 || !id_ok(d, e.x)) continue;
            const uint32_t v = e.x;
            d.out_adj[sb + j].x = TOMB;
            const uint64_t ib = d.in_beg[v];
            const uint32_t id = d.in_deg[v];
            if (in_list_ok(d, ib, id))
                for (uint32_t k = 0; k < id; ++k)
                    if (d.in_adj[ib + k].x == s) {
                        d.in_adj[ib + k].x = TOMB;
                        break;
                    }
            ++l_pruned;
            any = true;
            if (atomicExch(&pmark[v], stamp) != stamp) dirty[atomicAdd(&ctl->nDirty, 1u)] = v;
        }
        if (__any_sync(FULL, any) && lane == 0 && atomicExch(&pmark[s], stamp) != stamp)
            dirty[atomicAdd(&ctl->nDirty, 1u)] = s;
    }
    for (int o = 16; o > 0; o >>= 1) l_pruned += __shfl_xor_sync(FULL, l_pruned, o);
    if (lane == 0 && l_pruned) atomicAdd(&ctl->pruned, l_pruned);
}

// One warp per listed vertex: drop the tombstones from its out- and in-lists
// (at this point of a round no vertex carries the round's level, so the
// shared compaction drops nothing else).
__global__ void k_compact_dirty(Dev d, const uint32_t *X, const uint32_t *nX_dev, uint32_t r) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nX = *nX_dev;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nX; i += nwarps) {
        const uint32_t x = X[i];
        if (!id_ok(d, x)) continue;
        const uint64_t ob = d.out_beg[x], ib = d.in_beg[x];
        const uint32_t od = d.out_deg[x], id = d.in_deg[x];
        if (out_list_ok(d, ob, od)) {
            const uint32_t k = warp_compact_list(d, d.out_adj, ob, od, r);
            if (lane == 0) d.out_deg[x] = k;
        }
        if (in_list_ok(d, ib, id)) {
            const uint32_t k = warp_compact_list(d, d.in_adj, ib, id, r);
            if (lane == 0) d.in_deg[x] = k;
        }
    }
}

// One warp per rescored vertex u (eligible): its score on the pruned overlay
// from the recorded distances, P[u] = #{(v1, v2) kept} - (|N_in| + |N_out|).
__global__ void k_score_map(Dev d, DMap dm, const uint32_t *A, uint32_t nA, uint32_t r) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nA; i += nwarps) {
        const uint32_t u = A[i];
        if (!id_ok(d, u) || d.amark[u] != r) continue;
        const uint64_t ob = d.out_beg[u], ib = d.in_beg[u];
        const uint32_t od = d.out_deg[u], id = d.in_deg[u];
        if (!out_list_ok(d, ob, od) || !in_list_ok(d, ib, id)) continue;
        uint32_t kept = 0;
        bool miss = false;
        const uint64_t pairs = (uint64_t)od * id;
        for (uint64_t q = lane; q < pairs; q += 32) {
            const uint2 e1 = d.in_adj[ib + q / od];
            const uint2 e2 = d.out_adj[ob + q % od];
            if (e1.x == e2.x) continue;
            const uint32_t via = sat_add(e1.y, e2.y);
            uint32_t dv;
            if (!dmap_get(dm, dmap_key(e1.x, e2.x), &dv)) {
                miss = true;
                continue;
            }
            kept += via != INF && via <= dv;
        }
        kept = warp_sum(kept);
        if (__any_sync(FULL, miss) && lane == 0) atomicOr(&d.ctl->err, ERR_BOUND);
        if (lane == 0) d.P[u] = (int32_t)kept - (int32_t)(od + id);
    }
}

// One warp per affected vertex x: drop this round's contracted vertices from
// its out- and in-lists.
__global__ void k_compact_lists(Dev d, const uint32_t *X, uint32_t nX, uint32_t r) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nX; i += nwarps) {
        const uint32_t x = X[i];
        if (!id_ok(d, x)) continue;
        const uint64_t ob = d.out_beg[x], ib = d.in_beg[x];
        const uint32_t od = d.out_deg[x], id = d.in_deg[x];
        if (out_list_ok(d, ob, od)) {
            const uint32_t k = warp_compact_list(d, d.out_adj, ob, od, r);
            if (lane == 0) d.out_deg[x] = k;
        }
        if (in_list_ok(d, ib, id)) {
            const uint32_t k = warp_compact_list(d, d.in_adj, ib, id, r);
            if (lane == 0) d.in_deg[x] = k;
        }
    }
}

__global__ void k_reserve(Dev d, const uint32_t *X, uint32_t nX, uint64_t *reqO,
                          uint64_t *reqI) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nX;
         i += gridDim.x * blockDim.x) {
        const uint32_t x = X[i];
        const uint32_t no = d.new_out[x], ni = d.new_in[x];
        d.new_out[x] = 0;
        d.new_in[x] = 0;
        const uint32_t needO = d.out_deg[x] + no, needI = d.in_deg[x] + ni;
        reqO[i] = needO > d.out_cap[x] ? (uint64_t)max(2u * needO, 4u) : 0;
        reqI[i] = needI > d.in_cap[x] ? (uint64_t)max(2u * needI, 4u) : 0;
    }
}

// One warp per affected vertex whose list outgrew its capacity: copy it to
// its new place at the arena tail.
__global__ void k_relocate(Dev d, const uint32_t *X, uint32_t nX, const uint64_t *reqO,
                           const uint64_t *posO, const uint64_t *reqI, const uint64_t *posI) {
    const uint64_t to = d.ctl->out_tail, ti = d.ctl->in_tail;
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nX; i += nwarps) {
        const uint32_t x = X[i];
        if (reqO[i]) {
            const uint64_t nb = to + posO[i], ob = d.out_beg[x];
            const uint32_t dg = d.out_deg[x];
            if (out_list_ok(d, nb, (uint32_t)reqO[i]) && out_list_ok(d, ob, dg)) {
                for (uint32_t j = lane; j < dg; j += 32) d.out_adj[nb + j] = d.out_adj[ob + j];
                if (lane == 0) {
                    d.out_beg[x] = nb;
                    d.out_cap[x] = (uint32_t)reqO[i];
                }
            }
        }
        if (reqI[i]) {
            const uint64_t nb = ti + posI[i], ob = d.in_beg[x];
            const uint32_t dg = d.in_deg[x];
            if (in_list_ok(d, nb, (uint32_t)reqI[i]) && in_list_ok(d, ob, dg)) {
                for (uint32_t j = lane; j < dg; j += 32) d.in_adj[nb + j] = d.in_adj[ob + j];
                if (lane == 0) {
                    d.in_beg[x] = nb;
                    d.in_cap[x] = (uint32_t)reqI[i];
                }
            }
        }
    }
}


// Start of a round: its counters, and the score phase's witness work
// counters, start from zero.
__global__ void k_round_begin(Ctl *ctl) {
    ctl->nS = ctl->nS2 = ctl->nF = ctl->nAnext = ctl->nOvf = ctl->nRec = 0;
    ctl->candBound = ctl->degFout = ctl->degFin = ctl->degAnext = 0;
    ctl->pruned = 0;
    ctl->nDirty = 0;
    ctl->work = ctl->work2 = ctl->work3 = ctl->nOvf2 = 0;
}

// Start of a round's contraction phase: its counters and its witness work
// counters start from zero.
__global__ void k_contract_begin(Ctl *ctl) {
    ctl->cand = ctl->kept = ctl->merged = ctl->inserted = ctl->newEdges = 0;
    ctl->nOvf = 0;
    ctl->work = ctl->work2 = ctl->work3 = ctl->nOvf2 = 0;
}

// End of a round: the arena tails pass the lists relocated this round (when
// any were), the next round's live count takes the compacted one, the
// round's contraction counters are kept for the host's next read, and the
// shortcut log advances past the round's records.
__global__ void k_round_end(Ctl *ctl, int advance_tails) {
    if (advance_tails) {
        ctl->out_tail += ctl->relocOut;
        ctl->in_tail += ctl->relocIn;
    }
    ctl->nVO = ctl->nVO2;
    ctl->s_cand = ctl->cand;
    ctl->s_kept = ctl->kept;
    ctl->s_merged = ctl->merged;
    ctl->s_inserted = ctl->inserted;
    ctl->s_newEdges = ctl->newEdges;
    ctl->s_nRec = ctl->nRec;
    ctl->s_dm_count = ctl->dm_count;
    ctl->log_tail += ctl->nRec;
}

__global__ void k_insert(Dev d, const uint4 *rec, const uint8_t *flag, uint32_t r,
                         uint4 *log, uint32_t *log_round) {
    const uint32_t nRec = d.ctl->nRec;
    const uint64_t log_base = d.ctl->log_tail;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nRec;
         i += gridDim.x * blockDim.x) {
        const uint4 c = rec[i];  // (v1, v2, w, via)
        if (!id_ok(d, c.x) || !id_ok(d, c.y)) continue;
        if (flag[i]) {
            // Lower an existing edge. It sits among the list's entries from
            // before this kernel, ahead of anything appended concurrently.
            const uint64_t ob = d.out_beg[c.x];
            const uint32_t oc = out_list_ok(d, ob, d.out_cap[c.x]) ? d.out_cap[c.x] : 0;
            for (uint32_t j = 0; j < oc; ++j)
                if (d.out_adj[ob + j].x == c.y) {
                    d.out_adj[ob + j].y = c.z;
                    break;
                }
            const uint64_t ib = d.in_beg[c.y];
            const uint32_t ic = in_list_ok(d, ib, d.in_cap[c.y]) ? d.in_cap[c.y] : 0;
            for (uint32_t j = 0; j < ic; ++j)
                if (d.in_adj[ib + j].x == c.x) {
                    d.in_adj[ib + j].y = c.z;
                    break;
                }
        } else {
            const uint32_t p = atomicAdd(&d.out_deg[c.x], 1u);
            if (p < d.out_cap[c.x] && out_list_ok(d, d.out_beg[c.x], p + 1))
                d.out_adj[d.out_beg[c.x] + p] = make_uint2(c.y, c.z);
            else
                atomicOr(&d.ctl->err, ERR_BOUND);
            const uint32_t q = atomicAdd(&d.in_deg[c.y], 1u);
            if (q < d.in_cap[c.y] && in_list_ok(d, d.in_beg[c.y], q + 1))
                d.in_adj[d.in_beg[c.y] + q] = make_uint2(c.x, c.z);
            else
                atomicOr(&d.ctl->err, ERR_BOUND);
        }
        log[log_base + i] = c;
        log_round[log_base + i] = r;
    }
}

// --------------------------------------------------------------------------
// Postprocess: rank by (level, score, id) and the rank-ordered CSRs
// --------------------------------------------------------------------------

__global__ void k_rank_keys(const uint32_t *level, const int32_t *P, uint32_t n, uint64_t *keys,
                            uint32_t *vals) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        keys[v] = ((uint64_t)level[v] << 32) | ((uint32_t)P[v] ^ 0x80000000u);
        vals[v] = v;
    }
}

__global__ void k_rank_from_perm(const uint32_t *perm, uint32_t n, uint32_t *rank) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        rank[perm[i]] = i;
}

__global__ void k_ranked_deg(const uint32_t *perm, uint32_t n, const uint32_t *deg,
                             uint32_t *rdeg) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        rdeg[i] = deg[perm[i]];
    if (blockIdx.x == 0 && threadIdx.x == 0) rdeg[n] = 0;
}

constexpr uint32_t RANKED_SORT_MAX = 64;  // longest row a thread insertion-sorts

// Keys of every entry of a rank-ordered CSR for the radix sort of its rows:
// row << 32 | target rank (one warp per row), the weight as the value.
__global__ void k_row_keys(const uint32_t *off, uint32_t n, const uint2 *adj, uint64_t *keys, uint32_t *vals) {
    const uint32_t lane = lane_id();
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const uint32_t b = off[i], e = off[i + 1];
        for (uint32_t j = b + lane; j < e; j += 32) {
            const uint2 a = adj[j];
            keys[j] = ((uint64_t)i << 32) | a.x;
            vals[j] = a.y;
        }
    }
}

// The sorted keys back into the CSR's (target rank, weight) entries.
__global__ void k_row_unpack(const uint64_t *keys, const uint32_t *vals, uint64_t m, uint2 *adj) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < m;
         j += (uint64_t)gridDim.x * blockDim.x)
        adj[j] = make_uint2((uint32_t)keys[j], vals[j]);
}

__global__ void k_ranked_fill(const uint32_t *perm, const uint32_t *rank, uint32_t n,
                              const uint64_t *beg, const uint32_t *deg, const uint2 *src,
                              uint64_t src_count, const uint32_t *off, uint64_t dst_count,
                              uint2 *dst, Ctl *ctl) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t v = perm[i];
        if (v >= n) {
            atomicOr(&ctl->err, ERR_BOUND);
            continue;
        }
        const uint32_t dg = deg[v];
        const uint64_t b = beg[v];
        if (b + dg > src_count || (uint64_t)off[i] + dg > dst_count || off[i + 1] - off[i] != dg) {
            atomicOr(&ctl->err, ERR_BOUND);
            continue;
        }
        uint2 *out = dst + off[i];
        for (uint32_t j = 0; j < dg; ++j) {
            const uint2 e = src[b + j];
            if (e.x >= n) {
                atomicOr(&ctl->err, ERR_BOUND);
                out[j] = make_uint2(0, INF);
                continue;
            }
            out[j] = make_uint2(rank[e.x], e.y);
        }
        // rows are sorted by target rank, which makes the list order
        // canonical: short rows here (insertion sort), longer ones by the
        // radix sort of the whole CSR that a set flag asks for
        if (dg > RANKED_SORT_MAX) {
            ctl->longRows = 1;
            continue;
        }
        for (uint32_t j = 1; j < dg; ++j) {
            const uint2 t = out[j];
            uint32_t k = j;
            while (k > 0 && out[k - 1].x > t.x) {
                out[k] = out[k - 1];
                --k;
            }
            out[k] = t;
        }
    }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------

int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

struct EventPool {
    std::vector<cudaEvent_t> evs;
    size_t used = 0;
    cudaEvent_t get() {
        if (used == evs.size()) {
            cudaEvent_t e;
            CH_CUDA_TRY(cudaEventCreate(&e));
            evs.push_back(e);
        }
        return evs[used++];
    }
    ~EventPool() {
        for (auto e : evs) cudaEventDestroy(e);
    }
};

struct Span {
    cudaEvent_t a, b;
    double *acc;
    int round, phase;  // phase: index into the per-round timing row, or -1
};

struct Builder {
    ch_s *h;
    cudaStream_t st = nullptr;
    uint32_t n;
    uint64_t m_in;
    Dev d{};
    // overlay storage
    DevBuf<uint64_t> out_beg, in_beg;
    DevBuf<uint32_t> out_deg, in_deg, out_cap, in_cap;
    DevBuf<uint2> out_adj, in_adj;
    DevBuf<uint32_t> level, amark, smark, new_out, new_in, kround;
    DevBuf<uint8_t> inel;
    DevBuf<unsigned long long> emask;  // one word per out-arena entry
    DevBuf<int32_t> P;
    DevBuf<Ctl> ctl;
    Ctl *hctl = nullptr;  // pinned
    // lists
    DevBuf<uint32_t> VO, VO2, A, Anext, S, S2, F, ovf, ovf2, tmp;
    int blk_blocks = 152;
    uint32_t route_deg = 64;  // witness sources above this middle-degree sum go to the block tier
    DevBuf<uint64_t> reqO, reqI, posO, posI;
    DevBuf<uint32_t> scan32;
    DevBuf<uint64_t> scan64;
    // records and log
    DevBuf<uint4> rec;
    DevBuf<uint8_t> rec_flag;
    DevBuf<uint4> log;
    DevBuf<uint32_t> log_round;
    uint64_t log_count = 0;
    // CH edges per vertex (id order)
    DevBuf<uint2> ch_up, ch_dn;
    DevBuf<uint64_t> ch_up_beg, ch_dn_beg;
    DevBuf<uint32_t> ch_up_deg, ch_dn_deg;
    // learned priority
    DevBuf<uint32_t> cn, depth, rescore, orig_deg;
    DevBuf<int32_t> ed_last, label;
    DevBuf<long long> trace;     // 14 int64 per rescoring
    DevBuf<int32_t> trace_prio;  // priority per rescoring
    uint64_t trace_count = 0;
    bool tracing = false, learned = false, composite = false;
    MlpDevice mlp;
    DevBuf<float> fx, fy;
    // dense fallback
    DevBuf<uint32_t> dn32;
    DevBuf<unsigned long long> dn64;
    Dense dense{};
    // memoised witness distances across rounds (witness_memo_limit > 0)
    DevBuf<unsigned long long> dm_keys;
    DevBuf<uint32_t> dm_vals;
    DMap dm{};
    uint64_t dm_limit = 0;
    bool xm = false;              // the map is in use (memoisation or pruning)
    bool prune = false;           // overlay-edge pruning after the rescoring searches
    bool dm_phase_clear = false;  // pruning without memoisation: the map holds one phase
    DevBuf<uint32_t> pmark, dirty;
    void dmap_reserve(uint64_t keys);
    int sms = 152;
    EventPool pool;
    std::vector<Span> spans;

    int cur_round = -1;
    // The build's buffers go back to the library's cache when the builder is
    // destroyed; on an error path its kernels may still be running.
    ~Builder() { cudaStreamSynchronize(st); }
    void mark(double *acc, cudaEvent_t a, int phase = -1) {
        cudaEvent_t b = pool.get();
        CH_CUDA_TRY(cudaEventRecord(b, st));
        spans.push_back({a, b, acc, cur_round, phase});
    }
    cudaEvent_t start() {
        cudaEvent_t a = pool.get();
        CH_CUDA_TRY(cudaEventRecord(a, st));
        return a;
    }

    void sync_ctl() {
        CH_CUDA_TRY(cudaMemcpyAsync(hctl, ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CH_CUDA_TRY(cudaStreamSynchronize(st));
        if (hctl->err & ERR_INPUT) throw Error{CH_EINVAL, "graph has a malformed offset, id or weight"};
        if (hctl->err & ERR_BOUND) throw Error{CH_ECUDA, "internal index check failed"};
        if (hctl->err & ERR_MAP_FULL)
            throw Error{CH_ENOMEM, "the memoised witness-distance map is full (witness_memo_limit)"};
        if (hctl->err) throw Error{CH_ECUDA, "internal capacity error " + std::to_string(hctl->err)};
    }

    void normalise(const ch_graph_t *g);
    void emit_core(uint32_t r, uint32_t nVO, uint64_t live_edges);
    void run_rounds();
    void postprocess();
    template <int MODE>
    void witness(const uint32_t *Sl, const uint32_t *nS_dev, uint32_t nS_max, uint32_t r);
    template <int MODE, int FEAT>
    void launch_witness(const WArgs &a, int blocks);
    unsigned long long level_work = ~0ull;  // F_LW bound; all ones = off
    uint32_t theta = 0;                     // F_TH settled-vertex cap; 0 = off
};

#define CTL_OFF(field) offsetof(Ctl, field)

void Builder::normalise(const ch_graph_t *g) {
    const uint64_t m = g->m;
    if (m >= 0xFFFFFFFFull) throw Error{CH_ERANGE, "more than 2^32 - 2 input edges"};
    DevBuf<uint64_t> off_d;
    DevBuf<uint32_t> tgt_d, w_d;
    const uint64_t *off = g->offsets;
    const uint32_t *tgt = g->targets, *wt = g->weights;
    if (!g->on_device) {
        off_d.alloc(n + 1);
        tgt_d.alloc(m);
        w_d.alloc(m);
        CH_CUDA_TRY(cudaMemcpyAsync(off_d.ptr, off, (n + 1) * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, st));
        if (m) {
            CH_CUDA_TRY(cudaMemcpyAsync(tgt_d.ptr, tgt, m * 4, cudaMemcpyHostToDevice, st));
            CH_CUDA_TRY(cudaMemcpyAsync(w_d.ptr, wt, m * 4, cudaMemcpyHostToDevice, st));
        }
        off = off_d.ptr;
        tgt = tgt_d.ptr;
        wt = w_d.ptr;
    }
    k_validate_offsets<<<grid_for(n, 256, sms * 8), 256, 0, st>>>(off, n, m, ctl.ptr);
    CH_CHECK_LAUNCH();
    sync_ctl();

    DevBuf<uint64_t> keys, tkeys;
    DevBuf<uint32_t> vals, tvals, flags;
    keys.alloc(m);
    vals.alloc(m);
    tkeys.alloc(m);
    tvals.alloc(m);
    flags.alloc(m);
    const int gm = grid_for(m, 256, sms * 16);
    if (m) {
        k_edge_keys<<<gm, 256, 0, st>>>(off, tgt, wt, n, m, keys.ptr, vals.ptr, ctl.ptr);
        CH_CHECK_LAUNCH();
    }
    sync_ctl();
    off_d.release();
    tgt_d.release();
    w_d.release();
    const int vb = bits_for(n ? n - 1 : 0);
    std::vector<int> digits;
    append_digits(digits, 0, vb);
    append_digits(digits, 32, vb);
    radix_sort_pairs(keys.ptr, vals.ptr, tkeys.ptr, tvals.ptr, m, digits, st);
    uint64_t m1 = 0;
    if (m) {
        k_norm_flags<<<gm, 256, 0, st>>>(keys.ptr, m, flags.ptr);
        CH_CHECK_LAUNCH();
        exclusive_scan<uint32_t>(flags.ptr, flags.ptr, nullptr, m, &ctl.ptr->nVO2, scan32.ptr, st);
        sync_ctl();
        m1 = hctl->nVO2;
        k_norm_scatter<<<gm, 256, 0, st>>>(keys.ptr, vals.ptr, m, flags.ptr, tkeys.ptr, tvals.ptr);
        CH_CHECK_LAUNCH();
    }
    h->m_input = m1;
    flags.release();
    // tkeys/tvals now hold the normalised (u, v)-sorted edges
    out_deg.alloc(n);
    in_deg.alloc(n);
    out_cap.alloc(n);
    in_cap.alloc(n);
    out_beg.alloc(n + 1);
    in_beg.alloc(n + 1);
    DevBuf<uint64_t> first;
    first.alloc(n);
    const int gn = grid_for(n, 256, sms * 8);
    const int gm1 = grid_for(m1, 256, sms * 16);
    for (int dir = 0; dir < 2; ++dir) {
        DevBuf<uint32_t> &deg = dir == 0 ? out_deg : in_deg;
        DevBuf<uint32_t> &cap = dir == 0 ? out_cap : in_cap;
        DevBuf<uint64_t> &beg = dir == 0 ? out_beg : in_beg;
        DevBuf<uint2> &adj = dir == 0 ? out_adj : in_adj;
        if (dir == 1 && m1) {
            k_swap_key_halves<<<gm1, 256, 0, st>>>(tkeys.ptr, m1);
            CH_CHECK_LAUNCH();
            radix_sort_pairs(tkeys.ptr, tvals.ptr, keys.ptr, vals.ptr, m1, digits, st);
        }
        deg.zero(st);
        if (m1) {
            k_seg_heads<<<gm1, 256, 0, st>>>(tkeys.ptr, m1, first.ptr);
            CH_CHECK_LAUNCH();
            k_seg_deg<<<gm1, 256, 0, st>>>(tkeys.ptr, m1, first.ptr, deg.ptr);
            CH_CHECK_LAUNCH();
        }
        k_caps<<<gn, 256, 0, st>>>(deg.ptr, n, cap.ptr, beg.ptr);
        CH_CHECK_LAUNCH();
        exclusive_scan<uint64_t>(beg.ptr, beg.ptr, nullptr, n, beg.ptr + n, scan64.ptr, st);
        uint64_t total = 0;
        CH_CUDA_TRY(cudaMemcpyAsync(&total, beg.ptr + n, 8, cudaMemcpyDeviceToHost, st));
        CH_CUDA_TRY(cudaStreamSynchronize(st));
        adj.alloc(total + total / 2 + 1024);
        if (m1) {
            k_fill_adj<<<gm1, 256, 0, st>>>(tkeys.ptr, tvals.ptr, m1, first.ptr, beg.ptr, adj.ptr);
            CH_CHECK_LAUNCH();
        }
        if (dir == 0) hctl->out_tail = total; else hctl->in_tail = total;
    }
    CH_CUDA_TRY(cudaMemcpyAsync(&ctl.ptr->out_tail, &hctl->out_tail, 16, cudaMemcpyHostToDevice, st));
    CH_CUDA_TRY(cudaStreamSynchronize(st));
}

template <int MODE>
void Builder::witness(const uint32_t *Sl, const uint32_t *nS_dev, uint32_t nS_max, uint32_t r) {
    // the tiers' work counters (work, work2, work3, nOvf, nOvf2) are zeroed
    // by k_round_begin / k_contract_begin before each phase
    WArgs a;
    a.d = d;
    a.S = Sl;
    a.nS = nS_dev;
    a.work = &ctl.ptr->work;
    a.round = r;
    a.ovf = ovf.ptr;
    a.ovf2 = ovf2.ptr;
    a.rec = rec.ptr;
    a.rec_flag = rec_flag.ptr;
    a.rec_cap = rec.count;
    a.route_all = (uint32_t)blk_blocks * 16;
    a.route_deg = route_deg;
    a.dm = dm;
    a.level_work = level_work;
    a.theta = theta;
    if (dm_phase_clear) {
        CH_CUDA_TRY(cudaMemsetAsync(dm_keys.ptr, 0xFF, dm_keys.count * sizeof(unsigned long long), st));
        CH_CUDA_TRY(cudaMemsetAsync(&ctl.ptr->dm_count, 0, sizeof(unsigned long long), st));
    }
    cudaEvent_t e0 = start();
    const int blocks = grid_for((uint64_t)nS_max, WIT_WARPS, sms * 8);
    const int feat = (xm ? F_XM : 0) | (level_work != ~0ull && !theta ? F_LW : 0) | (prune ? F_PR : 0) |
                     (theta ? F_TH : 0);
    switch (feat) {
        case 0: launch_witness<MODE, 0>(a, blocks); break;
        case F_XM: launch_witness<MODE, F_XM>(a, blocks); break;
        case F_LW: launch_witness<MODE, F_LW>(a, blocks); break;
        case F_XM | F_LW: launch_witness<MODE, F_XM | F_LW>(a, blocks); break;
        case F_XM | F_PR: launch_witness<MODE, F_XM | F_PR>(a, blocks); break;
        case F_XM | F_LW | F_PR: launch_witness<MODE, F_XM | F_LW | F_PR>(a, blocks); break;
        case F_TH: launch_witness<MODE, F_TH>(a, blocks); break;
        case F_TH | F_XM: launch_witness<MODE, F_TH | F_XM>(a, blocks); break;
        case F_TH | F_XM | F_PR: launch_witness<MODE, F_TH | F_XM | F_PR>(a, blocks); break;
        default: throw Error{CH_EINVAL, "internal: unsupported witness feature set"};
    }
    mark(&h->t_witness_ms, e0, 5);
    h->witness_launches += 3;
}

// The three tiers of one phase, in order (each takes the sources the one
// before it could not hold).
template <int MODE, int FEAT>
void Builder::launch_witness(const WArgs &a, int blocks) {
    k_witness<MODE, FEAT><<<blocks, WIT_WARPS * 32, 0, st>>>(a);
    CH_CHECK_LAUNCH();
    k_witness_block<MODE, FEAT><<<blk_blocks, WB_THREADS, sizeof(BlkSmem), st>>>(a);
    CH_CHECK_LAUNCH();
    k_witness_dense<MODE, FEAT><<<dense.nslots, 256, 0, st>>>(a, dense);
    CH_CHECK_LAUNCH();
}

// Keeps the memoised-distance map at most half full with `keys` keys plus one
// round's new keys (at most one per candidate pair of the round, taken as 8
// per input edge), growing it by a rehash into a map at least twice as large.
// A round that still overfills it fails with CH_ENOMEM.
void Builder::dmap_reserve(uint64_t keys) {
    const uint64_t want = 2 * (keys + 8 * h->m_input + 1024);
    if (dm_keys.count >= want) return;
    uint64_t cap = std::max<uint64_t>(1024, dm_keys.count * 2);
    while (cap < want) cap <<= 1;
    DevBuf<unsigned long long> nk;
    DevBuf<uint32_t> nv;
    nk.alloc(cap);
    nv.alloc(cap);
    nk.fill_ff(st);
    DMap to = dm;
    to.keys = nk.ptr;
    to.vals = nv.ptr;
    to.mask = cap - 1;
    if (dm_keys.count) {
        k_dmap_rehash<<<grid_for(dm_keys.count, 256, sms * 8), 256, 0, st>>>(dm, to, ctl.ptr);
        CH_CHECK_LAUNCH();
    }
    CH_CUDA_TRY(cudaStreamSynchronize(st));
    dm_keys = std::move(nk);
    dm_vals = std::move(nv);
    dm = to;
}

void Builder::emit_core(uint32_t r, uint32_t nVO, uint64_t live_edges) {
    cudaEvent_t e0 = start();
    const Ctl c = *hctl;
    if (ch_up.count < c.ch_up_tail + live_edges)
        ch_up.grow(c.ch_up_tail + live_edges, c.ch_up_tail, st);
    if (ch_dn.count < c.ch_dn_tail + live_edges)
        ch_dn.grow(c.ch_dn_tail + live_edges, c.ch_dn_tail, st);
    k_emit_ch<<<grid_for((uint64_t)nVO * 32, 256, sms * 8), 256, 0, st>>>(
        d, VO.ptr, nVO, ch_up.ptr, ch_dn.ptr, ch_up_beg.ptr, ch_up_deg.ptr, ch_dn_beg.ptr,
        ch_dn_deg.ptr, ch_up.count, ch_dn.count, true, r);
    CH_CHECK_LAUNCH();
    mark(&h->t_update_ms, e0);
    sync_ctl();
    h->core_size = nVO;
}

void Builder::run_rounds() {
    const int gn = grid_for(n, 256, sms * 8);
    // live vertex list and A_0 = V
    k_iota<<<gn, 256, 0, st>>>(VO.ptr, n);
    CH_CHECK_LAUNCH();
    k_iota<<<gn, 256, 0, st>>>(A.ptr, n);
    CH_CHECK_LAUNCH();
    hctl->nVO = n;
    CH_CUDA_TRY(cudaMemcpyAsync(&ctl.ptr->nVO, &hctl->nVO, 4, cudaMemcpyHostToDevice, st));
    uint32_t nA = n, nVO = n;
    uint64_t live_edges = h->m_input;
    // The statistics row of a round is finished at the next read of the
    // control block, which also brings the round's contraction counters
    // (k_round_end): one host synchronisation per round.
    bool pending = false;
    std::array<uint64_t, CH_NSTAT> row{};
    uint64_t row_drop = 0;  // live edges the pending round removed (its V_F's and pruned ones)
    auto finish_row = [&]() {
        if (!pending) return;
        const Ctl &c = *hctl;
        row[4] = c.s_cand;
        row[5] = c.s_kept;
        row[6] = c.s_merged;
        row[7] = c.s_inserted;
        live_edges = live_edges - row_drop + c.s_newEdges;
        row[9] = live_edges;
        h->round_stats.push_back(row);
        if (c.s_nRec > rec.count) throw Error{CH_ECUDA, "internal: record overflow"};
        log_count = c.log_tail;
        pending = false;
    };
    for (uint32_t r = 0; nVO > 0; ++r) {
        if (r > 0x7FFFFFF0u) throw Error{CH_ERANGE, "too many rounds"};
        cur_round = (int)r;
        // reset per-round counters
        k_round_begin<<<1, 1, 0, st>>>(ctl.ptr);
        CH_CHECK_LAUNCH();
        // 1-2: score the affected set
        cudaEvent_t e0 = start();
        const uint32_t sstamp = 2 * r + 1, cstamp = 2 * r + 2;
        if (nA) {
            k_score_prep<<<grid_for((uint64_t)nA * 32, 256, sms * 8), 256, 0, st>>>(d, A.ptr, nA, sstamp,
                                                                                    S.ptr, r);
            CH_CHECK_LAUNCH();
            witness<MODE_SCORE>(S.ptr, &ctl.ptr->nS, nA * 4 + 32 > n ? n : nA * 4 + 32, r);
            if (prune) {
                // Alg. 3's pruning, then the scores on the pruned overlay from
                // the recorded distances
                k_prune_find<<<sms * 8, 256, 0, st>>>(d, dm, S.ptr, &ctl.ptr->nS, r);
                CH_CHECK_LAUNCH();
                k_prune_apply<<<sms * 8, 256, 0, st>>>(d, S.ptr, &ctl.ptr->nS, dirty.ptr, pmark.ptr, r + 1);
                CH_CHECK_LAUNCH();
                k_compact_dirty<<<sms * 8, 256, 0, st>>>(d, dirty.ptr, &ctl.ptr->nDirty, r);
                CH_CHECK_LAUNCH();
                k_score_map<<<grid_for((uint64_t)nA * 32, 256, sms * 8), 256, 0, st>>>(d, dm, A.ptr, nA, r);
                CH_CHECK_LAUNCH();
            }
            if (tracing || learned || composite) {
                if (tracing && trace.count < (trace_count + nA) * 14) {
                    const uint64_t want = std::max<uint64_t>(trace_count + nA, trace.count / 14 * 2);
                    trace.grow(want * 14, trace_count * 14, st);
                    trace_prio.grow(want, trace_count, st);
                }
                long long *rows = tracing ? trace.ptr + trace_count * 14 : nullptr;
                int32_t *plog = tracing ? trace_prio.ptr + trace_count : nullptr;
                const int ga = grid_for(nA, 256, sms * 8);
                if (tracing || learned) {
                    k_features<<<ga, 256, 0, st>>>(d, A.ptr, nA, r, rows, learned ? fx.ptr : nullptr);
                    CH_CHECK_LAUNCH();
                }
                if (learned) {
                    mlp.infer(fx.ptr, nA, fy.ptr, st);
                    k_apply_learned<<<ga, 256, 0, st>>>(d, A.ptr, nA, fy.ptr, plog);
                    CH_CHECK_LAUNCH();
                } else if (composite) {
                    k_composite<<<ga, 256, 0, st>>>(d, A.ptr, nA);
                    CH_CHECK_LAUNCH();
                }
                if (!learned && plog) {
                    k_log_priority<<<ga, 256, 0, st>>>(d, A.ptr, nA, plog);
                    CH_CHECK_LAUNCH();
                }
                if (tracing) trace_count += nA;
            }
        }
        mark(&h->t_score_ms, e0, 0);
        // 3: select
        e0 = start();
        k_select<<<grid_for((uint64_t)nVO, 256, sms * 8), 256, 0, st>>>(d, VO.ptr, nVO, r, F.ptr);
        CH_CHECK_LAUNCH();
        mark(&h->t_select_ms, e0, 1);
        // 4: contraction bookkeeping
        e0 = start();
        k_contract_prep<<<grid_for((uint64_t)nVO * 32, 256, sms * 8), 256, 0, st>>>(
            d, F.ptr, cstamp, r + 1, S2.ptr, Anext.ptr);
        CH_CHECK_LAUNCH();
        mark(&h->t_prep_ms, e0, 2);
        sync_ctl();
        finish_row();  // the round before
        const Ctl c = *hctl;
        const uint32_t nF = c.nF, nS2 = c.nS2, nAnext = c.nAnext;
        if (nF == 0) {
            // no eligible vertex left (only possible with a finite bound):
            // the live vertices are the core
            if (d.cmax == UINT64_MAX) throw Error{CH_ECUDA, "internal: empty selection"};
            emit_core(r, nVO, live_edges);
            break;
        }
        // capacities for this round's contraction
        const uint64_t cb = c.candBound;
        if (rec.count < cb) {
            rec.grow(std::max<uint64_t>(cb, rec.count * 2), 0, st);
            rec_flag.grow(rec.count, 0, st);
        }
        if (log.count < log_count + cb) {
            const uint64_t want = std::max<uint64_t>(log_count + cb, log.count * 2);
            log.grow(want, log_count, st);
            log_round.grow(want, log_count, st);
        }
        if (ch_up.count < c.ch_up_tail + c.degFout)
            ch_up.grow(std::max<uint64_t>(c.ch_up_tail + c.degFout, ch_up.count * 2), c.ch_up_tail, st);
        if (ch_dn.count < c.ch_dn_tail + c.degFin)
            ch_dn.grow(std::max<uint64_t>(c.ch_dn_tail + c.degFin, ch_dn.count * 2), c.ch_dn_tail, st);
        const uint64_t grow_bound = 2 * c.degAnext + 2 * cb + 4ull * nAnext;
        bool regrow = false;
        if (out_adj.count < c.out_tail + grow_bound) {
            out_adj.grow(std::max<uint64_t>(c.out_tail + grow_bound, out_adj.count * 2), c.out_tail, st);
            // the score phase's memo words stay with their arena positions
            emask.grow(out_adj.count, c.out_tail, st);
            regrow = true;
        }
        if (in_adj.count < c.in_tail + grow_bound) {
            in_adj.grow(std::max<uint64_t>(c.in_tail + grow_bound, in_adj.count * 2), c.in_tail, st);
            regrow = true;
        }
        if (regrow) {
            d.out_adj = out_adj.ptr;
            d.in_adj = in_adj.ptr;
            d.emask = emask.ptr;
            d.out_arena = out_adj.count;
            d.in_arena = in_adj.count;
        }
        k_contract_begin<<<1, 1, 0, st>>>(ctl.ptr);
        CH_CHECK_LAUNCH();
        // 5: witness searches for V_F's candidates
        e0 = start();
        if (nS2) witness<MODE_PRUNE>(S2.ptr, &ctl.ptr->nS2, nS2, r);
        mark(&h->t_contract_ms, e0, 3);
        // 6-10
        e0 = start();
        k_emit_ch<<<grid_for((uint64_t)nF * 32, 256, sms * 8), 256, 0, st>>>(
            d, F.ptr, nF, ch_up.ptr, ch_dn.ptr, ch_up_beg.ptr, ch_up_deg.ptr, ch_dn_beg.ptr,
            ch_dn_deg.ptr, ch_up.count, ch_dn.count, false, r);
        CH_CHECK_LAUNCH();
        if (nAnext) {
            const int ga = grid_for(nAnext, 256, sms * 8);
            const int gw = grid_for((uint64_t)nAnext * 32, 256, sms * 8);
            k_compact_lists<<<gw, 256, 0, st>>>(d, Anext.ptr, nAnext, r);
            CH_CHECK_LAUNCH();
            k_reserve<<<ga, 256, 0, st>>>(d, Anext.ptr, nAnext, reqO.ptr, reqI.ptr);
            CH_CHECK_LAUNCH();
            exclusive_scan<uint64_t>(reqO.ptr, posO.ptr, nullptr, nAnext, reinterpret_cast<uint64_t *>(&ctl.ptr->relocOut),
                                     scan64.ptr, st);
            exclusive_scan<uint64_t>(reqI.ptr, posI.ptr, nullptr, nAnext, reinterpret_cast<uint64_t *>(&ctl.ptr->relocIn),
                                     scan64.ptr, st);
            k_relocate<<<gw, 256, 0, st>>>(d, Anext.ptr, nAnext, reqO.ptr, posO.ptr, reqI.ptr,
                                           posI.ptr);
            CH_CHECK_LAUNCH();
        }
        const uint64_t rec_bound = std::max<uint64_t>(cb, 1);
        k_insert<<<grid_for(rec_bound, 256, sms * 8), 256, 0, st>>>(
            d, rec.ptr, rec_flag.ptr, r, log.ptr, log_round.ptr);
        CH_CHECK_LAUNCH();
        compact_alive(VO.ptr, &ctl.ptr->nVO, nVO, level.ptr, VO2.ptr, &ctl.ptr->nVO2, tmp.ptr,
                      scan32.ptr, st);
        std::swap(VO, VO2);
        k_round_end<<<1, 1, 0, st>>>(ctl.ptr, nAnext ? 1 : 0);
        CH_CHECK_LAUNCH();
        std::swap(A, Anext);
        mark(&h->t_update_ms, e0, 4);
        // this round's row: what is known now; its contraction counters
        // arrive with the next read of the control block
        row = {};
        row[0] = nA;
        row[1] = c.nS;
        row[2] = nF;
        row[3] = nS2;
        nVO -= nF;
        row[8] = nVO;
        row_drop = c.degFout + c.degFin + c.pruned;
        pending = true;
        nA = nAnext;
        if (dm_limit) {
            // memoised distances are cleared lazily: only after a round that
            // leaves more keys than the limit; otherwise the map keeps room
            // for another round's keys. The decision needs this round's
            // count before the next round's searches.
            sync_ctl();
            const uint64_t dm_count = hctl->s_dm_count;
            finish_row();
            if (dm_count > dm_limit) {
                CH_CUDA_TRY(cudaMemsetAsync(dm_keys.ptr, 0xFF, dm_keys.count * sizeof(unsigned long long), st));
                CH_CUDA_TRY(cudaMemsetAsync(&ctl.ptr->dm_count, 0, sizeof(unsigned long long), st));
            } else {
                dmap_reserve(dm_count);
            }
        }
    }
    if (pending) {
        sync_ctl();
        finish_row();
    }
    h->n_shortcuts = log_count;
    h->witness_bytes = 0;
}

void Builder::postprocess() {
    const int gn = grid_for(n, 256, sms * 8);
    DevBuf<uint64_t> keys, tkeys;
    DevBuf<uint32_t> vals, tvals;
    keys.alloc(n);
    tkeys.alloc(n);
    vals.alloc(n);
    tvals.alloc(n);
    k_rank_keys<<<gn, 256, 0, st>>>(level.ptr, P.ptr, n, keys.ptr, vals.ptr);
    CH_CHECK_LAUNCH();
    std::vector<int> digits;
    append_digits(digits, 0, 32);
    append_digits(digits, 32, bits_for(h->round_stats.size()));
    radix_sort_pairs(keys.ptr, vals.ptr, tkeys.ptr, tvals.ptr, n, digits, st);
    h->perm = std::move(vals);
    h->rank.alloc(n);
    k_rank_from_perm<<<gn, 256, 0, st>>>(h->perm.ptr, n, h->rank.ptr);
    CH_CHECK_LAUNCH();
    const uint64_t n_up = hctl->ch_up_tail, n_dn = hctl->ch_dn_tail;
    if (n_up >= 0xFFFFFFFFull || n_dn >= 0xFFFFFFFFull)
        throw Error{CH_ERANGE, "hierarchy has 2^32 - 1 or more edges in one direction"};
    h->n_up = n_up;
    h->n_down = n_dn;
    for (int dir = 0; dir < 2; ++dir) {
        DevBuf<uint32_t> &off = dir == 0 ? h->up_off : h->dn_off;
        DevBuf<uint2> &adj = dir == 0 ? h->up_adj : h->dn_adj;
        off.alloc(n + 1);
        adj.alloc(dir == 0 ? n_up : n_dn);
        k_ranked_deg<<<gn, 256, 0, st>>>(h->perm.ptr, n, dir == 0 ? ch_up_deg.ptr : ch_dn_deg.ptr,
                                         off.ptr);
        CH_CHECK_LAUNCH();
        exclusive_scan<uint32_t>(off.ptr, off.ptr, nullptr, (uint64_t)n + 1, nullptr, scan32.ptr, st);
        k_ranked_fill<<<gn, 256, 0, st>>>(h->perm.ptr, h->rank.ptr, n,
                                          dir == 0 ? ch_up_beg.ptr : ch_dn_beg.ptr,
                                          dir == 0 ? ch_up_deg.ptr : ch_dn_deg.ptr,
                                          dir == 0 ? ch_up.ptr : ch_dn.ptr,
                                          dir == 0 ? hctl->ch_up_tail : hctl->ch_dn_tail, off.ptr,
                                          dir == 0 ? n_up : n_dn, adj.ptr, ctl.ptr);
        CH_CHECK_LAUNCH();
    }
    sync_ctl();
    if (hctl->longRows) {
        // some row is longer than a thread sorts: sort every row of both
        // CSRs at once by (row, target rank)
        std::vector<int> rd;
        append_digits(rd, 0, bits_for(n));
        append_digits(rd, 32, bits_for(n));
        for (int dir = 0; dir < 2; ++dir) {
            DevBuf<uint32_t> &off = dir == 0 ? h->up_off : h->dn_off;
            DevBuf<uint2> &adj = dir == 0 ? h->up_adj : h->dn_adj;
            const uint64_t m = dir == 0 ? n_up : n_dn;
            if (m < 2) continue;
            DevBuf<uint64_t> k1, k2;
            DevBuf<uint32_t> v1, v2;
            k1.alloc(m);
            k2.alloc(m);
            v1.alloc(m);
            v2.alloc(m);
            k_row_keys<<<grid_for((uint64_t)n * 32, 256, sms * 8), 256, 0, st>>>(off.ptr, n, adj.ptr, k1.ptr,
                                                                                 v1.ptr);
            CH_CHECK_LAUNCH();
            radix_sort_pairs(k1.ptr, v1.ptr, k2.ptr, v2.ptr, m, rd, st);
            k_row_unpack<<<grid_for(m, 256, sms * 8), 256, 0, st>>>(k1.ptr, v1.ptr, m, adj.ptr);
            CH_CHECK_LAUNCH();
            CH_CUDA_TRY(cudaStreamSynchronize(st));
        }
    }
}

}  // namespace

void build_hierarchy(ch_s *h, const ch_graph_t *g, const ch_params_t *p) {
    Builder b;
    b.h = h;
    b.st = (cudaStream_t)p->stream;
    b.n = g->n;
    b.m_in = g->m;
    b.sms = device_sm_count();
    if (p->witness_route_deg) b.route_deg = p->witness_route_deg;
    const uint32_t n = g->n;
    h->n = n;
    h->hop_limit = p->hop_limit;
    CH_CUDA_TRY(cudaMallocHost(&b.hctl, sizeof(Ctl)));
    struct PinnedFree {
        Ctl *p;
        ~PinnedFree() {
            if (p) cudaFreeHost(p);
        }
    } pf{b.hctl};
    std::memset(b.hctl, 0, sizeof(Ctl));
    b.ctl.alloc(1);
    b.ctl.zero(b.st);
    b.scan32.alloc(kScanScratch);
    b.scan64.alloc(kScanScratch);

    cudaEvent_t t0 = b.start();
    if (n == 0) {
        if (g->m != 0) throw Error{CH_EINVAL, "n = 0 with m > 0"};
        h->level.alloc(0);
        h->prio.alloc(0);
        h->rank.alloc(0);
        h->perm.alloc(0);
        h->up_off.alloc(1);
        h->dn_off.alloc(1);
        h->up_off.zero(b.st);
        h->dn_off.zero(b.st);
        h->up_adj.alloc(0);
        h->dn_adj.alloc(0);
        h->sc.alloc(0);
        h->sc_round.alloc(0);
        CH_CUDA_TRY(cudaStreamSynchronize(b.st));
        return;
    }
    b.normalise(g);
    b.mark(&h->t_norm_ms, t0);

    b.level.alloc(n);
    b.level.fill_ff(b.st);
    b.P.alloc(n);
    b.P.zero(b.st);
    b.amark.alloc(n);
    b.amark.zero(b.st);
    b.inel.alloc(n);
    b.inel.zero(b.st);
    b.kround.alloc(n);
    b.kround.zero(b.st);
    b.smark.alloc(n);
    b.smark.zero(b.st);
    b.new_out.alloc(n);
    b.new_out.zero(b.st);
    b.new_in.alloc(n);
    b.new_in.zero(b.st);
    for (auto *l : {&b.VO, &b.VO2, &b.A, &b.Anext, &b.S, &b.S2, &b.F, &b.ovf, &b.ovf2}) l->alloc(n);
    {
        const int smem = (int)sizeof(BlkSmem);
        CH_CUDA_TRY(cudaFuncSetAttribute(k_witness_block<MODE_SCORE, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        CH_CUDA_TRY(cudaFuncSetAttribute(k_witness_block<MODE_PRUNE, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        const int feat = (p->witness_memo_limit || p->witness_prune ? F_XM : 0) |
                         (p->witness_level_work && !p->witness_settle_cap ? F_LW : 0) |
                         (p->witness_prune ? F_PR : 0) | (p->witness_settle_cap ? F_TH : 0);
        auto set_smem = [&](auto score_kernel, auto prune_kernel) {
            CH_CUDA_TRY(cudaFuncSetAttribute(score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            CH_CUDA_TRY(cudaFuncSetAttribute(prune_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        };
        if (feat == F_XM) set_smem(k_witness_block<MODE_SCORE, F_XM>, k_witness_block<MODE_PRUNE, F_XM>);
        if (feat == F_LW) set_smem(k_witness_block<MODE_SCORE, F_LW>, k_witness_block<MODE_PRUNE, F_LW>);
        if (feat == (F_XM | F_LW))
            set_smem(k_witness_block<MODE_SCORE, F_XM | F_LW>, k_witness_block<MODE_PRUNE, F_XM | F_LW>);
        if (feat == (F_XM | F_PR))
            set_smem(k_witness_block<MODE_SCORE, F_XM | F_PR>, k_witness_block<MODE_PRUNE, F_XM | F_PR>);
        if (feat == (F_XM | F_LW | F_PR))
            set_smem(k_witness_block<MODE_SCORE, F_XM | F_LW | F_PR>,
                     k_witness_block<MODE_PRUNE, F_XM | F_LW | F_PR>);
        if (feat == F_TH) set_smem(k_witness_block<MODE_SCORE, F_TH>, k_witness_block<MODE_PRUNE, F_TH>);
        if (feat == (F_TH | F_XM))
            set_smem(k_witness_block<MODE_SCORE, F_TH | F_XM>, k_witness_block<MODE_PRUNE, F_TH | F_XM>);
        if (feat == (F_TH | F_XM | F_PR))
            set_smem(k_witness_block<MODE_SCORE, F_TH | F_XM | F_PR>,
                     k_witness_block<MODE_PRUNE, F_TH | F_XM | F_PR>);
        int per_sm = 0;
        CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_witness_block<MODE_PRUNE, 0>,
                                                                  WB_THREADS, smem));
        b.blk_blocks = b.sms * std::max(1, per_sm);
    }
    b.tmp.alloc((size_t)n + 1);
    b.reqO.alloc(n);
    b.reqI.alloc(n);
    b.posO.alloc(n);
    b.posI.alloc(n);
    const uint64_t m1 = h->m_input;
    b.rec.alloc(std::max<uint64_t>(1024, m1));
    b.rec_flag.alloc(b.rec.count);
    b.log.alloc(std::max<uint64_t>(1024, m1));
    b.log_round.alloc(b.log.count);
    b.ch_up.alloc(m1 + 1024);
    b.ch_dn.alloc(m1 + 1024);
    b.ch_up_beg.alloc(n);
    b.ch_dn_beg.alloc(n);
    b.ch_up_deg.alloc(n);
    b.ch_dn_deg.alloc(n);
    // dense fallback slots: 9 uint32 + 1 uint64 arrays of n per slot; the
    // pool is 1 GiB, or 128 B per input edge up to 8 GiB (graphs with hubs
    // send many sources here), with 2 to 256 slots
    const uint64_t per_slot = (uint64_t)n * (9 * 4 + 8);
    const uint64_t pool_bytes = std::min<uint64_t>(8ull << 30, std::max<uint64_t>(1ull << 30, 128 * m1));
    uint32_t slots = (uint32_t)std::max<uint64_t>(2, std::min<uint64_t>(256, pool_bytes / per_slot));
    b.dense.nslots = slots;
    b.dn32.alloc((size_t)slots * n * 9);
    b.dn64.alloc((size_t)slots * n);
    {
        const size_t sn = (size_t)slots * n;
        uint32_t *p32 = b.dn32.ptr;
        b.dense.dist = p32;
        b.dense.fst = p32 + sn;
        b.dense.fa = p32 + 2 * sn;
        b.dense.fb = p32 + 3 * sn;
        b.dense.fda = p32 + 4 * sn;
        b.dense.fdb = p32 + 5 * sn;
        b.dense.touched = p32 + 6 * sn;
        b.dense.mt = p32 + 7 * sn;
        b.dense.direct = p32 + 8 * sn;
        b.dense.merge = b.dn64.ptr;
        CH_CUDA_TRY(cudaMemsetAsync(b.dense.direct, 0xFF, sn * 4, b.st));
        CH_CUDA_TRY(cudaMemsetAsync(b.dense.dist, 0xFF, sn * 4, b.st));
        CH_CUDA_TRY(cudaMemsetAsync(b.dense.fst, 0, sn * 4, b.st));
        CH_CUDA_TRY(cudaMemsetAsync(b.dense.merge, 0xFF, sn * 8, b.st));
    }

    b.cn.alloc(n);
    b.cn.zero(b.st);
    b.depth.alloc(n);
    b.depth.zero(b.st);
    b.rescore.alloc(n);
    b.rescore.zero(b.st);
    b.orig_deg.alloc(n);
    b.ed_last.alloc(n);
    b.ed_last.zero(b.st);
    b.label.alloc(n);
    b.label.zero(b.st);
    b.tracing = p->trace != 0;
    b.learned = p->priority == CH_PRIO_LEARNED;
    b.composite = p->priority == CH_PRIO_COMPOSITE;
    if (b.learned) {
        b.mlp.load(p->mlp_weights, b.st);
        b.fx.alloc((size_t)n * 16);
        b.fy.alloc(n);
    }
    if (b.tracing) {
        b.trace.alloc((size_t)n * 14 * 2);
        b.trace_prio.alloc((size_t)n * 2);
    }

    Dev &d = b.d;
    d.n = n;
    d.H = p->hop_limit;
    d.tie_mode = p->tie_break;
    d.tie_seed = p->tie_seed;
    d.out_beg = b.out_beg.ptr;
    d.in_beg = b.in_beg.ptr;
    d.out_deg = b.out_deg.ptr;
    d.in_deg = b.in_deg.ptr;
    d.out_cap = b.out_cap.ptr;
    d.in_cap = b.in_cap.ptr;
    d.out_adj = b.out_adj.ptr;
    d.in_adj = b.in_adj.ptr;
    d.out_arena = b.out_adj.count;
    d.in_arena = b.in_adj.count;
    d.level = b.level.ptr;
    d.P = b.P.ptr;
    d.amark = b.amark.ptr;
    d.smark = b.smark.ptr;
    d.new_out = b.new_out.ptr;
    d.new_in = b.new_in.ptr;
    d.ctl = b.ctl.ptr;
    d.cn = b.cn.ptr;
    d.depth = b.depth.ptr;
    d.rescore = b.rescore.ptr;
    d.orig_deg = b.orig_deg.ptr;
    d.ed_last = b.ed_last.ptr;
    d.label = b.label.ptr;
    d.cmax = p->max_candidates_per_vertex;
    d.inel = b.inel.ptr;
    d.ball = p->witness_ball_limit ? p->witness_ball_limit : 0xFFFFFFFFu;
    // memoised in-round decisions need both phases to decide alike, which a
    // ball bound or a level-work bound breaks (their cut levels depend on
    // each phase's own weight bound, through the labels it keeps); the
    // memoised distances across rounds replace them
    d.memo = p->witness_ball_limit == 0 && p->witness_memo_limit == 0 && p->witness_prune == 0 &&
             (p->witness_level_work == 0 || p->witness_settle_cap != 0);
    if (p->witness_level_work) b.level_work = p->witness_level_work;
    b.theta = p->witness_settle_cap;
    if (p->witness_memo_limit || p->witness_prune) {
        b.xm = true;
        b.dm.count = &b.ctl.ptr->dm_count;
        b.dm_limit = p->witness_memo_limit;
        b.dm_phase_clear = p->witness_memo_limit == 0;
        b.dmap_reserve(0);
    }
    if (p->witness_prune) {
        b.prune = true;
        b.pmark.alloc(n);
        b.pmark.zero(b.st);
        b.dirty.alloc(n);
    }
    b.emask.alloc(b.out_adj.count);
    d.emask = b.emask.ptr;
    d.kround = b.kround.ptr;
    k_orig_deg<<<grid_for(n, 256, b.sms * 8), 256, 0, b.st>>>(d);
    CH_CHECK_LAUNCH();

    b.run_rounds();
    b.cur_round = -1;
    cudaEvent_t t1 = b.start();
    b.postprocess();
    b.mark(&h->t_post_ms, t1);
    b.mark(&h->stats.build_ms, t0);
    CH_CUDA_TRY(cudaStreamSynchronize(b.st));

    h->round_times.assign(h->round_stats.size(), {});
    for (const Span &s : b.spans) {
        float ms = 0;
        CH_CUDA_TRY(cudaEventElapsedTime(&ms, s.a, s.b));
        *s.acc += ms;
        if (s.round >= 0 && s.phase >= 0 && (size_t)s.round < h->round_times.size())
            h->round_times[s.round][s.phase] += ms;
    }
    const Ctl &c = *b.hctl;
    h->stats.witness_sources = c.wit_sources + c.wit_block + c.wit_fallback;
    h->stats.witness_fallback = c.wit_block + c.wit_fallback;
    h->stats.witness_dense = c.wit_fallback;
    // Algorithmic bytes of the witness kernels: per search the source id
    // (4 B); per vertex whose out-list is read its offset and degree (12 B);
    // per adjacency entry read (id + weight, 8 B).
    h->witness_bytes = 4 * (c.wit_sources + c.wit_block + c.wit_fallback) + 12 * c.wit_vertices +
                       8 * c.wit_edges + 12 * c.wit_middles + 8 * c.wit_midedges;

    h->level = std::move(b.level);
    h->prio = std::move(b.P);
    h->labels = std::move(b.label);
    h->trace = std::move(b.trace);
    h->trace_prio = std::move(b.trace_prio);
    h->trace_rows = b.trace_count;          // row slots, marked ones included
    h->trace_valid = c.trace_valid;
    h->sc = std::move(b.log);
    h->sc_round = std::move(b.log_round);
}

}  // namespace gbch
