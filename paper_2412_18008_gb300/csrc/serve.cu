// Device-resident query server with continuous batching (no counterpart in
// the paper, which runs queries one after another).
//
// A persistent kernel keeps its blocks busy with requests published by the
// host into mapped pinned memory: a source and 1..k targets (k = 1 is an
// s-t query, k > 1 one-to-many). The unit of work is one (source, target)
// pair: a request's targets occupy consecutive positions of a pool, and
// blocks take pool positions in order from a device counter, so the
// targets of one large request are spread over every free block, and
// requests that arrive while others are on the device start as soon as a
// block frees. The block that finishes a request's last target publishes its
// completion. Admission is by memory: the host publishes a request only
// when the ring and the pool have room for it (ch_server_submit returns
// CH_EAGAIN otherwise).
//
// Each pair runs the batch kernel's shared-memory search (the same
// bidirectional upward search with the same pruning); a pair whose search
// spaces overflow the shared table is redone in the same block on a per-block
// hash table in global memory, so a request never needs a second kernel.
//
// Waits are bounded: a block that finds no work sleeps in short steps and
// gives up after the idle limit (device globaltimer), which closes the loop
// for every block and records a timeout; the host's stop call waits a
// bounded time for the kernel.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <new>
#include <thread>

#include "handle.cuh"
#include "qsearch.cuh"

namespace gbch {
namespace {

struct SvDesc {  // one request, written by the host before publication
    uint32_t s, k;
    uint64_t pos;  // pool position (monotone) of its first target
    uint64_t seq;  // its ticket
};

struct SvCtl {  // mapped host memory, written by the host only
    uint64_t published;  // pool positions [0, published) are readable
    uint32_t stop;
    uint32_t pad;
};

struct SvArgs {
    QArgs q;                     // hierarchy and the error word (status)
    SvCtl *ctl;                  // mapped
    const SvDesc *desc;          // mapped ring
    const uint32_t *item_req;    // mapped pool: ticket + 1 of the request owning each entry
    const uint32_t *targets;     // mapped pool
    uint32_t *answers;           // mapped pool
    uint32_t *done;              // mapped ring: ticket + 1 when served
    unsigned long long *t_begin, *t_end;  // mapped ring: device time (ns)
    uint32_t ring;
    uint64_t pool;
    unsigned long long *claimed;  // device: pool positions taken so far (all published)
    uint32_t *finished;           // device: targets served per ring slot
    uint32_t *closing;            // device: epoch of the launch a block closed
    uint32_t epoch;               // this launch (1, 2, ...)
    unsigned *status;             // device: SV_IDLE | QERR_BOUND | SV_UNMATCHED
    unsigned long long *diag;     // device: the first failure (SvDiag layout)
    unsigned long long idle_ns;
    // per-block fallback tables (global memory)
    uint32_t tbits;               // table of 2^tbits slots
    uint32_t fcap;                // frontier capacity
    uint32_t *key, *df, *db, *fst, *front, *touched;
};

// Status bits of the device loop (QERR_BOUND = 2 is an index check).
constexpr unsigned SV_IDLE = 1u;       // a launch ended after the idle limit without a published position
constexpr unsigned SV_UNMATCHED = 4u;  // a published entry never matched its descriptor

// What the loop saw when it gave up, for the host's messages: the first
// idle exit (words [0, DG_ERR)) and the last failure (words [DG_ERR, 2 DG_ERR)).
enum SvDiag : int {
    DG_CODE = 0,  // SV_IDLE or SV_UNMATCHED (0: none)
    DG_POS,       // idle: the claim counter; failure: the position taken
    DG_PUB,       // the published count last read
    DG_CLAIMED,   // idle: the launch epoch; failure: the claim counter
    DG_ITEM,      // failure: the entry's ticket + 1
    DG_SEQ,       // failure: the descriptor's ticket
    DG_DPOS,      // failure: the descriptor's first position
    DG_DK,        // failure: the descriptor's target count
    DG_ERR,       // offset of the failure record
    DG_WORDS = 2 * DG_ERR
};

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Relaxed system-scope loads of host-written (mapped) data.
__device__ __forceinline__ uint32_t ld_sys(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_sys(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

struct Tab {
    uint32_t *key, *df, *db, *fst, *front, *touched;
    uint32_t mask, fcap;
};

__device__ __forceinline__ uint32_t sv_insert(const Tab &t, uint32_t v, uint32_t bits, uint32_t *ntouch) {
    uint32_t h = (v * 2654435761u) >> (32 - bits);
    for (uint32_t probe = 0; probe <= t.mask; ++probe) {
        const uint32_t k = t.key[h];
        if (k == v) return h;
        if (k == EMPTY) {
            const uint32_t old = atomicCAS(&t.key[h], EMPTY, v);
            if (old == EMPTY) {
                t.touched[atomicAdd(ntouch, 1u)] = h;
                return h;
            }
            if (old == v) return h;
        }
        h = (h + 1) & t.mask;
    }
    return EMPTY;
}

__device__ __forceinline__ bool sv_claim(uint32_t *fst, uint32_t slot, uint32_t dir, uint32_t lvl) {
    const uint32_t shift = dir ? 16u : 0u;
    uint32_t old = fst[slot];
    while (true) {
        if (((old >> shift) & 0xFFFFu) == lvl) return false;
        const uint32_t want = (old & ~(0xFFFFu << shift)) | (lvl << shift);
        const uint32_t prev = atomicCAS(&fst[slot], old, want);
        if (prev == old) return true;
        old = prev;
    }
}

// Fallback for a pair whose search spaces overflow the shared table: the
// same search (warp-flattened levels, no stalling), labels in the block's
// global hash table. Control values (s_cnt3, s_ovf) are read between two
// barriers as in block_search. Returns INF when unreachable.
__device__ uint32_t sv_query(const SvArgs &a, const Tab &t, uint32_t rs, uint32_t rt,
                             uint32_t *s_cnt3, uint32_t *s_ovf, uint32_t *s_mu, uint32_t *s_nt) {
    const QArgs &g = a.q;
    const uint32_t tid = threadIdx.x;
    __syncthreads();
    if (tid == 0) {
        *s_nt = 0;
        const uint32_t ss = sv_insert(t, rs, a.tbits, s_nt);
        const uint32_t st = sv_insert(t, rt, a.tbits, s_nt);
        t.df[ss] = 0;
        t.db[st] = 0;
        t.front[0] = ss;
        t.front[1] = st | 0x80000000u;
        s_cnt3[0] = 2;
        s_cnt3[1] = 0;
        s_cnt3[2] = 0;
        *s_ovf = 0;
        *s_mu = ss == st ? 0u : INF;
    }
    for (uint32_t lvl = 1;; ++lvl) {
        __syncthreads();
        const uint32_t cur = (lvl - 1) & 1u;
        const uint32_t nfront = s_cnt3[(lvl - 1) % 3];
        const uint32_t ovf = *s_ovf;
        if (ovf || nfront == 0 || lvl >= 0xFFFFu) break;
        if (tid == 0) s_cnt3[(lvl + 1) % 3] = 0;
        const uint32_t *fr = t.front + (size_t)cur * t.fcap;
        uint32_t *fn = t.front + (size_t)(cur ^ 1u) * t.fcap;
        // frontier entries dealt to warps round-robin; each warp spreads its
        // entries' out-edges over its lanes
        const uint32_t lane = lane_id(), warp = tid >> 5, nwarps = blockDim.x >> 5;
        for (uint32_t p0 = 0; p0 < nfront; p0 += blockDim.x) {
            const uint32_t fi = p0 + warp + nwarps * lane;
            const bool fv = fi < nfront && fi < t.fcap;
            const uint32_t ent = fv ? fr[fi] : 0;
            const uint32_t dir = ent >> 31, slot = ent & 0x7FFFFFFFu;
            bool ok = fv;
            if (ok && slot > t.mask) {
                atomicOr(a.status, QERR_BOUND);
                ok = false;
            }
            const uint32_t x = ok ? t.key[slot] : 0;
            if (ok && x >= g.n) {
                atomicOr(a.status, QERR_BOUND);
                ok = false;
            }
            const uint32_t *off = dir ? g.dn_off : g.up_off;
            const uint32_t ne = dir ? g.n_dn : g.n_up;
            const uint32_t b = ok ? off[x] : 0, e_end = ok ? off[x + 1] : 0;
            if (ok && (b > e_end || e_end > ne)) {
                atomicOr(a.status, QERR_BOUND);
                ok = false;
            }
            const uint32_t cnt = ok ? e_end - b : 0;
            const uint32_t dx = cnt ? (dir ? t.db[slot] : t.df[slot]) : INF;
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
                if (e0 >= total) continue;
                const uint2 e = (odir ? g.dn_adj : g.up_adj)[ob + (e0 - oex)];
                const uint32_t nd = sat_add(odx, e.y);
                if (e.x >= g.n) {
                    atomicOr(a.status, QERR_BOUND);
                    continue;
                }
                if (nd == INF || nd >= *(volatile uint32_t *)s_mu) continue;
                const uint32_t ys = sv_insert(t, e.x, a.tbits, s_nt);
                if (ys == EMPTY) {
                    *s_ovf = 1;
                    continue;
                }
                uint32_t *dist = odir ? t.db : t.df;
                const uint32_t old = atomicMin(&dist[ys], nd);
                if (nd >= old) continue;
                const uint32_t other = odir ? t.df[ys] : t.db[ys];
                if (other != INF) atomicMin(s_mu, sat_add(nd, other));
                if (sv_claim(t.fst, ys, odir, lvl)) {
                    const uint32_t p = atomicAdd(&s_cnt3[lvl % 3], 1u);
                    if (p < t.fcap) fn[p] = ys | (odir << 31);
                    else *s_ovf = 1;
                }
            }
        }
    }
    __syncthreads();
    if (*s_ovf && tid == 0) atomicOr(a.status, QERR_BOUND);
    // the answer: least meeting sum over the reached vertices
    const uint32_t nt = *s_nt;
    uint32_t mu = INF;
    for (uint32_t p = tid; p < nt; p += blockDim.x) {
        const uint32_t sl = t.touched[p];
        mu = min(mu, sat_add(t.df[sl], t.db[sl]));
    }
    __syncthreads();
    if (tid == 0) *s_mu = INF;
    __syncthreads();
    atomicMin(s_mu, mu);
    __syncthreads();
    const uint32_t res = *s_mu;
    // reset the slots this query touched
    for (uint32_t p = tid; p < nt; p += blockDim.x) {
        const uint32_t sl = t.touched[p];
        t.key[sl] = EMPTY;
        t.df[sl] = INF;
        t.db[sl] = INF;
        t.fst[sl] = 0;
    }
    __syncthreads();
    return res;
}

template <bool WARP, bool STALL, bool DELTA = false>
__global__ void __launch_bounds__(QB_THREADS) k_serve(SvArgs a) {
    extern __shared__ __align__(16) unsigned char qb_raw[];
    QBSmem<12> &q = *reinterpret_cast<QBSmem<12> *>(qb_raw);
    QStat stat;  // not reported
    qb_clear(q);
    __shared__ uint32_t s_go, s_src, s_tgt, s_k, s_slot, s_first;
    __shared__ unsigned long long s_seq;
    __shared__ uint64_t s_e;
    const uint32_t tid = threadIdx.x;
    const QArgs &g = a.q;
    Tab t;
    const size_t tsz = (size_t)1 << a.tbits;
    t.key = a.key + blockIdx.x * tsz;
    t.df = a.df + blockIdx.x * tsz;
    t.db = a.db + blockIdx.x * tsz;
    t.fst = a.fst + blockIdx.x * tsz;
    t.touched = a.touched + blockIdx.x * tsz;
    t.front = a.front + blockIdx.x * (size_t)a.fcap * 2;
    t.mask = (uint32_t)tsz - 1;
    t.fcap = a.fcap;
    while (true) {
        __syncthreads();
        // Thread 0 takes the next published pool position. A position is
        // taken only once the host has published it, so a block that gives
        // up waiting holds nothing: after the idle limit the first block to
        // reach it closes this launch, every block leaves at its next look,
        // and what is published later waits for the host to launch the loop
        // again.
        if (tid == 0) {
            s_go = 0;
            const unsigned long long t0 = globaltimer();
            unsigned sleep_ns = 256;
            unsigned long long pos = 0;
            while (true) {
                if (*(volatile uint32_t *)a.closing == a.epoch) break;
                const unsigned long long pub = ld_acquire_sys(&a.ctl->published);
                const unsigned long long c = *(volatile unsigned long long *)a.claimed;
                if (c < pub) {
                    if (atomicCAS(a.claimed, c, c + 1ull) == c) {
                        pos = c;
                        s_go = 1;
                        break;
                    }
                    continue;  // another block took it: look again at once
                }
                // stop is set after the last publication: look again first
                if (ld_acquire_sys(&a.ctl->stop)) {
                    if (*(volatile unsigned long long *)a.claimed < ld_acquire_sys(&a.ctl->published)) continue;
                    break;
                }
                if (globaltimer() - t0 > a.idle_ns) {
                    if (atomicCAS(&a.diag[DG_CODE], 0ull, (unsigned long long)SV_IDLE) == 0ull) {
                        a.diag[DG_POS] = c;
                        a.diag[DG_PUB] = pub;
                        a.diag[DG_CLAIMED] = a.epoch;
                    }
                    atomicOr(a.status, SV_IDLE);
                    atomicExch(a.closing, a.epoch);
                    break;
                }
                __nanosleep(sleep_ns);
                sleep_ns = min(2u * sleep_ns, 8192u);
            }
            if (s_go) {
                // The entry names its request (ticket + 1); the request's
                // descriptor must carry that ticket and cover this position.
                // Both were written before the publication, so they match at
                // once; the re-read only guards against seeing them late. A
                // taken position is never dropped: a block that cannot match
                // it within the idle limit records what it saw and fails the
                // loop, which the host reports.
                const uint64_t e = pos % a.pool;
                const unsigned long long t1 = globaltimer();
                uint32_t v = 0, dk = 0;
                uint64_t dseq = 0, dpos = 0;
                while (true) {
                    v = ld_sys(a.item_req + e);
                    if (v != 0) {
                        const uint32_t slot = (v - 1) % a.ring;
                        const SvDesc *d = a.desc + slot;
                        dseq = ld_sys(&d->seq);
                        dpos = ld_sys(&d->pos);
                        dk = ld_sys(&d->k);
                        if ((uint32_t)(dseq + 1) == v && dpos <= pos && pos < dpos + dk) {
                            s_src = ld_sys(&d->s);
                            s_k = dk;
                            s_seq = dseq;
                            s_first = dpos == pos;
                            s_tgt = ld_sys(a.targets + e);
                            s_slot = slot;
                            s_e = e;
                            if (s_first) a.t_begin[slot] = globaltimer();
                            break;
                        }
                    }
                    if (globaltimer() - t1 > a.idle_ns) {
                        a.diag[DG_ERR + DG_CODE] = SV_UNMATCHED;
                        a.diag[DG_ERR + DG_POS] = pos;
                        a.diag[DG_ERR + DG_PUB] = ld_sys(&a.ctl->published);
                        a.diag[DG_ERR + DG_CLAIMED] = *(volatile unsigned long long *)a.claimed;
                        a.diag[DG_ERR + DG_ITEM] = v;
                        a.diag[DG_ERR + DG_SEQ] = dseq;
                        a.diag[DG_ERR + DG_DPOS] = dpos;
                        a.diag[DG_ERR + DG_DK] = dk;
                        atomicOr(a.status, SV_UNMATCHED);
                        atomicExch(a.closing, a.epoch);
                        s_go = 0;
                        break;
                    }
                    __nanosleep(256);
                }
            }
        }
        __syncthreads();
        if (!s_go) break;
        const uint32_t s = s_src, tv = s_tgt;
        uint32_t ans = INF;
        if (s < g.n && tv < g.n) {
            const uint32_t rs = g.rank[s], rt = g.rank[tv];
            if (rs < g.n && rt < g.n) {
                uint32_t cnt;
                if (!block_query<true, WARP, 12, STALL, DELTA>(q, g, rs, rt, ans, cnt, stat))
                    ans = sv_query(a, t, rs, rt, q.cnt3, &q.ovf, &q.mu, &q.cnt);
            } else if (tid == 0) {
                atomicOr(a.status, QERR_BOUND);
            }
        }
        if (tid == 0) {
            const uint32_t slot = s_slot;
            ((volatile uint32_t *)a.answers)[s_e] = ans;
            __threadfence_system();
            if (atomicAdd(&a.finished[slot], 1u) + 1u == s_k) {
                // last target of the request: publish its completion
                atomicExch(&a.finished[slot], 0u);
                a.t_end[slot] = globaltimer();
                __threadfence_system();
                ((volatile uint32_t *)a.done)[slot] = (uint32_t)(s_seq + 1);
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

template <class T>
struct Mapped {
    T *h = nullptr;
    T *d = nullptr;
    void alloc(size_t n) {
        void *p = nullptr;
        if (cudaHostAlloc(&p, std::max<size_t>(n, 1) * sizeof(T), cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            throw Error{CH_ENOMEM, "mapped host allocation failed"};
        }
        h = static_cast<T *>(p);
        std::memset(p, 0, std::max<size_t>(n, 1) * sizeof(T));
        void *dp = nullptr;
        CH_CUDA_TRY(cudaHostGetDevicePointer(&dp, p, 0));
        d = static_cast<T *>(dp);
    }
    ~Mapped() {
        if (h) cudaFreeHost(h);
    }
};

}  // namespace gbch

struct ch_server_s {
    ch_s *h = nullptr;
    cudaStream_t st = nullptr;
    uint32_t nblocks = 0, ring = 0;
    uint64_t pool = 0;
    unsigned long long idle_ns = 0;
    gbch::Mapped<gbch::SvCtl> ctl;
    gbch::Mapped<gbch::SvDesc> desc;
    gbch::Mapped<uint32_t> item_req, targets, answers, done;
    gbch::Mapped<unsigned long long> t_begin, t_end;
    gbch::DevBuf<uint32_t> scratch;
    gbch::DevBuf<unsigned long long> claimed;
    gbch::DevBuf<uint32_t> finished, closing;
    gbch::DevBuf<unsigned> status;
    gbch::DevBuf<unsigned long long> diag;
    // host-side ring and pool state
    uint64_t next_seq = 0, retired = 0, pool_head = 0, pool_tail = 0;
    std::vector<uint64_t> slot_pos;
    std::vector<uint32_t> slot_k;
    std::vector<char> consumed;
    bool running = false;
    // the loop's launch: kernel, block size and arguments; a launch that
    // ended at the idle limit is launched again (next epoch) when needed
    gbch::SvArgs args{};
    void (*kern)(gbch::SvArgs) = nullptr;
    int threads = 0;
    uint32_t launches = 0;
};

namespace gbch {

// Launches the device loop for the next epoch.
void server_launch(ch_server_s *sv) {
    sv->args.epoch = ++sv->launches;
    sv->kern<<<sv->nblocks, sv->threads, sizeof(QBSmem<12>), sv->st>>>(sv->args);
    CH_CHECK_LAUNCH();
}

void server_start(ch_server_s *sv, ch_s *h, const ch_server_params_t *p) {
    sv->h = h;
    sv->ring = p->ring;
    sv->pool = p->pool;
    sv->idle_ns = (unsigned long long)p->idle_ms * 1000000ull;
    const int sms = device_sm_count();
    // the handle's query configuration (layout and block size)
    const bool warp = h->q_layout == CH_QUERY_WARP_FLAT;
    const int threads = (int)h->q_threads;
    auto kern = warp ? (h->q_stall ? (h->q_delta ? k_serve<true, true, true> : k_serve<true, true>)
                                   : k_serve<true, false>)
                     : k_serve<false, false>;
    CH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(QBSmem<12>)));
    int per_sm = 0;
    CH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sizeof(QBSmem<12>)));
    sv->nblocks = p->blocks ? p->blocks : (uint32_t)sms * (uint32_t)std::max(per_sm, 1);
    uint32_t tbits = 10;
    while (tbits < 24 && ((1u << tbits) < std::min<uint32_t>(h->n, 1u << 17))) ++tbits;
    const size_t T = (size_t)1 << tbits;
    const size_t fcap = 2 * T;
    sv->ctl.alloc(1);
    sv->desc.alloc(sv->ring);
    sv->item_req.alloc(sv->pool);
    sv->targets.alloc(sv->pool);
    sv->answers.alloc(sv->pool);
    sv->done.alloc(sv->ring);
    sv->t_begin.alloc(sv->ring);
    sv->t_end.alloc(sv->ring);
    sv->slot_pos.assign(sv->ring, 0);
    sv->slot_k.assign(sv->ring, 0);
    sv->consumed.assign(sv->ring, 0);
    // per block: key, df, db, fst, touched (T each) and two frontiers (fcap each)
    const size_t per_block = 5 * T + 2 * fcap;
    sv->scratch.alloc(per_block * sv->nblocks);
    uint32_t *base = sv->scratch.ptr;
    const size_t NB = sv->nblocks;
    CH_CUDA_TRY(cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking));
    CH_CUDA_TRY(cudaMemsetAsync(base, 0xFF, 3 * T * NB * 4, sv->st));           // key, df, db
    CH_CUDA_TRY(cudaMemsetAsync(base + 3 * T * NB, 0, T * NB * 4, sv->st));      // fst
    sv->claimed.alloc(1);
    sv->claimed.zero(sv->st);
    sv->finished.alloc(sv->ring);
    sv->finished.zero(sv->st);
    sv->closing.alloc(1);
    sv->closing.zero(sv->st);
    sv->status.alloc(1);
    sv->status.zero(sv->st);
    sv->diag.alloc(DG_WORDS);
    sv->diag.zero(sv->st);
    SvArgs a{};
    a.q.n = h->n;
    a.q.n_up = (uint32_t)h->n_up;
    a.q.n_dn = (uint32_t)h->n_down;
    a.q.rank = h->rank.ptr;
    a.q.up_off = h->up_off.ptr;
    a.q.dn_off = h->dn_off.ptr;
    a.q.up_adj = h->up_adj.ptr;
    a.q.dn_adj = h->dn_adj.ptr;
    a.q.err = sv->status.ptr;
    a.q.delta = h->q_delta ? h->q_delta : INF;
    a.ctl = sv->ctl.d;
    a.desc = sv->desc.d;
    a.item_req = sv->item_req.d;
    a.targets = sv->targets.d;
    a.answers = sv->answers.d;
    a.done = sv->done.d;
    a.t_begin = sv->t_begin.d;
    a.t_end = sv->t_end.d;
    a.ring = sv->ring;
    a.pool = sv->pool;
    a.claimed = sv->claimed.ptr;
    a.finished = sv->finished.ptr;
    a.closing = sv->closing.ptr;
    a.status = sv->status.ptr;
    a.diag = sv->diag.ptr;
    a.idle_ns = sv->idle_ns;
    a.tbits = tbits;
    a.fcap = (uint32_t)fcap;
    a.key = base;
    a.df = base + T * NB;
    a.db = base + 2 * T * NB;
    a.fst = base + 3 * T * NB;
    a.touched = base + 4 * T * NB;
    a.front = base + 5 * T * NB;
    sv->args = a;
    sv->kern = kern;
    sv->threads = threads;
    server_launch(sv);
    sv->running = true;
}

// Reserve k consecutive pool positions (a ring; a request may wrap around
// the end of the pool); false if no room.
bool pool_reserve(ch_server_s *sv, uint32_t k, uint64_t &pos) {
    if (sv->pool_head + k - sv->pool_tail > sv->pool) return false;
    pos = sv->pool_head;
    sv->pool_head += k;
    return true;
}

// Copies n entries between a host array and the pool ring at position pos.
template <class F>
void pool_span(uint64_t P, uint64_t pos, uint64_t n, F &&f) {
    const uint64_t e = pos % P;
    const uint64_t n1 = std::min<uint64_t>(n, P - e);
    f(e, 0, n1);
    if (n1 < n) f(0, n1, n - n1);
}

// The loop's status word (device), read on the legacy stream, which does not
// wait for the loop's non-blocking stream.
unsigned server_status_word(ch_server_s *sv) {
    unsigned st = 0;
    CH_CUDA_TRY(cudaMemcpy(&st, sv->status.ptr, sizeof st, cudaMemcpyDeviceToHost));
    return st;
}

// The loop's status word and records, with the host's ring and pool
// counters, as one line for messages.
std::string server_state(ch_server_s *sv) {
    unsigned st = 0;
    unsigned long long dg[DG_WORDS] = {};
    if (cudaMemcpy(&st, sv->status.ptr, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(dg, sv->diag.ptr, sizeof dg, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return "device status unreadable";
    }
    const unsigned long long *e = dg + DG_ERR;
    char buf[640];
    std::snprintf(buf, sizeof buf,
                  "device status %u (1 idle exit, 2 index check, 4 unmatched entry); launches %u; "
                  "first idle exit: taken %llu published %llu epoch %llu; "
                  "failure: code %llu pos %llu published %llu taken %llu entry %llu desc seq %llu pos %llu k %llu; "
                  "host: next ticket %llu retired %llu pool head %llu tail %llu published %llu",
                  st, sv->launches, dg[DG_POS], dg[DG_PUB], dg[DG_CLAIMED], e[DG_CODE], e[DG_POS], e[DG_PUB],
                  e[DG_CLAIMED], e[DG_ITEM], e[DG_SEQ], e[DG_DPOS], e[DG_DK],
                  (unsigned long long)sv->next_seq, (unsigned long long)sv->retired,
                  (unsigned long long)sv->pool_head, (unsigned long long)sv->pool_tail,
                  (unsigned long long)sv->ctl.h->published);
    return buf;
}

// True while the loop's kernel runs.
bool server_alive(ch_server_s *sv) {
    const cudaError_t e = cudaStreamQuery(sv->st);
    if (e == cudaErrorNotReady) return true;
    if (e != cudaSuccess) throw Error{CH_ECUDA, std::string("server kernel: ") + cudaGetErrorString(e)};
    return false;
}

// Makes sure the loop runs: a launch that ended at the idle limit is
// launched again (its blocks held no position, so nothing was lost and the
// device counters carry over). A launch that ended on a failed check is an
// error, reported with the loop's state.
void server_resume(ch_server_s *sv) {
    if (server_alive(sv)) return;
    const unsigned st = server_status_word(sv);
    if (st & ~SV_IDLE) throw Error{CH_ECUDA, "server loop failed; " + server_state(sv)};
    server_launch(sv);
}

int server_submit(ch_server_s *sv, uint32_t s, const uint32_t *targets, uint32_t k, uint64_t *ticket) {
    if (!sv->running) return CH_EINVAL;
    if (k == 0) return CH_EINVAL;
    if (sv->next_seq - sv->retired >= sv->ring) {
        server_resume(sv);  // full: the loop must be serving before the caller retries
        return CH_EAGAIN;
    }
    if (k > sv->pool) return CH_EINVAL;
    uint64_t pos = 0;
    if (!pool_reserve(sv, k, pos)) {
        server_resume(sv);
        return CH_EAGAIN;
    }
    const uint64_t seq = sv->next_seq;
    const uint32_t slot = (uint32_t)(seq % sv->ring);
    pool_span(sv->pool, pos, k, [&](uint64_t e, uint64_t j, uint64_t n) {
        std::memcpy(sv->targets.h + e, targets + j, n * sizeof(uint32_t));
        std::fill(sv->item_req.h + e, sv->item_req.h + e + n, (uint32_t)(seq + 1));
    });
    sv->desc.h[slot] = SvDesc{s, k, pos, seq};
    sv->done.h[slot] = 0;
    sv->slot_pos[slot] = pos;
    sv->slot_k[slot] = k;
    sv->consumed[slot] = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *(volatile uint64_t *)&sv->ctl.h->published = pos + k;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    sv->next_seq = seq + 1;
    *ticket = seq;
    server_resume(sv);
    return CH_OK;
}

bool server_poll(ch_server_s *sv, uint64_t ticket, uint32_t *out, uint64_t *dev_ns) {
    const uint32_t slot = (uint32_t)(ticket % sv->ring);
    if (ticket < sv->retired || ticket >= sv->next_seq) throw Error{CH_EINVAL, "unknown ticket"};
    if (*(volatile uint32_t *)&sv->done.h[slot] != (uint32_t)(ticket + 1)) {
        server_resume(sv);  // not served yet: the loop must be running
        return false;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    if (out)
        pool_span(sv->pool, sv->slot_pos[slot], sv->slot_k[slot], [&](uint64_t e, uint64_t j, uint64_t n) {
            std::memcpy(out + j, sv->answers.h + e, n * sizeof(uint32_t));
        });
    if (dev_ns) *dev_ns = sv->t_end.h[slot] - sv->t_begin.h[slot];
    sv->consumed[slot] = 1;
    while (sv->retired < sv->next_seq && sv->consumed[sv->retired % sv->ring]) {
        const uint32_t rs = (uint32_t)(sv->retired % sv->ring);
        sv->pool_tail = sv->slot_pos[rs] + sv->slot_k[rs];
        sv->consumed[rs] = 0;
        ++sv->retired;
    }
    return true;
}

int server_stop(ch_server_s *sv, uint32_t *status) {
    if (!sv->running) return CH_OK;
    *(volatile uint32_t *)&sv->ctl.h->stop = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    // a launch that ended idle is launched once more, so that what was
    // published since is served; with stop set it ends once nothing is left
    if (!server_alive(sv) && server_status_word(sv) == SV_IDLE) server_launch(sv);
    // bounded wait: the kernel ends once no request is left, or at the idle limit
    const auto t0 = std::chrono::steady_clock::now();
    const double limit_s = (double)sv->idle_ns * 1e-9 + 30.0;
    while (true) {
        const cudaError_t e = cudaStreamQuery(sv->st);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) throw Error{CH_ECUDA, std::string("server kernel: ") + cudaGetErrorString(e)};
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit_s)
            return CH_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    sv->running = false;
    *status = server_status_word(sv);
    return CH_OK;
}

uint32_t server_blocks(const ch_server_s *sv) { return sv->nblocks; }

int server_running(ch_server_s *sv) {
    if (!sv->running) return 0;
    if (server_alive(sv)) return 1;
    if (server_status_word(sv) & ~SV_IDLE) throw Error{CH_ECUDA, "server loop failed; " + server_state(sv)};
    return 0;
}

ch_server_s *server_new() { return new (std::nothrow) ch_server_s(); }
void server_delete(ch_server_s *sv) { delete sv; }

void server_free(ch_server_s *sv) {
    if (sv->running) {
        uint32_t st = 0;
        server_stop(sv, &st);
    }
    // the loop's buffers go back to the library's cache: wait for the
    // kernel (it ends at its idle limit at the latest)
    if (sv->st) {
        cudaStreamSynchronize(sv->st);
        cudaStreamDestroy(sv->st);
    }
}

// Replays a request schedule against the server: request i is submitted at
// start + arrival_ns[i] (or as soon as there is room), completions are
// polled in between, and each request's latency is the time from its
// scheduled arrival to the moment its answers were seen on the host.
void server_replay(ch_server_s *sv, uint64_t nreq, const uint32_t *src, const uint32_t *k,
                   const uint64_t *toff, const uint32_t *targets, const uint64_t *arrival_ns,
                   uint32_t *answers, uint64_t *latency_ns, uint64_t *service_ns, double limit_s) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_ns = [&] {
        return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clk::now() - t0).count();
    };
    std::vector<uint64_t> ticket(nreq);
    std::vector<uint64_t> inflight;  // request indices submitted, not yet seen done
    inflight.reserve(sv->ring);
    uint64_t next = 0, finished = 0;
    while (finished < nreq) {
        // submit what is due
        while (next < nreq && arrival_ns[next] <= now_ns()) {
            const int rc = server_submit(sv, src[next], targets + toff[next], k[next], &ticket[next]);
            if (rc == CH_EAGAIN) break;
            if (rc != CH_OK) throw Error{rc, "server refused a request during the replay; " + server_state(sv)};
            inflight.push_back(next);
            ++next;
        }
        // poll completions
        size_t w = 0;
        for (size_t q = 0; q < inflight.size(); ++q) {
            const uint64_t i = inflight[q];
            uint64_t dev = 0;
            if (server_poll(sv, ticket[i], answers + toff[i], &dev)) {
                latency_ns[i] = now_ns() - arrival_ns[i];
                if (service_ns) service_ns[i] = dev;
                ++finished;
            } else {
                inflight[w++] = i;
            }
        }
        inflight.resize(w);
        if (std::chrono::duration<double>(clk::now() - t0).count() > limit_s)
            throw Error{CH_ETIMEOUT, "replay exceeded its time limit; " + server_state(sv)};
        server_resume(sv);
    }
}

}  // namespace gbch
