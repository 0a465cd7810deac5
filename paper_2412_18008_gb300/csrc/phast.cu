// One-to-all distances on a built hierarchy (ch_one_to_all), the PHAST scheme
// the paper cites for single-source distances on a CH (Sec. 5).
//
// A vertex's distance from s is the least d_up(x) + (a downward path x -> v)
// over the vertices x of s's upward search. Both parts are sweeps over the
// rank order, whose levels are contiguous rank ranges (rank sorts by level
// first):
//   upward    levels ascending. A level's labels are final once every lower
//             level has pushed along its E_up edges, because an E_up edge
//             leaves a vertex for a later-contracted one (its live
//             neighbours were outside the independent set V_F). A level
//             pushes its finite labels with atomicMin. The core, whose E_up
//             holds the edges among its own vertices, repeats its pushes
//             until a pass changes nothing (Bellman-Ford, at most core-size
//             passes).
//   downward  levels descending, core excluded (its labels are exact after
//             the upward part). d(u) = min(d(u), d(x) + w) over u's E_down
//             edges (x, u); x lies in a higher level, so d(x) is final. No
//             atomics: each vertex is written by its own thread.
//
// Layout: the labels of PK = 64 sources are interleaved per vertex in rank
// order, D[r * PK + i], so the 64 threads that serve one vertex read and
// write one 256-byte row and every gather along an edge is one coalesced
// 256-byte segment. A pass costs a chain of dependent level steps whatever
// its width, so the wider pass spreads that latency over more sources.
// Levels with more than TAIL_MAX vertices get a launch
// each; the run of smaller levels at the top of the hierarchy (where levels
// hold a handful of vertices) is walked by one block with a barrier between
// levels. The result leaves D through one permuting pass, out[i * n + v] =
// D[rank[v] * PK + i].
//
// Algorithmic bytes per batch of PK sources, both sweeps: the label rows
// (4 * PK B read and written per vertex and sweep), 8 B per E_up / E_down
// entry plus a 4 * PK-B label row per entry, and the offsets; then 4 * PK B
// read and 4 * PK B written per vertex for the output.

#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace gbch {
namespace {

constexpr uint32_t PK = 64;            // sources per pass (labels interleaved per vertex)
constexpr uint32_t TAIL_MAX = 512;     // largest level the one-block tail walks
constexpr int TAIL_THREADS = 1024;
constexpr uint32_t PERR_RANGE = 1u;    // a source id >= n (same bit as the query kernels)
constexpr uint32_t PERR_BOUND = 2u;    // an index check failed; the access was skipped

__global__ void k_phast_seed(uint32_t *D, const uint32_t *src, uint32_t nsrc, const uint32_t *rank,
                             uint32_t n, uint32_t *err) {
    const uint32_t i = threadIdx.x;
    if (i >= nsrc || i >= PK) return;
    const uint32_t s = src[i];
    if (s >= n) {
        atomicOr(err, PERR_RANGE);
        return;
    }
    const uint32_t r = rank[s];
    if (r >= n) {
        atomicOr(err, PERR_BOUND);
        return;
    }
    D[(uint64_t)r * PK + i] = 0;
}

// Pushes of one (vertex, source) pair along its E_up edges. Returns whether
// a label went down (for the core's fixpoint). A stale read of the target
// only costs an extra atomicMin: labels only ever decrease.
__device__ __forceinline__ bool phast_push(uint32_t *D, uint32_t r, uint32_t i, const uint32_t *up_off,
                                           const uint2 *up_adj, uint32_t n, uint32_t *err) {
    const uint32_t d = D[(uint64_t)r * PK + i];
    if (d == INF) return false;
    bool lowered = false;
    const uint32_t e1 = up_off[r + 1];
    for (uint32_t e = up_off[r]; e < e1; ++e) {
        const uint2 a = up_adj[e];
        if (a.x >= n) {
            atomicOr(err, PERR_BOUND);
            continue;
        }
        const uint32_t nd = sat_add(d, a.y);
        uint32_t *p = D + (uint64_t)a.x * PK + i;
        if (nd < *p && atomicMin(p, nd) > nd) lowered = true;
    }
    return lowered;
}

// Pull of one (vertex, source) pair over its E_down edges.
__device__ __forceinline__ void phast_pull(uint32_t *D, uint32_t r, uint32_t i, const uint32_t *dn_off,
                                           const uint2 *dn_adj, uint32_t n, uint32_t *err) {
    uint32_t d = D[(uint64_t)r * PK + i];
    const uint32_t e1 = dn_off[r + 1];
    for (uint32_t e = dn_off[r]; e < e1; ++e) {
        const uint2 a = dn_adj[e];
        if (a.x >= n) {
            atomicOr(err, PERR_BOUND);
            continue;
        }
        d = min(d, sat_add(D[(uint64_t)a.x * PK + i], a.y));
    }
    D[(uint64_t)r * PK + i] = d;
}

// One level [r0, r1) of the upward sweep, or (changed != nullptr) one pass
// over the core.
__global__ void k_phast_up(uint32_t *D, uint32_t r0, uint32_t r1, const uint32_t *up_off,
                           const uint2 *up_adj, uint32_t n, uint32_t *changed, uint32_t *err) {
    const uint64_t total = (uint64_t)(r1 - r0) * PK;
    bool lowered = false;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x)
        lowered |= phast_push(D, r0 + (uint32_t)(t / PK), (uint32_t)(t % PK), up_off, up_adj, n, err);
    if (changed && lowered) *changed = 1u;
}

// One level [r0, r1) of the downward sweep.
__global__ void k_phast_down(uint32_t *D, uint32_t r0, uint32_t r1, const uint32_t *dn_off,
                             const uint2 *dn_adj, uint32_t n, uint32_t *err) {
    const uint64_t total = (uint64_t)(r1 - r0) * PK;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x)
        phast_pull(D, r0 + (uint32_t)(t / PK), (uint32_t)(t % PK), dn_off, dn_adj, n, err);
}

// The small levels [l0, l1) in one block: upward (ascending) or downward
// (descending), a barrier between levels. A barrier makes the block's global
// writes visible to all of its threads.
__global__ void k_phast_tail(uint32_t *D, const uint32_t *lv, uint32_t l0, uint32_t l1, int upward,
                             const uint32_t *off, const uint2 *adj, uint32_t n, uint32_t *err) {
    for (uint32_t k = 0; k < l1 - l0; ++k) {
        const uint32_t l = upward ? l0 + k : l1 - 1 - k;
        const uint32_t r0 = lv[l], r1 = lv[l + 1];
        if (r0 > r1 || r1 > n) {
            if (threadIdx.x == 0) atomicOr(err, PERR_BOUND);
            return;  // uniform: every thread reads the same bounds
        }
        const uint32_t total = (r1 - r0) * PK;
        for (uint32_t t = threadIdx.x; t < total; t += blockDim.x) {
            if (upward)
                phast_push(D, r0 + t / PK, t % PK, off, adj, n, err);
            else
                phast_pull(D, r0 + t / PK, t % PK, off, adj, n, err);
        }
        __syncthreads();
    }
}

// out[i * n + v] = D[rank[v] * PK + i] for the batch's nsrc sources.
__global__ void k_phast_out(const uint32_t *D, const uint32_t *rank, uint32_t n, uint32_t nsrc,
                            uint32_t *out, uint32_t *err) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = rank[v];
        if (r >= n) {
            atomicOr(err, PERR_BOUND);
            continue;
        }
        const uint4 *row = reinterpret_cast<const uint4 *>(D + (uint64_t)r * PK);
        for (uint32_t q = 0; q < PK / 4 && 4 * q < nsrc; ++q) {
            const uint4 x = row[q];
            const uint32_t lab[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j)
                if (4 * q + j < nsrc) out[(uint64_t)(4 * q + j) * n + v] = lab[j];
        }
    }
}

}  // namespace

void one_to_all(ch_s *h, const uint32_t *src, uint64_t k, uint32_t *dist_out, cudaStream_t st) {
    if (k == 0 || h->n == 0) return;
    const uint32_t n = h->n;
    // Level boundaries in rank order: round r's selected count, then the core.
    const size_t L = h->round_stats.size();
    std::vector<uint32_t> lv(L + 2);
    uint64_t acc = 0;
    for (size_t l = 0; l < L; ++l) {
        lv[l] = (uint32_t)std::min<uint64_t>(acc, n);
        acc += h->round_stats[l][2];  // |V_F| of round l
    }
    lv[L] = (uint32_t)std::min<uint64_t>(acc, n);
    lv[L + 1] = n;
    if (acc + h->core_size != n) throw Error{CH_EINVAL, "the hierarchy's level sizes do not add up to n"};
    // The tail: the longest run of small levels right below the core.
    size_t tail = L;
    while (tail > 0 && lv[tail] - lv[tail - 1] <= TAIL_MAX) --tail;

    if (h->phast_d.count < (size_t)n * PK) h->phast_d.alloc((size_t)n * PK);
    if (h->phast_lv.count < L + 2) h->phast_lv.alloc(L + 2);
    if (h->phast_flag.count < 1) h->phast_flag.alloc(1);
    CH_CUDA_TRY(cudaMemcpyAsync(h->phast_lv.ptr, lv.data(), (L + 2) * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, st));
    uint32_t *D = h->phast_d.ptr;
    uint32_t *err = h->qerr.ptr;
    const int sms = device_sm_count();
    auto grid = [&](uint64_t pairs) { return grid_for(pairs, 256, sms * 8); };

    for (uint64_t b = 0; b < k; b += PK) {
        const uint32_t nsrc = (uint32_t)std::min<uint64_t>(PK, k - b);
        CH_CUDA_TRY(cudaMemsetAsync(D, 0xFF, (size_t)n * PK * sizeof(uint32_t), st));
        k_phast_seed<<<1, PK, 0, st>>>(D, src + b, nsrc, h->rank.ptr, n, err);
        CH_CHECK_LAUNCH();
        // upward: big levels one launch each, the small top levels in one
        // block, then the core to its fixpoint
        for (size_t l = 0; l < tail; ++l) {
            if (lv[l + 1] == lv[l]) continue;
            k_phast_up<<<grid((uint64_t)(lv[l + 1] - lv[l]) * PK), 256, 0, st>>>(
                D, lv[l], lv[l + 1], h->up_off.ptr, h->up_adj.ptr, n, nullptr, err);
            CH_CHECK_LAUNCH();
        }
        if (tail < L) {
            k_phast_tail<<<1, TAIL_THREADS, 0, st>>>(D, h->phast_lv.ptr, (uint32_t)tail, (uint32_t)L, 1,
                                                     h->up_off.ptr, h->up_adj.ptr, n, err);
            CH_CHECK_LAUNCH();
        }
        const uint32_t core_lo = lv[L];
        if (core_lo < n) {
            // at most (core size) passes change a label; one more finds none
            for (uint64_t pass = 0; pass <= (uint64_t)(n - core_lo); ++pass) {
                uint32_t changed = 0;
                CH_CUDA_TRY(cudaMemsetAsync(h->phast_flag.ptr, 0, sizeof(uint32_t), st));
                k_phast_up<<<grid((uint64_t)(n - core_lo) * PK), 256, 0, st>>>(
                    D, core_lo, n, h->up_off.ptr, h->up_adj.ptr, n, h->phast_flag.ptr, err);
                CH_CHECK_LAUNCH();
                CH_CUDA_TRY(cudaMemcpyAsync(&changed, h->phast_flag.ptr, sizeof(uint32_t),
                                            cudaMemcpyDeviceToHost, st));
                CH_CUDA_TRY(cudaStreamSynchronize(st));
                if (!changed) break;
            }
        }
        // downward: the small top levels in one block, then the big levels
        if (tail < L) {
            k_phast_tail<<<1, TAIL_THREADS, 0, st>>>(D, h->phast_lv.ptr, (uint32_t)tail, (uint32_t)L, 0,
                                                     h->dn_off.ptr, h->dn_adj.ptr, n, err);
            CH_CHECK_LAUNCH();
        }
        for (size_t l = tail; l-- > 0;) {
            if (lv[l + 1] == lv[l]) continue;
            k_phast_down<<<grid((uint64_t)(lv[l + 1] - lv[l]) * PK), 256, 0, st>>>(
                D, lv[l], lv[l + 1], h->dn_off.ptr, h->dn_adj.ptr, n, err);
            CH_CHECK_LAUNCH();
        }
        k_phast_out<<<grid(n), 256, 0, st>>>(D, h->rank.ptr, n, nsrc, dist_out + b * (uint64_t)n, err);
        CH_CHECK_LAUNCH();
    }
}

}  // namespace gbch
