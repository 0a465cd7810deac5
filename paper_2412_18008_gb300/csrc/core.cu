// Distance table of the core (the partial hierarchy's top, Sec. 3's
// candidate-bounded contraction): for every pair of core vertices, the
// length of the shortest path between them, so that a query stops its two
// upward searches at the core and joins them through the table instead of
// searching inside the core.
//
// The core vertices are the last core_size ranks; their E_up rows hold the
// core's own edges (a core vertex keeps its overlay out-edges, all to other
// core vertices). One block per core source runs a label-correcting search
// over those rows, with the source's table row as its label array: a
// frontier of the vertices whose label dropped in the level before, each
// queued once per level (a per-block stamp array). Distances between
// surviving vertices are those of the input graph, so row i is the
// shortest-path distance from core vertex i to every core vertex.
#include <algorithm>

#include "handle.cuh"

namespace gbch {
namespace {

constexpr uint32_t CORE_ERR_BOUND = 2u;

__global__ void __launch_bounds__(256) k_core_table(const uint32_t *up_off, const uint2 *up_adj, uint32_t n,
                                                     uint32_t n_up, uint32_t core_lo, uint32_t C,
                                                     uint32_t *tab, uint32_t *front, uint32_t *mark,
                                                     uint32_t *work, uint32_t *err) {
    __shared__ uint32_t s_item, s_nf[2];
    const uint32_t tid = threadIdx.x;
    uint32_t *fa = front + (size_t)blockIdx.x * 2 * C;
    uint32_t *fb = fa + C;
    uint32_t *mk = mark + (size_t)blockIdx.x * C;
    uint32_t stamp = 0;  // per level, never reused within this block
    while (true) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t src = s_item;
        if (src >= C) break;
        uint32_t *row = tab + (size_t)src * C;
        for (uint32_t j = tid; j < C; j += blockDim.x) row[j] = INF;
        __syncthreads();
        if (tid == 0) {
            row[src] = 0;
            fa[0] = src;
            s_nf[0] = 1;
        }
        uint32_t cur = 0;
        while (true) {
            __syncthreads();
            const uint32_t nf = s_nf[cur];
            __syncthreads();  // every thread has read the count
            if (nf == 0) break;
            ++stamp;
            if (tid == 0) s_nf[cur ^ 1] = 0;
            __syncthreads();
            const uint32_t *fr = cur ? fb : fa;
            uint32_t *nx = cur ? fa : fb;
            for (uint32_t f = tid; f < nf && f < C; f += blockDim.x) {
                const uint32_t x = fr[f];
                if (x >= C) {
                    atomicOr(err, CORE_ERR_BOUND);
                    continue;
                }
                const uint32_t dx = row[x];
                const uint32_t b = up_off[core_lo + x], e = up_off[core_lo + x + 1];
                if (b > e || e > n_up) {
                    atomicOr(err, CORE_ERR_BOUND);
                    continue;
                }
                for (uint32_t j = b; j < e; ++j) {
                    const uint2 a = up_adj[j];
                    if (a.x < core_lo || a.x >= n) {
                        atomicOr(err, CORE_ERR_BOUND);
                        continue;
                    }
                    const uint32_t y = a.x - core_lo;
                    const uint32_t nd = sat_add(dx, a.y);
                    if (nd >= row[y]) continue;
                    if (atomicMin(&row[y], nd) <= nd) continue;
                    if (atomicExch(&mk[y], stamp) == stamp) continue;
                    const uint32_t p = atomicAdd(&s_nf[cur ^ 1], 1u);
                    if (p < C) nx[p] = y;
                    else atomicOr(err, CORE_ERR_BOUND);
                }
            }
            cur ^= 1;
        }
    }
}

}  // namespace

void core_table(ch_s *h, uint64_t max_bytes, cudaStream_t st) {
    const uint64_t C = h->core_size;
    h->core_tab.release();
    h->core_n = 0;
    h->core_lo = h->n;
    if (C == 0) return;
    if (C >= (1ull << 32) || C > max_bytes / 4 / C)  // C^2 * 4 > max_bytes, without overflow
        throw Error{CH_ERANGE, "core distance table of " + std::to_string(C) + "^2 entries exceeds the byte limit"};
    const uint32_t n = h->n;
    const uint32_t core_lo = (uint32_t)(n - C);
    const int grid = device_sm_count() * 2;
    DevBuf<uint32_t> tab, front, mark, ctl;
    tab.alloc(C * C);
    front.alloc((size_t)grid * 2 * C);
    mark.alloc((size_t)grid * C);
    ctl.alloc(2);  // [0] work counter, [1] error word
    mark.zero(st);
    ctl.zero(st);
    k_core_table<<<grid, 256, 0, st>>>(h->up_off.ptr, h->up_adj.ptr, n, (uint32_t)h->n_up, core_lo,
                                       (uint32_t)C, tab.ptr, front.ptr, mark.ptr, ctl.ptr, ctl.ptr + 1);
    CH_CHECK_LAUNCH();
    uint32_t err = 0;
    CH_CUDA_TRY(cudaMemcpyAsync(&err, ctl.ptr + 1, 4, cudaMemcpyDeviceToHost, st));
    CH_CUDA_TRY(cudaStreamSynchronize(st));
    if (err) throw Error{CH_ECUDA, "internal index check failed in the core table"};
    h->core_tab = std::move(tab);
    h->core_lo = core_lo;
    h->core_n = (uint32_t)C;
}

}  // namespace gbch
