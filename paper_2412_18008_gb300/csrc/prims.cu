// Device-wide scan, compaction and radix sort used by the build.
#include "prims.cuh"

namespace gbch {

namespace {

constexpr int SCAN_BLOCKS = 608;   // 4 x 152 SMs; second pass is one block
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;

template <class T>
__device__ __forceinline__ T warp_incl_scan_t(T v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL, v, o);
        if (lane >= (uint32_t)o) v += t;
    }
    return v;
}

// Exclusive block scan of one value per thread; `total` gets the block sum.
template <class T>
__device__ T block_excl_scan(T v, T &total) {
    __shared__ T warp_tot[33];
    const uint32_t lane = lane_id(), wid = threadIdx.x >> 5;
    const uint32_t nwarps = (blockDim.x + 31) >> 5;
    T incl = warp_incl_scan_t<T>(v);
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T t = lane < nwarps ? warp_tot[lane] : T(0);
        T ti = warp_incl_scan_t<T>(t);
        if (lane < nwarps) warp_tot[lane] = ti - t;
        if (lane == 31) warp_tot[32] = ti;
    }
    __syncthreads();
    T res = incl - v + warp_tot[wid];
    total = warp_tot[32];
    __syncthreads();
    return res;
}

template <class T>
__global__ void scan_reduce_kernel(const T *in, const uint32_t *d_count, uint64_t host_count,
                                   T *block_sums) {
    uint64_t count = d_count ? *d_count : host_count;
    uint64_t chunk = (count + gridDim.x - 1) / gridDim.x;
    uint64_t beg = blockIdx.x * chunk;
    uint64_t end = beg + chunk < count ? beg + chunk : count;
    T s = 0;
    for (uint64_t i = beg + threadIdx.x; i < end; i += blockDim.x) s += in[i];
    T tot;
    block_excl_scan<T>(s, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

template <class T>
__global__ void scan_blocksums_kernel(T *block_sums, int nb, T *d_total) {
    T v = (int)threadIdx.x < nb ? block_sums[threadIdx.x] : T(0);
    T tot;
    T ex = block_excl_scan<T>(v, tot);
    if ((int)threadIdx.x < nb) block_sums[threadIdx.x] = ex;
    if (threadIdx.x == 0 && d_total) *d_total = tot;
}

template <class T>
__global__ void scan_apply_kernel(const T *in, T *out, const uint32_t *d_count,
                                  uint64_t host_count, const T *block_offsets) {
    uint64_t count = d_count ? *d_count : host_count;
    uint64_t chunk = (count + gridDim.x - 1) / gridDim.x;
    uint64_t beg = blockIdx.x * chunk;
    uint64_t end = beg + chunk < count ? beg + chunk : count;
    T carry = block_offsets[blockIdx.x];
    const uint64_t tile_items = (uint64_t)blockDim.x * SCAN_ITEMS;
    for (uint64_t tile = beg; tile < end; tile += tile_items) {
        T v[SCAN_ITEMS];
        T local = 0;
        uint64_t first = tile + (uint64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            uint64_t idx = first + k;
            v[k] = idx < end ? in[idx] : T(0);
            local += v[k];
        }
        T tile_total;
        T run = carry + block_excl_scan<T>(local, tile_total);
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            uint64_t idx = first + k;
            if (idx < end) out[idx] = run;
            run += v[k];
        }
        carry += tile_total;
    }
}

__global__ void alive_flags_kernel(const uint32_t *in, const uint32_t *d_count,
                                   const uint32_t *level, uint32_t *flags) {
    uint32_t count = *d_count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += gridDim.x * blockDim.x)
        flags[i] = level[in[i]] == INF ? 1u : 0u;
}

__global__ void alive_scatter_kernel(const uint32_t *in, const uint32_t *d_count,
                                     const uint32_t *level, const uint32_t *pos,
                                     uint32_t *out) {
    uint32_t count = *d_count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += gridDim.x * blockDim.x) {
        uint32_t v = in[i];
        if (level[v] == INF) out[pos[i]] = v;
    }
}

constexpr int RS_THREADS = 256;

__global__ void radix_hist_kernel(const uint64_t *keys, uint64_t n, int shift,
                                  uint32_t *hist) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    uint64_t beg = blockIdx.x * chunk;
    uint64_t end = beg + chunk < n ? beg + chunk : n;
    for (uint64_t i = beg + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d * gridDim.x + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(RS_THREADS)
radix_scatter_kernel(const uint64_t *keys, const uint32_t *vals, uint64_t n, int shift,
                     const uint32_t *hist_offsets, uint64_t *out_keys, uint32_t *out_vals) {
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t running[256];
    __shared__ uint32_t wc[NW][257];
    const uint32_t tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    for (int d = tid; d < 256; d += RS_THREADS)
        running[d] = hist_offsets[d * gridDim.x + blockIdx.x];
    for (int i = tid; i < NW * 257; i += RS_THREADS) (&wc[0][0])[i] = 0;
    __syncthreads();
    uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    uint64_t beg = blockIdx.x * chunk;
    uint64_t end = beg + chunk < n ? beg + chunk : n;
    for (uint64_t tile = beg; tile < end; tile += RS_THREADS) {
        uint64_t i = tile + tid;
        bool valid = i < end;
        uint64_t key = valid ? keys[i] : 0;
        uint32_t val = valid ? vals[i] : 0;
        uint32_t digit = valid ? (uint32_t)((key >> shift) & 0xFF) : 256u;
        uint32_t peers = __match_any_sync(FULL, digit);
        uint32_t rank_w = __popc(peers & ((1u << lane) - 1u));
        if (lane == (uint32_t)(__ffs(peers) - 1)) wc[wid][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = running[digit];
            for (uint32_t w = 0; w < wid; ++w) off += wc[w][digit];
            out_keys[off + rank_w] = key;
            out_vals[off + rank_w] = val;
        }
        __syncthreads();
        for (int d = tid; d < 256; d += RS_THREADS) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                s += wc[w][d];
                wc[w][d] = 0;
            }
            running[d] += s;
        }
        if (tid < NW) wc[tid][256] = 0;
        __syncthreads();
    }
}

}  // namespace

template <class T>
void exclusive_scan(const T *in, T *out, const uint32_t *d_count, uint64_t host_count,
                    T *d_total, T *scratch, cudaStream_t st) {
    static_assert(SCAN_BLOCKS <= 1024, "second pass is a single block");
    static_assert(SCAN_BLOCKS <= kScanScratch, "scratch too small");
    scan_reduce_kernel<T><<<SCAN_BLOCKS, SCAN_THREADS, 0, st>>>(in, d_count, host_count,
                                                                 scratch);
    CH_CHECK_LAUNCH();
    scan_blocksums_kernel<T><<<1, 1024, 0, st>>>(scratch, SCAN_BLOCKS, d_total);
    CH_CHECK_LAUNCH();
    scan_apply_kernel<T><<<SCAN_BLOCKS, SCAN_THREADS, 0, st>>>(in, out, d_count, host_count,
                                                                scratch);
    CH_CHECK_LAUNCH();
}

template void exclusive_scan<uint32_t>(const uint32_t *, uint32_t *, const uint32_t *, uint64_t,
                                       uint32_t *, uint32_t *, cudaStream_t);
template void exclusive_scan<uint64_t>(const uint64_t *, uint64_t *, const uint32_t *, uint64_t,
                                       uint64_t *, uint64_t *, cudaStream_t);

void compact_alive(const uint32_t *in, const uint32_t *d_in_count, uint64_t max_count,
                   const uint32_t *level, uint32_t *out, uint32_t *d_out_count,
                   uint32_t *tmp, uint32_t *scratch, cudaStream_t st) {
    int g = grid_for(max_count, 256, 4 * 152 * 4);
    alive_flags_kernel<<<g, 256, 0, st>>>(in, d_in_count, level, tmp);
    CH_CHECK_LAUNCH();
    exclusive_scan<uint32_t>(tmp, tmp, d_in_count, 0, d_out_count, scratch, st);
    alive_scatter_kernel<<<g, 256, 0, st>>>(in, d_in_count, level, tmp, out);
    CH_CHECK_LAUNCH();
}

void append_digits(std::vector<int> &digits, int lo_bit, int nbits) {
    if (nbits <= 0) return;
    int first = lo_bit / 8, last = (lo_bit + nbits - 1) / 8;
    for (int d = first; d <= last; ++d)
        if (digits.empty() || digits.back() < d) digits.push_back(d);
}

void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *tmp_keys,
                      uint32_t *tmp_vals, uint64_t n, const std::vector<int> &digits,
                      cudaStream_t st) {
    if (n <= 1 || digits.empty()) return;
    int G = (int)std::min<uint64_t>(1024, std::max<uint64_t>(1, n / (RS_THREADS * 16)));
    DevBuf<uint32_t> hist, scratch;
    hist.alloc((size_t)256 * G);
    scratch.alloc(kScanScratch);
    uint64_t *ka = keys, *kb = tmp_keys;
    uint32_t *va = vals, *vb = tmp_vals;
    for (int d : digits) {
        int shift = 8 * d;
        radix_hist_kernel<<<G, RS_THREADS, 0, st>>>(ka, n, shift, hist.ptr);
        CH_CHECK_LAUNCH();
        exclusive_scan<uint32_t>(hist.ptr, hist.ptr, nullptr, (uint64_t)256 * G, nullptr,
                                 scratch.ptr, st);
        radix_scatter_kernel<<<G, RS_THREADS, 0, st>>>(ka, va, n, shift, hist.ptr, kb, vb);
        CH_CHECK_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        CH_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        CH_CUDA_TRY(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    CH_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace gbch
