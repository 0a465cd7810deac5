// Shared device helpers and host plumbing of the CUDA path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <exception>
#include <string>
#include <vector>

#include "ch.h"

namespace gbch {

constexpr uint32_t INF = 0xFFFFFFFFu;
constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int NUM_SMS_HINT = 152;

// ---------------------------------------------------------------------------
// Error reporting
// ---------------------------------------------------------------------------

struct Error {
    int code;
    std::string msg;
};

void set_last_error(const char *fmt, ...);

#define CH_CUDA_TRY(expr)                                                        \
    do {                                                                         \
        cudaError_t err__ = (expr);                                              \
        if (err__ != cudaSuccess)                                                \
            throw ::gbch::Error{CH_ECUDA, std::string(#expr " failed: ") +       \
                                              cudaGetErrorString(err__)};        \
    } while (0)

// Every kernel launch of the library is followed by this check, which also
// counts the launch (reported by ch_kernel_launches()).
void count_launch();
// Adds to the launch count (negative: removes), e.g. for graph replays.
void kernel_launch_add(int64_t d);
#define CH_CHECK_LAUNCH()                    \
    do {                                     \
        ::gbch::count_launch();              \
        CH_CUDA_TRY(cudaGetLastError());     \
    } while (0)

// ---------------------------------------------------------------------------
// Device memory owned by the library
// ---------------------------------------------------------------------------

// Failure injection for the error paths (ch_debug_fail_alloc): true when
// this allocation is the one chosen to fail. Off unless armed.
bool inject_alloc_failure();

// The library's device allocator (alloc.cu): blocks come from a per-device
// cache of freed blocks in size classes, else from cudaMalloc. *got receives
// the block's class size, which dev_release needs. A block may be released
// only once the device no longer uses it. dev_trim waits for the device and
// frees the cached blocks of the current device (returns their bytes).
void *dev_alloc(size_t bytes, size_t *got);
void dev_release(void *p, size_t cls);
size_t dev_trim();

// A device array owned by the library (memory from dev_alloc). Releasing it
// (destruction, alloc, move-assignment) hands the block back to the cache,
// so the device must be done with it by then.
template <class T>
struct DevBuf {
    T *ptr = nullptr;
    size_t count = 0;
    size_t cls = 0;  // class size of the block

    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : ptr(o.ptr), count(o.count), cls(o.cls) {
        o.ptr = nullptr;
        o.count = 0;
        o.cls = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            ptr = o.ptr;
            count = o.count;
            cls = o.cls;
            o.ptr = nullptr;
            o.count = 0;
            o.cls = 0;
        }
        return *this;
    }
    // Destroyed while an exception unwinds, the array may still be in use by
    // work the failed call had enqueued: wait for the device first.
    ~DevBuf() {
        if (ptr && std::uncaught_exceptions() > 0) cudaDeviceSynchronize();
        release();
    }

    void release() {
        if (ptr) dev_release(ptr, cls);
        ptr = nullptr;
        count = 0;
        cls = 0;
    }
    // (Re)allocates n elements. An array that held memory before may still
    // be read by work in flight on any stream: the device is waited for
    // before its block goes back to the cache.
    void alloc(size_t n) {
        if (ptr) cudaDeviceSynchronize();
        release();
        if (n == 0) n = 1;
        if (inject_alloc_failure())
            throw Error{CH_ENOMEM, "injected failure of a " + std::to_string(n * sizeof(T)) +
                                       "-byte device allocation"};
        ptr = static_cast<T *>(dev_alloc(n * sizeof(T), &cls));
        count = n;
    }
    // Grow to at least n elements keeping the first `keep` elements.
    void grow(size_t n, size_t keep, cudaStream_t st) {
        if (n <= count) return;
        DevBuf<T> nb;
        nb.alloc(n);
        if (keep && ptr)
            CH_CUDA_TRY(cudaMemcpyAsync(nb.ptr, ptr, keep * sizeof(T),
                                        cudaMemcpyDeviceToDevice, st));
        CH_CUDA_TRY(cudaStreamSynchronize(st));
        *this = std::move(nb);
    }
    void zero(cudaStream_t st) {
        if (count) CH_CUDA_TRY(cudaMemsetAsync(ptr, 0, count * sizeof(T), st));
    }
    void fill_ff(cudaStream_t st) {
        if (count) CH_CUDA_TRY(cudaMemsetAsync(ptr, 0xFF, count * sizeof(T), st));
    }
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    uint32_t s = a + b;
    return (s < a || s == INF) ? INF : s;
}

// MurmurHash3 fmix32 finaliser (Appleby), a bijection on 32-bit words.
__host__ __device__ __forceinline__ uint32_t murmur_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= (uint32_t)o) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Owner lane of flattened item `idx` given each lane's exclusive prefix
// `excl` of a per-lane count: the largest lane l with excl_l <= idx.
__device__ __forceinline__ uint32_t warp_owner(uint32_t excl, uint32_t idx) {
    uint32_t lo = 0;
#pragma unroll
    for (uint32_t step = 16; step > 0; step >>= 1) {
        uint32_t cand = lo + step;
        uint32_t ex = __shfl_sync(FULL, excl, cand & 31u);
        if (cand < 32 && ex <= idx) lo = cand;
    }
    return lo;
}

// Warp-aggregated append of one element per active predicate lane to a
// global list; returns the slot for this lane (valid only where pred).
__device__ __forceinline__ uint32_t warp_append(bool pred, uint32_t *counter) {
    uint32_t mask = __ballot_sync(FULL, pred);
    uint32_t base = 0;
    if (mask) {
        uint32_t leader = __ffs(mask) - 1;
        if (lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
        base = __shfl_sync(FULL, base, leader);
    }
    return base + __popc(mask & ((1u << lane_id()) - 1u));
}

inline int grid_for(uint64_t work, int block, int max_blocks) {
    uint64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (uint64_t)max_blocks) g = max_blocks;
    return (int)g;
}

int device_sm_count();

}  // namespace gbch
