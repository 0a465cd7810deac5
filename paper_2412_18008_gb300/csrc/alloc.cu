// Device memory for the library's buffers: a per-device cache of freed
// blocks in size classes, so that repeated builds and queries reuse memory
// instead of paying cudaMalloc, and cudaFree's implicit device-wide
// synchronisation, on every call.
//
// A block is handed back to the cache only when the device no longer uses
// it: every entry point waits for its own work before its temporaries are
// released (ch_build and the other synchronous calls), and ch_free waits for
// the device before a hierarchy's memory is released. A cached block is
// therefore free to reuse on any stream. When cudaMalloc fails, the cache of
// that device is emptied (cudaFree of every block) and the allocation is
// tried once more.
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gbch {

namespace {

constexpr int kMaxDevices = 64;

struct Cache {
    std::map<size_t, std::vector<void *>> free_blocks;  // size class -> blocks
    size_t bytes = 0;                                   // bytes held in free_blocks
};

std::mutex g_cache_mu;
Cache g_cache[kMaxDevices];

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return dev >= 0 && dev < kMaxDevices ? dev : -1;
}

// Frees every cached block of device `dev` (lock held by the caller).
void empty_cache(int dev) {
    Cache &c = g_cache[dev];
    for (auto &kv : c.free_blocks)
        for (void *p : kv.second) cudaFree(p);
    c.free_blocks.clear();
    c.bytes = 0;
}

}  // namespace

// Size class of a request: at least 512 bytes, rounded up to an eighth of
// its power of two (at most 12.5% over the request).
size_t alloc_class(size_t bytes) {
    if (bytes <= 512) return 512;
    int lg = 63 - __builtin_clzll((unsigned long long)bytes);
    const size_t step = (size_t)1 << (lg > 3 ? lg - 3 : 0);
    return (bytes + step - 1) / step * step;
}

void *dev_alloc(size_t bytes, size_t *got) {
    const size_t cls = alloc_class(bytes);
    const int dev = current_device();
    if (dev >= 0) {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        Cache &c = g_cache[dev];
        auto it = c.free_blocks.find(cls);
        if (it != c.free_blocks.end() && !it->second.empty()) {
            void *p = it->second.back();
            it->second.pop_back();
            c.bytes -= cls;
            *got = cls;
            return p;
        }
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, cls);
    if (e != cudaSuccess && dev >= 0) {
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lock(g_cache_mu);
            empty_cache(dev);
        }
        e = cudaMalloc(&p, cls);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{CH_ENOMEM, "cudaMalloc of " + std::to_string(cls) + " bytes failed: " +
                                   cudaGetErrorString(e)};
    }
    *got = cls;
    return p;
}

void dev_release(void *p, size_t cls) {
    if (!p) return;
    const int dev = current_device();
    if (dev < 0) {
        cudaFree(p);
        return;
    }
    std::lock_guard<std::mutex> lock(g_cache_mu);
    Cache &c = g_cache[dev];
    c.free_blocks[cls].push_back(p);
    c.bytes += cls;
}

size_t dev_trim() {
    const int dev = current_device();
    if (dev < 0) return 0;
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lock(g_cache_mu);
    const size_t b = g_cache[dev].bytes;
    empty_cache(dev);
    return b;
}

}  // namespace gbch
