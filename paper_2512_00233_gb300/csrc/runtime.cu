// Device memory for the library: one stream-ordered memory pool per device,
// owned by the library, that keeps freed blocks cached (release threshold at
// its maximum) so that creating and destroying graphs of similar size does not
// go back to the driver.  kcore_release_cached_memory() trims the pools.
// Small pinned host buffers (copies of the sweep control block) are recycled
// through a free list instead of being allocated per graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "kc_common.cuh"

namespace kc {

namespace {

std::mutex g_pool_mu;
std::vector<cudaMemPool_t> g_pools;  // by device ordinal, null until first use

std::mutex g_pin_mu;
std::vector<void*> g_pinned_free;

cudaError_t device_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t threshold = UINT64_MAX;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), pool, st);
}

kcore_status dmalloc(void** p, size_t bytes, std::string* err, cudaStream_t st) {
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), pool, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        *err = std::string("device allocation of ") + std::to_string(bytes) + " bytes: " +
               cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? KCORE_ERR_OOM : KCORE_ERR_CUDA;
    }
    return KCORE_OK;
}

void dfree(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

cudaError_t pinned_get(void** p, size_t bytes) {
    if (bytes > kPinnedBlock) return cudaErrorInvalidValue;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pinned_free.empty()) {
            *p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return cudaSuccess;
        }
    }
    return cudaMallocHost(p, kPinnedBlock);
}

void pinned_put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pinned_free.push_back(p);
}

void release_cached() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (cudaMemPool_t pool : g_pools)
        if (pool) cudaMemPoolTrimTo(pool, 0);
}

}  // namespace kc

extern "C" void kcore_release_cached_memory(void) { kc::release_cached(); }
