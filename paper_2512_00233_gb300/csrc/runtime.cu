// Device memory for the library: one stream-ordered memory pool per device,
// owned by the library, that keeps freed blocks cached (release threshold at
// its maximum) so that creating and destroying graphs of similar size does not
// go back to the driver.  kcore_release_cached_memory() trims the pools.
// Small pinned host buffers (copies of the sweep control block) are recycled
// through a free list instead of being allocated per graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "kc_common.cuh"
#include "kcore_test.h"

namespace kc {

kcore_status cuda_status(cudaError_t e, const char* what);

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

// Test hook (kcore_test.h): fail the k-th allocation request as out of memory.
std::atomic<long long> g_fail_at{0};
std::atomic<long long> g_alloc_requests{0};

}  // namespace

bool alloc_fault() {
    const long long c = g_alloc_requests.fetch_add(1, std::memory_order_relaxed) + 1;
    const long long k = g_fail_at.load(std::memory_order_relaxed);
    return k > 0 && c == k;
}

namespace {

cudaMemPool_t pool_if_created() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    return dev < (int)g_pools.size() ? g_pools[dev] : nullptr;
}

}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
    if (alloc_fault()) return cudaErrorMemoryAllocation;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), pool, st);
}

kcore_status dmalloc(void** p, size_t bytes, std::string* err, cudaStream_t st) {
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = alloc_fault() ? cudaErrorMemoryAllocation : device_pool(&pool);
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
    if (alloc_fault()) return cudaErrorMemoryAllocation;
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

int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

void release_cached() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (cudaMemPool_t pool : g_pools)
        if (pool) cudaMemPoolTrimTo(pool, 0);
}

}  // namespace kc

extern "C" {

void kcore_release_cached_memory(void) { kc::release_cached(); }

void kcore_test_fail_alloc(int64_t k) {
    kc::g_alloc_requests.store(0);
    kc::g_fail_at.store(k > 0 ? k : 0);
}

int64_t kcore_test_alloc_count(void) { return kc::g_alloc_requests.load(); }

kcore_status kcore_test_pool_usage(int64_t* used, int64_t* reserved) {
    if (used) *used = 0;
    if (reserved) *reserved = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return kc::cuda_status(e, "kcore_test_pool_usage");
    cudaMemPool_t pool = kc::pool_if_created();
    if (!pool) return KCORE_OK;
    uint64_t u = 0, r = 0;
    e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
    if (e != cudaSuccess) return kc::cuda_status(e, "kcore_test_pool_usage");
    if (used) *used = (int64_t)u;
    if (reserved) *reserved = (int64_t)r;
    return KCORE_OK;
}

}  // extern "C"
