// Host-side launch helpers: per-kernel attributes set once per device, and
// occupancy queries cached, so that a launch costs the launch itself.
#pragma once

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda_runtime.h>

namespace qap {

// Raises kernel K's dynamic shared-memory limit to the most the device allows next
// to K's static shared memory, and prefers all of the unified L1 / shared storage as
// shared memory, once per device.
template <auto K>
cudaError_t configure_once() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, K);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// cudaOccupancyMaxActiveBlocksPerMultiprocessor for kernel K, cached by (device,
// threads per CTA, dynamic shared memory)
template <auto K>
int occupancy_cached(int threads, size_t smem) {
    static std::mutex lock;
    static std::map<std::tuple<int, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, threads, smem);
    {
        std::lock_guard<std::mutex> g(lock);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, K, threads, smem) != cudaSuccess) n = 0;
    std::lock_guard<std::mutex> g(lock);
    cache[key] = n;
    return n;
}

// registers per thread of kernel K (cached; 0 if the query fails)
template <auto K>
int kernel_regs() {
    static std::atomic<int> regs{-1};
    int v = regs.load(std::memory_order_relaxed);
    if (v >= 0) return v;
    cudaFuncAttributes fa{};
    v = cudaFuncGetAttributes(&fa, K) == cudaSuccess ? fa.numRegs : 0;
    regs.store(v, std::memory_order_relaxed);
    return v;
}

// shared memory per SM and reserved shared memory per CTA of the current device
inline void smem_limits(int* per_sm, int* reserved) {
    static std::atomic<int> cached_sm[64], cached_res[64];
    int dev = 0;
    cudaGetDevice(&dev);
    int a = cached_sm[dev & 63].load(std::memory_order_relaxed);
    int b = cached_res[dev & 63].load(std::memory_order_relaxed);
    if (a <= 0) {
        cudaDeviceGetAttribute(&a, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&b, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        cached_res[dev & 63].store(b, std::memory_order_relaxed);
        cached_sm[dev & 63].store(a, std::memory_order_relaxed);
    }
    *per_sm = a;
    *reserved = b;
}

// number of SMs of the current device (cached per device)
inline int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    int v = cached[dev & 63].load(std::memory_order_relaxed);
    if (v > 0) return v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev & 63].store(v, std::memory_order_relaxed);
    return v;
}

}  // namespace qap
