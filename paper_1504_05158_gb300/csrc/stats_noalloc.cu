// Population statistics of caller-provided device costs without any device
// allocation: the sort scratch and the result slots live in one file-scope device
// array that every GPU loading this library holds until the process exits.
#include <mutex>

#include "../../include/qap_pso.h"
#include "kernels.h"

namespace {

constexpr int kSortLen = QAP_NOALLOC_MAX_COUNT;  // power of two
constexpr int kResult = 8;                        // 6 percentiles, the 128-bit sum

// The only device memory this entry point uses. In host code this name is a
// host-side stand-in: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) int64_t g_noalloc_scratch[kSortLen + kResult];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

// Resolves the array's device address once per device (the device must be current).
cudaError_t scratch_for_current_device(int64_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<int64_t*>(g_addr[dev]);
    return cudaSuccess;
}

}  // namespace

extern "C" int qap_cost_stats_noalloc(const int64_t* costs, int32_t count, void* stream,
                                      int64_t* out6, double* mean) {
    if (!costs || !out6 || !mean) return QAP_ERR_INVALID_ARG;
    if (count < 1 || count > QAP_NOALLOC_MAX_COUNT) return QAP_ERR_INVALID_ARG;
    int64_t* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return QAP_ERR_CUDA;
    int len = 1;
    while (len < count) len <<= 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t* res = scratch + kSortLen;
    // the kernel rewrites scratch[0, len) and the result slots on every call, so
    // nothing left by an earlier call is read
    e = qap::launch_stats(costs, count, scratch, len, res, st);
    int64_t host[kResult];
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return QAP_ERR_CUDA;
    for (int i = 0; i < 6; ++i) out6[i] = host[i];
    *mean = qap::mean_of_sum(host[6], host[7], count);
    return QAP_OK;
}
