// Integer throughput of the SMs, measured on the device this process runs on: the
// denominator of the integer-bound kernels' roofline. Every thread runs eight
// independent chains of 32-bit multiply-adds (mad.lo, counted as two operations:
// the multiply and the add) or of add pairs (two operations), enough warps to fill
// every SM, timed with CUDA events; the best of a few runs is reported.
#include "../../include/qap_pso.h"
#include "kernels.h"
#include "launch.cuh"

namespace qap {
namespace {

constexpr int kUnroll = 16;
constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) k_int_peak(int iters, int a, int b, int* out) {
    int x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (int)threadIdx.x * (c + 3) + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == 0)
                    asm volatile("mad.lo.s32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(a), "r"(b));
                else
                    asm volatile("add.s32 %0, %0, %1;\n\tadd.s32 %0, %0, %2;" : "+r"(x[c]) : "r"(a), "r"(b));
            }
        }
    }
    int r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r ^= x[c];
    if (r == 0x7FFFFFFF) out[blockIdx.x] = r;  // keeps the chains alive; practically never stored
}

template <int KIND>
cudaError_t time_kind(cudaStream_t st, int* sink, double* ops_per_s) {
    const int sms = sm_count();
    int per_sm = occupancy_cached<k_int_peak<KIND>>(256, 0);
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * per_sm;
    const int iters = 2048;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            k_int_peak<KIND><<<grid, 256, 0, st>>>(iters, 3, 5, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) {  // the first run warms up
            const double ops = 2.0 * (double)grid * 256 * iters * kUnroll * kChains;
            const double r = ops / (ms * 1e-3);
            if (r > best) best = r;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) *ops_per_s = best;
    return e;
}

}  // namespace
}  // namespace qap

extern "C" int qap_int32_peak(void* stream, double* mad_ops_per_s, double* add_ops_per_s) {
    if (!mad_ops_per_s || !add_ops_per_s) return QAP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(int) * 65536);
    double mad = 0.0, add = 0.0;
    if (e == cudaSuccess) e = qap::time_kind<0>(st, sink, &mad);
    if (e == cudaSuccess) e = qap::time_kind<1>(st, sink, &add);
    cudaFree(sink);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? QAP_ERR_OOM : QAP_ERR_CUDA;
    *mad_ops_per_s = mad;
    *add_ops_per_s = add;
    return QAP_OK;
}
