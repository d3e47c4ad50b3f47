// The swap-value table of one permutation, for checking and inspection.
//
// Delta(r, s) = f(p o (r s)) - f(p) for every pair r < s, by the general O(n)
// formula for a swap (any F and D; section 2.1's goal function):
//   (F_rr - F_ss)(D_{p_s p_s} - D_{p_r p_r}) + (F_rs - F_sr)(D_{p_s p_r} - D_{p_r p_s})
//   + sum_{k != r, s} (F_kr - F_ks)(D_{p_k p_s} - D_{p_k p_r})
//                   + (F_rk - F_sk)(D_{p_s p_k} - D_{p_r p_k}),
// accumulated in int64. One thread per pair; F and D are read through the cache.
// Also the histogram of costs (the probability mass function of section 4.2).
#include "kernels.h"

namespace qap {
namespace {

__global__ void k_delta_table(const int32_t* __restrict__ F, const int32_t* __restrict__ D, int n,
                              const int32_t* __restrict__ perm, int64_t* __restrict__ out) {
    const int r = blockIdx.x;
    const int s = blockIdx.y * blockDim.x + threadIdx.x;
    if (s <= r || s >= n) return;
    const int pr = perm[r], pss = perm[s];
    long long d = (long long)(F[r * n + r] - F[s * n + s]) * (D[pss * n + pss] - D[pr * n + pr]) +
                  (long long)(F[r * n + s] - F[s * n + r]) * (D[pss * n + pr] - D[pr * n + pss]);
    for (int k = 0; k < n; ++k) {
        if (k == r || k == s) continue;
        const int pk = perm[k];
        d += (long long)(F[k * n + r] - F[k * n + s]) * (D[pk * n + pss] - D[pk * n + pr]) +
             (long long)(F[r * n + k] - F[s * n + k]) * (D[pss * n + pk] - D[pr * n + pk]);
    }
    const long long idx = (long long)r * n - (long long)r * (r + 1) / 2 + (s - r - 1);  // r-major
    out[idx] = d;
}

// Costs binned by b = floor((cost - lo) bins / (hi - lo)) (exact 128-bit integer
// arithmetic); counts[0]: below lo, counts[1 + b], counts[bins + 1]: at or above hi.
__global__ void k_histogram(const int64_t* __restrict__ cost, int count, int64_t lo, int64_t hi, int bins,
                            unsigned long long* __restrict__ counts) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int64_t c = cost[i];
        int slot;
        if (c < lo) {
            slot = 0;
        } else if (c >= hi) {
            slot = bins + 1;
        } else {
            const unsigned __int128 num = (unsigned __int128)(uint64_t)(c - lo) * (uint64_t)bins;
            slot = 1 + (int)(num / (unsigned __int128)(uint64_t)(hi - lo));
        }
        atomicAdd(counts + slot, 1ull);
    }
}

}  // namespace

cudaError_t launch_histogram(const int64_t* cost, int count, int64_t lo, int64_t hi, int bins,
                             unsigned long long* counts, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int grid = (count + 255) / 256 < 1024 ? (count + 255) / 256 : 1024;
    k_histogram<<<grid, 256, 0, st>>>(cost, count, lo, hi, bins, counts);
    return cudaGetLastError();
}

cudaError_t launch_delta_table(const int32_t* F, const int32_t* D, int n, const int32_t* perm, int64_t* out,
                               cudaStream_t st) {
    if (n < 2) return cudaSuccess;
    const dim3 grid((unsigned)n, (unsigned)((n + 127) / 128));
    k_delta_table<<<grid, 128, 0, st>>>(F, D, n, perm, out);
    return cudaGetLastError();
}

}  // namespace qap
