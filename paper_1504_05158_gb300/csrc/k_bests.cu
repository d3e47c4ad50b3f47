// End-of-iteration bookkeeping (one CTA per population) and population statistics.
//
// Bests (section 2.2 and 3.3): each swarm's best current particle (lowest cost,
// lowest index on ties) replaces P^G[k] only if strictly better; the global best
// ever is tracked separately because migration may make P^G worse.
// Migration (section 3.2):
//   rank (Algorithm 2): order swarms by P^G value (ties by index); for k < d the
//     k-th worst swarm's P^G becomes a randomly chosen current solution of the k-th
//     best swarm (Philox tag 4, counter (k, 0, t)), accepted even if worse; d < m/2
//     keeps donors and targets apart;
//   ring: every mig_period iterations swarm k's P^G goes to swarm k+1 (mod m), all
//     read from a snapshot.
// The device iteration counter advances here, so replayed graphs see fresh counters.
#include <climits>

#include "kernels.h"

namespace qap {
namespace {

constexpr int kThreads = 1024;
constexpr int kMaxSwarms = 4096;

__device__ __forceinline__ void warp_copy(uint8_t* dst, const uint8_t* src, int n, int lane) {
    for (int i = lane; i < n; i += 32) dst[i] = src[i];
}

// one CTA per population of the table
__global__ void __launch_bounds__(kThreads) k_bests(const StateView* __restrict__ views, int init_mode) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const StateView s = views[blockIdx.x];
    const int m = s.m, ss = s.ss, n = s.n;
    long long* sb_cost = reinterpret_cast<long long*>(smem);
    int* sb_idx = reinterpret_cast<int*>(sb_cost + m);
    int* ord = sb_idx + m;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int t = *s.t;
    // the search of this iteration has used the update kernel's buckets: empty them
    if (s.ord_cnt)
        for (int i = threadIdx.x; i < s.ord_resets; i += blockDim.x) s.ord_cnt[i] = 0;

    // each swarm's best current particle
    for (int k = warp; k < m; k += nwarps) {
        long long bc = LLONG_MAX;
        int bi = INT_MAX;
        for (int i = lane; i < ss; i += 32) {
            const long long c = s.cost[(size_t)k * ss + i];
            if (c < bc) {
                bc = c;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long oc = __shfl_xor_sync(FULL, bc, o);
            const int oi = __shfl_xor_sync(FULL, bi, o);
            if (oc < bc || (oc == bc && oi < bi)) {
                bc = oc;
                bi = oi;
            }
        }
        const int src = k * ss + bi;
        if (lane == 0) {
            sb_cost[k] = bc;
            sb_idx[k] = src;
        }
        const bool upd = init_mode || bc < s.costG[k];
        __syncwarp();
        if (upd) {
            warp_copy(s.PG + (size_t)k * s.ps, s.X + (size_t)src * s.ps, n, lane);
            if (lane == 0) s.costG[k] = bc;
        }
    }
    __syncthreads();
    // the global best ever
    if (warp == 0) {
        long long bc = LLONG_MAX;
        int bi = INT_MAX;
        for (int k = lane; k < m; k += 32) {
            if (sb_cost[k] < bc || (sb_cost[k] == bc && sb_idx[k] < bi)) {
                bc = sb_cost[k];
                bi = sb_idx[k];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long oc = __shfl_xor_sync(FULL, bc, o);
            const int oi = __shfl_xor_sync(FULL, bi, o);
            if (oc < bc || (oc == bc && oi < bi)) {
                bc = oc;
                bi = oi;
            }
        }
        const bool upd = init_mode || bc < *s.best_cost;
        __syncwarp();
        if (upd) {
            warp_copy(s.best, s.X + (size_t)bi * s.ps, n, lane);
            if (lane == 0) {
                *s.best_cost = bc;
                *s.best_iter = init_mode ? 0 : t + 1;
            }
        }
    }
    __syncthreads();
    if (!init_mode) {
        const int period = s.mig_period > 0 ? s.mig_period : 1;
        if ((t + 1) % period == 0) {
            if (s.mig_kind == 1 && s.mig_depth > 0) {
                for (int k = threadIdx.x; k < m; k += blockDim.x) {
                    const long long ck = s.costG[k];
                    int rank = 0;
                    for (int j = 0; j < m; ++j) {
                        const long long cj = s.costG[j];
                        rank += (cj < ck) || (cj == ck && j < k);
                    }
                    ord[rank] = k;
                }
                __syncthreads();
                for (int k = warp; k < s.mig_depth; k += nwarps) {
                    const int donor = ord[k], target = ord[m - 1 - k];
                    const U4 u = draw(s.seed, (uint32_t)k, 0u, (uint32_t)t, TAG_MIG, 0u);
                    const int src = donor * ss + (int)below(u.x, (uint32_t)ss);
                    warp_copy(s.PG + (size_t)target * s.ps, s.X + (size_t)src * s.ps, n, lane);
                    if (lane == 0) s.costG[target] = s.cost[src];
                }
            } else if (s.mig_kind == 2) {
                for (int i = threadIdx.x; i < m * s.ps; i += blockDim.x) s.PG2[i] = s.PG[i];
                for (int k = threadIdx.x; k < m; k += blockDim.x) s.costG2[k] = s.costG[k];
                __syncthreads();
                for (int k = warp; k < m; k += nwarps) {
                    const int dst = (k + 1) % m;
                    if (s.ring_if_better && !(s.costG2[k] < s.costG2[dst])) continue;
                    warp_copy(s.PG + (size_t)dst * s.ps, s.PG2 + (size_t)k * s.ps, n, lane);
                    if (lane == 0) s.costG[dst] = s.costG2[k];
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) *s.t = t + 1;
    }
}

// ---------------------------------------------------------------- statistics
// Nearest-rank percentiles of the current costs (section 4.2 reports 75/50/25/5 %
// ranks): P_q = sorted[ceil(q N) - 1], from an in-CTA bitonic sort of a padded copy;
// and the exact sum of the costs as a 128-bit integer (two int64 words), from which
// the host forms the mean (no floating point on the device).
__global__ void __launch_bounds__(kThreads) k_stats(const int64_t* cost, int count, int64_t* buf,
                                                     int len, int64_t* out8) {
    __shared__ long long part[kThreads / 32][2];
    __int128 sum = 0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const long long c = i < count ? cost[i] : LLONG_MAX;
        buf[i] = c;
        if (i < count) sum += c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long lo = __shfl_xor_sync(FULL, (long long)(unsigned long long)sum, o);
        const long long hi = __shfl_xor_sync(FULL, (long long)(sum >> 64), o);
        sum += (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | (unsigned long long)lo);
    }
    if ((threadIdx.x & 31) == 0) {
        part[threadIdx.x >> 5][0] = (long long)(unsigned long long)sum;
        part[threadIdx.x >> 5][1] = (long long)(sum >> 64);
    }
    __syncthreads();
    for (int k = 2; k <= len; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const int q = i ^ j;
                if (q > i) {
                    const long long x = buf[i], y = buf[q];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        buf[i] = y;
                        buf[q] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        __int128 tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            tot += (__int128)(((unsigned __int128)(unsigned long long)part[w][1] << 64) |
                              (unsigned long long)part[w][0]);
        const int pct[4] = {5, 25, 50, 75};
        out8[0] = buf[0];
        for (int q = 0; q < 4; ++q) {
            const long long rank = ((long long)pct[q] * count + 99) / 100;
            out8[1 + q] = buf[rank - 1];
        }
        out8[5] = buf[count - 1];
        out8[6] = (long long)(unsigned long long)tot;
        out8[7] = (long long)(tot >> 64);
    }
}

}  // namespace

int bests_max_swarms() { return kMaxSwarms; }

cudaError_t launch_bests(const StateView* d_views, int count, int m_max, int init_mode, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (m_max > kMaxSwarms) return cudaErrorInvalidValue;
    const size_t smem = (size_t)m_max * (8 + 4 + 4);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_bests, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_bests<<<count, kThreads, smem, st>>>(d_views, init_mode);
    return cudaGetLastError();
}

cudaError_t launch_stats(const int64_t* cost, int32_t count, int64_t* scratch, int32_t scratch_len,
                         int64_t* out8, cudaStream_t st) {
    if (count < 1 || scratch_len < count || (scratch_len & (scratch_len - 1))) return cudaErrorInvalidValue;
    k_stats<<<1, kThreads, 0, st>>>(cost, count, scratch, scratch_len, out8);
    return cudaGetLastError();
}

double mean_of_sum(int64_t sum_lo, int64_t sum_hi, int32_t count) {
    const __int128 sum = (__int128)(((unsigned __int128)(uint64_t)sum_hi << 64) | (uint64_t)sum_lo);
    const __int128 q = sum / count, r = sum % count;  // truncated: r has the sign of sum
    return (double)(int64_t)q + (double)(int64_t)r / (double)count;
}

}  // namespace qap
