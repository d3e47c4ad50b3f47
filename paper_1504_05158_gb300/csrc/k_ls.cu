// Goal function and best-improvement swap local search, one warp per particle.
//
// Goal function (section 2.1, Eq. 1): f(p) = sum_ij F[i][j] D[p(i)][p(j)].
// The paper names no local search; this is the swap neighbourhood N(p) =
// {p o (r s)} searched best-improvement (smallest move value, lowest (r, s) in
// r-major order on ties) until no move improves, as in Taillard's robust tabu
// search for the QAP. For symmetric F and D with zero diagonal, every move value
// comes from one matrix per particle,
//     G[k][l] = sum_j F[k][j] D[p(j)][l]            (location-indexed columns),
//     delta(r, s) = 2 (G[r][p(s)] + G[s][p(r)] - G[r][p(r)] - G[s][p(s)])
//                   + 4 F[r][s] D[p(r)][p(s)],
//     f(p) = sum_k G[k][p(k)],
// and applying swap (r, s) is a rank-1 update of G,
//     G[k][l] += (F[k][r] - F[k][s]) (D[p(s)][l] - D[p(r)][l])   (p before the swap),
// so a round costs O(1) per pair after an O(n^3) set-up per iteration.
//
// Layout: F (int32, rows padded to fs) and D (uint16) are staged once per CTA in
// shared memory; each warp owns one particle's G (n rows of n+1 int32, the odd
// stride keeps column gathers free of bank conflicts), G[k][p(k)] and p.
#include <climits>

#include "kernels.h"

namespace qap {
namespace {

constexpr int kMaxWarpsPerCta = 8;
constexpr int kSafetyMoves = 1 << 16;  // upper bound on moves of one search (never reached)
constexpr size_t kSmemLimit = 227 * 1024;

__host__ __device__ inline int round_up(int x, int a) { return (x + a - 1) / a * a; }
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t shared_part(int n) {
    return align16((size_t)n * round_up(n, 4) * 4) + align16((size_t)n * n * 2);
}
__host__ __device__ inline size_t warp_part(int n) {
    return align16((size_t)n * (n + 1) * 4) + align16((size_t)n * 4) * 2;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <int NW>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) k_ls(LsArgs a, int wpc) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n, fs = round_up(n, 4), gs = n + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t* sF = reinterpret_cast<int32_t*>(smem);
    uint16_t* sD = reinterpret_cast<uint16_t*>(smem + align16((size_t)n * fs * 4));
    unsigned char* wb = smem + shared_part(n) + (size_t)warp * warp_part(n);
    int32_t* G = reinterpret_cast<int32_t*>(wb);
    int32_t* gd = reinterpret_cast<int32_t*>(wb + align16((size_t)n * gs * 4));
    int32_t* pi = gd + align16((size_t)n * 4) / 4;

    for (int i = threadIdx.x; i < n * fs; i += blockDim.x) {
        const int r = i / fs, c = i % fs;
        sF[i] = c < n ? a.F[r * n + c] : 0;
    }
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sD[i] = (uint16_t)a.D[i];
    __syncthreads();
    if (warp >= wpc) return;

    const long long npairs = (long long)n * (n - 1) / 2;
    const int nv = n / 2;  // virtual rows: row t joined with row n-2-t

    for (int p = blockIdx.x * wpc + warp; p < a.count; p += gridDim.x * wpc) {
        for (int m = lane; m < n; m += 32) pi[m] = a.in[(size_t)p * a.ps_in + m];
        __syncwarp();
        int pm[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int m = lane + 32 * w;
            pm[w] = m < n ? pi[m] : 0;
        }
        long long cost = 0;
        int moves = 0, rounds = 0;
        if (a.max_moves < 0) {
            // goal function alone: lane sums its columns j, then the warp adds up
            long long part = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int j = lane + 32 * w;
                if (j < n) {
                    int col = 0;
                    for (int i = 0; i < n; ++i) col += sF[i * fs + j] * (int)sD[pi[i] * n + pm[w]];
                    part += col;
                }
            }
            cost = warp_sum64(part);
        } else {
            // ---- set-up: G = F * D_p (rows of D gathered by p) ----
            constexpr int KC = NW <= 2 ? 32 : 16;
            for (int kc = 0; kc < n; kc += KC) {
                int acc[KC][NW];
#pragma unroll
                for (int kk = 0; kk < KC; ++kk)
#pragma unroll
                    for (int w = 0; w < NW; ++w) acc[kk][w] = 0;
                for (int j = 0; j < n; ++j) {
                    const int pj = pi[j];
                    int dv[NW];
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const int l = lane + 32 * w;
                        dv[w] = l < n ? (int)sD[pj * n + l] : 0;
                    }
                    // F[k][j] = F[j][k] (symmetric): a contiguous, broadcast row slice
                    const int32_t* frow = sF + j * fs + kc;
#pragma unroll
                    for (int q = 0; q < KC / 4; ++q) {
                        int4 f4 = make_int4(0, 0, 0, 0);
                        if (kc + 4 * q < fs) f4 = *reinterpret_cast<const int4*>(frow + 4 * q);
#pragma unroll
                        for (int w = 0; w < NW; ++w) {
                            acc[4 * q + 0][w] += f4.x * dv[w];
                            acc[4 * q + 1][w] += f4.y * dv[w];
                            acc[4 * q + 2][w] += f4.z * dv[w];
                            acc[4 * q + 3][w] += f4.w * dv[w];
                        }
                    }
                }
#pragma unroll
                for (int kk = 0; kk < KC; ++kk) {
                    if (kc + kk < n) {
#pragma unroll
                        for (int w = 0; w < NW; ++w) {
                            const int l = lane + 32 * w;
                            if (l < n) G[(kc + kk) * gs + l] = acc[kk][w];
                        }
                    }
                }
            }
            __syncwarp();
            long long part = 0;
            for (int m = lane; m < n; m += 32) {
                gd[m] = G[m * gs + pi[m]];
                part += gd[m];
            }
            cost = warp_sum64(part);
            __syncwarp();

            // ---- rounds: evaluate every pair, apply the best improving swap ----
            for (;;) {
                if (a.max_moves > 0 && moves >= a.max_moves) break;
                if (moves >= kSafetyMoves) {  // a true descent never gets here; bounded anyway
                    if (lane == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                    break;
                }
                int best = INT_MAX;
                unsigned bkey = 0xFFFFFFFFu;
                for (int t = 0; t < nv; ++t) {
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const int e = lane + 32 * w;
                        if (e >= n) continue;
                        int k, m;
                        if (e < n - 1 - t) {
                            k = t;
                            m = t + 1 + e;
                        } else {
                            k = n - 2 - t;
                            m = e;
                            if (k == t) continue;
                        }
                        const int pk = pi[k], pmm = pi[m];
                        const int d = 2 * (G[k * gs + pmm] + G[m * gs + pk] - gd[k] - gd[m]) +
                                      4 * sF[k * fs + m] * (int)sD[pk * n + pmm];
                        const unsigned key = ((unsigned)k << 8) | (unsigned)m;
                        if (d < best || (d == best && key < bkey)) {
                            best = d;
                            bkey = key;
                        }
                    }
                }
                ++rounds;
                const int mn = __reduce_min_sync(FULL, best);
                const unsigned kmin = __reduce_min_sync(FULL, best == mn ? bkey : 0xFFFFFFFFu);
                if (mn >= 0) break;
                const int r = (int)(kmin >> 8), s = (int)(kmin & 255u);
                if (r >= n || s >= n || r >= s) {  // cannot happen; never index with it
                    if (lane == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                    break;
                }
                const int pr = pi[r], pss = pi[s];
                int bt[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int l = lane + 32 * w;
                    bt[w] = l < n ? (int)sD[pss * n + l] - (int)sD[pr * n + l] : 0;
                }
                for (int k = 0; k < n; ++k) {
                    const int ak = sF[r * fs + k] - sF[s * fs + k];
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const int l = lane + 32 * w;
                        if (l < n) G[k * gs + l] += ak * bt[w];
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    pi[r] = pss;
                    pi[s] = pr;
                }
                __syncwarp();
                for (int m = lane; m < n; m += 32) gd[m] = G[m * gs + pi[m]];
                __syncwarp();
                cost += mn;
                ++moves;
            }
        }
        // ---- outputs ----
        for (int m = lane; m < n; m += 32) a.out[(size_t)p * a.ps_out + m] = (uint8_t)pi[m];
        if (a.PL) {
            const long long old = a.costL[p];
            if (cost < old) {
                for (int m = lane; m < n; m += 32) a.PL[(size_t)p * a.ps_out + m] = (uint8_t)pi[m];
                if (lane == 0) a.costL[p] = cost;
            }
        }
        if (lane == 0) {
            a.cost[p] = cost;
            if (a.moves) a.moves[p] = moves;
            if (a.rounds) a.rounds[p] = rounds;
            if (a.counters) {
                atomicAdd(a.counters + CNT_PIT, 1ull);
                atomicAdd(a.counters + CNT_MOVES, (unsigned long long)moves);
                atomicAdd(a.counters + CNT_ROUNDS, (unsigned long long)rounds);
                if (rounds > 0) {
                    atomicAdd(a.counters + CNT_DELTA_FULL, (unsigned long long)npairs);
                    atomicAdd(a.counters + CNT_DELTA_INCR,
                              (unsigned long long)((rounds - 1) * npairs));
                }
            }
        }
        __syncwarp();
    }
}

template <int NW>
cudaError_t launch_nw(const LsArgs& a, cudaStream_t st) {
    const int n = a.n;
    int wpc = kMaxWarpsPerCta;
    while (wpc > 1 && shared_part(n) + wpc * warp_part(n) > kSmemLimit) --wpc;
    const size_t smem = shared_part(n) + wpc * warp_part(n);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_ls<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ls<NW>, wpc * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    const int need = (a.count + wpc - 1) / wpc;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_ls<NW><<<grid, wpc * 32, smem, st>>>(a, wpc);
    return cudaGetLastError();
}

}  // namespace

int ls_max_n() {
    int n = 2;
    while (n < 256 && shared_part(n + 1) + warp_part(n + 1) <= kSmemLimit) ++n;
    return n < 160 ? n : 160;
}

cudaError_t launch_ls(const LsArgs& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (a.n < 2 || a.n > ls_max_n()) return cudaErrorInvalidValue;
    switch ((a.n + 31) / 32) {
        case 1: return launch_nw<1>(a, st);
        case 2: return launch_nw<2>(a, st);
        case 3: return launch_nw<3>(a, st);
        case 4: return launch_nw<4>(a, st);
        case 5: return launch_nw<5>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qap
