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
// The set-up G = F * D_p is a dense product. Two kernels form it:
//   k_ls_tc (n <= 64, entries <= 2048, n max_f max_d < 2^24): on the tensor cores
//     (tcgen05, fp16 operands, fp32 accumulation in tensor memory). Every operand
//     and partial sum is an integer below 2^24, so the fp32 result is exact. With
//     G[k][l] = sum_j' F[k][p^-1(j')] D[j'][l], the A operand is F with its columns
//     gathered by p^-1 (per particle; 2 or 4 particles stacked to M = 128 rows) and
//     the B operand is D itself (symmetric, shared by every particle).
//   k_ls (any n up to the shared-memory limit): integer multiply-adds on the SIMT
//     cores.
// Layout: F (int32, rows padded to fs) and D (uint16) are staged once per CTA in
// shared memory; each warp owns one particle's G (n rows of n+1 int32, the odd
// stride keeps column gathers free of bank conflicts), G[k][p(k)] and p.
#include <climits>
#include <cstdlib>
#include <cstring>

#include <cuda_fp16.h>

#include "kernels.h"
#include "tc.cuh"

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
__host__ __device__ inline size_t g_bytes(int n) { return align16((size_t)n * (n + 1) * 4); }
__host__ __device__ inline size_t warp_part(int n) {
    return g_bytes(n) + align16((size_t)n * 4) * 2;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Stages F (int32, rows padded to fs) and D (uint16) for the searches.
__device__ __forceinline__ void stage_fd(const LsArgs& a, int32_t* sF, uint16_t* sD, int fs) {
    const int n = a.n;
    for (int i = threadIdx.x; i < n * fs; i += blockDim.x) {
        const int r = i / fs, c = i % fs;
        sF[i] = c < n ? a.F[r * n + c] : 0;
    }
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sD[i] = (uint16_t)a.D[i];
}

// Best-improvement descent of particle p from a complete G (rounds of all pairs,
// rank-1 updates), then its outputs: position, cost, counters, local best.
template <int NW>
__device__ __forceinline__ void descend_and_store(const LsArgs& a, int p, const int32_t* sF,
                                                  const uint16_t* sD, int32_t* G, int32_t* gd,
                                                  int32_t* pi, int lane) {
    const int n = a.n, fs = round_up(n, 4), gs = n + 1;
    const long long npairs = (long long)n * (n - 1) / 2;
    const int nv = n / 2;  // virtual rows: row t joined with row n-2-t
    long long part = 0;
    for (int m = lane; m < n; m += 32) {
        gd[m] = G[m * gs + pi[m]];
        part += gd[m];
    }
    long long cost = warp_sum64(part);
    __syncwarp();
    int moves = 0, rounds = 0;
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
                atomicAdd(a.counters + CNT_DELTA_INCR, (unsigned long long)((rounds - 1) * npairs));
            }
        }
    }
    __syncwarp();
}

// Outputs of the goal function alone (no local search).
__device__ __forceinline__ void store_cost_only(const LsArgs& a, int p, long long cost, const int32_t* pi,
                                                int lane) {
    const int n = a.n;
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
        if (a.moves) a.moves[p] = 0;
        if (a.rounds) a.rounds[p] = 0;
        if (a.counters) atomicAdd(a.counters + CNT_PIT, 1ull);
    }
    __syncwarp();
}

// ------------------------------------------------------------ SIMT set-up
template <int NW>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) k_ls(LsArgs a, int wpc) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n, fs = round_up(n, 4), gs = n + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t* sF = reinterpret_cast<int32_t*>(smem);
    uint16_t* sD = reinterpret_cast<uint16_t*>(smem + align16((size_t)n * fs * 4));
    unsigned char* wb = smem + shared_part(n) + (size_t)warp * warp_part(n);
    int32_t* G = reinterpret_cast<int32_t*>(wb);
    int32_t* gd = reinterpret_cast<int32_t*>(wb + g_bytes(n));
    int32_t* pi = gd + align16((size_t)n * 4) / 4;

    stage_fd(a, sF, sD, fs);
    __syncthreads();
    if (warp >= wpc) return;

    for (int p = blockIdx.x * wpc + warp; p < a.count; p += gridDim.x * wpc) {
        for (int m = lane; m < n; m += 32) pi[m] = a.in[(size_t)p * a.ps_in + m];
        __syncwarp();
        int pm[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int m = lane + 32 * w;
            pm[w] = m < n ? pi[m] : 0;
        }
        if (a.max_moves < 0) {
            // goal function alone: lane sums its columns j, then the warp adds up
            long long part = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int j = lane + 32 * w;
                if (j < n) {
                    long long col = 0;
                    for (int i = 0; i < n; ++i) col += (long long)sF[i * fs + j] * (int)sD[pi[i] * n + pm[w]];
                    part += col;
                }
            }
            store_cost_only(a, p, warp_sum64(part), pi, lane);
            continue;
        }
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
        descend_and_store<NW>(a, p, sF, sD, G, gd, pi, lane);
    }
}

// ------------------------------------------------------ tensor-core set-up
// One CTA of 8 warps takes 8 particles at a time. R rows per particle (32 or 64)
// stack 128 / R particles into one M = 128 tile; KP = NP = n rounded up to 16.
struct TcLayout {
    int n, R, KP, NP, tiles, fhs;
    size_t oF, oD, oFh, oB, oPin, oGd, oPi, oBar, oT, oU, total;
};

__host__ __device__ inline TcLayout tc_layout(int n) {
    TcLayout L{};
    L.n = n;
    L.R = n <= 32 ? 32 : 64;
    L.KP = round_up(n, 16);
    L.NP = L.KP;
    L.tiles = 8 * L.R / 128;
    L.fhs = round_up(n, 4) + 2;  // odd word stride: column gathers free of bank conflicts
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = (o + b + 127) & ~size_t(127);
        return r;
    };
    L.oF = take((size_t)n * round_up(n, 4) * 4);
    L.oD = take((size_t)n * n * 2);
    L.oFh = take((size_t)n * L.fhs * 2);
    L.oB = take((size_t)L.NP * L.KP * 2);
    L.oPin = take(8 * 64);
    L.oGd = take(8 * align16((size_t)n * 4));
    L.oPi = take(8 * align16((size_t)n * 4));
    L.oBar = take(16);
    L.oT = take(16);
    const size_t a_bytes = (size_t)L.tiles * 128 * L.KP * 2;
    const size_t gbytes = 8 * g_bytes(n);
    L.oU = take(a_bytes > gbytes ? a_bytes : gbytes);
    L.total = o;
    return L;
}

template <int NW>
__global__ void __launch_bounds__(256) k_ls_tc(LsArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int n = a.n, fs = round_up(n, 4);
    const TcLayout L = tc_layout(n);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int32_t* sF = reinterpret_cast<int32_t*>(smem + L.oF);
    uint16_t* sD = reinterpret_cast<uint16_t*>(smem + L.oD);
    __half* sFh = reinterpret_cast<__half*>(smem + L.oFh);
    unsigned char* sB = smem + L.oB;
    uint8_t* pinv = smem + L.oPin;
    int32_t* gd = reinterpret_cast<int32_t*>(smem + L.oGd + warp * align16((size_t)n * 4));
    int32_t* pi = reinterpret_cast<int32_t*>(smem + L.oPi + warp * align16((size_t)n * 4));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.oBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.oT);
    unsigned char* U = smem + L.oU;
    int32_t* G = reinterpret_cast<int32_t*>(U + warp * g_bytes(n));

    stage_fd(a, sF, sD, fs);
    for (int i = tid; i < n * L.fhs; i += blockDim.x) {
        const int r = i / L.fhs, c = i % L.fhs;
        sFh[i] = __int2half_rn(c < n ? a.F[r * n + c] : 0);
    }
    // B = D (symmetric): row l of the N x K operand is row l of D, zero padded
    for (int i = tid; i < L.NP * L.KP; i += blockDim.x) {
        const int l = i / L.KP, j = i % L.KP;
        const int v = (l < n && j < n) ? a.D[l * n + j] : 0;
        *reinterpret_cast<__half*>(sB + tc::tile_offset(l, j, L.KP)) = __int2half_rn(v);
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(L.tiles * L.NP)) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (tid == 0) mbar_init(bar, 1);
    fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = tc::idesc_f16_f32(128, L.NP);
    const uint32_t sbo = (uint32_t)(L.KP / 8) * 128;
    uint32_t phase = 0;
    bool healthy = true;
    const int groups = (a.count + 7) / 8;

    for (int g = blockIdx.x; g < groups && healthy; g += gridDim.x) {
        const int p = g * 8 + warp;
        const bool mine = p < a.count;
        // positions and their inverses
        for (int m = lane; m < n; m += 32) {
            const int v = mine ? a.in[(size_t)p * a.ps_in + m] : m;
            pi[m] = v;
            pinv[warp * 64 + v] = (uint8_t)m;
        }
        __syncthreads();
        // A operands: tile T row r is particle q = T * (128 / R) + r / R, facility k =
        // r % R; column j' holds F[k][p_q^-1(j')]
        const int rows = L.tiles * 128;
        for (int row = tid; row < rows; row += blockDim.x) {
            const int T = row >> 7, r = row & 127;
            const int q = T * (128 / L.R) + r / L.R, k = r % L.R;
            unsigned char* At = U + (size_t)T * 128 * L.KP * 2;
            const uint8_t* inv = pinv + q * 64;
            for (int c = 0; c < L.KP; c += 8) {
                __align__(16) __half h[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = c + e;
                    h[e] = (k < n && j < n) ? sFh[k * L.fhs + inv[j]] : __int2half_rn(0);
                }
                *reinterpret_cast<uint4*>(At + tc::tile_offset(r, c, L.KP)) = *reinterpret_cast<uint4*>(h);
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t b0 = smem_u32(sB);
            for (int T = 0; T < L.tiles; ++T) {
                const uint32_t a0 = smem_u32(U + (size_t)T * 128 * L.KP * 2);
                for (int s = 0; s < L.KP / 16; ++s)
                    tc::mma_f16(tbase + (uint32_t)(T * L.NP), tc::smem_desc(a0 + s * 256, 128, sbo),
                                tc::smem_desc(b0 + s * 256, 128, sbo), idesc, s > 0);
            }
            tc::mma_commit(bar);
        }
        const bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {  // the products never completed: record and stop
            if (tid == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
            healthy = false;
            break;
        }
        tc::fence_after_sync();
        // G from tensor memory: warp w reads lane quarter w % 4 of tiles w/4, w/4 + 2, ...
        for (int T = warp >> 2; T < L.tiles; T += 2) {
            const int r = 32 * (warp & 3) + lane;
            const int q = T * (128 / L.R) + r / L.R, k = r % L.R;
            int32_t* Gq = reinterpret_cast<int32_t*>(U + (size_t)q * g_bytes(n));
            const bool valid = k < n && g * 8 + q < a.count;
            for (int c = 0; c < L.NP; c += 16) {
                uint32_t v[16];
                tc::tmem_ld16(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(T * L.NP + c), v);
                tc::tmem_wait_ld();
                // G region overlaps the A tiles, which the finished products no longer read
                if (valid) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (c + e < n) Gq[k * (n + 1) + c + e] = __float2int_rn(__uint_as_float(v[e]));
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        if (mine) {
            if (a.max_moves < 0) {
                long long part = 0;
                for (int m = lane; m < n; m += 32) part += G[m * (n + 1) + pi[m]];
                store_cost_only(a, p, warp_sum64(part), pi, lane);
            } else {
                descend_and_store<NW>(a, p, sF, sD, G, gd, pi, lane);
            }
        }
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

bool use_tensor_cores(const LsArgs& a) {
    if (!a.tc_exact || a.n > 64) return false;
    const char* env = getenv("QAP_PSO_LS_SETUP");
    return !(env && strcmp(env, "simt") == 0);
}

template <int NW>
cudaError_t launch_tc(const LsArgs& a, cudaStream_t st) {
    const TcLayout L = tc_layout(a.n);
    if (L.total > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_ls_tc<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.total);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ls_tc<NW>, 256, L.total);
    // co-resident CTAs must fit the 512 tensor-memory columns together
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(L.tiles * L.NP)) ncols <<= 1;
    const int tmem_cap = (int)(512 / ncols);
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    const int need = (a.count + 7) / 8;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_ls_tc<NW><<<grid, 256, L.total, st>>>(a);
    return cudaGetLastError();
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
    if (use_tensor_cores(a)) return a.n <= 32 ? launch_tc<1>(a, st) : launch_tc<2>(a, st);
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
