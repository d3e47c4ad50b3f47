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
//   k_ls_team (symmetric, entries <= 2048, n max_f max_d < 2^24; n <= 128, or
//     n <= 160 with entries <= 255): on the tensor cores (tcgen05, fp16 operands,
//     fp32 accumulation in tensor memory). Every operand and partial sum is an
//     integer below 2^24, so the fp32 result is exact (details at the kernel).
//   k_ls (any n up to the shared-memory limit): integer multiply-adds on the SIMT
//     cores.
// Layout: F (int32, rows padded to fs) and D (uint16) are staged once per CTA in
// shared memory; each warp owns one particle's G (n rows of n+1 int32, the odd
// stride keeps column gathers free of bank conflicts), G[k][p(k)] and p.
#include <climits>

#include <cuda_fp16.h>

#include "kernels.h"
#include "launch.cuh"
#include "tc.cuh"

namespace qap {
namespace {

constexpr int kMaxWarpsPerCta = 8;
constexpr int kSafetyMoves = 1 << 16;  // upper bound on moves of one search (never reached)
constexpr size_t kSmemLimit = 227 * 1024;

__host__ __device__ inline int round_up(int x, int a) { return (x + a - 1) / a * a; }
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared memory of the SIMT searches. GT is the integer type of the table G (int32
// when every swap value fits, int64 otherwise), DT the staged type of D (uint16 or
// int32). F (int32, rows padded to fs = n rounded up to 4) and D are staged in
// shared memory when they fit beside the warps' tables, else read from global
// memory through the cache (fs = n); per warp: G (n rows of n + 1), G[k][p(k)], p.
template <typename GT, typename DT>
__host__ __device__ inline size_t simt_fd_bytes(int n) {
    return align16((size_t)n * round_up(n, 4) * 4) + align16((size_t)n * n * sizeof(DT));
}
template <typename GT>
__host__ __device__ inline size_t simt_warp_bytes(int n) {
    return align16((size_t)n * (n + 1) * sizeof(GT)) + align16((size_t)n * sizeof(GT)) + align16((size_t)n * 4);
}
// F and D go to shared memory when they fit beside `wpc` warps in `smem` bytes
template <typename GT, typename DT>
__host__ __device__ inline bool simt_staged(int n, int wpc, size_t smem) {
    return simt_fd_bytes<GT, DT>(n) + (size_t)wpc * simt_warp_bytes<GT>(n) <= smem;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// warp-wide lexicographic minimum of (value, key)
template <typename GT>
__device__ __forceinline__ void warp_min2(GT& v, unsigned& key) {
    if constexpr (sizeof(GT) == 4) {
        const int mv = __reduce_min_sync(FULL, (int)v);
        key = __reduce_min_sync(FULL, (int)v == mv ? key : 0xFFFFFFFFu);
        v = (GT)mv;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const GT ov = __shfl_xor_sync(FULL, v, o);
            const unsigned ok = __shfl_xor_sync(FULL, key, o);
            if (ov < v || (ov == v && ok < key)) {
                v = ov;
                key = ok;
            }
        }
    }
}

template <typename GT>
__device__ __forceinline__ GT gt_max() {
    return sizeof(GT) == 4 ? (GT)INT_MAX : (GT)LLONG_MAX;
}

// Best-improvement descent of particle p from a complete G (rounds of all pairs,
// rank-1 updates), then its outputs: position, cost, counters, local best. F has
// row stride fs; Dm is D (n x n) in shared or global memory.
template <int NW, typename GT, typename DT>
__device__ __forceinline__ void descend_and_store(const LsArgs& a, int p, const int32_t* F, int fs,
                                                  const DT* Dm, GT* G, GT* gd, int32_t* pi, int lane) {
    const int n = a.n, gs = n + 1;
    const long long npairs = (long long)n * (n - 1) / 2;
    const int nv = n / 2;  // virtual rows: row t joined with row n-2-t
    long long part = 0;
    for (int m = lane; m < n; m += 32) {
        gd[m] = G[m * gs + pi[m]];
        part += (long long)gd[m];
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
        GT best = gt_max<GT>();
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
                const GT d = 2 * (G[k * gs + pmm] + G[m * gs + pk] - gd[k] - gd[m]) +
                             4 * (GT)F[k * fs + m] * (GT)Dm[pk * n + pmm];
                const unsigned key = ((unsigned)k << 8) | (unsigned)m;
                if (d < best || (d == best && key < bkey)) {
                    best = d;
                    bkey = key;
                }
            }
        }
        ++rounds;
        warp_min2<GT>(best, bkey);
        if (best >= 0) break;
        const int r = (int)(bkey >> 8), s = (int)(bkey & 255u);
        if (r >= n || s >= n || r >= s) {  // cannot happen; never index with it
            if (lane == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
            break;
        }
        const int pr = pi[r], pss = pi[s];
        GT bt[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int l = lane + 32 * w;
            bt[w] = l < n ? (GT)((long long)Dm[pss * n + l] - (long long)Dm[pr * n + l]) : (GT)0;
        }
        for (int k = 0; k < n; ++k) {
            const GT ak = (GT)((long long)F[r * fs + k] - (long long)F[s * fs + k]);
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
        cost += (long long)best;
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

// Whether the update kernel's buckets hold every particle of the population exactly
// once (their counts add up to the population), so that the hand-out can follow them.
__device__ __forceinline__ bool ord_ready(const LsArgs& a) {
    if (!a.ord_cnt || !a.ord_list) return false;
    int tot = 0;
#pragma unroll
    for (int b = 0; b < kOrdBuckets; ++b) tot += a.ord_cnt[b];
    return tot == a.count;
}
// The q-th particle handed out: the buckets from the highest down (particles that S_x
// moved farthest first), else index order.
__device__ __forceinline__ int ord_pick(const LsArgs& a, bool ready, int q) {
    if (!ready || q >= a.count) return q;
    int rem = q;
    for (int b = kOrdBuckets - 1; b >= 0; --b) {
        const int c = a.ord_cnt[b];
        if (rem < c) return a.ord_list[(size_t)b * a.count + rem];
        rem -= c;
    }
    return q;
}

// the next particle of warp-per-particle kernels: from the population's counter (in
// the update kernel's order when it is ready), else a fixed stride
__device__ __forceinline__ int next_particle(const LsArgs& a, bool ready, int& p, int stride, int lane) {
    if (a.work) {
        int q = 0;
        if (lane == 0) q = ord_pick(a, ready, atomicAdd(a.work, 1));
        return __shfl_sync(FULL, q, 0);
    }
    const int cur = p;
    p += stride;
    return cur;
}

// ------------------------------------------------------------ SIMT set-up
// G = F * D_p by integer multiply-adds, one warp per particle; cpi CTAs per
// population of the table (CTA b serves population b / cpi), wpc warps per CTA,
// `smem` bytes of dynamic shared memory (sized for the largest n of the table).
// GT = int32 when every value of G and every swap value fits (n max_f max_d <
// 2^27) and D fits 16 bits (DT = uint16); else GT = int64 with DT = int32 (exact
// while (n^2 + 8 n + 4) max_f max_d < 2^62).
template <int NW, typename GT, typename DT>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) k_ls(const LsArgs* __restrict__ args, int cpi, int wpc,
                                                             int smem) {
    extern __shared__ __align__(1024) unsigned char smem_buf[];
    const LsArgs a = args[blockIdx.x / cpi];
    const int cb = blockIdx.x % cpi;
    const int n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool staged = simt_staged<GT, DT>(n, wpc, (size_t)smem);
    const int fs = staged ? round_up(n, 4) : n;
    const int32_t* F = a.F;
    const DT* Dm = nullptr;
    unsigned char* wb0 = smem_buf;
    if (staged) {
        int32_t* sF = reinterpret_cast<int32_t*>(smem_buf);
        DT* sD = reinterpret_cast<DT*>(smem_buf + align16((size_t)n * fs * 4));
        for (int i = threadIdx.x; i < n * fs; i += blockDim.x) {
            const int r = i / fs, c = i % fs;
            sF[i] = c < n ? a.F[r * n + c] : 0;
        }
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) sD[i] = (DT)a.D[i];
        F = sF;
        Dm = sD;
        wb0 += simt_fd_bytes<GT, DT>(n);
    } else {
        if constexpr (sizeof(DT) == 4) Dm = reinterpret_cast<const DT*>(a.D);
    }
    __syncthreads();
    if (warp >= wpc || !Dm) return;  // (the launcher stages 16-bit D always)
    unsigned char* wb = wb0 + (size_t)warp * simt_warp_bytes<GT>(n);
    GT* G = reinterpret_cast<GT*>(wb);
    GT* gd = reinterpret_cast<GT*>(wb + align16((size_t)n * (n + 1) * sizeof(GT)));
    int32_t* pi = reinterpret_cast<int32_t*>(wb + align16((size_t)n * (n + 1) * sizeof(GT)) +
                                             align16((size_t)n * sizeof(GT)));
    const int gs = n + 1;

    int pnext = cb * wpc + warp;
    const bool ready = ord_ready(a);
    for (;;) {
        const int pcur = next_particle(a, ready, pnext, cpi * wpc, lane);
        if (pcur >= a.count) break;
        for (int m = lane; m < n; m += 32) pi[m] = a.in[(size_t)pcur * a.ps_in + m];
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
                    for (int i = 0; i < n; ++i) col += (long long)F[i * fs + j] * (long long)Dm[pi[i] * n + pm[w]];
                    part += col;
                }
            }
            store_cost_only(a, pcur, warp_sum64(part), pi, lane);
            continue;
        }
        // ---- set-up: G = F * D_p (rows of D gathered by p) ----
        constexpr int KC = sizeof(GT) == 8 ? 8 : (NW <= 2 ? 32 : 16);
        for (int kc = 0; kc < n; kc += KC) {
            GT acc[KC][NW];
#pragma unroll
            for (int kk = 0; kk < KC; ++kk)
#pragma unroll
                for (int w = 0; w < NW; ++w) acc[kk][w] = 0;
            for (int j = 0; j < n; ++j) {
                const int pj = pi[j];
                GT dv[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int l = lane + 32 * w;
                    dv[w] = l < n ? (GT)Dm[pj * n + l] : (GT)0;
                }
                // F[k][j] = F[j][k] (symmetric): a contiguous, broadcast row slice
                const int32_t* frow = F + j * fs + kc;
                if (staged) {
#pragma unroll
                    for (int q = 0; q < KC / 4; ++q) {
                        int4 f4 = make_int4(0, 0, 0, 0);
                        if (kc + 4 * q < fs) f4 = *reinterpret_cast<const int4*>(frow + 4 * q);
#pragma unroll
                        for (int w = 0; w < NW; ++w) {
                            acc[4 * q + 0][w] += (GT)f4.x * dv[w];
                            acc[4 * q + 1][w] += (GT)f4.y * dv[w];
                            acc[4 * q + 2][w] += (GT)f4.z * dv[w];
                            acc[4 * q + 3][w] += (GT)f4.w * dv[w];
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < KC; ++q) {
                        const GT f = kc + q < n ? (GT)__ldg(frow + q) : (GT)0;
#pragma unroll
                        for (int w = 0; w < NW; ++w) acc[q][w] += f * dv[w];
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
        descend_and_store<NW, GT, DT>(a, pcur, F, fs, Dm, G, gd, pi, lane);
    }
}

// ------------------------------------------------- direct search (any instance)
// The goal function and the swap search for any F and D (not symmetric, nonzero
// diagonal, entries up to 2^31 - 1) in exact int64 arithmetic: every round takes
// each pair's value from the general O(n) formula (the terms of the double sum whose
// row or column index is r or s), so nothing but p is kept per particle. One warp per
// particle; F and D (int32) in shared memory when they fit, else read through the
// cache. Exact while (n^2 + 8 n + 4) max_f max_d < 2^62.
__device__ __forceinline__ long long delta_general(const int32_t* F, const int32_t* D, const int32_t* pi, int n,
                                                   int r, int s) {
    const int pr = pi[r], ps = pi[s];
    long long d = (long long)(F[r * n + r] - F[s * n + s]) * (long long)(D[ps * n + ps] - D[pr * n + pr]) +
                  (long long)(F[r * n + s] - F[s * n + r]) * (long long)(D[ps * n + pr] - D[pr * n + ps]);
    for (int k = 0; k < n; ++k) {
        if (k == r || k == s) continue;
        const int pk = pi[k];
        d += (long long)(F[k * n + r] - F[k * n + s]) * (long long)(D[pk * n + ps] - D[pk * n + pr]);
        d += (long long)(F[r * n + k] - F[s * n + k]) * (long long)(D[ps * n + pk] - D[pr * n + pk]);
    }
    return d;
}

__host__ __device__ inline size_t direct_fd_bytes(int n) { return 2 * align16((size_t)n * n * 4); }
__host__ __device__ inline size_t direct_warp_bytes(int n) { return align16((size_t)n * 4); }

__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) k_ls_direct(const LsArgs* __restrict__ args, int cpi,
                                                                    int wpc, int smem) {
    extern __shared__ __align__(1024) unsigned char smem_buf[];
    const LsArgs a = args[blockIdx.x / cpi];
    const int cb = blockIdx.x % cpi;
    const int n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool staged = direct_fd_bytes(n) + (size_t)wpc * direct_warp_bytes(n) <= (size_t)smem;
    const int32_t* F = a.F;
    const int32_t* D = a.D;
    unsigned char* wb0 = smem_buf;
    if (staged) {
        int32_t* sF = reinterpret_cast<int32_t*>(smem_buf);
        int32_t* sD = reinterpret_cast<int32_t*>(smem_buf + align16((size_t)n * n * 4));
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
            sF[i] = a.F[i];
            sD[i] = a.D[i];
        }
        F = sF;
        D = sD;
        wb0 += direct_fd_bytes(n);
    }
    __syncthreads();
    if (warp >= wpc) return;
    int32_t* pi = reinterpret_cast<int32_t*>(wb0 + (size_t)warp * direct_warp_bytes(n));
    const long long npairs = (long long)n * (n - 1) / 2;
    int pnext = cb * wpc + warp;
    const bool ready = ord_ready(a);
    for (;;) {
        const int p = next_particle(a, ready, pnext, cpi * wpc, lane);
        if (p >= a.count) break;
        for (int m = lane; m < n; m += 32) pi[m] = a.in[(size_t)p * a.ps_in + m];
        __syncwarp();
        long long part = 0;
        for (int i = lane; i < n; i += 32)
            for (int j = 0; j < n; ++j) part += (long long)F[i * n + j] * (long long)D[pi[i] * n + pi[j]];
        long long cost = warp_sum64(part);
        if (a.max_moves < 0) {
            store_cost_only(a, p, cost, pi, lane);
            continue;
        }
        int moves = 0, rounds = 0;
        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= kSafetyMoves) {
                if (lane == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            long long best = LLONG_MAX;
            unsigned bkey = 0xFFFFFFFFu;
            for (int r = 0; r < n - 1; ++r)
                for (int s = r + 1 + lane; s < n; s += 32) {
                    const long long d = delta_general(F, D, pi, n, r, s);
                    const unsigned key = ((unsigned)r << 8) | (unsigned)s;
                    if (d < best || (d == best && key < bkey)) {
                        best = d;
                        bkey = key;
                    }
                }
            ++rounds;
            warp_min2<long long>(best, bkey);
            if (best >= 0) break;
            const int r = (int)(bkey >> 8), s = (int)(bkey & 255u);
            if (r >= n || s >= n || r >= s) {  // cannot happen; never index with it
                if (lane == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            __syncwarp();
            if (lane == 0) {
                const int t = pi[r];
                pi[r] = pi[s];
                pi[s] = t;
            }
            __syncwarp();
            cost += best;
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
                atomicAdd(a.counters + CNT_DELTA_FULL, (unsigned long long)(rounds * npairs));
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------ tensor-core set-up
// Teams of WPP warps (1 for n <= 32, 2 for n <= 64, 8 for n <= 128) search one
// particle at a time, independently of the other teams of the CTA, taking
// particles from a per-population counter. Per particle the team keeps, instead
// of G, the matrix
//     H[k][m] = G[k][p(m)] - G[k][p(k)]      (zero diagonal)
// and the permuted distances Dp[k][m] = D[p(k)][p(m)], so that
//     delta(k, m) = 2 (H[k][m] + H[m][k]) + 4 F[k][m] Dp[k][m];
// the table stores H + F o Dp (F, Dp symmetric), so that delta(k, m) is twice the
// sum of two of its words. A swap (r, s) changes G by the rank-1 term
// fd e^T (fd[k] = F[k][r] - F[k][s], e[x] = Dp[s][x] - Dp[r][x], p before the
// swap), hence
//     H[k][m] += fd[k] (e[m] - e[k])                       k, m not in {r, s},
// rows and columns r, s exchange with their own corrections, and Dp exchanges
// rows and columns r and s.
//
// The set-up is the dense product G_p = F Dp (G_p[k][m] = G[k][p(m)]) on the
// tensor cores: A = F (shared by every particle of the CTA), B = Dp (per
// particle; symmetric, so its N x K operand is Dp itself), fp16 operands, fp32
// accumulation in tensor memory, exact because every term and partial sum is an
// integer below 2^24. A team's particle occupies the rows of the M = 128
// accumulator that sit in the tensor-memory lane quarters of its own warps; the
// A tile holds the n rows of F once, and a team whose quarters start at row
// `rowbase` points its A descriptor rowbase rows before the tile (those rows of
// the product are never read back).
template <int WPP, typename ET>
struct TeamLayout {
    int n, KP, NP, gs, dps, arows, mrows, groups, teams;
    bool smem_d;
    size_t tU, tDp, tPi, tFd, tEv, tX, tBar, team_bytes;  // offsets inside a team's block
    size_t oTeamLo, oA, oTeamHi, oF, oD, oT, total;
};

constexpr int kXchBytes = 256;  // per team: reduction slots and the next particle

__host__ __device__ inline size_t round128(size_t x) { return (x + 127) & ~size_t(127); }

template <typename ET>
__host__ __device__ constexpr int team_groups() {
    return sizeof(ET) == 1 ? 2 : 1;
}

// two integers (exact in fp16: |v| <= 2048) as a half2 word, a in the low half
__device__ __forceinline__ uint32_t pack_h2(int a, int b) {
    return (uint32_t)__half_as_ushort(__int2half_rn(a)) | ((uint32_t)__half_as_ushort(__int2half_rn(b)) << 16);
}

template <int WPP, typename ET>
__host__ __device__ inline TeamLayout<WPP, ET> team_layout(int n, bool allow_smem_d = true) {
    TeamLayout<WPP, ET> L{};
    constexpr int TEAMS = WPP == 8 ? 1 : 8;
    constexpr int ES = (int)sizeof(ET);
    L.n = n;
    L.teams = TEAMS;
    L.KP = round_up(n, 16);
    L.NP = L.KP;
    L.gs = n | 1;            // odd word stride: column accesses of H free of bank conflicts
    L.dps = L.KP + 4 / ES;   // odd word stride of the rows of Dp
    // accumulator rows: one M = 128 product with 16-bit staging (n <= 128); the 8-bit
    // variant serves 128 < n <= 160 with two (A rows 128.. in the second)
    L.groups = team_groups<ET>();
    L.mrows = 128 * L.groups;
    L.arows = WPP >= 4 ? (L.groups == 2 ? L.KP : 128) : 32 * WPP;
    // team block: union(B tile, H), Dp, then the small arrays
    const size_t b_bytes = (size_t)L.NP * L.KP * 2, h_bytes = (size_t)n * L.gs * 4;
    L.tU = 0;
    size_t o = round128(b_bytes > h_bytes ? b_bytes : h_bytes);
    L.tDp = o;
    o += round128((size_t)n * L.dps * ES);
    L.tPi = o;                       // p as bytes, KP entries (zero padded)
    L.tFd = L.tPi + align16(L.KP);   // the compacted rows of a move: int4 per row, then a count per warp
    L.tEv = L.tFd + align16((size_t)round_up(n, 32) * 16 + 32);
    L.tX = L.tEv + align16((size_t)n * 4);
    L.tBar = L.tX + kXchBytes;
    L.team_bytes = round128(L.tBar + 8);
    // CTA: low teams, A tile, high teams, F, (D), tensor-memory slot. The MMA of a
    // team reads 128 rows of A from (rowbase rows before) the tile: keep that many
    // bytes of the allocation on both sides of it.
    const size_t arow_bytes = (size_t)L.KP * 2;
    const size_t reach = (size_t)(128 - (L.arows < 128 ? L.arows : 128)) * arow_bytes;  // before A
    const size_t reach_after = (size_t)(L.mrows - L.arows) * arow_bytes;               // after A's rows
    const int lo = TEAMS / 2;
    L.oTeamLo = 0;
    size_t c = (size_t)lo * L.team_bytes;
    if (c < reach) c = round128(reach);
    L.oA = c;
    c += round128((size_t)L.arows * arow_bytes);
    L.oTeamHi = c;
    const size_t after_a = (size_t)(TEAMS - lo) * L.team_bytes;
    c += after_a > reach_after ? after_a : round128(reach_after);
    L.oF = c;
    c += round128((size_t)n * n * ES);
    L.oT = c;
    c += 128;
    L.oD = c;
    L.smem_d = allow_smem_d && c + round128((size_t)n * n * ES) <= kSmemLimit;
    if (L.smem_d) c += round128((size_t)n * n * ES);
    L.total = c;
    return L;
}

template <int WPP>
__device__ __forceinline__ void team_sync(int team) {
    if (WPP == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(32 * WPP) : "memory");
}

// true on every thread of the team iff v is true on every thread of the team
template <int WPP>
__device__ __forceinline__ bool team_all(bool v, int team) {
    if (WPP == 1) return __all_sync(FULL, v);
    uint32_t r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, %2, %3, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + team), "r"(32 * WPP)
        : "memory");
    return r != 0;
}

// team-wide lexicographic minimum of (value, key); xch ints [0, 4 WPP) used
// alternately (`parity`) so consecutive reductions need a single barrier each
template <int WPP>
__device__ __forceinline__ void team_min2(int& v, unsigned& key, int* xch, int parity, int team, int lane,
                                          int wi) {
    const int mv = __reduce_min_sync(FULL, v);
    const unsigned mk = __reduce_min_sync(FULL, v == mv ? key : 0xFFFFFFFFu);
    if (WPP == 1) {
        v = mv;
        key = mk;
        return;
    }
    int* x = xch + parity * 2 * WPP;
    if (lane == 0) {
        x[2 * wi] = mv;
        x[2 * wi + 1] = (int)mk;
    }
    team_sync<WPP>(team);
    int bv = x[0];
    unsigned bk = (unsigned)x[1];
#pragma unroll
    for (int w = 1; w < WPP; ++w) {
        const int ov = x[2 * w];
        const unsigned ok = (unsigned)x[2 * w + 1];
        if (ov < bv || (ov == bv && ok < bk)) {
            bv = ov;
            bk = ok;
        }
    }
    v = bv;
    key = bk;
}

template <int WPP>
__device__ __forceinline__ long long team_sum64(long long v, long long* xch, int team, int lane, int wi) {
    v = warp_sum64(v);
    if (WPP == 1) return v;
    if (lane == 0) xch[wi] = v;
    team_sync<WPP>(team);
    long long t = 0;
#pragma unroll
    for (int w = 0; w < WPP; ++w) t += xch[w];
    team_sync<WPP>(team);
    return t;
}

// Best-improvement descent of particle p by one team from a complete table H + F o Dp
// (called H below). The team's
// threads form `nph` phases of `slotw` threads: thread (ph, e) evaluates pair slot e
// of virtual rows ph, ph + nph, ... (row t joined with row n-2-t) and, after a move,
// updates column e of H in rows ph, ph + nph, ...
// When the instance bounds the swap values enough for 32-bit keys (key_l = kl > 0), the
// table holds every word scaled by 2^(2 kl), and the words above the diagonal also hold
// their pair's index (k << kl | m): the two words of a pair then add up to its search
// key S 2^(2 kl) + (k << kl | m), with nothing else to form per pair.
template <int WPP, typename ET>
__device__ __forceinline__ void descend_team(const LsArgs& a, int p, const ET* sF, int32_t* H, ET* Dp,
                                             uint8_t* pi8, int4* seg, int32_t* ev, int* xch, long long cost,
                                             int gs, int dps, int tt, int team) {
    constexpr int TT = 32 * WPP;
    const int n = a.n;
    const int lane = tt & 31, wi = tt >> 5;
    const int slotw = round_up(n, 32) < TT ? round_up(n, 32) : TT;
    const int nph = TT / slotw, ph = tt / slotw, e = tt % slotw;
    const bool on = ph < nph && e < n;
    const long long npairs = (long long)n * (n - 1) / 2;
    const int nv = n / 2;
    const int nseg = (n + 31) >> 5;  // warps whose threads hold rows in A
    int* segc = reinterpret_cast<int*>(seg + 32 * nseg);
    int moves = 0, rounds = 0;
    if (a.max_moves >= 0) {
        const int kl = a.key_l, sh = 2 * kl;
        const int pmask = (1 << kl) - 1;
        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= kSafetyMoves) {
                if (tt == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            // pair (k, m), k < m, of virtual row t for this thread; S = H[k][m] + H[m][k]
            // (the swap value is 2 S); k == t on the second half is row t's own pair
            auto pair_of = [&](int t, int& k, int& m) {
                const bool first = e < n - 1 - t;
                k = first ? t : n - 2 - t;
                m = first ? t + 1 + e : e;
                return first || k != t;
            };
            // the minimum of (S, k, m), lowest pair on ties: 32-bit keys S 2^(2 kl) +
            // (k << kl | m) when the instance bounds |S| (kl > 0), else 64-bit keys
            // S 2^16 + (k << 8 | m); four independent running minima per thread
            int sbest;
            unsigned bkey;
            if (kl > 0) {
                int b0 = INT_MAX, b1 = INT_MAX, b2 = INT_MAX, b3 = INT_MAX;
                if (on) {
                    // the pair's two table words add up to its key
                    auto pv = [&](int t) -> int {
                        int k, m;
                        const bool ok = pair_of(t, k, m);
                        const int v = H[k * gs + m] + H[m * gs + k];
                        return ok ? v : INT_MAX;
                    };
                    int t = ph;
                    for (; t + 3 * nph < nv; t += 4 * nph) {
                        b0 = min(b0, pv(t));
                        b1 = min(b1, pv(t + nph));
                        b2 = min(b2, pv(t + 2 * nph));
                        b3 = min(b3, pv(t + 3 * nph));
                    }
                    for (; t < nv; t += nph) b0 = min(b0, pv(t));
                }
                int kv = min(min(b0, b1), min(b2, b3));
                bkey = 0u;
                team_min2<WPP>(kv, bkey, xch, rounds & 1, team, lane, wi);
                sbest = kv == INT_MAX ? INT_MAX : (kv >> sh);
                bkey = (unsigned)((((kv >> kl) & pmask) << 8) | (kv & pmask));
            } else {
                long long b0 = LLONG_MAX, b1 = LLONG_MAX, b2 = LLONG_MAX, b3 = LLONG_MAX;
                if (on) {
                    auto pv = [&](int t) -> long long {
                        int k, m;
                        const bool ok = pair_of(t, k, m);
                        const int sv = H[k * gs + m] + H[m * gs + k];
                        const long long v = (long long)sv * 65536 + ((k << 8) | m);
                        return ok ? v : LLONG_MAX;
                    };
                    int t = ph;
                    for (; t + 3 * nph < nv; t += 4 * nph) {
                        const long long v0 = pv(t), v1 = pv(t + nph);
                        const long long v2 = pv(t + 2 * nph), v3 = pv(t + 3 * nph);
                        b0 = v0 < b0 ? v0 : b0;
                        b1 = v1 < b1 ? v1 : b1;
                        b2 = v2 < b2 ? v2 : b2;
                        b3 = v3 < b3 ? v3 : b3;
                    }
                    for (; t < nv; t += nph) {
                        const long long v0 = pv(t);
                        b0 = v0 < b0 ? v0 : b0;
                    }
                }
                b0 = b1 < b0 ? b1 : b0;
                b2 = b3 < b2 ? b3 : b2;
                const long long bv = b2 < b0 ? b2 : b0;
                sbest = bv == LLONG_MAX ? INT_MAX : (int)(bv >> 16);
                bkey = bv == LLONG_MAX ? 0xFFFFFFFFu : (unsigned)(bv & 0xFFFF);
                team_min2<WPP>(sbest, bkey, xch, rounds & 1, team, lane, wi);
            }
            ++rounds;
            if (sbest >= 0) break;
            const int best = 2 * sbest;
            const int r = (int)(bkey >> 8), s = (int)(bkey & 255u);
            if (r >= n || s >= n || r >= s) {  // cannot happen; never index with it
                if (tt == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            // A: the move's vectors and the old rows and columns r, s of H (the table
            // holds H + F o Dp)
            const int Frs = sF[r * n + s], Drs = Dp[r * dps + s];
            const int frd = Frs * Drs;
            // table words back to values (the pair index sits below bit sh); values to words
            auto val = [&](int wv) { return wv >> sh; };
            auto word = [&](int v, int k, int m) {
                return (int)((unsigned)v << sh) + (k < m && kl > 0 ? ((k << kl) | m) : 0);
            };
            const int hrs = val(H[r * gs + s]) - frd, hsr = val(H[s * gs + r]) - frd;
            int fx = 0, ex = 0, drx = 0, dsx = 0, hxr = 0, hxs = 0, hrx = 0, hsx = 0, Fxr = 0, Fxs = 0;
            const int x = tt;
            if (x < n) {
                Fxr = sF[r * n + x];  // F[x][r] (symmetric)
                Fxs = sF[s * n + x];
                fx = Fxr - Fxs;
                drx = Dp[r * dps + x];
                dsx = Dp[s * dps + x];
                ex = dsx - drx;
                hxr = val(H[x * gs + r]) - Fxr * drx;
                hxs = val(H[x * gs + s]) - Fxs * dsx;
                hrx = val(H[r * gs + x]) - Fxr * drx;
                hsx = val(H[s * gs + x]) - Fxs * dsx;
                ev[x] = ex;
            }
            {
                // the rows B changes (fd != 0, outside {r, s}), compacted per warp: the row's
                // word offset and the rank-1 term in table words (fd scaled by 2^sh, the
                // pair index bits stay)
                const bool act = x < n && x != r && x != s && fx != 0;
                const unsigned bal = __ballot_sync(FULL, act);
                const int wseg = tt >> 5;
                if (act) {
                    const int fxs = (int)((unsigned)fx << sh);
                    seg[32 * wseg + __popc(bal & ((1u << lane) - 1u))] = make_int4(x * gs, fxs, fxs * ex, 0);
                }
                if (lane == 0 && wseg < nseg) segc[wseg] = __popc(bal);
            }
            team_sync<WPP>(team);
            // B: rows and columns outside {r, s} (F o Dp does not change there), over the
            // compacted rows whose fd is not zero (the others do not change)
            if (on && e != r && e != s) {
                const int ec = ev[e];
                int32_t* col = H + e;
                for (int w = 0; w < nseg; ++w) {
                    const int c = segc[w];
                    const int4* q = seg + 32 * w;
                    int i = ph;
                    for (; i + 3 * nph < c; i += 4 * nph) {
                        const int4 q0 = q[i], q1 = q[i + nph], q2 = q[i + 2 * nph], q3 = q[i + 3 * nph];
                        int32_t* h0 = col + q0.x;
                        int32_t* h1 = col + q1.x;
                        int32_t* h2 = col + q2.x;
                        int32_t* h3 = col + q3.x;
                        const int g0 = *h0, g1 = *h1, g2 = *h2, g3 = *h3;
                        *h0 = g0 + q0.y * ec - q0.z;
                        *h1 = g1 + q1.y * ec - q1.z;
                        *h2 = g2 + q2.y * ec - q2.z;
                        *h3 = g3 + q3.y * ec - q3.z;
                    }
                    for (; i < c; i += nph) {
                        const int4 q0 = q[i];
                        col[q0.x] += q0.y * ec - q0.z;
                    }
                }
            }
            // C: rows and columns r and s (e[r] = Drs, e[s] = -Drs, fd[r] = -Frs,
            // fd[s] = Frs), each with F o Dp of the swapped Dp (Dp[x][r] <- Dp[x][s])
            if (x < n && x != r && x != s) {
                H[x * gs + r] = word(hxs - fx * (Drs + ex) + Fxr * dsx, x, r);
                H[x * gs + s] = word(hxr + fx * (Drs - ex) + Fxs * drx, x, s);
                H[r * gs + x] = word(hrx - hrs - Frs * (ex + Drs) + Fxr * dsx, r, x);
                H[s * gs + x] = word(hsx - hsr + Frs * (ex - Drs) + Fxs * drx, s, x);
                Dp[x * dps + r] = (ET)dsx;
                Dp[x * dps + s] = (ET)drx;
                Dp[r * dps + x] = (ET)dsx;
                Dp[s * dps + x] = (ET)drx;
            }
            if (tt == 0) {
                H[r * gs + s] = word(-hrs - frd, r, s);  // -hrs - 2 Frs Drs, plus F[r][s] Dp[r][s] (unchanged)
                H[s * gs + r] = word(-hsr - frd, s, r);
                const uint8_t t8 = pi8[r];
                pi8[r] = pi8[s];
                pi8[s] = t8;
            }
            team_sync<WPP>(team);
            cost += best;
            ++moves;
        }
    }
    for (int m = tt; m < n; m += TT) a.out[(size_t)p * a.ps_out + m] = pi8[m];
    if (a.PL) {
        const long long old = a.costL[p];
        if (cost < old) {
            for (int m = tt; m < n; m += TT) a.PL[(size_t)p * a.ps_out + m] = pi8[m];
            if (tt == 0) a.costL[p] = cost;
        }
    }
    if (tt == 0) {
        a.cost[p] = cost;
        if (a.moves) a.moves[p] = moves;
        if (a.rounds) a.rounds[p] = rounds;
        if (a.counters) {
            atomicAdd(a.counters + CNT_PIT, 1ull);
            if (a.max_moves >= 0) {
                atomicAdd(a.counters + CNT_MOVES, (unsigned long long)moves);
                atomicAdd(a.counters + CNT_ROUNDS, (unsigned long long)rounds);
                if (rounds > 0) {
                    atomicAdd(a.counters + CNT_DELTA_FULL, (unsigned long long)npairs);
                    atomicAdd(a.counters + CNT_DELTA_INCR, (unsigned long long)((rounds - 1) * npairs));
                }
            }
        }
    }
}

// cpi CTAs per population of the table: CTA b serves population b / cpi. smem_d:
// D is staged in shared memory (else the Dp gathers read it through the cache).
template <int WPP, typename ET>
__global__ void __launch_bounds__(WPP == 2 ? 512 : 256, WPP == 1 ? 2 : 1)
    k_ls_team(const LsArgs* __restrict__ args, int cpi, int smem_d) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int TT = 32 * WPP;
    const LsArgs a = args[blockIdx.x / cpi];
    const int cb = blockIdx.x % cpi;
    const int n = a.n;
    const TeamLayout<WPP, ET> L = team_layout<WPP, ET>(n, smem_d != 0);
    const int TEAMS = L.teams;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int team = warp / WPP, tt = tid - team * TT;
    const int lo = TEAMS / 2;
    unsigned char* tb = smem + (team < lo ? L.oTeamLo + (size_t)team * L.team_bytes
                                          : L.oTeamHi + (size_t)(team - lo) * L.team_bytes);
    unsigned char* U = tb + L.tU;
    int32_t* H = reinterpret_cast<int32_t*>(U);
    ET* Dp = reinterpret_cast<ET*>(tb + L.tDp);
    uint8_t* pi8 = tb + L.tPi;
    int4* seg = reinterpret_cast<int4*>(tb + L.tFd);
    int32_t* ev = reinterpret_cast<int32_t*>(tb + L.tEv);
    int* xch = reinterpret_cast<int*>(tb + L.tX);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tb + L.tBar);
    unsigned char* sA = smem + L.oA;
    ET* sF = reinterpret_cast<ET*>(smem + L.oF);
    const ET* sD = reinterpret_cast<const ET*>(smem + L.oD);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.oT);
    const int KP = L.KP, gs = L.gs, dps = L.dps;

    // shared by every particle: F (uint16, row-major), D when it fits, the A tile
    // (row i < n holds F[i], rows up to `arows` are zero)
    for (int i = tid; i < n * n; i += blockDim.x) sF[i] = (ET)a.F[i];
    if (L.smem_d)
        for (int i = tid; i < n * n; i += blockDim.x) const_cast<ET*>(sD)[i] = (ET)a.D[i];
    for (int i = tid; i < L.arows * (KP / 8); i += blockDim.x) {
        const int r = i / (KP / 8), c = (i % (KP / 8)) * 8;
        uint32_t h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = c + 2 * q;
            h[q] = pack_h2(r < n && j < n ? a.F[r * n + j] : 0, r < n && j + 1 < n ? a.F[r * n + j + 1] : 0);
        }
        *reinterpret_cast<uint4*>(sA + tc::tile_offset(r, c, KP)) = make_uint4(h[0], h[1], h[2], h[3]);
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(TEAMS * team_groups<ET>() * L.NP)) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (tt == 0) mbar_init(bar, 1);
    fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tcol = *tslot + (uint32_t)(team * team_groups<ET>() * L.NP);
    const uint32_t idesc = tc::idesc_f16_f32(128, L.NP);
    const int tkl = a.key_l, tsh = 2 * tkl;  // the table's word format (descend_team)
    const uint32_t sbo = (uint32_t)(KP / 8) * 128;
    const int rowbase = 32 * ((team * WPP) & 3);  // the lane quarter of the team's first warp
    const uint32_t a_base = smem_u32(sA) - (uint32_t)(rowbase / 8) * sbo;
    const int wq = warp & 3;                      // this warp's lane quarter
    const bool reader = (warp % WPP) < 4;         // warps that read the team's rows back
    uint32_t phase = 0;
    int next = cb * TEAMS + team;
    const int stride = cpi * TEAMS;
    const bool ready = ord_ready(a);

    for (;;) {
        int p;
        if (a.work) {
            if (tt == 0) xch[60] = ord_pick(a, ready, atomicAdd(a.work, 1));
            team_sync<WPP>(team);
            p = xch[60];
            team_sync<WPP>(team);
        } else {
            p = next;
            next += stride;
        }
        if (p >= a.count) break;
        for (int m = tt; m < KP; m += TT) pi8[m] = m < n ? a.in[(size_t)p * a.ps_in + m] : 0;
        team_sync<WPP>(team);
        // Dp (ET rows) and the B tile (fp16, zero padded) of this particle. Dp is
        // symmetric, so thread (part, j) gathers column j of Dp, D[p(m)][p(j)] for the
        // rows m of its chunks (a warp reads one row of D at distinct columns), and
        // writes it as row j of Dp and of the B tile
        {
            const int parts = TT / L.NP;  // threads per row (NP <= TT)
            const bool packed = a.Dpk != nullptr && !L.smem_d;
            if (tt < parts * L.NP) {
                const int j = tt % L.NP, part = tt / L.NP;
                const int pjv = j < n ? (int)pi8[j] : 0;
                for (int c = 8 * part; c < KP; c += 8 * parts) {
                    uint32_t h[4] = {0u, 0u, 0u, 0u};
                    if (j < n) {
                        const uint2 pm8 = *reinterpret_cast<const uint2*>(pi8 + c);
                        int v[8];
                        if (packed) {  // fp16 bits and value in one word: no conversions
                            uint32_t w[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const int pmq = (int)(((q < 4 ? pm8.x : pm8.y) >> (8 * (q & 3))) & 0xFFu);
                                w[q] = c + q < n ? __ldg(a.Dpk + pmq * n + pjv) : 0u;
                                v[q] = (int)(w[q] & 0xFFFFu);
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) h[q] = __byte_perm(w[2 * q], w[2 * q + 1], 0x7632);
                        } else {
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const int pmq = (int)(((q < 4 ? pm8.x : pm8.y) >> (8 * (q & 3))) & 0xFFu);
                                v[q] = 0;
                                if (c + q < n) v[q] = L.smem_d ? (int)sD[pmq * n + pjv] : __ldg(a.D + pmq * n + pjv);
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) h[q] = pack_h2(v[2 * q], v[2 * q + 1]);
                        }
                        if (c + 8 <= n) {  // whole words of Dp (rows start on 4 bytes)
                            if (sizeof(ET) == 2) {
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    *reinterpret_cast<uint32_t*>(Dp + j * dps + c + 2 * q) =
                                        (uint32_t)v[2 * q] | ((uint32_t)v[2 * q + 1] << 16);
                            } else {
#pragma unroll
                                for (int q = 0; q < 2; ++q)
                                    *reinterpret_cast<uint32_t*>(Dp + j * dps + c + 4 * q) =
                                        (uint32_t)v[4 * q] | ((uint32_t)v[4 * q + 1] << 8) |
                                        ((uint32_t)v[4 * q + 2] << 16) | ((uint32_t)v[4 * q + 3] << 24);
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                if (c + q < n) Dp[j * dps + c + q] = (ET)v[q];
                        }
                    }
                    *reinterpret_cast<uint4*>(U + tc::tile_offset(j, c, KP)) = make_uint4(h[0], h[1], h[2], h[3]);
                }
            }
        }
        fence_proxy_async();
        team_sync<WPP>(team);
        if (tt == 0) {
            tc::fence_after_sync();
            const uint32_t b0 = smem_u32(U);
#pragma unroll
            for (int g = 0; g < team_groups<ET>(); ++g)  // accumulator rows 128 g .. 128 g + 127
                for (int s = 0; s < KP / 16; ++s)
                    tc::mma_f16(tcol + (uint32_t)(g * L.NP), tc::smem_desc(a_base + g * 16 * sbo + s * 256, 128, sbo),
                                tc::smem_desc(b0 + s * 256, 128, sbo), idesc, s > 0);
            tc::mma_commit(bar);
        }
        const bool ok = team_all<WPP>(mbar_wait(bar, phase), team);
        if (!ok) {  // the product did not complete in time: record and leave
            if (tt == 0) {
                if (a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                mbar_wait(bar, phase);  // one more bounded wait before the tensor memory is freed
            }
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // G_p from tensor memory, written as H + F o Dp (it overwrites the B tile,
        // which the completed product no longer reads): reader warp w holds rows
        // k = 32 (w % WPP) + lane; their diagonal G[k][p(k)] = G_p[k][k] sits in the
        // two 16-column chunks that start at the warp's first row. F and Dp are read
        // by symmetry (row c + q, column k: distinct banks across the lanes).
        if (reader) {
#pragma unroll
            for (int g = 0; g < team_groups<ET>(); ++g) {
                const int kb = 128 * g + 32 * (warp % WPP), k = kb + lane;
                const uint32_t tb = tcol + (uint32_t)(g * L.NP) + ((uint32_t)(32 * wq) << 16);
                float dg = 0.0f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cc = kb + 16 * h;
                    if (cc >= L.NP) continue;  // warp-uniform
                    uint32_t v[16];
                    tc::tmem_ld16(tb + (uint32_t)cc, v);
                    tc::tmem_wait_ld();
                    // element k - cc of v by a select tree on its bits (constant indices)
                    const int idx = k - cc;
                    uint32_t t8[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) t8[i] = (idx & 8) ? v[i + 8] : v[i];
#pragma unroll
                    for (int i = 0; i < 4; ++i) t8[i] = (idx & 4) ? t8[i + 4] : t8[i];
#pragma unroll
                    for (int i = 0; i < 2; ++i) t8[i] = (idx & 2) ? t8[i + 2] : t8[i];
                    const uint32_t pick = (idx & 1) ? t8[1] : t8[0];
                    if (idx >= 0 && idx < 16) dg = __uint_as_float(pick);
                }
                const int d = __float2int_rn(dg);
                if (k < n) ev[k] = d;
                for (int c = 0; c < L.NP; c += 16) {
                    uint32_t v[16];
                    tc::tmem_ld16(tb + (uint32_t)c, v);
                    tc::tmem_wait_ld();
                    if (k < n) {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (c + q < n) {
                                const int hv = __float2int_rn(__uint_as_float(v[q])) - d +
                                               (int)sF[(c + q) * n + k] * (int)Dp[(c + q) * dps + k];
                                // a table word (scaled, with the pair index above the diagonal)
                                H[k * gs + c + q] = (int)((unsigned)hv << tsh) +
                                                    (k < c + q && tkl > 0 ? ((k << tkl) | (c + q)) : 0);
                            }
                    }
                }
            }
        }
        tc::fence_before_sync();
        team_sync<WPP>(team);
        long long part = 0;
        for (int m = tt; m < n; m += TT) part += ev[m];
        const long long cost = team_sum64<WPP>(part, reinterpret_cast<long long*>(xch) + 16, team, lane, tt >> 5);
        team_sync<WPP>(team);
        descend_team<WPP, ET>(a, p, sF, H, Dp, pi8, seg, ev, xch, cost, gs, dps, tt, team);
        team_sync<WPP>(team);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(*tslot, ncols);
}

// CTAs of one launch that fit an SM: shared memory (all of the unified storage as
// shared memory), threads, and the 512 tensor-memory columns
template <int WPP, typename ET>
int team_ctas_per_sm(const TeamLayout<WPP, ET>& T) {
    int smem_sm = 0, reserved = 0;
    smem_limits(&smem_sm, &reserved);
    int c = smem_sm / (int)(T.total + reserved);
    const int threads = 32 * WPP * T.teams;
    const int by_threads = 2048 / threads;
    if (c > by_threads) c = by_threads;
    const int regs = kernel_regs<k_ls_team<WPP, ET>>();
    if (regs > 0 && c > 65536 / (regs * threads)) c = 65536 / (regs * threads);
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(T.teams * T.groups * T.NP)) ncols <<= 1;
    if (c > (int)(512 / ncols)) c = (int)(512 / ncols);
    return c < 1 ? 1 : c;
}

template <int WPP, typename ET>
cudaError_t launch_team(const LsLaunch& L, cudaStream_t st) {
    // D in shared memory when it fits, unless reading it through the cache lets
    // more CTAs share an SM
    TeamLayout<WPP, ET> T = team_layout<WPP, ET>(L.n_max, true);
    if (T.smem_d) {
        const TeamLayout<WPP, ET> T2 = team_layout<WPP, ET>(L.n_max, false);
        if (team_ctas_per_sm(T2) > team_ctas_per_sm(T)) T = T2;
    }
    if (T.total > kSmemLimit) return cudaErrorInvalidValue;
    const int threads = 32 * WPP * T.teams;
    cudaError_t e = configure_once<k_ls_team<WPP, ET>>();
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int per_sm = team_ctas_per_sm(T);
    int cpi = L.cpi;
    if (cpi <= 0) {  // one wave over the table, at least one CTA per population
        cpi = (sms * per_sm + L.count - 1) / L.count;
        const int per_pop = (L.total / L.count + T.teams - 1) / T.teams;
        if (cpi > per_pop) cpi = per_pop;
        if (cpi < 1) cpi = 1;
    }
    e = cudaMemsetAsync(L.d_work, 0, sizeof(int32_t) * L.count, st);
    if (e != cudaSuccess) return e;
    k_ls_team<WPP, ET><<<L.count * cpi, threads, T.total, st>>>(L.d_args, cpi, T.smem_d ? 1 : 0);
    return cudaGetLastError();
}

// one launch of a warp-per-particle search kernel K with wpc warps and smem bytes
template <auto K>
cudaError_t launch_warp_kernel(const LsLaunch& L, int wpc, size_t smem, cudaStream_t st) {
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = configure_once<K>();
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    int per_sm = occupancy_cached<K>(wpc * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int cpi = L.cpi;
    if (cpi <= 0) {
        cpi = (sms * per_sm + L.count - 1) / L.count;
        const int per_pop = (L.total / L.count + wpc - 1) / wpc;
        if (cpi > per_pop) cpi = per_pop;
        if (cpi < 1) cpi = 1;
    }
    e = cudaMemsetAsync(L.d_work, 0, sizeof(int32_t) * L.count, st);
    if (e != cudaSuccess) return e;
    K<<<L.count * cpi, wpc * 32, smem, st>>>(L.d_args, cpi, wpc, (int)smem);
    return cudaGetLastError();
}

// largest n whose SIMT search fits one warp in shared memory (with F and D staged
// when D has 16 bits: that variant always stages them)
template <typename GT, typename DT>
int simt_max_n() {
    int n = 2;
    while (n < 256) {
        const int m = n + 1;
        const size_t need = simt_warp_bytes<GT>(m) + (sizeof(DT) == 2 ? simt_fd_bytes<GT, DT>(m) : 0);
        if (need > kSmemLimit) break;
        n = m;
    }
    return n;
}

template <int NW, typename GT, typename DT>
cudaError_t launch_simt(const LsLaunch& L, cudaStream_t st) {
    const int n = L.n_max;
    const size_t fd = simt_fd_bytes<GT, DT>(n), pw = simt_warp_bytes<GT>(n);
    int w_staged = kMaxWarpsPerCta;
    while (w_staged > 0 && fd + w_staged * pw > kSmemLimit) --w_staged;
    int w_global = kMaxWarpsPerCta;
    while (w_global > 0 && w_global * pw > kSmemLimit) --w_global;
    // 16-bit D is always staged; 32-bit F and D are staged unless that halves the warps
    const bool staged = sizeof(DT) == 2 ? true : (w_staged >= 1 && 2 * w_staged >= w_global);
    const int wpc = staged ? w_staged : w_global;
    if (wpc < 1) return cudaErrorInvalidValue;
    return launch_warp_kernel<k_ls<NW, GT, DT>>(L, wpc, (staged ? fd : 0) + wpc * pw, st);
}

cudaError_t launch_direct(const LsLaunch& L, cudaStream_t st) {
    const int n = L.n_max;
    const int wpc = kMaxWarpsPerCta;
    const size_t fd = direct_fd_bytes(n), pw = direct_warp_bytes(n);
    const bool staged = fd + wpc * pw <= kSmemLimit;
    return launch_warp_kernel<k_ls_direct>(L, wpc, (staged ? fd : 0) + wpc * pw, st);
}

template <typename GT, typename DT>
cudaError_t launch_simt_t(const LsLaunch& L, cudaStream_t st) {
    switch ((L.n_max + 31) / 32) {
        case 1: return launch_simt<1, GT, DT>(L, st);
        case 2: return launch_simt<2, GT, DT>(L, st);
        case 3: return launch_simt<3, GT, DT>(L, st);
        case 4: return launch_simt<4, GT, DT>(L, st);
        case 5: return launch_simt<5, GT, DT>(L, st);
        case 6: return launch_simt<6, GT, DT>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------ general instances (any F, D)
// The same search for F and D that need not be symmetric nor have a zero diagonal
// (entries <= 2048, 2 n max_f max_d < 2^24; n <= 128). With Dp[k][m] = D[p(k)][p(m)],
// R = F Dp^T and C = F^T Dp (R[a][m] = sum_j F[a][j] D[p(m)][p(j)], C[a][m] = sum_i
// F[i][a] D[p(i)][p(m)]), the team keeps H[a][m] = (R + C)[a][m] - (R + C)[a][a];
// then f(p) = trace(R + C) / 2 and
//     delta(r, s) = H[r][s] + H[s][r] + K(r, s),
// K collecting the terms of the general swap formula whose indices are only r and s.
// A swap changes R and C by rank-1 terms (fR[k] = F[k][r] - F[k][s] against
// eR[x] = Dp[x][s] - Dp[x][r]; fC[k] = F[r][k] - F[s][k] against eC[x] = Dp[s][x] -
// Dp[r][x]); rows and columns r, s exchange with their own corrections, and Dp
// exchanges rows and columns r and s. The set-up accumulates F Dp^T and F^T Dp in one
// tensor-memory accumulator (two chains of tcgen05.mma, A = F and F^T shared by the
// CTA, B = Dp and Dp^T per particle). One 8-warp team per CTA.
struct GenLayout {
    int n, KP, NP, gs, dps;
    bool smem_d;
    size_t oA1, oA2, oF, oD, oU, oDp, oPi, oRow, oCol, oEv, oX, oBar, oT, total;
};

__host__ __device__ inline GenLayout gen_layout(int n, bool allow_smem_d = true) {
    GenLayout L{};
    L.n = n;
    L.KP = round_up(n, 16);
    L.NP = L.KP;
    L.gs = n | 1;
    L.dps = L.KP + 2;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = round128(o + b);
        return r;
    };
    const size_t a_bytes = (size_t)128 * L.KP * 2, b_bytes = (size_t)L.NP * L.KP * 2;
    const size_t h_bytes = (size_t)n * L.gs * 4;
    L.oA1 = take(a_bytes);
    L.oA2 = take(a_bytes);
    L.oF = take((size_t)n * n * 2);
    L.oU = take(2 * b_bytes > h_bytes ? 2 * b_bytes : h_bytes);  // B tiles, then H
    L.oDp = take((size_t)n * L.dps * 2);
    L.oPi = take(L.KP);
    L.oRow = take((size_t)n * 16);
    L.oCol = take((size_t)n * 8);
    L.oEv = take((size_t)n * 4);
    L.oX = take(kXchBytes);
    L.oBar = take(8);
    L.oT = take(16);
    L.oD = o;
    L.smem_d = allow_smem_d && o + round128((size_t)n * n * 2) <= kSmemLimit;
    if (L.smem_d) o = round128(o + (size_t)n * n * 2);
    L.total = o;
    return L;
}

__device__ __forceinline__ void descend_gen(const LsArgs& a, int p, const uint16_t* sF, int32_t* H, uint16_t* Dp,
                                            uint8_t* pi8, int4* rowv, int2* colv, int* xch, long long cost,
                                            int gs, int dps, int tt) {
    constexpr int TT = 256;
    const int n = a.n;
    const int lane = tt & 31, wi = tt >> 5;
    const int slotw = round_up(n, 32) < TT ? round_up(n, 32) : TT;
    const int nph = TT / slotw, ph = tt / slotw, e = tt % slotw;
    const bool on = ph < nph && e < n;
    const long long npairs = (long long)n * (n - 1) / 2;
    const int nv = n / 2;
    auto Fv = [&](int i, int j) { return (int)sF[i * n + j]; };
    auto Dv = [&](int i, int j) { return (int)Dp[i * dps + j]; };
    int moves = 0, rounds = 0;
    if (a.max_moves >= 0) {
        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= kSafetyMoves) {
                if (tt == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            long long b0 = LLONG_MAX, b1 = LLONG_MAX;
            if (on) {
                auto pair_value = [&](int t) -> long long {
                    const bool c1 = e < n - 1 - t;
                    const int k = c1 ? t : n - 2 - t;
                    const int m = c1 ? t + 1 + e : e;
                    const int Fkk = Fv(k, k), Fmm = Fv(m, m), Fkm = Fv(k, m), Fmk = Fv(m, k);
                    const int Dkk = Dv(k, k), Dmm = Dv(m, m), Dkm = Dv(k, m), Dmk = Dv(m, k);
                    // the terms of the general formula with indices in {k, m} only
                    const int corner = (Fkk - Fmm) * (Dmm - Dkk) + (Fkm - Fmk) * (Dmk - Dkm);
                    const int sub = (Fkk - Fmk) * (Dmk - Dkk) + (Fkm - Fmm) * (Dmm - Dkm) +
                                    (Fkk - Fkm) * (Dkm - Dkk) + (Fmk - Fmm) * (Dmm - Dmk);
                    const int d = H[k * gs + m] + H[m * gs + k] + corner - sub;
                    const long long v = (long long)d * 65536 + ((k << 8) | m);
                    return (c1 || k != t) ? v : LLONG_MAX;
                };
                int t = ph;
                for (; t + nph < nv; t += 2 * nph) {
                    const long long v0 = pair_value(t), v1 = pair_value(t + nph);
                    b0 = v0 < b0 ? v0 : b0;
                    b1 = v1 < b1 ? v1 : b1;
                }
                for (; t < nv; t += nph) {
                    const long long v0 = pair_value(t);
                    b0 = v0 < b0 ? v0 : b0;
                }
            }
            const long long bv = b1 < b0 ? b1 : b0;
            int best = bv == LLONG_MAX ? INT_MAX : (int)(bv >> 16);
            unsigned bkey = bv == LLONG_MAX ? 0xFFFFFFFFu : (unsigned)(bv & 0xFFFF);
            team_min2<8>(best, bkey, xch, rounds & 1, 0, lane, wi);
            ++rounds;
            if (best >= 0) break;
            const int r = (int)(bkey >> 8), s = (int)(bkey & 255u);
            if (r >= n || s >= n || r >= s) {  // cannot happen; never index with it
                if (tt == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            // A: the move's vectors and the old rows and columns r, s of H and Dp
            const int hrs = H[r * gs + s], hsr = H[s * gs + r];
            const int fRr = Fv(r, r) - Fv(r, s), fRs = Fv(s, r) - Fv(s, s);
            const int fCr = Fv(r, r) - Fv(s, r), fCs = Fv(r, s) - Fv(s, s);
            const int eRr = Dv(r, s) - Dv(r, r), eRs = Dv(s, s) - Dv(s, r);
            const int eCr = Dv(s, r) - Dv(r, r), eCs = Dv(s, s) - Dv(r, s);
            const int drr = Dv(r, r), dss = Dv(s, s), drs = Dv(r, s), dsr = Dv(s, r);
            const int x = tt;
            int fR = 0, fC = 0, eR = 0, eC = 0, hxr = 0, hxs = 0, hrx = 0, hsx = 0;
            int dxr = 0, dxs = 0, drx = 0, dsx = 0;
            if (x < n) {
                fR = Fv(x, r) - Fv(x, s);
                fC = Fv(r, x) - Fv(s, x);
                dxr = Dv(x, r);
                dxs = Dv(x, s);
                drx = Dv(r, x);
                dsx = Dv(s, x);
                eR = dxs - dxr;
                eC = dsx - drx;
                hxr = H[x * gs + r];
                hxs = H[x * gs + s];
                hrx = H[r * gs + x];
                hsx = H[s * gs + x];
                const bool rs = x == r || x == s;
                rowv[x] = make_int4(rs ? 0 : fR, rs ? 0 : fC, fR * eR + fC * eC, 0);
                colv[x] = make_int2(eR, eC);
            }
            team_sync<8>(0);
            // B: rows and columns outside {r, s}
            if (on && e != r && e != s) {
                const int2 ce = colv[e];
                for (int k = ph; k < n; k += nph) {
                    const int4 q = rowv[k];
                    if (q.x | q.y) H[k * gs + e] += q.x * ce.x + q.y * ce.y - q.z;
                }
            }
            // C: rows and columns r and s
            if (x < n && x != r && x != s) {
                H[x * gs + r] = hxs + fR * (eRs - eR) + fC * (eCs - eC);
                H[x * gs + s] = hxr + fR * (eRr - eR) + fC * (eCr - eC);
                H[r * gs + x] = hrx - hrs + fRr * (eR - eRs) + fCr * (eC - eCs);
                H[s * gs + x] = hsx - hsr + fRs * (eR - eRr) + fCs * (eC - eCr);
                Dp[x * dps + r] = (uint16_t)dxs;
                Dp[x * dps + s] = (uint16_t)dxr;
                Dp[r * dps + x] = (uint16_t)dsx;
                Dp[s * dps + x] = (uint16_t)drx;
            }
            if (tt == 0) {
                H[r * gs + s] = -hrs + fRr * (eRr - eRs) + fCr * (eCr - eCs);
                H[s * gs + r] = -hsr + fRs * (eRs - eRr) + fCs * (eCs - eCr);
                Dp[r * dps + r] = (uint16_t)dss;
                Dp[s * dps + s] = (uint16_t)drr;
                Dp[r * dps + s] = (uint16_t)dsr;
                Dp[s * dps + r] = (uint16_t)drs;
                const uint8_t t8 = pi8[r];
                pi8[r] = pi8[s];
                pi8[s] = t8;
            }
            team_sync<8>(0);
            cost += best;
            ++moves;
        }
    }
    for (int m = tt; m < n; m += TT) a.out[(size_t)p * a.ps_out + m] = pi8[m];
    if (a.PL) {
        const long long old = a.costL[p];
        if (cost < old) {
            for (int m = tt; m < n; m += TT) a.PL[(size_t)p * a.ps_out + m] = pi8[m];
            if (tt == 0) a.costL[p] = cost;
        }
    }
    if (tt == 0) {
        a.cost[p] = cost;
        if (a.moves) a.moves[p] = moves;
        if (a.rounds) a.rounds[p] = rounds;
        if (a.counters) {
            atomicAdd(a.counters + CNT_PIT, 1ull);
            if (a.max_moves >= 0) {
                atomicAdd(a.counters + CNT_MOVES, (unsigned long long)moves);
                atomicAdd(a.counters + CNT_ROUNDS, (unsigned long long)rounds);
                if (rounds > 0) {
                    atomicAdd(a.counters + CNT_DELTA_FULL, (unsigned long long)npairs);
                    atomicAdd(a.counters + CNT_DELTA_INCR, (unsigned long long)((rounds - 1) * npairs));
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256, 2) k_ls_gen(const LsArgs* __restrict__ args, int cpi, int smem_d) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const LsArgs a = args[blockIdx.x / cpi];
    const int cb = blockIdx.x % cpi;
    const int n = a.n;
    const GenLayout L = gen_layout(n, smem_d != 0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sA1 = smem + L.oA1;
    unsigned char* sA2 = smem + L.oA2;
    uint16_t* sF = reinterpret_cast<uint16_t*>(smem + L.oF);
    const uint16_t* sD = reinterpret_cast<const uint16_t*>(smem + L.oD);
    unsigned char* U = smem + L.oU;
    unsigned char* B2 = U + (size_t)L.NP * L.KP * 2;
    int32_t* H = reinterpret_cast<int32_t*>(U);
    uint16_t* Dp = reinterpret_cast<uint16_t*>(smem + L.oDp);
    uint8_t* pi8 = smem + L.oPi;
    int4* rowv = reinterpret_cast<int4*>(smem + L.oRow);
    int2* colv = reinterpret_cast<int2*>(smem + L.oCol);
    int32_t* ev = reinterpret_cast<int32_t*>(smem + L.oEv);
    int* xch = reinterpret_cast<int*>(smem + L.oX);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.oBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.oT);
    const int KP = L.KP, gs = L.gs, dps = L.dps;

    for (int i = tid; i < n * n; i += blockDim.x) sF[i] = (uint16_t)a.F[i];
    if (L.smem_d)
        for (int i = tid; i < n * n; i += blockDim.x) const_cast<uint16_t*>(sD)[i] = (uint16_t)a.D[i];
    // A1 = F, A2 = F^T (rows >= n zero)
    for (int i = tid; i < 128 * (KP / 8); i += blockDim.x) {
        const int r = i / (KP / 8), c = (i % (KP / 8)) * 8;
        uint32_t h1[4], h2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = c + 2 * q;
            const bool r_in = r < n;
            h1[q] = pack_h2(r_in && j < n ? a.F[r * n + j] : 0, r_in && j + 1 < n ? a.F[r * n + j + 1] : 0);
            h2[q] = pack_h2(r_in && j < n ? a.F[j * n + r] : 0, r_in && j + 1 < n ? a.F[(j + 1) * n + r] : 0);
        }
        *reinterpret_cast<uint4*>(sA1 + tc::tile_offset(r, c, KP)) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
        *reinterpret_cast<uint4*>(sA2 + tc::tile_offset(r, c, KP)) = make_uint4(h2[0], h2[1], h2[2], h2[3]);
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)L.NP) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (tid == 0) mbar_init(bar, 1);
    fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tcol = *tslot;
    const uint32_t idesc = tc::idesc_f16_f32(128, L.NP);
    const uint32_t sbo = (uint32_t)(KP / 8) * 128;
    const int slotw = round_up(n, 32) < 256 ? round_up(n, 32) : 256;
    const int nph = 256 / slotw, ph = tid / slotw, col = tid % slotw;
    uint32_t phase = 0;
    int next = cb;
    const bool ready = ord_ready(a);

    for (;;) {
        int p;
        if (a.work) {
            if (tid == 0) xch[60] = ord_pick(a, ready, atomicAdd(a.work, 1));
            team_sync<8>(0);
            p = xch[60];
            team_sync<8>(0);
        } else {
            p = next;
            next += cpi;
        }
        if (p >= a.count) break;
        for (int m = tid; m < KP; m += 256) pi8[m] = m < n ? a.in[(size_t)p * a.ps_in + m] : 0;
        team_sync<8>(0);
        // Dp (uint16 rows) and the B tiles Dp and Dp^T (fp16, zero padded)
        for (int i = tid; i < L.NP * (KP / 8); i += 256) {
            const int m = i / (KP / 8), c = (i % (KP / 8)) * 8;
            uint32_t h1[4] = {0u, 0u, 0u, 0u}, h2[4] = {0u, 0u, 0u, 0u};
            if (m < n) {
                const int pm = pi8[m];
                int v1[8], v2[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = c + q;
                    v1[q] = 0;
                    v2[q] = 0;
                    if (j < n) {
                        const int pj = pi8[j];
                        v1[q] = L.smem_d ? (int)sD[pm * n + pj] : __ldg(a.D + pm * n + pj);  // Dp[m][j]
                        v2[q] = L.smem_d ? (int)sD[pj * n + pm] : __ldg(a.D + pj * n + pm);  // Dp[j][m]
                        Dp[m * dps + j] = (uint16_t)v1[q];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    h1[q] = pack_h2(v1[2 * q], v1[2 * q + 1]);
                    h2[q] = pack_h2(v2[2 * q], v2[2 * q + 1]);
                }
            }
            *reinterpret_cast<uint4*>(U + tc::tile_offset(m, c, KP)) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
            *reinterpret_cast<uint4*>(B2 + tc::tile_offset(m, c, KP)) = make_uint4(h2[0], h2[1], h2[2], h2[3]);
        }
        fence_proxy_async();
        team_sync<8>(0);
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a1 = smem_u32(sA1), a2 = smem_u32(sA2), b1 = smem_u32(U), b2 = smem_u32(B2);
            for (int s = 0; s < KP / 16; ++s)  // F Dp^T
                tc::mma_f16(tcol, tc::smem_desc(a1 + s * 256, 128, sbo), tc::smem_desc(b1 + s * 256, 128, sbo), idesc,
                            s > 0);
            for (int s = 0; s < KP / 16; ++s)  // + F^T Dp
                tc::mma_f16(tcol, tc::smem_desc(a2 + s * 256, 128, sbo), tc::smem_desc(b2 + s * 256, 128, sbo), idesc,
                            true);
            tc::mma_commit(bar);
        }
        const bool ok = team_all<8>(mbar_wait(bar, phase), 0);
        if (!ok) {  // the product did not complete in time: record and leave
            if (tid == 0) {
                if (a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                mbar_wait(bar, phase);  // one more bounded wait before the tensor memory is freed
            }
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        if (warp < 4) {  // rows k = 32 warp + lane, lane quarter = warp
            const int k = 32 * warp + lane;
            for (int c = 0; c < L.NP; c += 16) {
                uint32_t v[16];
                tc::tmem_ld16(tcol + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
                tc::tmem_wait_ld();
                if (k < n) {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (c + q < n) H[k * gs + c + q] = __float2int_rn(__uint_as_float(v[q]));
                }
            }
            if (k < n) ev[k] = H[k * gs + k];
        }
        tc::fence_before_sync();
        team_sync<8>(0);
        long long part = 0;
        for (int m = tid; m < n; m += 256) part += ev[m];
        const long long cost2 = team_sum64<8>(part, reinterpret_cast<long long*>(xch) + 16, 0, lane, tid >> 5);
        if (ph < nph && col < n)
            for (int k = ph; k < n; k += nph) H[k * gs + col] -= ev[k];
        team_sync<8>(0);
        descend_gen(a, p, sF, H, Dp, pi8, rowv, colv, xch, cost2 / 2, gs, dps, tid);
        team_sync<8>(0);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(*tslot, ncols);
}

cudaError_t launch_gen(const LsLaunch& L, cudaStream_t st) {
    GenLayout T = gen_layout(L.n_max, true);
    int smem_sm = 0, reserved = 0;
    smem_limits(&smem_sm, &reserved);
    auto ctas = [&](const GenLayout& G) {
        int c = smem_sm / (int)(G.total + reserved);
        const int regs = kernel_regs<k_ls_gen>();
        if (regs > 0 && c > 65536 / (regs * 256)) c = 65536 / (regs * 256);
        if (c > 8) c = 8;
        uint32_t ncols = 32;
        while (ncols < (uint32_t)G.NP) ncols <<= 1;
        if (c > (int)(512 / ncols)) c = (int)(512 / ncols);
        return c < 1 ? 1 : c;
    };
    if (T.smem_d) {
        const GenLayout T2 = gen_layout(L.n_max, false);
        if (ctas(T2) > ctas(T)) T = T2;
    }
    if (T.total > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = configure_once<k_ls_gen>();
    if (e != cudaSuccess) return e;
    const int per_sm = ctas(T);
    int cpi = L.cpi;
    if (cpi <= 0) {
        cpi = (sm_count() * per_sm + L.count - 1) / L.count;
        const int per_pop = L.total / L.count;
        if (cpi > per_pop) cpi = per_pop;
        if (cpi < 1) cpi = 1;
    }
    e = cudaMemsetAsync(L.d_work, 0, sizeof(int32_t) * L.count, st);
    if (e != cudaSuccess) return e;
    k_ls_gen<<<L.count * cpi, 256, T.total, st>>>(L.d_args, cpi, T.smem_d ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

int ls_max_n(LsKind kind) {
    switch (kind) {
        case LS_TEAM1: return 32;
        case LS_TEAM2: return 64;
        case LS_TEAM8: return 128;
        case LS_TEAM8N: return 160;
        case LS_GEN: return 128;
        case LS_SIMT: return simt_max_n<int32_t, uint16_t>();
        case LS_SIMT64: return simt_max_n<int64_t, int32_t>();
        case LS_DIRECT: return 256;
        default: return 0;
    }
}

LsKind ls_kind(const LsArgs& a) {
    if (a.force >= 0) return (LsKind)a.force;
    const int n = a.n;
    if (!a.sym) return (a.tc_exact & 4) && n <= ls_max_n(LS_GEN) ? LS_GEN : LS_DIRECT;
    if (a.tc_exact & 1) {
        if (n <= 32) return LS_TEAM1;
        if (n <= 64) return LS_TEAM2;
        if (n <= 128) return LS_TEAM8;
        // past 128 rows only the 8-bit staging of F and Dp (entries <= 255) fits shared memory
        if ((a.tc_exact & 2) && n <= 160) return LS_TEAM8N;
    }
    if (a.exact32 && n <= ls_max_n(LS_SIMT)) return LS_SIMT;
    if (n <= ls_max_n(LS_SIMT64)) return LS_SIMT64;
    return LS_DIRECT;
}

bool ls_kind_serves(LsKind kind, const LsArgs& a) {
    const int n = a.n;
    if (n < 2 || n > ls_max_n(kind)) return false;
    switch (kind) {
        case LS_TEAM1:
        case LS_TEAM2:
        case LS_TEAM8: return (a.tc_exact & 1) != 0;
        case LS_TEAM8N: return (a.tc_exact & 3) == 3 && n > 128;
        case LS_GEN: return (a.tc_exact & 4) != 0;
        case LS_SIMT: return a.sym && a.exact32;
        case LS_SIMT64: return a.sym != 0;
        case LS_DIRECT: return true;
        default: return false;
    }
}

cudaError_t launch_ls(const LsLaunch& L, cudaStream_t st) {
    if (L.count <= 0 || L.total <= 0) return cudaSuccess;
    if (L.n_max < 2 || L.n_max > ls_max_n((LsKind)L.kind)) return cudaErrorInvalidValue;
    switch (L.kind) {
        case LS_TEAM1: return launch_team<1, uint16_t>(L, st);
        case LS_TEAM2: return launch_team<2, uint16_t>(L, st);
        case LS_TEAM8: return launch_team<8, uint16_t>(L, st);
        case LS_TEAM8N: return launch_team<8, uint8_t>(L, st);
        case LS_GEN: return launch_gen(L, st);
        case LS_SIMT: return launch_simt_t<int32_t, uint16_t>(L, st);
        case LS_SIMT64: return launch_simt_t<int64_t, int32_t>(L, st);
        case LS_DIRECT: return launch_direct(L, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qap
