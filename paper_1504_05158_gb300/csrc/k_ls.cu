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
//   k_ls_team (n <= 128, symmetric, entries <= 2048, n max_f max_d < 2^24): on the
//     tensor cores (tcgen05, fp16 operands, fp32 accumulation in tensor memory).
//     Every operand and partial sum is an integer below 2^24, so the fp32 result is
//     exact. With G[k][l] = sum_j' F[k][p^-1(j')] D[j'][l], the A operand is F with
//     its columns gathered by p^-1 (one particle per M = 128 tile) and the B operand
//     is D itself (symmetric, shared by every particle).
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
// cpi CTAs per population of the table: CTA b serves population b / cpi
template <int NW>
__global__ void __launch_bounds__(kMaxWarpsPerCta * 32) k_ls(const LsArgs* __restrict__ args, int cpi,
                                                             int wpc) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const LsArgs a = args[blockIdx.x / cpi];
    const int cb = blockIdx.x % cpi;
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

    int p = cb * wpc + warp;
    for (;;) {
        if (a.work) {
            int q = 0;
            if (lane == 0) q = atomicAdd(a.work, 1);
            p = __shfl_sync(FULL, q, 0);
        }
        if (p >= a.count) break;
        const int pcur = p;
        if (!a.work) p += cpi * wpc;
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
                    for (int i = 0; i < n; ++i) col += (long long)sF[i * fs + j] * (int)sD[pi[i] * n + pm[w]];
                    part += col;
                }
            }
            store_cost_only(a, pcur, warp_sum64(part), pi, lane);
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
        descend_and_store<NW>(a, pcur, sF, sD, G, gd, pi, lane);
    }
}

// ------------------------------------------------------ tensor-core set-up
// Teams of WPP warps (1 for n <= 32, 2 for n <= 64, 8 for n <= 128) search one
// particle at a time, independently of the other teams of the CTA. A team's
// particle occupies the rows of an M = 128 A tile that sit in the tensor-memory
// lane quarters of the team's own warps (rows of other quarters are never read
// back), the team has its own tensor-memory columns and mbarrier, and particles come
// from a per-population counter, so no team waits for another team's search.
// KP = NP = n rounded up to 16. The search reads F from its fp16 copy (exact).
template <int WPP>
struct TeamLayout {
    int n, KP, NP, fhs;
    size_t oD, oFh, oB, oPin, oGd, oPi, oX, oBar, oT, oU, ubytes, total;
};

constexpr int kXchBytes = 256;  // per team: reduction slots and the next particle

template <int WPP>
__host__ __device__ inline TeamLayout<WPP> team_layout(int n) {
    TeamLayout<WPP> L{};
    constexpr int TEAMS = 8 / WPP;
    L.n = n;
    L.KP = round_up(n, 16);
    L.NP = L.KP;
    L.fhs = round_up(n, 4) + 2;  // odd word stride: column gathers free of bank conflicts
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = (o + b + 127) & ~size_t(127);
        return r;
    };
    L.oD = take((size_t)n * n * 2);
    L.oFh = take((size_t)n * L.fhs * 2);
    L.oB = take((size_t)L.NP * L.KP * 2);
    L.oPin = take(TEAMS * 128);
    L.oGd = take(TEAMS * align16((size_t)n * 4));
    L.oPi = take(TEAMS * align16((size_t)n * 4));
    L.oX = take(TEAMS * kXchBytes);
    L.oBar = take(TEAMS * 8);
    L.oT = take(16);
    const size_t a_bytes = (size_t)128 * L.KP * 2;
    L.ubytes = (a_bytes > g_bytes(n) ? a_bytes : g_bytes(n) + 127) & ~size_t(127);
    L.oU = take((size_t)TEAMS * L.ubytes);
    L.total = o;
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

__device__ __forceinline__ int fval(const __half* sFh, int fhs, int k, int m) {
    return __half2int_rn(sFh[k * fhs + m]);
}

// Best-improvement descent of particle p by one team from a complete G. The team's
// threads form `nph` phases of `slotw` threads: thread (ph, e) evaluates pair slot e
// of virtual rows ph, ph + nph, ... and, after a move, updates column e of G in rows
// ph, ph + nph, ...
template <int WPP>
__device__ __forceinline__ void descend_team(const LsArgs& a, int p, const __half* sFh, int fhs,
                                             const uint16_t* sD, int32_t* G, int32_t* gd, int32_t* pi,
                                             int* xch, int tt, int team) {
    constexpr int TT = 32 * WPP;
    const int n = a.n, gs = n + 1;
    const int lane = tt & 31, wi = tt >> 5;
    const int slotw = round_up(n, 32) < TT ? round_up(n, 32) : TT;
    const int nph = TT / slotw, ph = tt / slotw, e = tt % slotw;
    const bool on = ph < nph && e < n;
    const long long npairs = (long long)n * (n - 1) / 2;
    const int nv = n / 2;
    long long part = 0;
    for (int m = tt; m < n; m += TT) {
        gd[m] = G[m * gs + pi[m]];
        part += gd[m];
    }
    long long cost = team_sum64<WPP>(part, reinterpret_cast<long long*>(xch) + 16, team, lane, wi);
    int moves = 0, rounds = 0;
    if (a.max_moves >= 0) {
        for (;;) {
            if (a.max_moves > 0 && moves >= a.max_moves) break;
            if (moves >= kSafetyMoves) {
                if (tt == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            int best = INT_MAX;
            unsigned bkey = 0xFFFFFFFFu;
            if (on) {
                for (int t = ph; t < nv; t += nph) {
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
                                  4 * fval(sFh, fhs, k, m) * (int)sD[pk * n + pmm];
                    const unsigned key = ((unsigned)k << 8) | (unsigned)m;
                    if (d < best || (d == best && key < bkey)) {
                        best = d;
                        bkey = key;
                    }
                }
            }
            team_min2<WPP>(best, bkey, xch, rounds & 1, team, lane, wi);
            ++rounds;
            if (best >= 0) break;
            const int r = (int)(bkey >> 8), s = (int)(bkey & 255u);
            if (r >= n || s >= n || r >= s) {  // cannot happen; never index with it
                if (tt == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
                break;
            }
            const int pr = pi[r], pss = pi[s];
            if (on) {
                const int bt = (int)sD[pss * n + e] - (int)sD[pr * n + e];
                for (int k = ph; k < n; k += nph)
                    G[k * gs + e] += (fval(sFh, fhs, r, k) - fval(sFh, fhs, s, k)) * bt;
            }
            team_sync<WPP>(team);  // G complete; p itself is still the old one
            for (int m = tt; m < n; m += TT) {
                const int pm = m == r ? pss : (m == s ? pr : pi[m]);
                gd[m] = G[m * gs + pm];
                if (m == r || m == s) pi[m] = pm;
            }
            team_sync<WPP>(team);
            cost += best;
            ++moves;
        }
    }
    for (int m = tt; m < n; m += TT) a.out[(size_t)p * a.ps_out + m] = (uint8_t)pi[m];
    if (a.PL) {
        const long long old = a.costL[p];
        if (cost < old) {
            for (int m = tt; m < n; m += TT) a.PL[(size_t)p * a.ps_out + m] = (uint8_t)pi[m];
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

// cpi CTAs per population of the table: CTA b serves population b / cpi
template <int WPP>
__global__ void __launch_bounds__(256) k_ls_team(const LsArgs* __restrict__ args, int cpi) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int TT = 32 * WPP, TEAMS = 8 / WPP;
    const LsArgs a = args[blockIdx.x / cpi];
    const int cb = blockIdx.x % cpi;
    const int n = a.n;
    const TeamLayout<WPP> L = team_layout<WPP>(n);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int team = warp / WPP, tt = tid - team * TT;
    uint16_t* sD = reinterpret_cast<uint16_t*>(smem + L.oD);
    __half* sFh = reinterpret_cast<__half*>(smem + L.oFh);
    unsigned char* sB = smem + L.oB;
    uint8_t* pinv = smem + L.oPin + team * 128;
    int32_t* gd = reinterpret_cast<int32_t*>(smem + L.oGd + team * align16((size_t)n * 4));
    int32_t* pi = reinterpret_cast<int32_t*>(smem + L.oPi + team * align16((size_t)n * 4));
    int* xch = reinterpret_cast<int*>(smem + L.oX + team * kXchBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.oBar) + team;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.oT);
    unsigned char* U = smem + L.oU + (size_t)team * L.ubytes;
    int32_t* G = reinterpret_cast<int32_t*>(U);

    for (int i = tid; i < n * n; i += blockDim.x) sD[i] = (uint16_t)a.D[i];
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
    while (ncols < (uint32_t)(TEAMS * L.NP)) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (tt == 0) mbar_init(bar, 1);
    fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tcol = *tslot + (uint32_t)(team * L.NP);
    const uint32_t idesc = tc::idesc_f16_f32(128, L.NP);
    const uint32_t sbo = (uint32_t)(L.KP / 8) * 128;
    const int rowbase = 32 * ((team * WPP) & 3);  // the lane quarter of the team's first warp
    const int wq = warp & 3;                      // this warp's lane quarter
    const bool reader = (warp % WPP) < 4;         // warps that read the team's rows back
    uint32_t phase = 0;
    int next = cb * TEAMS + team;
    const int stride = cpi * TEAMS;

    for (;;) {
        int p;
        if (a.work) {
            if (tt == 0) xch[60] = atomicAdd(a.work, 1);
            team_sync<WPP>(team);
            p = xch[60];
            team_sync<WPP>(team);
        } else {
            p = next;
            next += stride;
        }
        if (p >= a.count) break;
        for (int m = tt; m < n; m += TT) {
            const int v = a.in[(size_t)p * a.ps_in + m];
            pi[m] = v;
            pinv[v] = (uint8_t)m;
        }
        team_sync<WPP>(team);
        // A rows of this particle: row rowbase + k holds F[k][p^-1(j')] in column j'
        for (int k = tt; k < n; k += TT) {
            for (int c = 0; c < L.KP; c += 8) {
                __align__(16) __half h[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = c + q;
                    h[q] = j < n ? sFh[k * L.fhs + pinv[j]] : __int2half_rn(0);
                }
                *reinterpret_cast<uint4*>(U + tc::tile_offset(rowbase + k, c, L.KP)) =
                    *reinterpret_cast<uint4*>(h);
            }
        }
        fence_proxy_async();
        team_sync<WPP>(team);
        if (tt == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = smem_u32(U), b0 = smem_u32(sB);
            for (int s = 0; s < L.KP / 16; ++s)
                tc::mma_f16(tcol, tc::smem_desc(a0 + s * 256, 128, sbo), tc::smem_desc(b0 + s * 256, 128, sbo),
                            idesc, s > 0);
            tc::mma_commit(bar);
        }
        const bool ok = team_all<WPP>(mbar_wait(bar, phase), team);
        phase ^= 1u;
        if (!ok) {  // the product never completed: record and leave (cannot be expected)
            if (tt == 0 && a.counters) atomicAdd(a.counters + CNT_ERR, 1ull);
            break;
        }
        tc::fence_after_sync();
        // G from tensor memory: reader warp w holds rows k = 32 (w % WPP) + lane of its quarter
        if (reader) {
            const int k = 32 * (warp % WPP) + lane;
            for (int c = 0; c < L.NP; c += 16) {
                uint32_t v[16];
                tc::tmem_ld16(tcol + ((uint32_t)(32 * wq) << 16) + (uint32_t)c, v);
                tc::tmem_wait_ld();
                // G overwrites the A tile, which the completed product no longer reads
                if (k < n) {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (c + q < n) G[k * (n + 1) + c + q] = __float2int_rn(__uint_as_float(v[q]));
                }
            }
        }
        tc::fence_before_sync();
        team_sync<WPP>(team);
        descend_team<WPP>(a, p, sFh, L.fhs, sD, G, gd, pi, xch, tt, team);
        team_sync<WPP>(team);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(*tslot, ncols);
}

template <int WPP>
cudaError_t launch_team(const LsLaunch& L, cudaStream_t st) {
    const TeamLayout<WPP> T = team_layout<WPP>(L.n_max);
    if (T.total > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_ls_team<WPP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)T.total);
    // all of the unified L1 / shared storage as shared memory, so two CTAs fit an SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ls_team<WPP>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ls_team<WPP>, 256, T.total);
    int smem_sm = 0, reserved = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int by_smem = smem_sm / (int)(T.total + reserved);
    if (by_smem > per_sm) per_sm = by_smem;  // the occupancy query can ignore the carveout request
    // co-resident CTAs must fit the 512 tensor-memory columns together
    uint32_t ncols = 32;
    while (ncols < (uint32_t)((8 / WPP) * T.NP)) ncols <<= 1;
    const int tmem_cap = (int)(512 / ncols);
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    if (per_sm < 1) per_sm = 1;
    int cpi = L.cpi;
    if (cpi <= 0) {  // one wave over the table, at least one CTA per population
        cpi = (sms * per_sm + L.count - 1) / L.count;
        const int per_pop = (L.total / L.count + (8 / WPP) - 1) / (8 / WPP);
        if (cpi > per_pop) cpi = per_pop;
        if (cpi < 1) cpi = 1;
    }
    e = cudaMemsetAsync(L.d_work, 0, sizeof(int32_t) * L.count, st);
    if (e != cudaSuccess) return e;
    k_ls_team<WPP><<<L.count * cpi, 256, T.total, st>>>(L.d_args, cpi);
    return cudaGetLastError();
}

template <int NW>
cudaError_t launch_nw(const LsLaunch& L, cudaStream_t st) {
    const int n = L.n_max;
    int wpc = kMaxWarpsPerCta;
    while (wpc > 1 && shared_part(n) + wpc * warp_part(n) > kSmemLimit) --wpc;
    const size_t smem = shared_part(n) + wpc * warp_part(n);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_ls<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ls<NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ls<NW>, wpc * 32, smem);
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
    k_ls<NW><<<L.count * cpi, wpc * 32, smem, st>>>(L.d_args, cpi, wpc);
    return cudaGetLastError();
}

}  // namespace

int ls_max_n() {
    int n = 2;
    while (n < 256 && shared_part(n + 1) + warp_part(n + 1) <= kSmemLimit) ++n;
    return n < 160 ? n : 160;
}

LsKind ls_kind(const LsArgs& a) {
    const char* env = getenv("QAP_PSO_LS_SETUP");
    const bool simt = env && strcmp(env, "simt") == 0;
    if (!a.tc_exact || a.n > 128 || simt) return LS_SIMT;
    return a.n <= 32 ? LS_TEAM1 : (a.n <= 64 ? LS_TEAM2 : LS_TEAM8);
}

cudaError_t launch_ls(const LsLaunch& L, cudaStream_t st) {
    if (L.count <= 0 || L.total <= 0) return cudaSuccess;
    if (L.n_max < 2 || L.n_max > ls_max_n()) return cudaErrorInvalidValue;
    if (L.kind == LS_TEAM1) return launch_team<1>(L, st);
    if (L.kind == LS_TEAM2) return launch_team<2>(L, st);
    if (L.kind == LS_TEAM8) return launch_team<8>(L, st);
    switch ((L.n_max + 31) / 32) {
        case 1: return launch_nw<1>(L, st);
        case 2: return launch_nw<2>(L, st);
        case 3: return launch_nw<3>(L, st);
        case 4: return launch_nw<4>(L, st);
        case 5: return launch_nw<5>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qap
