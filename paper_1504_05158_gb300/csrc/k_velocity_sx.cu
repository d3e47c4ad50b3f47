// Initialisation, and the velocity and position updates of every particle in one
// kernel (k_update), one warp per particle: the particle's n x n tile of V is staged in
// shared memory with one bulk copy, S_x reads it, the velocity replaces it in place and
// one bulk copy stores it back, so V is read and written once per iteration.
//
// Velocity (section 3.1, Eq. 4): W = c1 V(t) + c2 r2 (P^L - X(t)) + c3 r3 (P^G - X(t)),
// V(t+1) = S_v(W); S_v Raw clamps to [-v_max, v_max], Norm then divides column j by
// n_j = sum_i |W_ij| (columns with n_j = 0 stay 0). Arithmetic in fp32, V stored
// in fp32 or bf16 (round to nearest even).
//
// Position (Eq. 5): X(t+1) = S_x(X(t) + V(t)) with S_x = SecondTarget(Y, Z = X(t),
// depth) (Algorithm 1): n greedy steps, each taking an element of the set M of the
// largest remaining elements of Y, assigning its column (facility) to its row
// (location) and deleting both; in the first `depth` steps some elements equal to
// 1 in Z are ignored (all of them as Algorithm 1 prints, or only the `depth`
// largest, the reading that reproduces the pictures of Eq. 6). M is ordered by
// column then row; with random ties the k-th element is taken, k = floor(u |M| /
// 2^32) with u from Philox. Lanes own columns and keep each column's maximum, its
// multiplicity and the rows holding it (a bit mask) over the remaining rows, so a
// step costs a warp reduction, a few ballots and one mask word per owned column;
// steps that all draw from one set of equal maxima run as a tie group, and X(t)
// cells above every remaining plain value are assigned together in a round.
#include <climits>

#include "kernels.h"
#include "launch.cuh"

namespace qap {
namespace {

constexpr int kWarps = 4;
constexpr size_t kBarBytes = 64;  // one mbarrier per warp, ahead of the tiles
constexpr size_t kSmemLimit = 227 * 1024;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename VT>
__host__ __device__ inline size_t tile_bytes(int n) {
    return align16((size_t)n * n * sizeof(VT));
}
// The row masks of the column caches of SecondTarget: word wi of column slot w of a
// lane at em[(w nwr + wi) 32 + lane], nwr = the row words of the largest n served.
__host__ __device__ inline size_t mask_bytes(int n) {
    const size_t w = (size_t)(n + 31) / 32;
    return w * w * 32 * sizeof(uint32_t);
}
__host__ __device__ inline size_t lists_bytes(int n) { return align16((size_t)(n > 128 ? n : 128)); }
// The cells of a tie group (tie_group): up to 32 kGroupSlots per warp.
constexpr int kGroupSlots = 4;
constexpr size_t kGroupBytes = 32 * kGroupSlots * sizeof(uint32_t);
template <typename VT>
__host__ __device__ inline size_t warp_bytes(int n) {
    // + deleted-row bits (8 words) + the tail's row/column lists or PickColumn's order
    // + the row masks + the tie group's cells
    return tile_bytes<VT>(n) + 32 + lists_bytes(n) + mask_bytes(n) + kGroupBytes;
}

// --------------------------------------------------------------------- init
// X(0): Fisher-Yates shuffle (i = n-1 .. 1, j = below(u, i+1), Philox tag 2, draw q =
// n-1-i is word q mod 4 of block q / 4); V(0)[e] = v_max (2 u - 1) formed in fp32
// (tag 3, element e = i n + j is word e mod 4 of block e / 4).
template <typename VT>
__global__ void k_init(StateView s) {
    __shared__ uint8_t perm[kWarps][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = s.n;
    for (int p = blockIdx.x * kWarps + warp; p < s.P; p += gridDim.x * kWarps) {
        // draws are keyed by the swarm's index in the whole run (swarm_base + local)
        const uint32_t swarm = (uint32_t)(s.swarm_base + p / s.ss), pis = (uint32_t)(p % s.ss);
        if (lane == 0) {
            uint8_t* q = perm[warp];
            for (int i = 0; i < n; ++i) q[i] = (uint8_t)i;
            U4 u{0, 0, 0, 0};
            for (int i = n - 1; i >= 1; --i) {
                const int d = n - 1 - i;
                if ((d & 3) == 0) u = draw(s.seed, pis, swarm, 0u, TAG_INIT_X, (uint32_t)(d >> 2));
                const int j = (int)below(word_of(u, d & 3), (uint32_t)(i + 1));
                const uint8_t tmp = q[i];
                q[i] = q[j];
                q[j] = tmp;
            }
        }
        __syncwarp();
        for (int m = lane; m < n; m += 32) s.Xsx[(size_t)p * s.ps + m] = perm[warp][m];
        VT* V = reinterpret_cast<VT*>(s.V) + (size_t)p * s.vstride;
        const int nn = n * n, nblocks = (nn + 3) / 4;
        for (int b = lane; b < nblocks; b += 32) {
            const U4 u = draw(s.seed, pis, swarm, 0u, TAG_INIT_V, (uint32_t)b);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = 4 * b + i;
                if (e < nn) {
                    const float v = s.v_max * (2.0f * u01f(word_of(u, i)) - 1.0f);
                    V[e] = VStore<VT>::from_f(v);
                }
            }
        }
        if (lane == 0) {
            s.costL[p] = LLONG_MAX;
            s.moves[p] = 0;
        }
        __syncwarp();
    }
}

// --------------------------------------------------------- velocity and S_x
// Per-column cache of the largest plain velocity value V[i][c] over the remaining
// rows i other than the column's X(t) row pz: the value, its multiplicity and the
// rows holding it (a bit mask over the rows, in shared memory). The X(t) cell itself,
// Y[pz][c] = V[pz][c] + 1, is kept apart, so ignoring it (the first `depth` steps) or
// losing it (row pz assigned) never forces a rescan. A deleted row leaves every
// mask; once the rows holding the maximum have all gone, the cache keeps the
// largest value the scan saw below the maximum as an upper bound of the remaining
// rows (count 0) and is rescanned only when that bound could matter; +inf means never
// scanned, -inf means no rows left. Deleted rows are bits of `dead` (shared memory,
// one word per 32 rows).
struct ColMax {
    float v;
    int cnt;
    float v2;  // the largest value below v over the scanned rows (-inf if none)
};

// The maximum of column c over the remaining rows other than pz; em (the column's
// mask, words 32 apart) receives the rows holding it. Two passes over the column: the
// maximum first, then the rows equal to it and the value below it. Each reads kScanU
// rows at a time with independent loads into kScanU partial results: few registers
// (the scan sets the update kernel's register budget) and little code (a small loop
// body keeps the kernel's hot code in the instruction cache).
constexpr int kScanU = 4;
template <typename VT>
__device__ __forceinline__ ColMax vscan(const VT* tile, const uint32_t* dead, int n, int c, int pz, uint32_t* em) {
    const float kNegInf = __int_as_float(0xff800000);
    const int nw = (n + 31) >> 5;
    auto okbits = [&](int wi) {
        uint32_t ok = ~dead[wi];
        if ((pz >> 5) == wi) ok &= ~(1u << (pz & 31));
        const int lim = n - 32 * wi;
        if (lim < 32) ok &= (1u << lim) - 1u;
        return ok;
    };
    float mu[kScanU];
#pragma unroll
    for (int u = 0; u < kScanU; ++u) mu[u] = kNegInf;
    for (int wi = 0; wi < nw; ++wi) {
        const uint32_t ok = okbits(wi);
        const VT* col = tile + (size_t)(32 * wi) * n + c;
#pragma unroll 1
        for (int b = 0; b < 32; b += kScanU) {
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const float v = ((ok >> (b + u)) & 1u) ? VStore<VT>::to_f(col[(b + u) * n]) : kNegInf;
                mu[u] = fmaxf(mu[u], v);
            }
        }
    }
    float mx = mu[0];
#pragma unroll
    for (int u = 1; u < kScanU; ++u) mx = fmaxf(mx, mu[u]);
#pragma unroll
    for (int u = 0; u < kScanU; ++u) mu[u] = kNegInf;
    int cnt = 0;
    for (int wi = 0; wi < nw; ++wi) {
        const uint32_t ok = okbits(wi);
        const VT* col = tile + (size_t)(32 * wi) * n + c;
        uint32_t eq = 0u;
#pragma unroll 1
        for (int b = 0; b < 32; b += kScanU) {
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const bool in = (ok >> (b + u)) & 1u;
                const float v = in ? VStore<VT>::to_f(col[(b + u) * n]) : kNegInf;
                eq |= (in && v == mx) ? (1u << (b + u)) : 0u;
                mu[u] = fmaxf(mu[u], v < mx ? v : kNegInf);
            }
        }
        em[32 * wi] = eq;
        cnt += __popc(eq);
    }
    float v2 = mu[0];
#pragma unroll
    for (int u = 1; u < kScanU; ++u) v2 = fmaxf(v2, mu[u]);
    return ColMax{cnt ? mx : kNegInf, cnt, v2};
}

// The float of an order key (fkey's inverse; +0 for the key of +-0).
__device__ __forceinline__ float unkey(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// The cache vscan forms, for one column c whose scan the whole warp shares: lane l reads
// rows l, l + 32, ...; the maximum and the largest value below it are warp reductions of
// the order keys, the rows holding the maximum are ballots (bit l of word q = row
// 32 q + l, the mask layout). Every lane receives the result; lane q writes word q of
// the column's mask (em: the column's first word, words 32 apart). A rebuild of a few
// columns costs a few warp-wide instructions each instead of a whole scan by one lane
// while the others wait.
template <int NW, typename VT>
__device__ __forceinline__ ColMax coscan(const VT* tile, const uint32_t* dead, int n, int lane, int c, int pz,
                                         uint32_t* em) {
    uint32_t key[NW];
    uint32_t lm = 0u;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int i = 32 * q + lane;
        const bool ok = i < n && i != pz && !((dead[q] >> lane) & 1u);
        key[q] = ok ? fkey(VStore<VT>::to_f(tile[i * n + c])) : 0u;
        lm = max(lm, key[q]);
    }
    const uint32_t km = __reduce_max_sync(FULL, lm);
    uint32_t l2 = 0u;
#pragma unroll
    for (int q = 0; q < NW; ++q) l2 = max(l2, key[q] < km ? key[q] : 0u);
    const uint32_t k2 = __reduce_max_sync(FULL, l2);
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        if (32 * q >= n) continue;
        const unsigned m = __ballot_sync(FULL, key[q] != 0u && key[q] == km);
        cnt += __popc(m);
        if (lane == q) em[32 * q] = m;
    }
    const float kNegInf = __int_as_float(0xff800000);
    return ColMax{km ? unkey(km) : kNegInf, km ? cnt : 0, k2 ? unkey(k2) : kNegInf};
}

// Two adjacent elements of a tile row as floats (8-byte fp32 or 4-byte bf16 accesses).
template <typename VT>
struct Pair;
template <>
struct Pair<float> {
    static __device__ __forceinline__ void get(const float* p, float& a, float& b) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void put(float* p, float a, float b) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
};
template <>
struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ void get(const __nv_bfloat16* p, float& a, float& b) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
        a = __low2float(v);
        b = __high2float(v);
    }
    static __device__ __forceinline__ void put(__nv_bfloat16* p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
};

// The first cache build of SecondTarget, before any row is deleted: every owned
// column at once, the columns' X(t) cells holding -inf in the tile (second_target
// hides them), so no row needs a test. Pass 1 forms each column's maximum, pass 2 its
// rows and the largest value below it; kScanU rows of every owned column per loop
// step.
template <int NW, typename VT>
__device__ __forceinline__ void first_scan(const VT* tile, uint32_t* em, int nwr, int n, int lane,
                                           const bool (&alive)[NW], float (&vm)[NW], int (&vc)[NW],
                                           float (&v2)[NW]) {
    const float kNegInf = __int_as_float(0xff800000);
    float mu[NW][kScanU];
#pragma unroll
    for (int w = 0; w < NW; ++w)
#pragma unroll
        for (int u = 0; u < kScanU; ++u) mu[w][u] = kNegInf;
    const int nfull = n - n % kScanU;
#pragma unroll 1
    for (int i = 0; i < nfull; i += kScanU) {
#pragma unroll
        for (int u = 0; u < kScanU; ++u)
#pragma unroll
            for (int w = 0; w < NW; ++w)
                if (alive[w]) mu[w][u] = fmaxf(mu[w][u], VStore<VT>::to_f(tile[(i + u) * n + lane + 32 * w]));
    }
    for (int i = nfull; i < n; ++i)
#pragma unroll
        for (int w = 0; w < NW; ++w)
            if (alive[w]) mu[w][0] = fmaxf(mu[w][0], VStore<VT>::to_f(tile[i * n + lane + 32 * w]));
    float mx[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        mx[w] = mu[w][0];
#pragma unroll
        for (int u = 1; u < kScanU; ++u) mx[w] = fmaxf(mx[w], mu[w][u]);
#pragma unroll
        for (int u = 0; u < kScanU; ++u) mu[w][u] = kNegInf;
    }
    int cnt[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) cnt[w] = 0;
    for (int wi = 0; 32 * wi < n; ++wi) {
        uint32_t eq[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) eq[w] = 0u;
        const int i1 = n < 32 * wi + 32 ? n : 32 * wi + 32;
        const int i1f = i1 - (i1 - 32 * wi) % kScanU;
#pragma unroll 1
        for (int i = 32 * wi; i < i1f; i += kScanU) {
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const uint32_t bit = 1u << ((i + u) & 31);
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (!alive[w]) continue;
                    const float v = VStore<VT>::to_f(tile[(i + u) * n + lane + 32 * w]);
                    const bool at = v == mx[w];
                    eq[w] |= at ? bit : 0u;
                    mu[w][u] = fmaxf(mu[w][u], at ? kNegInf : v);
                }
            }
        }
        for (int i = i1f; i < i1; ++i) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (!alive[w]) continue;
                const float v = VStore<VT>::to_f(tile[i * n + lane + 32 * w]);
                const bool at = v == mx[w];
                eq[w] |= at ? 1u << (i & 31) : 0u;
                mu[w][0] = fmaxf(mu[w][0], at ? kNegInf : v);
            }
        }
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            if (!alive[w]) continue;
            em[(w * nwr + wi) * 32 + lane] = eq[w];
            cnt[w] += __popc(eq[w]);
        }
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (!alive[w]) continue;
        float b = mu[w][0];
#pragma unroll
        for (int u = 1; u < kScanU; ++u) b = fmaxf(b, mu[w][u]);
        vm[w] = cnt[w] ? mx[w] : kNegInf;
        vc[w] = cnt[w];
        v2[w] = b;
    }
}

// The first cache build for fp32 tiles when n is even and n <= 64: lane L reads
// columns 2L and 2L + 1 of every row with one 8-byte access, forms their maxima, rows
// and values below them as first_scan does, writes the row masks into the owning
// lanes' mask slots and hands each column's results to its owner (column c = lane +
// 32 w). (With bf16 tiles the column-per-lane scan measured faster.)
template <int NW, typename VT>
__device__ __forceinline__ void first_scan_pairs(const VT* tile, uint32_t* em, int nwr, int n, int lane,
                                                 const bool (&alive)[NW], float (&vm)[NW], int (&vc)[NW],
                                                 float (&v2)[NW]) {
    const float kNegInf = __int_as_float(0xff800000);
    const int c0 = 2 * lane;
    const bool on = c0 < n;  // n even: column c0 + 1 exists too
    const VT* col = tile + c0;
    const int nfull = n - n % kScanU;
    float ma[kScanU], mb[kScanU];
#pragma unroll
    for (int u = 0; u < kScanU; ++u) ma[u] = mb[u] = kNegInf;
    if (on) {
#pragma unroll 1
        for (int i = 0; i < nfull; i += kScanU) {
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                float x, y;
                Pair<VT>::get(col + (i + u) * n, x, y);
                ma[u] = fmaxf(ma[u], x);
                mb[u] = fmaxf(mb[u], y);
            }
        }
        for (int i = nfull; i < n; ++i) {
            float x, y;
            Pair<VT>::get(col + i * n, x, y);
            ma[0] = fmaxf(ma[0], x);
            mb[0] = fmaxf(mb[0], y);
        }
    }
    float mxa = ma[0], mxb = mb[0];
#pragma unroll
    for (int u = 1; u < kScanU; ++u) {
        mxa = fmaxf(mxa, ma[u]);
        mxb = fmaxf(mxb, mb[u]);
    }
#pragma unroll
    for (int u = 0; u < kScanU; ++u) ma[u] = mb[u] = kNegInf;
    int ca = 0, cb = 0;
    for (int wi = 0; 32 * wi < n; ++wi) {
        uint32_t ea = 0u, eb = 0u;
        const int i1 = n < 32 * wi + 32 ? n : 32 * wi + 32;
        const int i1f = i1 - (i1 - 32 * wi) % kScanU;
        if (on) {
#pragma unroll 1
            for (int i = 32 * wi; i < i1f; i += kScanU) {
#pragma unroll
                for (int u = 0; u < kScanU; ++u) {
                    float x, y;
                    Pair<VT>::get(col + (i + u) * n, x, y);
                    const uint32_t bit = 1u << ((i + u) & 31);
                    const bool ax = x == mxa, by = y == mxb;
                    ea |= ax ? bit : 0u;
                    eb |= by ? bit : 0u;
                    ma[u] = fmaxf(ma[u], ax ? kNegInf : x);
                    mb[u] = fmaxf(mb[u], by ? kNegInf : y);
                }
            }
            for (int i = i1f; i < i1; ++i) {
                float x, y;
                Pair<VT>::get(col + i * n, x, y);
                const uint32_t bit = 1u << (i & 31);
                const bool ax = x == mxa, by = y == mxb;
                ea |= ax ? bit : 0u;
                eb |= by ? bit : 0u;
                ma[0] = fmaxf(ma[0], ax ? kNegInf : x);
                mb[0] = fmaxf(mb[0], by ? kNegInf : y);
            }
            em[((c0 >> 5) * nwr + wi) * 32 + (c0 & 31)] = ea;
            em[(((c0 + 1) >> 5) * nwr + wi) * 32 + ((c0 + 1) & 31)] = eb;
            ca += __popc(ea);
            cb += __popc(eb);
        }
    }
    float va = ma[0], vb = mb[0];
#pragma unroll
    for (int u = 1; u < kScanU; ++u) {
        va = fmaxf(va, ma[u]);
        vb = fmaxf(vb, mb[u]);
    }
    // column c's results sit in lane c / 2 (as its a or b column)
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int c = lane + 32 * w;
        const int src = (c >> 1) & 31;
        const float m_a = __shfl_sync(FULL, mxa, src), m_b = __shfl_sync(FULL, mxb, src);
        const int k_a = __shfl_sync(FULL, ca, src), k_b = __shfl_sync(FULL, cb, src);
        const float w_a = __shfl_sync(FULL, va, src), w_b = __shfl_sync(FULL, vb, src);
        if (alive[w]) {
            const bool odd = c & 1;
            const int cnt = odd ? k_b : k_a;
            vm[w] = cnt ? (odd ? m_b : m_a) : kNegInf;
            vc[w] = cnt;
            v2[w] = odd ? w_b : w_a;
        }
    }
    __syncwarp();  // the masks other lanes wrote
}

// Rebuilds the caches of the owned columns that need it (need[w]): by the warp together
// (coscan) when at most kCoopMax columns of a slot need it, else by each lane alone
// (vscan, every lane scanning its own column at once).
constexpr int kCoopMax = 8;
template <int NW, typename VT>
__device__ __forceinline__ void rebuild(const VT* tile, const uint32_t* dead, uint32_t* em, int nwr, int n, int lane,
                                        const int (&pic)[NW], const bool (&need)[NW], float (&vm)[NW],
                                        int (&vc)[NW], float (&v2)[NW]) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const unsigned who = __ballot_sync(FULL, need[w]);
        if (!who) continue;
        if (__popc(who) > kCoopMax) {
            if (need[w]) {
                const ColMax cm = vscan<VT>(tile, dead, n, lane + 32 * w, pic[w], &em[(w * nwr) * 32 + lane]);
                vm[w] = cm.v;
                vc[w] = cm.cnt;
                v2[w] = cm.v2;
            }
            continue;
        }
        unsigned rem = who;
        while (rem) {
            const int L = __ffs(rem) - 1;
            rem &= rem - 1u;
            const int pz = __shfl_sync(FULL, pic[w], L);
            const ColMax cm = coscan<NW, VT>(tile, dead, n, lane, L + 32 * w, pz, &em[(w * nwr) * 32 + L]);
            if (lane == L) {
                vm[w] = cm.v;
                vc[w] = cm.cnt;
                v2[w] = cm.v2;
            }
        }
    }
}

// The last steps of SecondTarget once at most kTailCols columns are left and the
// exclusion phase is over: the remaining A x A cells (at most kTailSlots per lane)
// run the greedy directly, one maximum and one ballot count per step. Cells are
// numbered q = (column index) A + (row index) over the remaining columns and rows,
// both ascending, which is the column-major order of M that the tie draw uses.
constexpr int kTailSlots = 1;
constexpr int kTailCols = 5;   // kTailCols^2 <= 32 kTailSlots

template <int NW, typename VT>
__device__ __forceinline__ int sx_tail(const StateView& s, const VT* tile, const uint32_t* dead, uint8_t* lists,
                                       int n, int lane, const int (&pic)[NW], const bool (&alive)[NW],
                                       const float (&zv)[NW], uint32_t pis, uint32_t swarm, uint32_t t, int step,
                                       int A, U4& tu, int& tblk, int (&newp)[NW]) {
    uint8_t* rows = lists;       // remaining rows, ascending
    uint8_t* cols = lists + 16;  // remaining columns, ascending
    uint8_t* xrow = lists + 32;  // their X(t) rows
    float* xval = reinterpret_cast<float*>(lists + 64);  // and the Y values of their X(t) cells
    const unsigned below_me = (1u << lane) - 1u;
    int base = 0;
#pragma unroll
    for (int wi = 0; wi < NW; ++wi) {
        const int lim = n - 32 * wi;  // rows of this word (none past n when NW is wider than n needs)
        uint32_t m = lim <= 0 ? 0u : ~dead[wi];
        if (lim > 0 && lim < 32) m &= (1u << lim) - 1u;
        if ((m >> lane) & 1u) rows[base + __popc(m & below_me)] = (uint8_t)(32 * wi + lane);
        base += __popc(m);
    }
    base = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const unsigned am = __ballot_sync(FULL, alive[w]);
        if (alive[w]) {
            const int pos = base + __popc(am & below_me);
            cols[pos] = (uint8_t)(lane + 32 * w);
            xrow[pos] = (uint8_t)pic[w];
            xval[pos] = zv[w];
        }
        base += __popc(am);
    }
    __syncwarp();
    uint32_t key[kTailSlots];
    int rc[kTailSlots];  // (row index << 8) | column index
    // q / A as (q ceil(2^16 / A)) >> 16: exact for every q < A^2 with A <= kTailCols
    const int inv_a = (65536 + A - 1) / A;
#pragma unroll
    for (int sl = 0; sl < kTailSlots; ++sl) {
        const int q = lane + 32 * sl;
        key[sl] = 0u;  // no cell (every finite value has a nonzero key)
        rc[sl] = 0;
        if (q < A * A) {
            const int ci = (q * inv_a) >> 16, ri = q - ci * A;  // q / A, q % A
            const int r = rows[ri], c = cols[ci];
            const float y = r == xrow[ci] ? xval[ci] : VStore<VT>::to_f(tile[r * n + c]);
            key[sl] = fkey(y);
            rc[sl] = (ri << 8) | ci;
        }
    }
    int ties = 0;
    for (int k = 0; k < A; ++k, ++step) {
        uint32_t lm = 0u;
#pragma unroll
        for (int sl = 0; sl < kTailSlots; ++sl) lm = max(lm, key[sl]);
        const uint32_t gm = __reduce_max_sync(FULL, lm);
        unsigned b[kTailSlots];
        int tot = 0;
#pragma unroll
        for (int sl = 0; sl < kTailSlots; ++sl) {
            b[sl] = __ballot_sync(FULL, key[sl] != 0u && key[sl] == gm);
            tot += __popc(b[sl]);
        }
        int kk = 0;
        if (tot > 1) {
            ++ties;
            if (s.tie_rule == 0) {
                if ((step >> 2) != tblk) {  // one block of draws serves four steps
                    tu = draw(s.seed, pis, swarm, t, TAG_TIE, (uint32_t)(step >> 2));
                    tblk = step >> 2;
                }
                kk = (int)below(word_of(tu, step & 3), (uint32_t)tot);
            }
        }
        // the kk-th cell of M in cell order (slot, then lane)
        int src = 0, val = 0;
        bool found = false;
#pragma unroll
        for (int sl = 0; sl < kTailSlots; ++sl) {
            const int c = __popc(b[sl]);
            if (!found && kk < c) {
                unsigned m = b[sl];
                for (int j = 0; j < kk; ++j) m &= m - 1u;  // drop the kk lower members
                src = __ffs(m) - 1;
                val = rc[sl];
                found = true;
            } else if (!found) {
                kk -= c;
            }
        }
        const int pick = __shfl_sync(FULL, val, src);
        const int ri = pick >> 8, ci = pick & 0xFF;
        const int r = rows[ri], c = cols[ci];
#pragma unroll
        for (int w = 0; w < NW; ++w)
            if (lane + 32 * w == c) newp[w] = r;
#pragma unroll
        for (int sl = 0; sl < kTailSlots; ++sl)
            if ((rc[sl] >> 8) == ri || (rc[sl] & 0xFF) == ci) key[sl] = 0u;
    }
    return ties;
}

// PickColumn (section 3.1) on Y for one particle: the columns in a Fisher-Yates
// order (Philox tag 7; lane 0 shuffles into shared memory), each taking its largest
// element over the free rows; a maximum shared by several rows is resolved like a
// tie of Algorithm 1 (rows ascending, element k of the tie draw, or the first).
// Rows are spread over the lanes (row i = lane + 32 w). Returns the number of ties.
template <int NW, typename VT>
__device__ __forceinline__ int pick_column(const StateView& s, const VT* tile, uint32_t* dead, uint8_t* order,
                                           int n, int lane, const int (&pic)[NW], uint32_t pis, uint32_t swarm,
                                           uint32_t t, float zadd, int (&newp)[NW]) {
    if (lane == 0) {
        for (int c = 0; c < n; ++c) order[c] = (uint8_t)c;
        U4 u{0, 0, 0, 0};
        for (int i = n - 1; i >= 1; --i) {
            const int d = n - 1 - i;
            if ((d & 3) == 0) u = draw(s.seed, pis, swarm, t, TAG_COLUMNS, (uint32_t)(d >> 2));
            const int j = (int)below(word_of(u, d & 3), (uint32_t)(i + 1));
            const uint8_t tmp = order[i];
            order[i] = order[j];
            order[j] = tmp;
        }
    }
    if (lane < NW) dead[lane] = 0u;
    __syncwarp();
    int ties = 0;
    U4 tu{0, 0, 0, 0};
    int tblk = -1;
    for (int step = 0; step < n; ++step) {
        const int c = order[step];
        int pz = -1;  // the X(t) row of column c (held by lane c mod 32, slot c / 32)
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int v = __shfl_sync(FULL, pic[w], c & 31);
            if (w == (c >> 5)) pz = v;
        }
        uint32_t key[NW];
        uint32_t lm = 0u;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int i = lane + 32 * w;
            key[w] = 0u;
            if (i < n && !((dead[w] >> lane) & 1u)) {
                float y = VStore<VT>::to_f(tile[i * n + c]);
                if (i == pz) y += zadd;
                key[w] = fkey(y);
            }
            lm = max(lm, key[w]);
        }
        const uint32_t gm = __reduce_max_sync(FULL, lm);
        unsigned b[NW];
        int tot = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            b[w] = __ballot_sync(FULL, key[w] != 0u && key[w] == gm);
            tot += __popc(b[w]);
        }
        int kk = 0;
        if (tot > 1) {
            ++ties;
            if (s.tie_rule == 0) {
                if ((step >> 2) != tblk) {
                    tu = draw(s.seed, pis, swarm, t, TAG_TIE, (uint32_t)(step >> 2));
                    tblk = step >> 2;
                }
                kk = (int)below(word_of(tu, step & 3), (uint32_t)tot);
            }
        }
        int r = -1;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int cw = __popc(b[w]);
            if (r < 0 && kk < cw) {
                unsigned m = b[w];
                for (int j = 0; j < kk; ++j) m &= m - 1u;  // drop the kk lower members
                r = 32 * w + __ffs(m) - 1;
            } else if (r < 0) {
                kk -= cw;
            }
        }
        if (r < 0 || r >= n) {  // cannot happen; never index with it
            if (lane == 0) atomicAdd(s.counters + CNT_ERR, 1ull);
            return ties;
        }
        if (lane == (c & 31)) {
#pragma unroll
            for (int w = 0; w < NW; ++w)
                if (w == (c >> 5)) newp[w] = r;
        }
        if (lane == 0) dead[r >> 5] |= 1u << (r & 31);
        __syncwarp();
    }
    return ties;
}

// A run of steps of SecondTarget at one value g. When a step's set M (the remaining
// cells equal to the largest remaining value g) has at least two and at most
// 32 kGroupSlots elements, no other cell can reach g while M is not empty, so the next
// steps draw from M alone until it is: M is listed once in its column-major order
// (column, then row), one cell per lane and slot, and each step takes the k-th live
// cell (k from the step's tie draw, as in a single step), deletes its row and column
// and drops the cells that lie in either, with a few ballots per step. The run stops
// when M is empty, at the end of the exclusion phase (the ignored X(t) cells return)
// or, past that phase, when only X(t) cells are left in M (a round then takes them
// together). Afterwards the caches of the remaining columns lose the deleted rows.
// Inputs: the step's per-column counts cm, modes (0 the X(t) cell alone, 1 the plain
// maximum and the X(t) cell, 2 the plain maximum alone), the three ballots of the
// counts' bits and the per-slot totals tw. Returns -1 on an inconsistent list (which
// cannot happen; counted as an error).
template <int NW>
__device__ __forceinline__ int tie_group(const StateView& s, uint32_t* dead, uint32_t* em, uint32_t* gl, int nwr,
                                         int n, int lane, const int (&pic)[NW], bool (&alive)[NW], bool (&zal)[NW],
                                         float (&vm)[NW], int (&vc)[NW], const float (&v2)[NW], int (&newp)[NW],
                                         const int (&cm)[NW], const int (&mode)[NW], const unsigned (&b0)[NW],
                                         const unsigned (&b1)[NW], const unsigned (&b2)[NW], const int (&tw)[NW],
                                         int tot, int depth, bool use_ex, uint32_t pis, uint32_t swarm, uint32_t t,
                                         int& step, int& ties, U4& tu, int& tblk) {
    auto emw = [&](int w, int wi) -> uint32_t& { return em[(w * nwr + wi) * 32 + lane]; };
    // list M: a column's cells go to positions [start, start + cm) in column order,
    // each cell (X flag << 16) | (row << 8) | column
    const unsigned le = (2u << lane) - 1u;
    int base = 0;
    bool bad = false;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int incl = __popc(b0[w] & le) + 2 * __popc(b1[w] & le) + 4 * __popc(b2[w] & le);
        if (cm[w] > 0) {
            const int c = lane + 32 * w;
            int o = base + incl - cm[w];
            const int end = base + incl;
            if (mode[w] == 0) {
                gl[o++] = (1u << 16) | ((uint32_t)pic[w] << 8) | (uint32_t)c;
            } else {
#pragma unroll
                for (int wi = 0; wi < NW; ++wi) {
                    if (32 * wi >= n) continue;
                    uint32_t m = emw(w, wi);
                    if (mode[w] == 1 && (pic[w] >> 5) == wi) m |= 1u << (pic[w] & 31);
                    while (m && o < end) {
                        const int r = 32 * wi + __ffs(m) - 1;
                        m &= m - 1u;
                        gl[o++] = (r == pic[w] ? (1u << 16) : 0u) | ((uint32_t)r << 8) | (uint32_t)c;
                    }
                }
            }
            bad = bad || o != end;
        }
        base += tw[w];
    }
    if (__any_sync(FULL, bad)) {
        if (lane == 0) atomicAdd(s.counters + CNT_ERR, 1ull);
        return -1;
    }
    __syncwarp();
    uint32_t cell[kGroupSlots];
    unsigned bq[kGroupSlots];
    const int nq = (tot + 31) >> 5;  // slots in use
#pragma unroll
    for (int q = 0; q < kGroupSlots; ++q) {
        const int e = 32 * q + lane;
        cell[q] = e < tot ? gl[e] : 0u;
        const int inq = tot - 32 * q;
        bq[q] = inq >= 32 ? FULL : inq > 0 ? (1u << inq) - 1u : 0u;
    }
    uint32_t gone[NW];
#pragma unroll
    for (int wi = 0; wi < NW; ++wi) gone[wi] = 0u;
    int left = tot;
    for (;;) {
        int k = 0;
        if (left > 1) {
            ++ties;
            if (s.tie_rule == 0) {
                if ((step >> 2) != tblk) {  // one block of draws serves four steps
                    tu = draw(s.seed, pis, swarm, t, TAG_TIE, (uint32_t)(step >> 2));
                    tblk = step >> 2;
                }
                k = (int)below(word_of(tu, step & 3), (uint32_t)left);
            }
        }
        // the k-th live cell in list order (slot, then lane)
        uint32_t mine = 0u, bsel = 0u;
        bool found = false;
#pragma unroll
        for (int q = 0; q < kGroupSlots; ++q) {
            const int cq = __popc(bq[q]);
            if (!found && k < cq) {
                mine = cell[q];
                bsel = bq[q];
                found = true;
            } else if (!found) {
                k -= cq;
            }
        }
        const bool me = ((bsel >> lane) & 1u) && __popc(bsel & (le >> 1)) == k;
        const int src = __ffs(__ballot_sync(FULL, me)) - 1;
        if (src < 0) {  // cannot happen
            if (lane == 0) atomicAdd(s.counters + CNT_ERR, 1ull);
            return -1;
        }
        const uint32_t pc = __shfl_sync(FULL, mine, src);
        const int r = (int)((pc >> 8) & 0xFFu), c = (int)(pc & 0xFFu);
        if (lane == (c & 31)) {
#pragma unroll
            for (int w = 0; w < NW; ++w)
                if (w == (c >> 5)) {
                    newp[w] = r;
                    alive[w] = false;
                }
        }
#pragma unroll
        for (int wi = 0; wi < NW; ++wi)
            if (wi == (r >> 5)) gone[wi] |= 1u << (r & 31);
        left = 0;
        bool plain = false;
#pragma unroll
        for (int q = 0; q < kGroupSlots; ++q) {
            if (q >= nq) continue;
            const bool live = ((bq[q] >> lane) & 1u) && (int)((cell[q] >> 8) & 0xFFu) != r &&
                              (int)(cell[q] & 0xFFu) != c;
            bq[q] = __ballot_sync(FULL, live);
            left += __popc(bq[q]);
            plain = plain || (live && !(cell[q] >> 16));
        }
        ++step;
        if (left == 0) break;
        if (use_ex ? step >= depth : !__any_sync(FULL, plain)) break;
    }
    // the deleted rows leave the remaining columns' caches
#pragma unroll
    for (int wi = 0; wi < NW; ++wi)
        if (lane == wi) dead[wi] |= gone[wi];
    __syncwarp();
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (!alive[w]) continue;
#pragma unroll
        for (int wi = 0; wi < NW; ++wi)
            if ((pic[w] >> 5) == wi && ((gone[wi] >> (pic[w] & 31)) & 1u)) zal[w] = false;
        if (vc[w] == 0) continue;
        int cnt = 0;
#pragma unroll
        for (int wi = 0; wi < NW; ++wi) {
            if (32 * wi >= n) continue;
            uint32_t& m = emw(w, wi);
            const uint32_t mv = m;
            if (mv & gone[wi]) m = mv & ~gone[wi];
            cnt += __popc(mv & ~gone[wi]);
        }
        vc[w] = cnt;
        if (cnt == 0) vm[w] = v2[w];  // the maximum's rows are gone: the bound below it
    }
    return 0;
}

// SecondTarget (Algorithm 1) on Y for one particle; returns the number of steps
// whose set M had more than one element and leaves the location chosen for each
// owned column (facility) in newp. The tile holds V with Y = X(t) + V (zadd = 1:
// the X(t) cell of column c is tile[pz][c] + 1, every other cell the tile value),
// or Y itself (zadd = 0).
//
// After the first `depth` steps, every X(t) cell that exceeds all remaining plain
// values (bound P0) is taken by the greedy in descending order over consecutive
// steps, each in its own row and column, so such cells are assigned together in
// one round; equal values among them only reorder those steps (each group of g
// equal values is g - 1 steps with a choice). Other steps run one at a time.
template <int NW, typename VT>
__device__ __forceinline__ int second_target(const StateView& s, VT* tile, uint32_t* dead, uint32_t* em,
                                             int nwr, int n, int lane, const int (&pic)[NW], uint32_t pis,
                                             uint32_t swarm, uint32_t t, float zadd, int (&newp)[NW]) {
    const int depth = s.depth;
    if (lane < NW) dead[lane] = 0u;
    __syncwarp();
    // word wi of column slot w's row mask
    auto emw = [&](int w, int wi) -> uint32_t& { return em[(w * nwr + wi) * 32 + lane]; };
    float zv[NW], vm[NW], v2[NW];
    int vc[NW];
    bool alive[NW], zal[NW], ex[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int c = lane + 32 * w;
        alive[w] = c < n;
        zal[w] = alive[w];
        ex[w] = false;
        zv[w] = alive[w] ? VStore<VT>::to_f(tile[pic[w] * n + c]) + zadd : 0.0f;
        vm[w] = __int_as_float(0x7f800000);
        v2[w] = vm[w];
        vc[w] = 0;
        newp[w] = 0;
    }
    // The X(t) cells' values are kept in zv; while S_x runs, the tile holds -inf in
    // their place, so that scans need no test for them; they are put back on return.
    VT zraw[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (!alive[w]) continue;
        VT& cell = tile[pic[w] * n + lane + 32 * w];
        zraw[w] = cell;
        cell = VStore<VT>::from_f(__int_as_float(0xff800000));
    }
    auto finish = [&](int ties_out) {
        __syncwarp();
#pragma unroll
        for (int w = 0; w < NW; ++w)
            if (lane + 32 * w < n) tile[pic[w] * n + lane + 32 * w] = zraw[w];
        __syncwarp();
        return ties_out;
    };
    __syncwarp();
    if (sizeof(VT) == 4 && NW <= 2 && (n & 1) == 0)
        first_scan_pairs<NW, VT>(tile, em, nwr, n, lane, alive, vm, vc, v2);
    else
        first_scan<NW, VT>(tile, em, nwr, n, lane, alive, vm, vc, v2);
    if (depth > 0) {
        if (s.sx_rule == 0) {
            // Algorithm 1 as printed: every element equal to 1 in Z = X(t) is ignored
#pragma unroll
            for (int w = 0; w < NW; ++w) ex[w] = alive[w];
        } else {
            // the `depth` largest of them (lower column first on ties)
            for (int d = 0; d < depth; ++d) {
                uint32_t lm = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    if (alive[w] && !ex[w]) lm = max(lm, fkey(zv[w]));
                const uint32_t gm = __reduce_max_sync(FULL, lm);
                bool done = false;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (done) continue;
                    const unsigned bal = __ballot_sync(FULL, alive[w] && !ex[w] && fkey(zv[w]) == gm);
                    if (bal) {
                        if (lane == __ffs(bal) - 1) ex[w] = true;
                        done = true;
                    }
                }
            }
        }
    }
    int ties = 0;
    U4 tu{0, 0, 0, 0};  // the block of tie draws of steps 4 tblk .. 4 tblk + 3
    int tblk = -1;
    // A round can only form after the greedy has just taken an X(t) cell (or at the
    // first step past the exclusion phase, or right after a round): when it takes a
    // plain cell instead, every X(t) cell was below the largest plain value, so the
    // test is skipped (single steps give the same result in every case).
    bool try_round = true;
    // Nonzero: the key of the maximum the next step is known to have. After a step at
    // value g that leaves a plain cell at g (its column's cache is exact), every other
    // remaining cell is at most g, so the next step has the same maximum: it skips the
    // round test (no X(t) cell can exceed a plain value g), the rebuilds (a stale bound
    // lies below g) and the warp maximum. Not carried across the end of the exclusion
    // phase, where ignored X(t) cells return.
    uint32_t cont_key = 0u;
    for (int step = 0; step < n;) {
        const bool use_ex = step < depth;
        if (!use_ex) {
            const int A = n - step;  // columns left
            if (A <= kTailCols) {
                ties += sx_tail<NW, VT>(s, tile, dead, reinterpret_cast<uint8_t*>(dead + 8), n, lane, pic, alive,
                                        zv, pis, swarm, t, step, A, tu, tblk, newp);
                break;
            }
        }
        bool zin[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) zin[w] = alive[w] && zal[w] && !(use_ex && ex[w]);

        if (!use_ex && try_round && !cont_key) {
            // ---- a round of X(t) cells above every remaining plain value ----
            {
                bool need[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) need[w] = alive[w] && !zin[w] && vc[w] == 0;
                rebuild<NW, VT>(tile, dead, em, nwr, n, lane, pic, need, vm, vc, v2);
            }
            uint32_t lp = 0u;
#pragma unroll
            for (int w = 0; w < NW; ++w)
                if (alive[w]) lp = max(lp, fkey(vm[w]));
            const uint32_t P0 = __reduce_max_sync(FULL, lp);
            bool inB[NW];
            uint32_t bkey[NW];
            unsigned any = 0u;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                bkey[w] = fkey(zv[w]);
                inB[w] = zin[w] && bkey[w] > P0;
                any |= __ballot_sync(FULL, inB[w]);
            }
            if (any) {
                // size of the round and the number of distinct values in it: a cell
                // is the first of its value group when no equal cell of the round sits
                // in a lower column (same register slot: lower lane; lower slot: any lane)
                int mine = 0, firsts = 0;
                // a round whose cells all hold one value (the converged swarm: every X(t)
                // cell of Y is 0.5) has one distinct value; no comparison across lanes needed
                uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    if (inB[w]) {
                        kmin = min(kmin, bkey[w]);
                        kmax = max(kmax, bkey[w]);
                    }
                const bool one_value = __reduce_min_sync(FULL, kmin) == __reduce_max_sync(FULL, kmax);
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (one_value) {
                        mine += inB[w] ? 1 : 0;
                        continue;
                    }
                    const unsigned grp = __match_any_sync(FULL, inB[w] ? bkey[w] : 0xFFFFFFFFu);
                    bool first = inB[w] && (__ffs(grp) - 1 == lane);
#pragma unroll
                    for (int w0 = 0; w0 < w; ++w0) {
                        const uint32_t mk = inB[w0] ? bkey[w0] : 0xFFFFFFFFu;
#pragma unroll 8
                        for (int L = 0; L < 32; ++L)
                            if (__shfl_sync(FULL, mk, L) == bkey[w]) first = false;
                    }
                    mine += inB[w] ? 1 : 0;
                    firsts += first ? 1 : 0;
                }
                const int nb = (int)__reduce_add_sync(FULL, (unsigned)mine);
                const int distinct = one_value ? 1 : (int)__reduce_add_sync(FULL, (unsigned)firsts);
                ties += nb - distinct;
                // assign, delete the rows, and let the other columns lose them
                uint32_t gone[NW];
#pragma unroll
                for (int wi = 0; wi < NW; ++wi) {
                    uint32_t bits = 0u;
#pragma unroll
                    for (int w = 0; w < NW; ++w)
                        if (inB[w] && (pic[w] >> 5) == wi) bits |= 1u << (pic[w] & 31);
                    gone[wi] = __reduce_or_sync(FULL, bits);
                }
#pragma unroll
                for (int wi = 0; wi < NW; ++wi)
                    if (lane == wi) dead[wi] |= gone[wi];
                __syncwarp();
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (inB[w]) {
                        newp[w] = pic[w];
                        alive[w] = false;
                    }
                }
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (!alive[w] || vc[w] == 0) continue;  // rows of the round are never pic[w]
                    int cnt = 0;
#pragma unroll
                    for (int wi = 0; wi < NW; ++wi) {
                        if (32 * wi >= n) continue;
                        uint32_t& m = emw(w, wi);
                        const uint32_t mv = m;
                        if (mv & gone[wi]) m = mv & ~gone[wi];
                        cnt += __popc(mv & ~gone[wi]);
                    }
                    vc[w] = cnt;
                    if (cnt == 0) vm[w] = v2[w];  // the maximum's rows are gone: the bound below it
                }
                step += nb;
                continue;
            }
        }

        // ---- one greedy step: the effective maximum of every owned column ----
        // mode: 0 the X(t) cell alone, 1 the plain maximum and the X(t) cell (equal),
        // 2 the plain maximum alone
        uint32_t key[NW];
        int cnt[NW], mode[NW];
        if (!cont_key) {
            bool need[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) need[w] = alive[w] && vc[w] == 0 && !(zin[w] && zv[w] > vm[w]);
            rebuild<NW, VT>(tile, dead, em, nwr, n, lane, pic, need, vm, vc, v2);
        }
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            key[w] = 0u;
            cnt[w] = 0;
            mode[w] = 0;
            if (!alive[w]) continue;
            float e;
            if (vc[w] == 0) {  // the X(t) cell above a stale bound, or nothing else left
                if (!zin[w]) continue;
                e = zv[w];
                cnt[w] = 1;
            } else if (zin[w] && zv[w] > vm[w]) {
                e = zv[w];
                cnt[w] = 1;
            } else if (zin[w] && zv[w] == vm[w]) {
                e = vm[w];
                cnt[w] = vc[w] + 1;
                mode[w] = 1;
            } else {
                e = vm[w];
                cnt[w] = vc[w];
                mode[w] = 2;
            }
            key[w] = fkey(e);
        }
        uint32_t lm = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) lm = max(lm, key[w]);
        const uint32_t gm = cont_key ? cont_key : __reduce_max_sync(FULL, lm);
        // the elements of M per column (c = lane + 32 w ascending); while every count
        // is below 8, three ballots of their low bits give each slot's total and every
        // lane's inclusive prefix without a shuffle scan
        int cm[NW];
        bool big = false;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            cm[w] = key[w] == gm ? cnt[w] : 0;
            big = big || cm[w] >= 8;
        }
        unsigned b0[NW], b1[NW], b2[NW];
        int tw[NW], tot = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            b0[w] = __ballot_sync(FULL, cm[w] & 1);
            b1[w] = __ballot_sync(FULL, cm[w] & 2);
            b2[w] = __ballot_sync(FULL, cm[w] & 4);
            tw[w] = __popc(b0[w]) + 2 * __popc(b1[w]) + 4 * __popc(b2[w]);
            tot += tw[w];
        }
        const bool wide = __any_sync(FULL, big);
        if (!wide && tot >= 2 && tot <= 32 * kGroupSlots) {
            // several cells at g: the steps at g run as one group
            if (tie_group<NW>(s, dead, em, em + nwr * nwr * 32, nwr, n, lane, pic, alive, zal, vm, vc, v2, newp, cm,
                              mode, b0, b1, b2, tw, tot, depth, use_ex, pis, swarm, t, step, ties, tu, tblk) < 0)
                return finish(ties);
            try_round = true;
            cont_key = 0u;
            continue;
        }
        int owner = -1, ow = 0, kk = 0;
        if (!wide) {
            int k = 0;
            if (tot > 1) {
                ++ties;
                if (s.tie_rule == 0) {
                    if ((step >> 2) != tblk) {  // one block of draws serves four steps
                        tu = draw(s.seed, pis, swarm, t, TAG_TIE, (uint32_t)(step >> 2));
                        tblk = step >> 2;
                    }
                    k = (int)below(word_of(tu, step & 3), (uint32_t)tot);
                }
            }
            int sel = -1;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (sel >= 0) continue;
                if (k < tw[w])
                    sel = w;
                else
                    k -= tw[w];
            }
            unsigned B0 = 0u, B1 = 0u, B2 = 0u;
            int c = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w)
                if (w == sel) {
                    B0 = b0[w];
                    B1 = b1[w];
                    B2 = b2[w];
                    c = cm[w];
                }
            const unsigned le = (2u << lane) - 1u;  // lanes 0 .. lane
            const int incl = __popc(B0 & le) + 2 * __popc(B1 & le) + 4 * __popc(B2 & le);
            owner = __ffs(__ballot_sync(FULL, sel >= 0 && incl > k)) - 1;
            ow = sel < 0 ? 0 : sel;
            kk = k - (incl - c);  // used by the owner only
        } else {
            tot = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) tot += (int)__reduce_add_sync(FULL, (unsigned)cm[w]);
            int k = 0;
            ++ties;
            if (s.tie_rule == 0) {
                if ((step >> 2) != tblk) {
                    tu = draw(s.seed, pis, swarm, t, TAG_TIE, (uint32_t)(step >> 2));
                    tblk = step >> 2;
                }
                k = (int)below(word_of(tu, step & 3), (uint32_t)tot);
            }
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (owner >= 0) continue;
                const int c = cm[w];
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                const int twid = __shfl_sync(FULL, incl, 31);
                if (k < twid) {
                    const unsigned bal = __ballot_sync(FULL, incl > k);
                    owner = __ffs(bal) - 1;
                    ow = w;
                    kk = __shfl_sync(FULL, k - (incl - c), owner);
                } else {
                    k -= twid;
                }
            }
        }
        // the owner takes the kk-th row (ascending) holding its column's maximum: the
        // rows of the mask, with the X(t) row when its cell is equal (mode 1)
        int r = -1, took_x = 0;
        if (lane == owner) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (w != ow) continue;
                if (mode[w] == 0) {
                    r = pic[w];
                } else {
                    int k = kk;
#pragma unroll
                    for (int wi = 0; wi < NW; ++wi) {
                        if (r >= 0 || 32 * wi >= n) continue;
                        uint32_t m = emw(w, wi);
                        if (mode[w] == 1 && (pic[w] >> 5) == wi) m |= 1u << (pic[w] & 31);
                        const int c = __popc(m);
                        if (k < c) {
                            for (int j = 0; j < k; ++j) m &= m - 1u;  // drop the k lower rows
                            r = 32 * wi + __ffs(m) - 1;
                        } else {
                            k -= c;
                        }
                    }
                }
                newp[w] = r;
                alive[w] = false;
                took_x = (zin[w] && r == pic[w]) ? 1 : 0;
                if (r >= 0 && r < n) dead[r >> 5] |= 1u << (r & 31);
            }
        }
        const int rx = __shfl_sync(FULL, (r & 0xFFFF) | (took_x << 16), owner < 0 ? 0 : owner);
        r = (int)(short)(rx & 0xFFFF);
        if (!use_ex) try_round = (rx >> 16) != 0;
        if (owner < 0 || r < 0 || r >= n) {  // cannot happen; never index with it
            if (lane == 0) atomicAdd(s.counters + CNT_ERR, 1ull);
            return finish(ties);
        }
        __syncwarp();
        // the other columns lose row r
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            if (!alive[w]) continue;
            if (r == pic[w]) {
                zal[w] = false;
            } else if (vc[w] > 0) {
                uint32_t& m = emw(w, r >> 5);
                const uint32_t bit = 1u << (r & 31), mv = m;
                if (mv & bit) {
                    m = mv & ~bit;
                    if (--vc[w] == 0) vm[w] = v2[w];  // the maximum's rows are gone: the bound below it
                }
            }
        }
        {
            bool plain_at_g = false;
#pragma unroll
            for (int w = 0; w < NW; ++w) plain_at_g = plain_at_g || (alive[w] && vc[w] > 0 && fkey(vm[w]) == gm);
            const bool same_ex = (step + 1 < depth) == use_ex;
            cont_key = (same_ex && __any_sync(FULL, plain_at_g)) ? gm : 0u;
        }
        ++step;
    }
    return finish(ties);
}

// The flat particle index f of a table of populations: the population and the
// particle inside it (f only grows along a warp's grid-stride loop).
struct TableCursor {
    int inst = 0;
    __device__ __forceinline__ int advance(const int32_t* prefix, int count, int f) {
        while (inst + 1 < count && prefix[inst + 1] <= f) ++inst;
        return f - prefix[inst];
    }
};

// Velocity (Eq. 4 + S_v) of one particle in its shared-memory tile, in place, by one
// warp: lane `lane` owns the columns j = lane + 32 c. W = clamp(c1 v) everywhere but
// at the rows X(t), P^L and P^G of a column (at most three), where the attraction
// terms enter; those cells are formed from exact splits and rounded once (eq4_cell),
// so they keep their relative accuracy when the terms cancel. Norm divides column j
// by the sum of |W| over the column (four interleaved partial sums, added pairwise);
// a zero column stays zero.
template <int NW, typename VT>
__device__ __noinline__ void velocity_in_tile(VT* tile, int n, int lane, const uint8_t* xrow, const uint8_t* plrow,
                                              const uint8_t* pgrow, float c1, float vmax, bool norm, Split a,
                                              Split b) {
    auto wgen = [&](float v) { return fminf(fmaxf(__fmul_rn(c1, v), -vmax), vmax); };
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        const int j = lane + 32 * c;
        if (j >= n) continue;
        const int px = xrow[j], pl = plrow[j], pg = pgrow[j];
        // the distinct special rows of the column and their values from V(t)
        int srow[3];
        float sval[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            int i = q == 0 ? px : (q == 1 ? pl : pg);
            if (q >= 1 && i == px) i = -1;
            if (q == 2 && i == pl) i = -1;
            srow[q] = i;
            sval[q] = 0.0f;
            if (i >= 0) {
                const int dl = (pl == i) - (px == i);
                const int dg = (pg == i) - (px == i);
                const float v = VStore<VT>::to_f(tile[i * n + j]);
                sval[q] = fminf(fmaxf(eq4_cell(exact_mul(c1, v), a, b, dl, dg), -vmax), vmax);
            }
        }
        float inv = 1.0f;
        if (norm) {
            float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
            int i = 0;
            for (; i + 3 < n; i += 4) {
                p0 += fabsf(wgen(VStore<VT>::to_f(tile[i * n + j])));
                p1 += fabsf(wgen(VStore<VT>::to_f(tile[(i + 1) * n + j])));
                p2 += fabsf(wgen(VStore<VT>::to_f(tile[(i + 2) * n + j])));
                p3 += fabsf(wgen(VStore<VT>::to_f(tile[(i + 3) * n + j])));
            }
            for (; i < n; ++i) p0 += fabsf(wgen(VStore<VT>::to_f(tile[i * n + j])));
            float sum = (p0 + p1) + (p2 + p3);
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (srow[q] >= 0) sum += fabsf(sval[q]) - fabsf(wgen(VStore<VT>::to_f(tile[srow[q] * n + j])));
            inv = sum > 0.0f ? 1.0f / sum : 1.0f;
        }
        for (int i = 0; i < n; ++i) {
            const float x = wgen(VStore<VT>::to_f(tile[i * n + j]));
            tile[i * n + j] = VStore<VT>::from_f(norm ? x * inv : x);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (srow[q] >= 0) tile[srow[q] * n + j] = VStore<VT>::from_f(norm ? sval[q] * inv : sval[q]);
    }
}

// Two adjacent columns per lane (n even): the same velocity as velocity_in_tile with
// 8-byte (fp32) or 4-byte (bf16) shared-memory accesses; lane `lane` owns columns
// 2 lane + 64 c and 2 lane + 64 c + 1. Column sums from four interleaved partial sums
// (rows mod 4, added pairwise); the write pass loads four rows before it stores them.
template <typename VT>
__device__ __noinline__ void velocity_pairs(VT* tile, int n, int lane, const uint8_t* xrow, const uint8_t* plrow,
                                            const uint8_t* pgrow, float c1, float vmax, bool norm, Split a,
                                            Split b) {
    auto wgen = [&](float v) { return fminf(fmaxf(__fmul_rn(c1, v), -vmax), vmax); };
    for (int j0 = 2 * lane; j0 < n; j0 += 64) {
        int srow[2][3];
        float sval[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + h;
            const int px = xrow[j], pl = plrow[j], pg = pgrow[j];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                int i = q == 0 ? px : (q == 1 ? pl : pg);
                if (q >= 1 && i == px) i = -1;
                if (q == 2 && i == pl) i = -1;
                srow[h][q] = i;
                sval[h][q] = 0.0f;
                if (i >= 0) {
                    const int dl = (pl == i) - (px == i);
                    const int dg = (pg == i) - (px == i);
                    const float v = VStore<VT>::to_f(tile[i * n + j]);
                    sval[h][q] = fminf(fmaxf(eq4_cell(exact_mul(c1, v), a, b, dl, dg), -vmax), vmax);
                }
            }
        }
        float inv0 = 1.0f, inv1 = 1.0f;
        // With Norm, the clamp of the plain cells is usually idle (|c1 v| <= v_max for
        // every v of the two columns): the first pass forms the column sums of |c1 v| and
        // the largest |c1 v|; only when that exceeds v_max are the sums formed again from
        // the clamped values. Either way the sums and the stored values are those of
        // clamp(c1 v).
        bool unclamped = false;
        if (norm) {
            float px[4] = {0.f, 0.f, 0.f, 0.f}, py[4] = {0.f, 0.f, 0.f, 0.f};
            float mxy = 0.0f;
            int i = 0;
            for (; i + 3 < n; i += 4) {
                float x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) Pair<VT>::get(tile + (i + u) * n + j0, x[u], y[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 g = fmul2_rn(make_float2(x[u], y[u]), make_float2(c1, c1));
                    const float gx = fabsf(g.x), gy = fabsf(g.y);
                    px[u] += gx;
                    py[u] += gy;
                    mxy = fmaxf(mxy, fmaxf(gx, gy));
                }
            }
            for (; i < n; ++i) {
                float x0, y0;
                Pair<VT>::get(tile + i * n + j0, x0, y0);
                const float gx = fabsf(__fmul_rn(c1, x0)), gy = fabsf(__fmul_rn(c1, y0));
                px[0] += gx;
                py[0] += gy;
                mxy = fmaxf(mxy, fmaxf(gx, gy));
            }
            unclamped = mxy <= vmax;
            if (!unclamped) {
#pragma unroll
                for (int u = 0; u < 4; ++u) px[u] = py[u] = 0.0f;
                i = 0;
                for (; i + 3 < n; i += 4) {
                    float x[4], y[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) Pair<VT>::get(tile + (i + u) * n + j0, x[u], y[u]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        px[u] += fabsf(wgen(x[u]));
                        py[u] += fabsf(wgen(y[u]));
                    }
                }
                for (; i < n; ++i) {
                    float x0, y0;
                    Pair<VT>::get(tile + i * n + j0, x0, y0);
                    px[0] += fabsf(wgen(x0));
                    py[0] += fabsf(wgen(y0));
                }
            }
            float s0 = (px[0] + px[1]) + (px[2] + px[3]), s1 = (py[0] + py[1]) + (py[2] + py[3]);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (srow[0][q] >= 0)
                    s0 += fabsf(sval[0][q]) - fabsf(wgen(VStore<VT>::to_f(tile[srow[0][q] * n + j0])));
                if (srow[1][q] >= 0)
                    s1 += fabsf(sval[1][q]) - fabsf(wgen(VStore<VT>::to_f(tile[srow[1][q] * n + j0 + 1])));
            }
            inv0 = s0 > 0.0f ? 1.0f / s0 : 1.0f;
            inv1 = s1 > 0.0f ? 1.0f / s1 : 1.0f;
        }
        int i = 0;
        if (unclamped) {
            for (; i + 3 < n; i += 4) {
                float x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) Pair<VT>::get(tile + (i + u) * n + j0, x[u], y[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 g = fmul2_rn(fmul2_rn(make_float2(x[u], y[u]), make_float2(c1, c1)),
                                              make_float2(inv0, inv1));
                    Pair<VT>::put(tile + (i + u) * n + j0, g.x, g.y);
                }
            }
        }
        for (; i + 3 < n; i += 4) {
            float x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) Pair<VT>::get(tile + (i + u) * n + j0, x[u], y[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float gx = wgen(x[u]), gy = wgen(y[u]);
                Pair<VT>::put(tile + (i + u) * n + j0, norm ? gx * inv0 : gx, norm ? gy * inv1 : gy);
            }
        }
        for (; i < n; ++i) {
            float x, y;
            Pair<VT>::get(tile + i * n + j0, x, y);
            x = wgen(x);
            y = wgen(y);
            Pair<VT>::put(tile + i * n + j0, norm ? x * inv0 : x, norm ? y * inv1 : y);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (srow[0][q] >= 0) tile[srow[0][q] * n + j0] = VStore<VT>::from_f(norm ? sval[0][q] * inv0 : sval[0][q]);
            if (srow[1][q] >= 0)
                tile[srow[1][q] * n + j0 + 1] = VStore<VT>::from_f(norm ? sval[1][q] * inv1 : sval[1][q]);
        }
    }
}

// One particle iteration's update of every particle of the table, one warp per
// particle: the V tile is staged in shared memory with one bulk copy; S_x
// (SecondTarget, Algorithm 1, or PickColumn) runs on Y = X(t) + V(t) and the velocity
// of Eq. 4 replaces the tile in place (the other order when the population forms
// X(t) + V(t+1)); one bulk copy stores V(t+1). V is read from memory once and written
// once per iteration. Shared-memory slots are sized for the largest n of the table;
// particles are handed out one at a time from a counter (their cost varies with the
// ties of the greedy), else in a fixed grid-stride order. The discretisation entry
// point (sx_only) runs S_x alone on Y.
// Blocks per SM the update kernel is compiled for (n <= 64): fp32 tiles (16 KB at
// n = 64) let shared memory hold three 4-warp blocks, and the registers are capped so
// that three fit; bf16 tiles (8 KB) leave room for more than four, so the registers
// are capped at 128 per thread to let four blocks (16 warps) run. Larger n keep the
// registers they need.
template <int NW, typename VT>
struct UpdBlocks {
    static constexpr int kMin = NW <= 2 ? 3 : 1;
};
template <int NW>
struct UpdBlocks<NW, __nv_bfloat16> {
    static constexpr int kMin = NW <= 2 ? 4 : 1;
};

template <int NW, typename VT>
__global__ void __launch_bounds__(kWarps * 32, UpdBlocks<NW, VT>::kMin)
    k_update(const StateView* __restrict__ views, const int32_t* __restrict__ prefix, int count, int n_max,
             int32_t* __restrict__ work) {
    const int wpc = blockDim.x >> 5;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem) + warp;
    unsigned char* wbase = smem + kBarBytes + warp * warp_bytes<VT>(n_max);
    VT* tile = reinterpret_cast<VT*>(wbase);
    uint32_t* dead = reinterpret_cast<uint32_t*>(wbase + tile_bytes<VT>(n_max));
    uint32_t* em = reinterpret_cast<uint32_t*>(wbase + tile_bytes<VT>(n_max) + 32 + lists_bytes(n_max));
    const int nwr = (n_max + 31) >> 5;
    if (lane == 0) mbar_init(bar, 1);
    __syncwarp();
    uint32_t phase = 0;
    const int total = prefix[count];
    TableCursor cur;

    auto grab = [&](int fixed) {
        if (!work) return fixed;
        int q = 0;
        if (lane == 0) q = atomicAdd(work, 1);
        return __shfl_sync(FULL, q, 0);
    };
    int fnext = total;
    for (int f = grab(blockIdx.x * wpc + warp); f < total; f = fnext) {
        const int p = cur.advance(prefix, count, f);
        const StateView s = views[cur.inst];
        const int n = s.n;
        const uint32_t t = (uint32_t)*s.t;
        const uint32_t tbytes = (uint32_t)tile_bytes<VT>(n);
        const bool sx_only = s.sx_only != 0;
        const int lsw = p / s.ss;  // the swarm in this population; draws use its index in the run
        const uint32_t swarm = sx_only ? (uint32_t)s.sx_swarm[p] : (uint32_t)(s.swarm_base + lsw);
        const uint32_t pis = sx_only ? (uint32_t)s.sx_pis[p] : (uint32_t)(p % s.ss);
        VT* Vg = reinterpret_cast<VT*>(s.V) + (size_t)p * s.vstride;
        // the tile -> shared memory with one bulk copy (tile padded to 16 bytes), once
        // the store of the previous particle has finished reading it
        __syncwarp();
        if (lane == 0) {
            bulk_wait_read();
            fence_proxy_async();
            bulk_load(tile, Vg, tbytes, bar);
        }
        int pic[NW], newp[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int j = lane + 32 * w;
            pic[w] = j < n ? s.X[(size_t)p * s.ps + j] : -1;
            newp[w] = 0;
        }
        // the velocity's inputs are loaded when it runs, so that nothing of it stays
        // live across S_x
        auto velocity = [&]() {
            const U4 ur = draw(s.seed, pis, swarm, t, TAG_R, 0u);  // r2, r3: one draw per particle
            const Split a = exact_mul(s.c2, u01f(ur.x)), b = exact_mul(s.c3, u01f(ur.y));
            if ((n & 1) == 0)  // rows start on 8 (fp32) or 4 (bf16) bytes: paired columns
                velocity_pairs<VT>(tile, n, lane, s.X + (size_t)p * s.ps, s.PL + (size_t)p * s.ps,
                                   s.PG + (size_t)lsw * s.ps, s.c1, s.v_max, s.sv_kind == 1, a, b);
            else
                velocity_in_tile<NW, VT>(tile, n, lane, s.X + (size_t)p * s.ps, s.PL + (size_t)p * s.ps,
                                         s.PG + (size_t)lsw * s.ps, s.c1, s.v_max, s.sv_kind == 1, a, b);
        };
        const bool ok = mbar_wait(bar, phase);
        if (!__all_sync(FULL, ok)) {  // the copy did not land in time: record, leave this warp
            if (lane == 0) {
                atomicAdd(s.counters + CNT_ERR, 1ull);
                mbar_wait(bar, phase);  // one more bounded wait for a load still in flight
                bulk_wait_all();
            }
            return;
        }
        phase ^= 1u;
        const bool new_v = !sx_only && s.pos_uses_new_v != 0;
        if (new_v) {  // X(t) + V(t+1): the velocity first
            velocity();
            __syncwarp();
        }
        // X(t) + V: the X(t) cell of each column is the tile value + 1; Y itself in
        // the discretisation entry point
        const float zadd = sx_only ? 0.0f : 1.0f;
        const int ties = s.sx_kind == 1
                             ? pick_column<NW, VT>(s, tile, dead, reinterpret_cast<uint8_t*>(dead + 8), n, lane, pic,
                                                   pis, swarm, t, zadd, newp)
                             : second_target<NW, VT>(s, tile, dead, em, nwr, n, lane, pic, pis, swarm, t, zadd,
                                                     newp);
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int j = lane + 32 * w;
            if (j < n) s.Xsx[(size_t)p * s.ps + j] = (uint8_t)newp[w];
        }
        if (lane == 0 && ties) atomicAdd(s.counters + CNT_TIES, (unsigned long long)ties);
        // the warp's next particle, taken once S_x is done: its tile is fetched into L2
        // while the velocity and the store of this one run
        fnext = grab(f + gridDim.x * wpc);
        if (lane == 0 && fnext < total) {
            TableCursor nc = cur;
            const int pn = nc.advance(prefix, count, fnext);
            const StateView* sv = views + nc.inst;
            bulk_prefetch_l2(reinterpret_cast<const VT*>(sv->V) + (size_t)pn * sv->vstride,
                             (uint32_t)tile_bytes<VT>(sv->n));
        }
        if (s.ord_cnt) {  // the search's hand-out order: bucket of the distance moved
            int d = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) d += __popc(__ballot_sync(FULL, lane + 32 * w < n && newp[w] != pic[w]));
            if (lane == 0) {
                const int b = ord_bucket(d);
                const int slot = atomicAdd(s.ord_cnt + b, 1);
                if (slot < s.P) s.ord_list[(size_t)b * s.P + slot] = p;  // else the search keeps index order
            }
        }
        if (!sx_only) {
            __syncwarp();  // S_x has read the tile
            if (!new_v) velocity();
            fence_proxy_async();  // this lane's tile writes, before the bulk store reads them
            __syncwarp();
            if (lane == 0) bulk_store(Vg, tile, tbytes);
        }
        __syncwarp();
    }
    if (lane == 0) bulk_wait_all();
}

template <int NW, typename VT>
cudaError_t launch_upd(const VsxLaunch& L, cudaStream_t st) {
    int wpc = L.warps > 0 ? L.warps : kWarps;  // warps (particles) per CTA
    if (wpc > kWarps) wpc = kWarps;
    while (wpc > 1 && kBarBytes + wpc * warp_bytes<VT>(L.n_max) > kSmemLimit) --wpc;
    const size_t smem = kBarBytes + wpc * warp_bytes<VT>(L.n_max);
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = configure_once<k_update<NW, VT>>();
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    int per_sm = occupancy_cached<k_update<NW, VT>>(wpc * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    const int need = (L.total + wpc - 1) / wpc;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (L.d_work) {
        e = cudaMemsetAsync(L.d_work, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return e;
    }
    k_update<NW, VT><<<grid, wpc * 32, smem, st>>>(L.d_views, L.d_prefix, L.count, L.n_max, L.d_work);
    return cudaGetLastError();
}

template <typename VT>
cudaError_t launch_upd_t(const VsxLaunch& L, cudaStream_t st) {
    switch ((L.n_max + 31) / 32) {
        case 1: return launch_upd<1, VT>(L, st);
        case 2: return launch_upd<2, VT>(L, st);
        case 3: return launch_upd<3, VT>(L, st);
        case 4: return launch_upd<4, VT>(L, st);
        case 5: return launch_upd<5, VT>(L, st);
        case 6:
        case 7:
        case 8: return launch_upd<8, VT>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int velocity_sx_max_n(int v_bf16) {
    int n = 2;
    while (n < 256 && kBarBytes + (v_bf16 ? warp_bytes<__nv_bfloat16>(n + 1) : warp_bytes<float>(n + 1)) <=
                          kSmemLimit)
        ++n;
    return n;
}

cudaError_t launch_init(const StateView& s, int v_bf16, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = (s.P + kWarps - 1) / kWarps;
    if (grid > sms * 8) grid = sms * 8;
    if (v_bf16)
        k_init<__nv_bfloat16><<<grid, kWarps * 32, 0, st>>>(s);
    else
        k_init<float><<<grid, kWarps * 32, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_velocity_sx(const VsxLaunch& L, cudaStream_t st) {
    if (L.total <= 0) return cudaSuccess;
    if (L.n_max > velocity_sx_max_n(L.v_bf16)) return cudaErrorInvalidValue;
    return L.v_bf16 ? launch_upd_t<__nv_bfloat16>(L, st) : launch_upd_t<float>(L, st);
}

}  // namespace qap
