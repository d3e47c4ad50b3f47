// Initialisation and the velocity/position update of every particle, one warp
// per particle, the particle's n x n velocity tile staged in shared memory.
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
// 2^32) with u from Philox. Lanes own columns and keep each column's maximum key
// and multiplicity over the remaining rows, so a step costs one warp reduction
// plus the columns whose maximum sat in the deleted row.
#include <climits>

#include "kernels.h"

namespace qap {
namespace {

constexpr int kWarps = 4;
constexpr size_t kSmemLimit = 227 * 1024;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename VT>
__host__ __device__ inline size_t tile_bytes(int n) {
    return align16((size_t)n * n * sizeof(VT));
}
template <typename VT>
__host__ __device__ inline size_t warp_bytes(int n) {
    return tile_bytes<VT>(n) + align16((size_t)n);
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
        const uint32_t swarm = (uint32_t)(p / s.ss), pis = (uint32_t)(p % s.ss);
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
template <int NW, typename VT>
__device__ __forceinline__ float yval(const VT* tile, int n, int i, int col, int pic) {
    return VStore<VT>::to_f(tile[i * n + col]) + (pic == i ? 1.0f : 0.0f);
}

// maximum key and its multiplicity over the remaining rows of one column
template <typename VT>
__device__ __forceinline__ void col_scan(const VT* tile, const uint8_t* rowdead, int n, int col,
                                         int pic, int exrow, uint32_t& key, int& cnt) {
    uint32_t mx = 0;
    int c = 0;
    for (int i = 0; i < n; ++i) {
        if (rowdead[i] || i == exrow) continue;
        const uint32_t k = fkey(VStore<VT>::to_f(tile[i * n + col]) + (pic == i ? 1.0f : 0.0f));
        if (k > mx) {
            mx = k;
            c = 1;
        } else if (k == mx) {
            ++c;
        }
    }
    key = mx;
    cnt = c;
}

template <int NW, typename VT>
__global__ void __launch_bounds__(kWarps * 32) k_velocity_sx(StateView s) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = s.n;
    VT* tile = reinterpret_cast<VT*>(smem + warp * warp_bytes<VT>(n));
    uint8_t* rowdead = smem + warp * warp_bytes<VT>(n) + tile_bytes<VT>(n);
    const uint32_t t = (uint32_t)*s.t;
    const bool norm = s.sv_kind == 1;

    for (int p = blockIdx.x * kWarps + warp; p < s.P; p += gridDim.x * kWarps) {
        const uint32_t swarm = (uint32_t)(p / s.ss), pis = (uint32_t)(p % s.ss);
        int pic[NW], plc[NW], pgc[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int j = lane + 32 * w;
            pic[w] = j < n ? s.X[(size_t)p * s.ps + j] : -1;
            plc[w] = j < n ? s.PL[(size_t)p * s.ps + j] : -1;
            pgc[w] = j < n ? s.PG[(size_t)swarm * s.ps + j] : -1;
        }
        // stage V(t) in shared memory (16-byte chunks; the tile is padded to 16 bytes)
        VT* Vg = reinterpret_cast<VT*>(s.V) + (size_t)p * s.vstride;
        {
            const uint4* src = reinterpret_cast<const uint4*>(Vg);
            uint4* dst = reinterpret_cast<uint4*>(tile);
            const int chunks = (int)(tile_bytes<VT>(n) / 16);
            for (int c = lane; c < chunks; c += 32) dst[c] = src[c];
        }
        for (int i = lane; i < n; i += 32) rowdead[i] = 0;
        __syncwarp();

        // ---- Eq. 4 ----
        const U4 ur = draw(s.seed, pis, swarm, t, TAG_R, 0u);
        const float a = s.c2 * u01f(ur.x), b = s.c3 * u01f(ur.y);
        float inv[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) inv[w] = 1.0f;
        if (norm) {
            float sum[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) sum[w] = 0.0f;
            for (int i = 0; i < n; ++i) {
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int j = lane + 32 * w;
                    if (j < n) {
                        const float v = VStore<VT>::to_f(tile[i * n + j]);
                        const float dl = (float)((plc[w] == i) - (pic[w] == i));
                        const float dg = (float)((pgc[w] == i) - (pic[w] == i));
                        float x = fmaf(s.c1, v, a * dl + b * dg);
                        x = fminf(fmaxf(x, -s.v_max), s.v_max);
                        sum[w] += fabsf(x);
                    }
                }
            }
#pragma unroll
            for (int w = 0; w < NW; ++w) inv[w] = sum[w] > 0.0f ? 1.0f / sum[w] : 1.0f;
        }
        const bool newv = s.pos_uses_new_v != 0;
        for (int i = 0; i < n; ++i) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int j = lane + 32 * w;
                if (j < n) {
                    const float v = VStore<VT>::to_f(tile[i * n + j]);
                    const float dl = (float)((plc[w] == i) - (pic[w] == i));
                    const float dg = (float)((pgc[w] == i) - (pic[w] == i));
                    float x = fmaf(s.c1, v, a * dl + b * dg);
                    x = fminf(fmaxf(x, -s.v_max), s.v_max);
                    if (norm) x *= inv[w];
                    const VT o = VStore<VT>::from_f(x);
                    Vg[i * n + j] = o;
                    if (newv) tile[i * n + j] = o;
                }
            }
        }
        __syncwarp();

        // ---- Eq. 5: SecondTarget on Y = X(t) + V ----
        const int depth = s.depth;
        int exrow[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) exrow[w] = -1;
        if (depth > 0) {
            if (s.sx_rule == 0) {
#pragma unroll
                for (int w = 0; w < NW; ++w) exrow[w] = pic[w];
            } else {
                uint32_t zk[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    zk[w] = pic[w] >= 0 ? fkey(yval<NW, VT>(tile, n, pic[w], lane + 32 * w, pic[w])) : 0u;
                for (int d = 0; d < depth; ++d) {
                    uint32_t lm = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w)
                        if (exrow[w] < 0 && zk[w] > lm) lm = zk[w];
                    const uint32_t gm = __reduce_max_sync(FULL, lm);
                    bool done = false;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        if (done) continue;
                        const unsigned bal = __ballot_sync(FULL, exrow[w] < 0 && pic[w] >= 0 && zk[w] == gm);
                        if (bal) {
                            if (lane == __ffs(bal) - 1) exrow[w] = pic[w];
                            done = true;
                        }
                    }
                }
            }
        }
        uint32_t ckey[NW];
        int ccnt[NW], newp[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            newp[w] = 0;
            ckey[w] = 0;
            ccnt[w] = 0;
            if (pic[w] >= 0)
                col_scan<VT>(tile, rowdead, n, lane + 32 * w, pic[w], depth > 0 ? exrow[w] : -1,
                             ckey[w], ccnt[w]);
        }
        int ties = 0;
        for (int step = 0; step < n; ++step) {
            if (step == depth && depth > 0) {
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    if (ckey[w]) col_scan<VT>(tile, rowdead, n, lane + 32 * w, pic[w], -1, ckey[w], ccnt[w]);
            }
            uint32_t lm = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) lm = ckey[w] > lm ? ckey[w] : lm;
            const uint32_t gm = __reduce_max_sync(FULL, lm);
            int lc = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) lc += (ckey[w] == gm) ? ccnt[w] : 0;
            const int tot = (int)__reduce_add_sync(FULL, (unsigned)lc);
            int k = 0;
            if (tot > 1) {
                ++ties;
                if (s.tie_rule == 0) {
                    const U4 u = draw(s.seed, pis, swarm, t, TAG_TIE, (uint32_t)(step >> 2));
                    k = (int)below(word_of(u, step & 3), (uint32_t)tot);
                }
            }
            // the column holding the k-th element of M (columns j = lane + 32 w ascending)
            int owner = -1, ow = 0, kk = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (owner >= 0) continue;
                const int c = (ckey[w] == gm) ? ccnt[w] : 0;
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                const int tw = __shfl_sync(FULL, incl, 31);
                if (k < tw) {
                    const unsigned bal = __ballot_sync(FULL, incl > k);
                    owner = __ffs(bal) - 1;
                    ow = w;
                    kk = __shfl_sync(FULL, k - (incl - c), owner);
                } else {
                    k -= tw;
                }
            }
            // the owner lane finds the kk-th such row (ascending)
            int r = -1;
            const bool use_ex = step < depth;
            if (lane == owner) {
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (w != ow) continue;
                    const int col = lane + 32 * w;
                    int seen = 0;
                    for (int i = 0; i < n; ++i) {
                        if (rowdead[i] || (use_ex && i == exrow[w])) continue;
                        if (fkey(yval<NW, VT>(tile, n, i, col, pic[w])) == gm) {
                            if (seen == kk) {
                                r = i;
                                break;
                            }
                            ++seen;
                        }
                    }
                    newp[w] = r;
                    ckey[w] = 0;
                    ccnt[w] = 0;
                }
            }
            r = __shfl_sync(FULL, r, owner < 0 ? 0 : owner);
            if (owner < 0 || r < 0 || r >= n) {  // cannot happen; never index with it
                if (lane == 0) atomicAdd(s.counters + CNT_ERR, 1ull);
                break;
            }
            if (lane == 0) rowdead[r] = 1;
            __syncwarp();
            // columns whose maximum sat in row r lose one of its copies
            if (!(step + 1 == depth)) {
                const bool ex_next = step + 1 < depth;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (!ckey[w]) continue;
                    if (ex_next && r == exrow[w]) continue;
                    const uint32_t kr = fkey(yval<NW, VT>(tile, n, r, lane + 32 * w, pic[w]));
                    if (kr == ckey[w] && --ccnt[w] == 0)
                        col_scan<VT>(tile, rowdead, n, lane + 32 * w, pic[w], ex_next ? exrow[w] : -1,
                                     ckey[w], ccnt[w]);
                }
            }
        }
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int j = lane + 32 * w;
            if (j < n) s.Xsx[(size_t)p * s.ps + j] = (uint8_t)newp[w];
        }
        if (lane == 0 && ties) atomicAdd(s.counters + CNT_TIES, (unsigned long long)ties);
        __syncwarp();
    }
}

template <int NW, typename VT>
cudaError_t launch_vsx(const StateView& s, cudaStream_t st) {
    const size_t smem = kWarps * warp_bytes<VT>(s.n);
    int warps = kWarps;
    if (smem > kSmemLimit) return cudaErrorInvalidValue;
    (void)warps;
    cudaError_t e = cudaFuncSetAttribute(k_velocity_sx<NW, VT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_velocity_sx<NW, VT>, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    const int need = (s.P + kWarps - 1) / kWarps;
    if (grid > need) grid = need;
    k_velocity_sx<NW, VT><<<grid, kWarps * 32, smem, st>>>(s);
    return cudaGetLastError();
}

template <typename VT>
cudaError_t launch_vsx_t(const StateView& s, cudaStream_t st) {
    switch ((s.n + 31) / 32) {
        case 1: return launch_vsx<1, VT>(s, st);
        case 2: return launch_vsx<2, VT>(s, st);
        case 3: return launch_vsx<3, VT>(s, st);
        case 4: return launch_vsx<4, VT>(s, st);
        case 5: return launch_vsx<5, VT>(s, st);
        case 6: return launch_vsx<6, VT>(s, st);
        case 7: return launch_vsx<7, VT>(s, st);
        case 8: return launch_vsx<8, VT>(s, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int velocity_sx_max_n(int v_bf16) {
    int n = 2;
    while (n < 256 && kWarps * (v_bf16 ? warp_bytes<__nv_bfloat16>(n + 1) : warp_bytes<float>(n + 1)) <=
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

cudaError_t launch_velocity_sx(const StateView& s, int v_bf16, cudaStream_t st) {
    if (s.n > velocity_sx_max_n(v_bf16)) return cudaErrorInvalidValue;
    return v_bf16 ? launch_vsx_t<__nv_bfloat16>(s, st) : launch_vsx_t<float>(s, st);
}

}  // namespace qap
