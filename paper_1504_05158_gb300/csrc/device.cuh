// Device-side building blocks shared by the kernels of the PSO iteration:
// the Philox4x32-10 counter-based generator, the float ordering key used by the
// S_x argmax, storage-format conversions, and the device view of a state.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace qap {

constexpr unsigned FULL = 0xFFFFFFFFu;

// ----------------------------------------------------------------------- RNG
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round takes
// the 64-bit products of words 0 and 2 with two odd constants, mixes their high
// halves with words 1 and 3 and the round key, and advances the key by two Weyl
// increments. key = (seed low, seed high); counter = (c0, c1, c2, tag<<24 | block).
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = mulhi32(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = mulhi32(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

enum : uint32_t { TAG_R = 0, TAG_TIE = 1, TAG_INIT_X = 2, TAG_INIT_V = 3, TAG_MIG = 4, TAG_COLUMNS = 7 };

__host__ __device__ __forceinline__ U4 draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                             uint32_t tag, uint32_t block) {
    return philox(c0, c1, c2, (tag << 24) | (block & 0xFFFFFFu), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(const U4& u, int i) {
    return i == 0 ? u.x : (i == 1 ? u.y : (i == 2 ? u.z : u.w));
}

// top 24 bits as a fraction in [0, 1); exact in fp32
__device__ __forceinline__ float u01f(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }
// floor(u * k / 2^32) in [0, k)
__host__ __device__ __forceinline__ uint32_t below(uint32_t u, uint32_t k) {
    return (uint32_t)(((uint64_t)u * (uint64_t)k) >> 32);
}

// ------------------------------------------------ Eq. 4 at one cell, exactly
// A product of two fp32 values held exactly as hi + lo (hi rounded, lo = the
// rounding error, recovered by one fused multiply-add).
struct Split {
    float hi, lo;
};
__device__ __forceinline__ Split exact_mul(float x, float y) {
    const float h = __fmul_rn(x, y);
    return Split{h, __fmaf_rn(x, y, -h)};
}
// s = fl(x + y) and the rounding error x + y - s (Knuth's two-sum, six additions).
__device__ __forceinline__ float two_sum(float x, float y, float& err) {
    const float s = __fadd_rn(x, y);
    const float bp = __fsub_rn(s, x);
    err = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bp)), __fsub_rn(y, bp));
    return s;
}
// c1 v + dl a + dg b for dl, dg in {-1, 0, 1} (the only values the differences of
// permutation-matrix entries take in Eq. 4), with c1 v, a and b given as exact
// splits: the hi parts are summed with error-free two-sums and every error term is
// added back before the one final rounding (Ogita, Rump and Oishi's Sum2). The
// result is the exact value rounded once, up to u^2 (u = 2^-24) of the terms, so it
// keeps its relative accuracy when the terms cancel.
__device__ __forceinline__ float eq4_cell(Split p, Split a, Split b, int dl, int dg) {
    const float ah = dl == 0 ? 0.0f : (dl > 0 ? a.hi : -a.hi);
    const float al = dl == 0 ? 0.0f : (dl > 0 ? a.lo : -a.lo);
    const float bh = dg == 0 ? 0.0f : (dg > 0 ? b.hi : -b.hi);
    const float bl = dg == 0 ? 0.0f : (dg > 0 ? b.lo : -b.lo);
    float e1, e2;
    const float s1 = two_sum(p.hi, ah, e1);
    const float s2 = two_sum(s1, bh, e2);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(p.lo, al), __fadd_rn(bl, e1)), e2);
    return __fadd_rn(s2, lo);
}

// --------------------------------------------------------------- float keys
// Monotone map float -> uint32 (larger float, larger key); +0 and -0 share a key;
// no finite float maps to 0, which marks "nothing".
__device__ __forceinline__ uint32_t fkey(float f) {
    uint32_t b = __float_as_uint(f == 0.0f ? 0.0f : f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// ---------------------------------------------------------- storage formats
template <typename VT>
struct VStore;
template <>
struct VStore<float> {
    static __device__ __forceinline__ float load(const float* p) { return *p; }
    static __device__ __forceinline__ float to_f(float v) { return v; }
    static __device__ __forceinline__ float from_f(float v) { return v; }
};
template <>
struct VStore<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
};

// ------------------------------------------------- mbarrier + 1-D bulk copies
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// orders this thread's earlier generic-proxy shared-memory accesses before later
// bulk (async-proxy) copies that touch the same bytes
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned); completion is signalled on `bar` as transaction bytes
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// shared -> global bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), committed as one bulk group of the issuing thread
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// waits until the issuing thread's bulk stores have finished reading shared memory
// (a.x b.x, a.y b.y), each product rounded to nearest like __fmul_rn, in one
// paired fp32 instruction
__device__ __forceinline__ float2 fmul2_rn(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x)),
          "l"(((unsigned long long)__float_as_uint(b.y) << 32) | __float_as_uint(b.x)));
    return make_float2(__uint_as_float((uint32_t)d), __uint_as_float((uint32_t)(d >> 32)));
}

// A hint that brings `bytes` (a multiple of 16, from a 16-byte aligned address) of
// global memory into L2 ahead of a later bulk load.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// waits until the issuing thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// waits for phase `parity` of `bar` to complete; gives up after a bounded number of
// polls and returns false (the caller records an error instead of hanging)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    uint32_t sleep_ns = 32;
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it >= 4) {  // back off: leave the issue slots to other warps
            __nanosleep(sleep_ns);
            if (sleep_ns < 256) sleep_ns <<= 1;
        }
    }
    return false;
}

// ------------------------------------------------------------ device state
// Everything one iteration touches, by value in each kernel's arguments. Pointers
// never change after pso_init, so captured graphs stay valid.
struct StateView {
    int32_t n, m, ss, P;
    int32_t swarm_base;  // index of swarm 0 of this population in the whole run (a part of a
                         // run split over processes); the Philox counters use base + local
    int32_t ps;       // bytes between consecutive permutations (>= n, multiple of 16)
    int64_t vstride;  // elements between consecutive particles' V tiles (multiple of 8)
    void* V;          // P tiles of n x n, row = location, column = facility
    uint8_t* X;       // current positions
    uint8_t* Xsx;     // S_x results of the running iteration
    uint8_t* PL;
    int64_t* costL;
    int64_t* cost;
    int32_t* moves;   // per particle, last iteration
    int32_t* rounds;  // per particle, last iteration
    uint8_t* PG;      // m swarm bests
    uint8_t* PG2;     // ring snapshot
    int64_t* costG;
    int64_t* costG2;
    uint8_t* best;
    int64_t* best_cost;
    int32_t* best_iter;
    int32_t* t;       // completed iterations (device-resident so graph replays advance it)
    unsigned long long* counters;
    uint64_t seed;
    float c1, c2, c3, v_max;
    int32_t sv_kind, sx_rule, depth, tie_rule, pos_uses_new_v, sx_kind;
    int32_t ls_max_moves, mig_kind, mig_depth, mig_period, ring_if_better;
    // S_x alone (the discretisation entry point): V holds Y itself, X holds Z, and
    // the Philox counters of particle p are (sx_pis[p], sx_swarm[p], *t)
    int32_t sx_only;
    const int32_t* sx_swarm;
    const int32_t* sx_pis;
    // The order in which the iteration's search hands out particles (null: index
    // order). The update kernel appends particle p to list ord_list[b P ..] of bucket
    // b = ord_bucket(d), d the number of positions where S_x moved p away from X(t);
    // the search takes the buckets from the highest down (a particle moved far from its
    // last local optimum tends to need many moves); k_bests zeroes the counts.
    int32_t* ord_cnt;   // kOrdBuckets counts
    int32_t* ord_list;  // kOrdBuckets x P particle indices
    int32_t ord_resets; // counts k_bests zeroes from ord_cnt on (those of the parts too)
};

constexpr int kOrdBuckets = 8;
__host__ __device__ inline int ord_bucket(int d) {
    return d <= 2 ? 0 : d <= 4 ? 1 : d <= 6 ? 2 : d <= 8 ? 3 : d <= 12 ? 4 : d <= 16 ? 5 : d <= 24 ? 6 : 7;
}

// counters[CNT_ERR] counts internal consistency failures (a kernel that detects one
// skips the access instead of faulting; the host reports it).
enum { CNT_PIT = 0, CNT_MOVES, CNT_ROUNDS, CNT_DELTA_FULL, CNT_DELTA_INCR, CNT_TIES, CNT_ERR, CNT_N };

}  // namespace qap
