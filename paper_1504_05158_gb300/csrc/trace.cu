// Per-iteration statistics of section 4.2 recorded on the device: after the
// bookkeeping of every iteration, the percentile ranks (nearest rank, 5/25/50/75 %)
// of the current costs of the whole population and of every swarm (Figs. 4 and 5),
// and the histogram of the population's costs (the probability mass function of
// Figs. 6 and 7, times the particle count), into a ring of records that the host
// reads once.
//
// Record layout (int64 words), len = 9 + 8 m + bins + 2:
//   [0]                 completed iterations t when recorded (the record's stamp)
//   [1 .. 8]            population: min, p5, p25, p50, p75, max, sum (low word, high word)
//   [9 + 8 k .. +8]     swarm k: the same eight words
//   [9 + 8 m ..]        histogram: below lo, bins equal-width bins of [lo, hi), at or above hi
// The record of iteration t goes to slot (t - 1) mod capacity; the host orders the
// slots by their stamps.
//
// One launch of m + 1 CTAs, none waiting for another: CTA k < m sorts swarm k's costs
// in shared memory (bitonic); CTA m computes the population's figures (percentiles by
// a radix selection over the costs) and its histogram.
#include <algorithm>
#include <climits>
#include <utility>
#include <vector>

#include "launch.cuh"
#include "state.h"

namespace qap {
namespace {

constexpr int kThreads = 1024;
constexpr int kMaxSort = 16384;  // swarm sizes up to this are sorted in shared memory
constexpr int kBuckets = 2048;

__device__ __forceinline__ __int128 block_sum128(__int128 v, long long* part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long lo = __shfl_xor_sync(FULL, (long long)(unsigned long long)v, o);
        const long long hi = __shfl_xor_sync(FULL, (long long)(v >> 64), o);
        v += (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | (unsigned long long)lo);
    }
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        part[2 * w] = (long long)(unsigned long long)v;
        part[2 * w + 1] = (long long)(v >> 64);
    }
    __syncthreads();
    __int128 t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
        t += (__int128)(((unsigned __int128)(unsigned long long)part[2 * i + 1] << 64) |
                        (unsigned long long)part[2 * i]);
    return t;
}

__device__ __forceinline__ long long rank_of(int pct, int count) {  // ceil(pct count / 100)
    return ((long long)pct * count + 99) / 100;
}

// The r-th smallest (1-based) of cost[0, count), all of them in [lo, hi]: each pass
// counts the values of the current window in kBuckets buckets and keeps the bucket
// that holds rank r.
__device__ long long select_rank(const int64_t* cost, int count, long long r, long long lo, long long hi,
                                 unsigned* hist, long long* bcast) {
    long long base = lo;
    unsigned long long span = (unsigned long long)(hi - lo);
    while (span > 0) {
        int bits = 64 - __clzll((long long)span);
        const int shift = bits > 11 ? bits - 11 : 0;
        for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < count; i += blockDim.x) {
            const long long v = cost[i];
            const unsigned long long d = (unsigned long long)(v - base);
            if (v >= base && d <= span) atomicAdd(&hist[d >> shift], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // warp 0: 64 buckets per lane, then a lane scan
            const int lane = threadIdx.x;
            unsigned long long mine = 0;
            for (int b = 0; b < kBuckets / 32; ++b) mine += hist[lane * (kBuckets / 32) + b];
            unsigned long long incl = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long x = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += x;
            }
            const unsigned ball = __ballot_sync(FULL, (long long)incl >= r);
            const int owner = __ffs(ball) - 1;
            if (lane == owner) {
                long long rr = r - (long long)(incl - mine);
                int b = lane * (kBuckets / 32);
                for (;; ++b) {
                    if ((long long)hist[b] >= rr) break;
                    rr -= hist[b];
                }
                bcast[0] = base + ((long long)b << shift);
                bcast[1] = rr;
            }
        }
        __syncthreads();
        const long long nb = bcast[0];
        r = bcast[1];
        const unsigned long long width = shift == 0 ? 0ull : ((1ull << shift) - 1ull);
        const unsigned long long rest = span - (unsigned long long)(nb - base);
        span = rest < width ? rest : width;
        base = nb;
        __syncthreads();
    }
    return base;
}

__device__ __forceinline__ int bin_of(long long c, long long lo, long long hi, int bins) {
    if (c < lo) return 0;
    if (c >= hi) return bins + 1;
    return 1 + (int)(((__int128)(c - lo) * bins) / (__int128)(hi - lo));
}

__global__ void __launch_bounds__(kThreads) k_trace(const StateView s, int64_t* ring, int capacity, int len,
                                                    long long lo, long long hi, int bins) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long part[2 * (kThreads / 32)];
    __shared__ long long bcast[2];
    const int m = s.m, ss = s.ss, P = s.P;
    const int t = *s.t;  // already advanced by the bookkeeping (>= 1)
    int64_t* rec = ring + (size_t)((t - 1) % capacity) * len;
    int64_t* hist_out = rec + 9 + 8 * m;
    if ((int)blockIdx.x < m) {
        // ---- swarm k: sort in shared memory, percentiles, histogram ----
        const int k = blockIdx.x;
        const int64_t* c = s.cost + (size_t)k * ss;
        long long* buf = reinterpret_cast<long long*>(smem);
        int len2 = 1;
        while (len2 < ss) len2 <<= 1;
        __int128 sum = 0;
        for (int i = threadIdx.x; i < len2; i += blockDim.x) {
            const long long v = i < ss ? c[i] : LLONG_MAX;
            buf[i] = v;
            if (i < ss) sum += v;
        }
        const __int128 tot = block_sum128(sum, part);
        __syncthreads();
        for (int kk = 2; kk <= len2; kk <<= 1)
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < len2; i += blockDim.x) {
                    const int q = i ^ j;
                    if (q > i) {
                        const long long x = buf[i], y = buf[q];
                        if ((x > y) == ((i & kk) == 0)) {
                            buf[i] = y;
                            buf[q] = x;
                        }
                    }
                }
                __syncthreads();
            }
        if (threadIdx.x == 0) {
            int64_t* o = rec + 9 + 8 * k;
            const int pct[4] = {5, 25, 50, 75};
            o[0] = buf[0];
            for (int q = 0; q < 4; ++q) o[1 + q] = buf[rank_of(pct[q], ss) - 1];
            o[5] = buf[ss - 1];
            o[6] = (long long)(unsigned long long)tot;
            o[7] = (long long)(tot >> 64);
        }
        return;
    }
    // ---- the population: histogram, min, max, sum, then the percentiles ----
    unsigned* hist = reinterpret_cast<unsigned*>(smem);
    for (int i = threadIdx.x; i < bins + 2; i += blockDim.x) hist_out[i] = 0;
    __syncthreads();
    long long mn = LLONG_MAX, mx = LLONG_MIN;
    __int128 sum = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const long long v = s.cost[i];
        mn = v < mn ? v : mn;
        mx = v > mx ? v : mx;
        sum += v;
        atomicAdd(reinterpret_cast<unsigned long long*>(hist_out) + bin_of(v, lo, hi, bins), 1ull);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long a = __shfl_xor_sync(FULL, mn, o), b = __shfl_xor_sync(FULL, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    __shared__ long long mm[2 * (kThreads / 32)];
    if ((threadIdx.x & 31) == 0) {
        mm[2 * (threadIdx.x >> 5)] = mn;
        mm[2 * (threadIdx.x >> 5) + 1] = mx;
    }
    const __int128 tot = block_sum128(sum, part);  // (its barriers also publish mm)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
        mn = mm[2 * i] < mn ? mm[2 * i] : mn;
        mx = mm[2 * i + 1] > mx ? mm[2 * i + 1] : mx;
    }
    const int pct[4] = {5, 25, 50, 75};
    long long pv[4];
    for (int q = 0; q < 4; ++q) pv[q] = select_rank(s.cost, P, rank_of(pct[q], P), mn, mx, hist, bcast);
    if (threadIdx.x == 0) {
        rec[0] = t;
        rec[1] = mn;
        for (int q = 0; q < 4; ++q) rec[2 + q] = pv[q];
        rec[6] = mx;
        rec[7] = (long long)(unsigned long long)tot;
        rec[8] = (long long)(tot >> 64);
    }
}

}  // namespace

int trace_max_swarm() { return kMaxSort; }

cudaError_t launch_trace(const StateView& s, const TraceBuf& tb, cudaStream_t st) {
    if (!tb.d || s.ss > kMaxSort) return cudaErrorInvalidValue;
    int len2 = 1;
    while (len2 < s.ss) len2 <<= 1;
    size_t smem = (size_t)len2 * 8;
    if (smem < kBuckets * 4) smem = kBuckets * 4;
    cudaError_t e = configure_once<k_trace>();
    if (e != cudaSuccess) return e;
    k_trace<<<s.m + 1, kThreads, smem, st>>>(s, tb.d, tb.capacity, tb.len, tb.lo, tb.hi, tb.bins);
    return cudaGetLastError();
}

}  // namespace qap

using namespace qap;

extern "C" {

int pso_trace_start(pso_state_t s, int32_t capacity, int64_t lo, int64_t hi, int32_t bins) {
    if (!s || capacity < 1 || bins < 1 || bins > (1 << 20) || hi <= lo) return QAP_ERR_INVALID_ARG;
    if (s->borrowed || s->sv.ss > trace_max_swarm()) return QAP_ERR_UNSUPPORTED;
    const int len = 9 + 8 * s->sv.m + bins + 2;
    const size_t bytes = 8 * (size_t)capacity * len;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    int64_t* d = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, bytes, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaFree(d);
        return status_of(e);
    }
    if (s->trace.d) cudaFree(s->trace.d);
    s->trace.d = d;
    s->trace.capacity = capacity;
    s->trace.len = len;
    s->trace.bins = bins;
    s->trace.lo = lo;
    s->trace.hi = hi;
    // the captured iterations change: capture them again at the next pso_step
    if (s->g1) cudaGraphExecDestroy(s->g1);
    if (s->g16) cudaGraphExecDestroy(s->g16);
    s->g1 = s->g16 = nullptr;
    return QAP_OK;
}

int pso_trace_record_len(pso_state_t s, int32_t* len) {
    if (!s || !len || !s->trace.d) return QAP_ERR_INVALID_ARG;
    *len = s->trace.len;
    return QAP_OK;
}

int pso_trace_read(pso_state_t s, int64_t* records, int32_t max_records, int32_t* count) {
    if (!s || !count || max_records < 0 || (max_records > 0 && !records) || !s->trace.d) return QAP_ERR_INVALID_ARG;
    const TraceBuf& tb = s->trace;
    std::vector<int64_t> h((size_t)tb.capacity * tb.len);
    cudaError_t e = cudaMemcpyAsync(h.data(), tb.d, h.size() * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return status_of(e);
    // the recorded slots (stamp >= 1) by stamp; the most recent max_records, oldest first
    std::vector<std::pair<int64_t, int>> slots;
    for (int i = 0; i < tb.capacity; ++i)
        if (h[(size_t)i * tb.len] >= 1) slots.push_back({h[(size_t)i * tb.len], i});
    std::sort(slots.begin(), slots.end());
    const size_t take = slots.size() < (size_t)max_records ? slots.size() : (size_t)max_records;
    for (size_t i = 0; i < take; ++i) {
        const int64_t* src = h.data() + (size_t)slots[slots.size() - take + i].second * tb.len;
        for (int w = 0; w < tb.len; ++w) records[i * tb.len + w] = src[w];
    }
    *count = (int32_t)take;
    return QAP_OK;
}

int pso_trace_stop(pso_state_t s) {
    if (!s) return QAP_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (s->trace.d) cudaFree(s->trace.d);
    s->trace = TraceBuf{};
    if (s->g1) cudaGraphExecDestroy(s->g1);
    if (s->g16) cudaGraphExecDestroy(s->g16);
    s->g1 = s->g16 = nullptr;
    return status_of(e);
}

}  // extern "C"
