// Host-side launchers of the PSO-iteration kernels (internal to the library).
//
// Every launcher covers a table of populations (one or many instances of possibly
// different n) in a single kernel launch: the kernels read each population's view
// or arguments from a small device table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"

namespace qap {

// Arguments of the goal-function / local-search kernels for one population.
// Permutations are uint8 rows (facility -> location) `ps_in` / `ps_out` bytes apart.
struct LsArgs {
    int32_t n, count;
    int32_t ps_in, ps_out;
    const int32_t* F;  // device n x n, symmetric with zero diagonal when max_moves >= 0
    const int32_t* D;  // device n x n
    const uint32_t* Dpk;  // D as (fp16 bits << 16) | value when every entry is <= 2048 (the
                          // tensor-core set-up gathers both from one word), else null
    const uint8_t* in;
    uint8_t* out;
    int64_t* cost;     // count
    int32_t* moves;    // count, may be null
    int32_t* rounds;   // count, may be null
    uint8_t* PL;       // local bests to update (may be null)
    int64_t* costL;
    unsigned long long* counters;  // may be null
    int32_t max_moves; // < 0: goal function only; 0: to a local optimum; > 0: cap
    int32_t tc_exact;  // bit 0: symmetric, zero diagonal, entries <= 2048 and n max_f max_d < 2^24:
                       // the tensor-core set-up is exact;
                       // bit 1: also every entry <= 255 (8-bit staging of F and D);
                       // bit 2: any F, D (not symmetric or not zero-diagonal) with entries
                       // <= 2048, 2 n max_f max_d < 2^24 and n <= 128: the general
                       // tensor-core search is exact
    int32_t* work;     // device counter handing out this population's particles (zeroed
                       // by the launcher before every launch)
    int32_t key_l;     // > 0: n <= 2^key_l and n max_f max_d < 2^(30 - 2 key_l), so the
                       // tensor-core search packs a swap value and its pair in 32 bits
    int32_t sym;       // F and D symmetric with zero diagonal
    int32_t exact32;   // n max_f max_d < 2^27 and max_d <= 65535: the int32 SIMT search is exact
    int32_t force;     // a LsKind chosen by the caller, or -1 (ls_kind decides)
    const int32_t* ord_cnt;   // the hand-out order of the iteration's particles (the
    const int32_t* ord_list;  // update kernel's buckets, StateView::ord_*), or null
};

// Which local-search kernel serves a population, and the launch shape.
//   TEAM1/2/8: symmetric, tensor-core set-up, teams of 1, 2, 8 warps (n <= 32, 64, 128)
//   TEAM8N:    the same with 8-bit staging (entries <= 255), 128 < n <= 160
//   GEN:       any F, D (small entries), tensor-core set-up of R + C, n <= 128
//   SIMT:      symmetric, int32 G from SIMT multiply-adds (n max_f max_d < 2^27)
//   SIMT64:    symmetric, int64 G (any entries whose costs fit int64)
//   DIRECT:    any F, D, int64, every swap value from the general O(n) formula
enum LsKind {
    LS_TEAM1 = 0, LS_TEAM2 = 1, LS_SIMT = 2, LS_TEAM8 = 3, LS_TEAM8N = 4, LS_GEN = 5,
    LS_SIMT64 = 6, LS_DIRECT = 7, LS_KINDS = 8
};
LsKind ls_kind(const LsArgs& a);
// whether `kind` is exact for the population described by `a` and serves its n
bool ls_kind_serves(LsKind kind, const LsArgs& a);

// One local-search launch over `count` populations of the same kind.
struct LsLaunch {
    const LsArgs* d_args;  // device table, `count` entries
    int32_t* d_work;       // the populations' counters (contiguous, `count` ints)
    int count;
    int n_max;             // largest n in the table (shared-memory layout)
    int kind;              // LsKind
    int cpi;               // CTAs per population (0 = automatic)
    int total;             // particles over the table (automatic shape)
};
cudaError_t launch_ls(const LsLaunch& L, cudaStream_t st);
// largest n a search kernel serves
int ls_max_n(LsKind kind);

// The update of every particle of `count` populations (flat index over particles):
// velocity (Eq. 4 + S_v) and position (Eq. 5, S_x) in one kernel, one warp per
// particle, V read and written once.
struct VsxLaunch {
    const StateView* d_views;
    const int32_t* d_prefix;  // count + 1 particle offsets
    int count;
    int n_max;
    int total;                // prefix[count]
    int v_bf16;               // every population of the table has the same storage
    int warps;                // warps per CTA (0 = automatic)
    int32_t* d_work;          // the kernel's particle counter (zeroed before each
                              // launch), or null for a fixed grid-stride order
};
cudaError_t launch_velocity_sx(const VsxLaunch& L, cudaStream_t st);
int velocity_sx_max_n(int v_bf16);

cudaError_t launch_init(const StateView& s, int v_bf16, cudaStream_t st);
// One CTA per population; init_mode: the bookkeeping after initialisation (no
// migration, t unchanged).
cudaError_t launch_bests(const StateView* d_views, int count, int m_max, int init_mode, cudaStream_t st);
int bests_max_swarms();

// Sorts `count` costs in `scratch` (>= next power of two entries) and writes
// {min, p5, p25, p50, p75, max, sum low word, sum high word} to out8 (device
// pointers; the sum of the costs as a 128-bit two's-complement integer).
cudaError_t launch_stats(const int64_t* cost, int32_t count, int64_t* scratch, int32_t scratch_len,
                         int64_t* out8, cudaStream_t st);
// Host: the mean of `count` values whose 128-bit sum is (sum_hi, sum_lo), as
// floor-quotient plus remainder / count.
double mean_of_sum(int64_t sum_lo, int64_t sum_hi, int32_t count);

// Per-iteration statistics of a population, recorded on the device into a ring of
// `capacity` records of `len` int64 words (layout in trace.cu).
struct TraceBuf {
    int64_t* d = nullptr;  // [0] records written, then capacity records
    int32_t capacity = 0, len = 0, bins = 0;
    int64_t lo = 0, hi = 0;
};
// After the iteration's bookkeeping (the iteration counter already advanced).
cudaError_t launch_trace(const StateView& s, const TraceBuf& tb, cudaStream_t st);
// largest swarm size the trace kernel sorts in shared memory
int trace_max_swarm();

// Histogram of `count` device costs: counts (device, bins + 2, zeroed by the caller)
// [0] below lo, [1 + b] for b = floor((cost - lo) bins / (hi - lo)), [bins + 1] >= hi.
cudaError_t launch_histogram(const int64_t* cost, int count, int64_t lo, int64_t hi, int bins,
                             unsigned long long* counts, cudaStream_t st);

// Delta(r, s) of every pair r < s of one permutation (device pointers; out holds
// n (n - 1) / 2 int64 in r-major pair order).
cudaError_t launch_delta_table(const int32_t* F, const int32_t* D, int n, const int32_t* perm, int64_t* out,
                               cudaStream_t st);

}  // namespace qap
