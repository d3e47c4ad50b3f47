// Internal definitions of the C-ABI handles, shared by the runtime and the batch
// engine (not part of the public header).
#pragma once

#include <cuda_runtime.h>

#include "../../include/qap_pso.h"
#include "kernels.h"

struct qap_instance {
    int32_t n;
    int32_t* dF;
    int32_t* dD;
    uint32_t* dDpk;  // tc_exact bit 0: D as (fp16 bits << 16) | value, else null
    int32_t sym_zd;
    int32_t max_f, max_d;
    int32_t exact32;    // n max_f max_d < 2^27
    int32_t exact64;    // (n^2 + 8 n + 4) max_f max_d < 2^62: every cost and swap value fits int64
    int32_t narrow_ok;  // every entry fits the uint16 staging of the kernels
    int32_t tc_exact;   // bit 0: the tensor-core set-up of the local search is exact; bit 1: and 8-bit staging fits
    int32_t key_l;      // pair-index bits of the 32-bit search keys, 0 when |delta| is not bounded enough
};

// One population. Its kernels read it through one-entry device tables (the same
// kernels serve a batch of many populations with longer tables).
constexpr int kMaxSplit = 2;

struct pso_state {
    qap_instance* inst;
    pso_params_t prm;
    uint64_t seed;
    cudaStream_t stream;
    bool own_stream;
    qap::StateView sv;
    void* dbase;
    int64_t* stats_buf;
    int32_t stats_len;
    int64_t* stats_out;       // 6 int64 + 1 double
    qap::StateView* d_view;   // 1 entry
    int32_t* d_prefix;        // {0, P}
    qap::LsArgs* d_ls;        // [0] iteration, [1] initialisation
    int32_t* d_work;          // their particle counters
    qap::LsArgs h_ls[2];      // host copies (sources of the uploads)
    int32_t h_prefix[2];
    qap::VsxLaunch vsx;
    qap::LsLaunch ls_iter, ls_init;
    // The captured iterations run the update and the search in `nsplit` parts of whole
    // swarms, each part on its own branch of the graph (part 0 on `stream`, part h on
    // aux[h - 1]), so the kernels of one part fill the SMs that the end of another
    // part's kernel leaves idle; bests and migration join them. nsplit 1: no parts.
    int nsplit;
    qap::StateView* d_pview;       // nsplit part views
    qap::LsArgs* d_pls;            // nsplit part searches
    int32_t* d_pprefix;            // nsplit x {0, part particles}
    int32_t* d_pwork;              // nsplit x {update, search} counters
    qap::VsxLaunch pvsx[kMaxSplit];
    qap::LsLaunch pls[kMaxSplit];
    cudaStream_t aux[kMaxSplit - 1];
    cudaEvent_t ev_fork, ev_join[kMaxSplit - 1];
    cudaGraphExec_t g1, g16;
    bool borrowed;            // a member of a batch (the batch runs its iterations)
    qap::TraceBuf trace;      // per-iteration statistics (off unless pso_trace_start)
    unsigned char* h_res;     // pinned: best cost, iteration and permutation (pso_best)
};

namespace qap {
// The launches of one iteration, for timing them one by one.
struct TimedParts {
    const VsxLaunch* vsx;
    const LsLaunch* ls;
    int nls;
    const StateView* views;
    int count;
    int m_max;
};
// Runs `iterations` iterations with events around every phase (after writing
// flush_bytes of flush_buf, when given) and adds the device milliseconds to ms_out:
// [0] the update (velocity and S_x, one kernel), [1] goal function + local search,
// [2] bests + migration, [3] whole iterations, [4] 0 (kept for the layout).
cudaError_t timed_iterations(cudaStream_t st, int iterations, void* flush_buf, size_t flush_bytes,
                             const TimedParts& T, float* ms_out);
int status_of(cudaError_t e);
LsArgs ls_args_for(const pso_state* s, bool init, int32_t* work);
cudaError_t reinit_state(pso_state* s, cudaStream_t st);
}  // namespace qap
