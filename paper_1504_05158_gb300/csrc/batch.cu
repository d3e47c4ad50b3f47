// Batches: many independent populations (instances of uneven n) advanced together.
// Each phase of an iteration is one kernel launch over the whole batch (the local
// search takes one launch per kernel kind present), the iterations are replayed
// from a captured CUDA graph, and launch shapes come from timing candidates on the
// batch itself (the autotuner), after which the members are re-initialised.
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "state.h"

using namespace qap;

namespace {

struct Group {
    LsLaunch launch;
    std::vector<LsArgs> host;
};

// Launch shapes found by the autotuner, by (v storage, n_max, members, particles)
// for the velocity kernel and (kind, n_max, members, particles) for the search.
std::mutex g_tune_lock;
std::map<std::tuple<int, int, int, int>, int> g_vsx_warps;
std::map<std::tuple<int, int, int, int>, int> g_ls_cpi;

}  // namespace

struct pso_batch {
    std::vector<pso_state*> members;
    cudaStream_t stream;
    bool own_stream;
    void* dbase;
    StateView* d_views;
    int32_t* d_prefix;
    std::vector<StateView> h_views;
    std::vector<int32_t> h_prefix;
    std::vector<Group> groups;
    VsxLaunch vsx;
    int m_max;
    cudaGraphExec_t g1, g16;
};

namespace {

cudaError_t enqueue(pso_batch* b) {
    cudaError_t e = launch_velocity_sx(b->vsx, b->stream);
    for (auto& g : b->groups)
        if (e == cudaSuccess) e = launch_ls(g.launch, b->stream);
    if (e == cudaSuccess) e = launch_bests(b->d_views, (int)b->members.size(), b->m_max, 0, b->stream);
    return e;
}

cudaError_t capture(pso_batch* b, int iters, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < iters && e == cudaSuccess; ++i) e = enqueue(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// milliseconds of `reps` runs of f() on the batch's stream
template <typename Fn>
float time_on(cudaStream_t st, int reps, Fn f) {
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    cudaEventRecord(a, st);
    for (int i = 0; i < reps; ++i) f();
    cudaEventRecord(z, st);
    cudaEventSynchronize(z);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, z);
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    return ms;
}

// Picks the velocity kernel's warps per CTA and each search group's CTAs per
// population by timing candidates on the batch's own data (the state advances
// while tuning; the caller re-initialises it afterwards).
cudaError_t autotune(pso_batch* b) {
    const int count = (int)b->members.size();
    const auto vkey = std::make_tuple(b->vsx.v_bf16, b->vsx.n_max, count, b->vsx.total);
    {
        std::lock_guard<std::mutex> g(g_tune_lock);
        auto it = g_vsx_warps.find(vkey);
        if (it != g_vsx_warps.end()) b->vsx.warps = it->second;
    }
    if (b->vsx.warps == 0) {
        float best = 1e30f;
        int pick = 4;
        for (int w : {1, 2, 4}) {
            VsxLaunch L = b->vsx;
            L.warps = w;
            if (launch_velocity_sx(L, b->stream) != cudaSuccess) continue;  // warm
            const float ms = time_on(b->stream, 2, [&] { launch_velocity_sx(L, b->stream); });
            if (ms < best) {
                best = ms;
                pick = w;
            }
        }
        b->vsx.warps = pick;
        std::lock_guard<std::mutex> g(g_tune_lock);
        g_vsx_warps[vkey] = pick;
    }
    for (auto& grp : b->groups) {
        LsLaunch& L = grp.launch;
        const auto key = std::make_tuple(L.kind, L.n_max, L.count, L.total);
        {
            std::lock_guard<std::mutex> g(g_tune_lock);
            auto it = g_ls_cpi.find(key);
            if (it != g_ls_cpi.end()) {
                L.cpi = it->second;
                continue;
            }
        }
        float best = 1e30f;
        int pick = 0;
        for (int c : {0, 1, 2, 4, 8, 16}) {
            LsLaunch T = L;
            T.cpi = c;
            if (launch_ls(T, b->stream) != cudaSuccess) continue;  // warm
            const float ms = time_on(b->stream, 2, [&] { launch_ls(T, b->stream); });
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        L.cpi = pick;
        std::lock_guard<std::mutex> g(g_tune_lock);
        g_ls_cpi[key] = pick;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int pso_batch_create(int32_t count, const qap_instance_t* insts, const pso_params_t* params,
                     const uint64_t* seeds, void* stream, int32_t autotune_shapes, pso_batch_t* out) {
    if (count < 1 || !insts || !params || !seeds || !out) return QAP_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!insts[i] || params[i].v_storage != params[0].v_storage) return QAP_ERR_INVALID_ARG;
    pso_batch* b = new (std::nothrow) pso_batch();
    if (!b) return QAP_ERR_OOM;
    if (stream) {
        b->stream = (cudaStream_t)stream;
        b->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return status_of(e);
        }
        b->own_stream = true;
    }
    for (int i = 0; i < count; ++i) {
        pso_state_t s = nullptr;
        const int st = pso_init(insts[i], &params[i], seeds[i], b->stream, &s);
        if (st != QAP_OK) {
            pso_batch_destroy(b);
            return st;
        }
        s->borrowed = true;
        b->members.push_back(s);
    }
    // tables over all members
    int total = 0, n_max = 0, m_max = 0;
    b->h_prefix.push_back(0);
    for (auto* s : b->members) {
        b->h_views.push_back(s->sv);
        total += s->sv.P;
        b->h_prefix.push_back(total);
        n_max = std::max(n_max, (int)s->sv.n);
        m_max = std::max(m_max, (int)s->sv.m);
    }
    b->m_max = m_max;
    int kind_count[LS_KINDS] = {};
    for (auto* s : b->members) ++kind_count[s->ls_iter.kind];
    size_t bytes = sizeof(StateView) * count + sizeof(int32_t) * (count + 1) + 1024 + 256;
    for (int k = 0; k < LS_KINDS; ++k) bytes += (sizeof(LsArgs) + sizeof(int32_t)) * kind_count[k] + 512;
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
        pso_batch_destroy(b);
        return status_of(e);
    }
    b->dbase = base;
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t o = off;
        off = (off + n + 255) & ~size_t(255);
        return base + o;
    };
    b->d_views = (StateView*)take(sizeof(StateView) * count);
    b->d_prefix = (int32_t*)take(sizeof(int32_t) * (count + 1));
    int32_t* d_pos_work = (int32_t*)take(sizeof(int32_t));
    e = cudaMemcpy(b->d_views, b->h_views.data(), sizeof(StateView) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_prefix, b->h_prefix.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice);
    for (int k = 0; k < LS_KINDS && e == cudaSuccess; ++k) {
        if (!kind_count[k]) continue;
        Group g;
        LsArgs* d_args = (LsArgs*)take(sizeof(LsArgs) * kind_count[k]);
        int32_t* d_work = (int32_t*)take(sizeof(int32_t) * kind_count[k]);
        int gn = 0, gtot = 0;
        for (auto* s : b->members) {
            if (s->ls_iter.kind != k) continue;
            LsArgs a = s->h_ls[0];
            a.work = d_work + g.host.size();
            g.host.push_back(a);
            gn = std::max(gn, (int)a.n);
            gtot += a.count;
        }
        g.launch = LsLaunch{d_args, d_work, kind_count[k], gn, k, 0, gtot};
        e = cudaMemcpy(d_args, g.host.data(), sizeof(LsArgs) * g.host.size(), cudaMemcpyHostToDevice);
        b->groups.push_back(g);
    }
    b->vsx = VsxLaunch{b->d_views, b->d_prefix, count, n_max, total, params[0].v_storage == PSO_V_BF16, 0,
                       d_pos_work};
    if (e == cudaSuccess && autotune_shapes) {
        e = autotune(b);
        // the tuning runs advanced the members: start them again from their seeds
        for (auto* s : b->members)
            if (e == cudaSuccess) e = reinit_state(s, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        pso_batch_destroy(b);
        return status_of(e);
    }
    *out = b;
    return QAP_OK;
}

int pso_batch_step(pso_batch_t b, int32_t iterations) {
    if (!b || iterations < 0) return QAP_ERR_INVALID_ARG;
    if (iterations == 0) return QAP_OK;
    cudaError_t e = cudaSuccess;
    if (!b->g1) e = capture(b, 1, &b->g1);
    if (e == cudaSuccess && iterations >= 16 && !b->g16) e = capture(b, 16, &b->g16);
    int left = iterations;
    while (left >= 16 && e == cudaSuccess) {
        e = cudaGraphLaunch(b->g16, b->stream);
        left -= 16;
    }
    while (left > 0 && e == cudaSuccess) {
        e = cudaGraphLaunch(b->g1, b->stream);
        --left;
    }
    return status_of(e);
}

int pso_batch_step_timed(pso_batch_t b, int32_t iterations, void* flush_buf, size_t flush_bytes,
                         float* ms_out) {
    if (!b || iterations < 0 || !ms_out) return QAP_ERR_INVALID_ARG;
    std::vector<LsLaunch> ls;
    for (auto& g : b->groups) ls.push_back(g.launch);
    const TimedParts T{&b->vsx, ls.data(), (int)ls.size(), b->d_views, (int)b->members.size(), b->m_max};
    return status_of(timed_iterations(b->stream, iterations, flush_buf, flush_bytes, T, ms_out));
}

int pso_batch_member(pso_batch_t b, int32_t index, pso_state_t* out) {
    if (!b || !out || index < 0 || index >= (int)b->members.size()) return QAP_ERR_INVALID_ARG;
    *out = b->members[index];
    return QAP_OK;
}

int pso_batch_size(pso_batch_t b, int32_t* count) {
    if (!b || !count) return QAP_ERR_INVALID_ARG;
    *count = (int32_t)b->members.size();
    return QAP_OK;
}

void pso_batch_destroy(pso_batch_t b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->g1) cudaGraphExecDestroy(b->g1);
    if (b->g16) cudaGraphExecDestroy(b->g16);
    for (auto* s : b->members) pso_destroy(s);
    cudaFree(b->dbase);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
