// C-ABI of the library (declared in include/qap_pso.h): instances, population
// state, the iteration loop as a captured CUDA graph, results, statistics,
// state export/import and the single-kernel entry points.
#include <climits>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "state.h"

using namespace qap;

namespace qap {

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return QAP_OK;
    if (e == cudaErrorMemoryAllocation) return QAP_ERR_OOM;
    return QAP_ERR_CUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// the result block of a state: the counters, then the best cost (8 bytes), its
// iteration (4), padding (4) and the best permutation
constexpr size_t kCntBytes = (CNT_N * 8 + 15) / 16 * 16;
constexpr size_t kResHead = kCntBytes + 16;

// fp16 bits of an integer 0 <= v <= 2048 (exact: at most 11 significant bits)
uint16_t half_bits_small(int v) {
    if (v <= 0) return 0;
    int e = 0;
    while ((v >> (e + 1)) != 0) ++e;  // floor(log2 v)
    const uint32_t mant = e >= 10 ? ((uint32_t)v >> (e - 10)) & 0x3FFu : ((uint32_t)v << (10 - e)) & 0x3FFu;
    return (uint16_t)(((uint32_t)(e + 15) << 10) | mant);
}

// host round-to-nearest-even float -> bfloat16 bits (finite inputs)
uint16_t host_bf16(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    if ((b & 0x7F800000u) == 0x7F800000u) return (uint16_t)(b >> 16);  // inf / nan kept
    const uint32_t lsb = (b >> 16) & 1u;
    b += 0x7FFFu + lsb;
    return (uint16_t)(b >> 16);
}
float host_from_bf16(uint16_t h) {
    uint32_t b = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

int validate(const qap_instance* inst, const pso_params_t* p) {
    const int n = inst->n;
    if (p->swarms < 1 || p->swarms > bests_max_swarms()) return QAP_ERR_INVALID_ARG;
    if (p->swarm_size < 1) return QAP_ERR_INVALID_ARG;
    if ((long long)p->swarms * p->swarm_size > (1LL << 26)) return QAP_ERR_INVALID_ARG;
    if (!(p->v_max > 0.0f)) return QAP_ERR_INVALID_ARG;
    if (p->sv_kind != PSO_SV_RAW && p->sv_kind != PSO_SV_NORM) return QAP_ERR_INVALID_ARG;
    if (p->sx_rule != PSO_SX_ALG1 && p->sx_rule != PSO_SX_TOPD) return QAP_ERR_INVALID_ARG;
    if (p->sx_kind == PSO_SXK_SECOND_TARGET && (p->depth < 0 || p->depth >= n))
        return QAP_ERR_INVALID_ARG;  // d < n (section 3.1); PickColumn has no depth
    if (p->tie_rule != PSO_TIE_RANDOM && p->tie_rule != PSO_TIE_FIRST) return QAP_ERR_INVALID_ARG;
    if (p->mig_kind < PSO_MIG_NONE || p->mig_kind > PSO_MIG_RING) return QAP_ERR_INVALID_ARG;
    if (p->mig_depth < 0 || 2 * p->mig_depth >= p->swarms + (p->mig_kind == PSO_MIG_RANK ? 0 : 1 << 30))
        return QAP_ERR_INVALID_ARG;  // d < m / 2 (Algorithm 2)
    if (p->mig_period < 1) return QAP_ERR_INVALID_ARG;
    if (p->v_storage != PSO_V_FP32 && p->v_storage != PSO_V_BF16) return QAP_ERR_INVALID_ARG;
    if (p->sx_kind != PSO_SXK_SECOND_TARGET && p->sx_kind != PSO_SXK_PICK_COLUMN) return QAP_ERR_INVALID_ARG;
    if (!inst->exact64) return QAP_ERR_OVERFLOW;  // costs or swap values could leave int64
    if (n > velocity_sx_max_n(p->v_storage)) return QAP_ERR_UNSUPPORTED;
    return QAP_OK;
}

LsArgs ls_args_for(const pso_state* s, bool init, int32_t* work) {
    LsArgs a{};
    a.n = s->sv.n;
    a.count = s->sv.P;
    a.ps_in = a.ps_out = s->sv.ps;
    a.F = s->inst->dF;
    a.D = s->inst->dD;
    a.Dpk = s->inst->dDpk;
    a.in = s->sv.Xsx;
    a.out = s->sv.X;
    a.cost = s->sv.cost;
    a.moves = s->sv.moves;
    a.rounds = s->sv.rounds;
    a.PL = s->sv.PL;
    a.costL = s->sv.costL;
    a.counters = init ? nullptr : s->sv.counters;
    a.max_moves = (init && !s->prm.ls_at_init) ? -1 : s->prm.ls_max_moves;
    a.tc_exact = s->inst->tc_exact;
    a.key_l = s->inst->key_l;
    a.sym = s->inst->sym_zd;
    a.exact32 = s->inst->exact32 && s->inst->narrow_ok;
    a.force = -1;
    a.work = work;
    if (!init) {  // the iteration's search follows the update kernel's order
        a.ord_cnt = s->sv.ord_cnt;
        a.ord_list = s->sv.ord_list;
    }
    return a;
}

// Random particles, costs, bests; iteration counter and counters back to zero.
cudaError_t reinit_state(pso_state* s, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(s->sv.counters, 0, CNT_N * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->sv.t, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_init(s->sv, s->prm.v_storage == PSO_V_BF16, st);
    if (e == cudaSuccess) e = launch_ls(s->ls_init, st);
    if (e == cudaSuccess) e = launch_bests(s->d_view, 1, s->sv.m, 1, st);
    return e;
}

cudaError_t timed_iterations(cudaStream_t st, int iterations, void* flush_buf, size_t flush_bytes,
                             const TimedParts& T, float* ms_out) {
    if (iterations <= 0) return cudaSuccess;
    constexpr int E = 4;  // update (velocity + S_x), search, bests
    std::vector<cudaEvent_t> ev((size_t)iterations * E, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    for (int i = 0; i < iterations && e == cudaSuccess; ++i) {
        cudaEvent_t* q = &ev[(size_t)i * E];
        if (flush_buf && flush_bytes) e = cudaMemsetAsync(flush_buf, i & 0xFF, flush_bytes, st);
        if (e == cudaSuccess) e = cudaEventRecord(q[0], st);
        if (e == cudaSuccess) e = launch_velocity_sx(*T.vsx, st);
        if (e == cudaSuccess) e = cudaEventRecord(q[1], st);
        for (int g = 0; g < T.nls && e == cudaSuccess; ++g) e = launch_ls(T.ls[g], st);
        if (e == cudaSuccess) e = cudaEventRecord(q[2], st);
        if (e == cudaSuccess) e = launch_bests(T.views, T.count, T.m_max, 0, st);
        if (e == cudaSuccess) e = cudaEventRecord(q[3], st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    auto span = [&](int i, int a, int b) {
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[(size_t)i * E + a], ev[(size_t)i * E + b]);
        return ms;
    };
    for (int i = 0; i < iterations && e == cudaSuccess; ++i) {
        acc[0] += span(i, 0, 1);
        acc[1] += span(i, 1, 2);
        acc[2] += span(i, 2, 3);
        acc[3] += span(i, 0, 3);
    }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (e == cudaSuccess)
        for (int k = 0; k < 5; ++k) ms_out[k] += acc[k];
    return e;
}

}  // namespace qap

namespace {

cudaError_t enqueue_iteration(pso_state* s) {
    cudaError_t e = cudaSuccess;
    if (s->nsplit > 1) {
        // fork: part h's update and search on its own stream; join before the bests
        e = cudaEventRecord(s->ev_fork, s->stream);
        for (int h = 1; h < s->nsplit && e == cudaSuccess; ++h) e = cudaStreamWaitEvent(s->aux[h - 1], s->ev_fork, 0);
        for (int h = 0; h < s->nsplit && e == cudaSuccess; ++h)
            e = launch_velocity_sx(s->pvsx[h], h ? s->aux[h - 1] : s->stream);
        for (int h = 0; h < s->nsplit && e == cudaSuccess; ++h) e = launch_ls(s->pls[h], h ? s->aux[h - 1] : s->stream);
        for (int h = 1; h < s->nsplit && e == cudaSuccess; ++h) {
            e = cudaEventRecord(s->ev_join[h - 1], s->aux[h - 1]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_join[h - 1], 0);
        }
    } else {
        e = launch_velocity_sx(s->vsx, s->stream);
        if (e == cudaSuccess) e = launch_ls(s->ls_iter, s->stream);
    }
    if (e != cudaSuccess) return e;
    e = launch_bests(s->d_view, 1, s->sv.m, 0, s->stream);
    if (e == cudaSuccess && s->trace.d) e = launch_trace(s->sv, s->trace, s->stream);
    return e;
}

cudaError_t capture(pso_state* s, int iters, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < iters; ++i) {
        e = enqueue_iteration(s);
        if (e != cudaSuccess) break;
    }
    cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

}  // namespace

static int init_state(qap_instance_t inst, const pso_params_t* params, uint64_t seed, int32_t first_swarm,
                      bool part, void* stream, pso_state_t* out);

extern "C" {

const char* qap_status_string(int status) {
    switch (status) {
        case QAP_OK: return "ok";
        case QAP_ERR_INVALID_ARG: return "invalid argument";
        case QAP_ERR_OOM: return "out of device memory";
        case QAP_ERR_CUDA: return "CUDA error";
        case QAP_ERR_TIMEOUT: return "device wait timed out";
        case QAP_ERR_OVERFLOW: return "instance values exceed the exact integer path";
        case QAP_ERR_UNSUPPORTED: return "unsupported by this build";
        default: return "unknown status";
    }
}

int qap_create_instance(int32_t n, const int32_t* F, const int32_t* D, qap_instance_t* out) {
    if (!out || !F || !D || n < 2 || n > 256) return QAP_ERR_INVALID_ARG;
    int32_t mf = 0, md = 0;
    int sym = 1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const int32_t f = F[i * n + j], d = D[i * n + j];
            if (f < 0 || d < 0) return QAP_ERR_INVALID_ARG;  // non-negative (section 2.1)
            if (f > mf) mf = f;
            if (d > md) md = d;
            if (f != F[j * n + i] || d != D[j * n + i]) sym = 0;
            if (i == j && (f != 0 || d != 0)) sym = 0;
        }
    qap_instance* q = new (std::nothrow) qap_instance();
    if (!q) return QAP_ERR_OOM;
    q->n = n;
    q->sym_zd = sym;
    q->max_f = mf;
    q->max_d = md;
    q->exact32 = ((long double)n * mf * md < (long double)(1 << 27)) ? 1 : 0;
    q->narrow_ok = md <= 65535 ? 1 : 0;
    // every cost (n^2 terms), every value of the search tables (n terms) and every swap
    // value (8 n + 4 such terms) stays below 2^62 in magnitude: exact in int64
    q->exact64 = ((long double)n * n + 8.0L * n + 4.0L) * mf * md < 4611686018427387904.0L ? 1 : 0;
    q->tc_exact = (sym && mf <= 2048 && md <= 2048 && (long double)n * mf * md < (long double)(1 << 24)) ? 1 : 0;
    if (q->tc_exact && mf <= 255 && md <= 255) q->tc_exact |= 2;
    if (!sym && n <= 128 && mf <= 2048 && md <= 2048 && 2.0L * n * mf * md < (long double)(1 << 24))
        q->tc_exact |= 4;  // the general search
    // symmetric, zero diagonal: |delta(r, s)| <= 2 (n - 2) max_f max_d, so half of it
    // (S) with the pair index (2 L bits, n <= 2^L) fits a 32-bit key when
    // n max_f max_d < 2^(30 - 2 L)
    {
        int L = 1;
        while ((1 << L) < n) ++L;
        q->key_l = (sym && 2 * L <= 16 && (long double)n * mf * md < (long double)(1u << (30 - 2 * L))) ? L : 0;
    }
    const size_t bytes = (size_t)n * n * 4;
    cudaError_t e = cudaMalloc(&q->dF, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&q->dD, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(q->dF, F, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q->dD, D, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && (q->tc_exact & 1)) {
        // D for the tensor-core set-up: each entry (<= 2048, exact in fp16) with its
        // fp16 bits in the high half
        std::vector<uint32_t> pk((size_t)n * n);
        for (size_t i = 0; i < pk.size(); ++i) pk[i] = ((uint32_t)half_bits_small(D[i]) << 16) | (uint32_t)D[i];
        e = cudaMalloc(&q->dDpk, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(q->dDpk, pk.data(), bytes, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(q->dF);
        cudaFree(q->dD);
        cudaFree(q->dDpk);
        delete q;
        return status_of(e);
    }
    *out = q;
    return QAP_OK;
}

void qap_destroy_instance(qap_instance_t inst) {
    if (!inst) return;
    cudaFree(inst->dF);
    cudaFree(inst->dD);
    cudaFree(inst->dDpk);
    delete inst;
}

int qap_instance_info(qap_instance_t inst, qap_instance_info_t* out) {
    if (!inst || !out) return QAP_ERR_INVALID_ARG;
    out->n = inst->n;
    out->symmetric_zero_diag = inst->sym_zd;
    out->max_f = inst->max_f;
    out->max_d = inst->max_d;
    out->exact_int32 = inst->exact32;
    out->exact_int64 = inst->exact64;
    return QAP_OK;
}

void pso_params_default(pso_params_t* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->swarms = 1;
    p->swarm_size = 32;
    p->c1 = 0.8f;
    p->c2 = 0.5f;
    p->c3 = 0.5f;
    p->sv_kind = PSO_SV_NORM;
    p->v_max = 1.0f;
    p->sx_rule = PSO_SX_ALG1;
    p->depth = 2;
    p->tie_rule = PSO_TIE_RANDOM;
    p->pos_uses_new_v = 0;
    p->ls_max_moves = 0;
    p->ls_at_init = 0;
    p->mig_kind = PSO_MIG_NONE;
    p->mig_depth = 0;
    p->mig_period = 1;
    p->ring_if_better = 0;
    p->v_storage = PSO_V_FP32;
}

int pso_init(qap_instance_t inst, const pso_params_t* params, uint64_t seed, void* stream,
             pso_state_t* out) {
    return init_state(inst, params, seed, 0, false, stream, out);
}

int pso_init_part(qap_instance_t inst, const pso_params_t* params, uint64_t seed, int32_t first_swarm,
                  void* stream, pso_state_t* out) {
    return init_state(inst, params, seed, first_swarm, true, stream, out);
}

}  // extern "C"

static int init_state(qap_instance_t inst, const pso_params_t* params, uint64_t seed, int32_t first_swarm,
                      bool part, void* stream, pso_state_t* out) {
    if (!inst || !params || !out || first_swarm < 0) return QAP_ERR_INVALID_ARG;
    pso_params_t prm = *params;
    if (part) {  // a part of a run: the caller migrates (the run's migration depth may exceed the part's)
        prm.mig_kind = PSO_MIG_NONE;
        prm.mig_depth = 0;
    }
    int v = validate(inst, &prm);
    if (v != QAP_OK) return v;
    pso_state* s = new (std::nothrow) pso_state();
    if (!s) return QAP_ERR_OOM;
    s->inst = inst;
    s->prm = prm;
    params = &s->prm;
    s->seed = seed;
    if (stream) {
        s->stream = (cudaStream_t)stream;
        s->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return status_of(e);
        }
        s->own_stream = true;
    }
    const int n = inst->n, m = params->swarms, ss = params->swarm_size;
    const int P = m * ss;
    StateView& sv = s->sv;
    sv.n = n;
    sv.m = m;
    sv.ss = ss;
    sv.P = P;
    sv.swarm_base = first_swarm;
    sv.ps = (int32_t)align_up(n, 16);
    sv.vstride = (int64_t)align_up((size_t)n * n, 8);
    const size_t esz = params->v_storage == PSO_V_BF16 ? 2 : 4;
    int sl = 1;
    while (sl < P) sl <<= 1;
    s->stats_len = sl;
    // one allocation, 256-byte aligned pieces
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t oV = take((size_t)P * sv.vstride * esz);
    const size_t oX = take((size_t)P * sv.ps), oXsx = take((size_t)P * sv.ps), oPL = take((size_t)P * sv.ps);
    const size_t ocostL = take((size_t)P * 8), ocost = take((size_t)P * 8);
    const size_t omoves = take((size_t)P * 4), orounds = take((size_t)P * 4);
    const size_t oPG = take((size_t)m * sv.ps), oPG2 = take((size_t)m * sv.ps);
    const size_t ocostG = take((size_t)m * 8), ocostG2 = take((size_t)m * 8);
    // the counters, the best cost, its iteration and the best permutation side by side:
    // pso_best reads them with one copy (and reports the kernels' error counter)
    const size_t ores = take(kResHead + (size_t)sv.ps), ocnt = ores, obc = ores + kCntBytes,
                 obi = obc + 8, obest = obc + 16;
    const size_t ot = take(4);
    const size_t ostb = take((size_t)sl * 8), osto = take(8 * 8);
    const size_t oview = take(sizeof(StateView)), opre = take(2 * 4), ols = take(2 * sizeof(LsArgs));
    const size_t owork = take(3 * 4);  // search (iteration, set-up), position
    // the search order: counts of the whole population, then of each part; one list area
    // (a part's lists lie in the range of its own particles)
    const size_t oordc = take(kOrdBuckets * 4 * (1 + kMaxSplit)), oordl = take((size_t)kOrdBuckets * P * 4);
    const size_t opview = take(kMaxSplit * sizeof(StateView)), opls = take(kMaxSplit * sizeof(LsArgs));
    const size_t opprefix = take(2 * kMaxSplit * 4), opwork = take(2 * kMaxSplit * 4);
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) {
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return status_of(e);
    }
    s->dbase = base;
    e = cudaMallocHost(&s->h_res, kResHead + (size_t)sv.ps);  // pinned: pso_best's read-back
    if (e != cudaSuccess) {
        s->h_res = nullptr;
        pso_destroy(s);
        return status_of(e);
    }
    sv.V = base + oV;
    sv.X = (uint8_t*)(base + oX);
    sv.Xsx = (uint8_t*)(base + oXsx);
    sv.PL = (uint8_t*)(base + oPL);
    sv.costL = (int64_t*)(base + ocostL);
    sv.cost = (int64_t*)(base + ocost);
    sv.moves = (int32_t*)(base + omoves);
    sv.rounds = (int32_t*)(base + orounds);
    sv.PG = (uint8_t*)(base + oPG);
    sv.PG2 = (uint8_t*)(base + oPG2);
    sv.costG = (int64_t*)(base + ocostG);
    sv.costG2 = (int64_t*)(base + ocostG2);
    sv.best = (uint8_t*)(base + obest);
    sv.best_cost = (int64_t*)(base + obc);
    sv.best_iter = (int32_t*)(base + obi);
    sv.t = (int32_t*)(base + ot);
    sv.counters = (unsigned long long*)(base + ocnt);
    s->stats_buf = (int64_t*)(base + ostb);
    s->stats_out = (int64_t*)(base + osto);
    s->d_view = (StateView*)(base + oview);
    s->d_prefix = (int32_t*)(base + opre);
    s->d_ls = (LsArgs*)(base + ols);
    s->d_work = (int32_t*)(base + owork);
    sv.ord_cnt = (int32_t*)(base + oordc);
    sv.ord_list = (int32_t*)(base + oordl);
    s->d_pview = (StateView*)(base + opview);
    s->d_pls = (LsArgs*)(base + opls);
    s->d_pprefix = (int32_t*)(base + opprefix);
    s->d_pwork = (int32_t*)(base + opwork);
    sv.seed = seed;
    sv.c1 = params->c1;
    sv.c2 = params->c2;
    sv.c3 = params->c3;
    sv.v_max = params->v_max;
    sv.sv_kind = params->sv_kind;
    sv.sx_rule = params->sx_rule;
    sv.depth = params->depth;
    sv.tie_rule = params->tie_rule;
    sv.sx_kind = params->sx_kind;
    sv.pos_uses_new_v = params->pos_uses_new_v;
    sv.ls_max_moves = params->ls_max_moves;
    sv.mig_kind = params->mig_kind;
    sv.mig_depth = params->mig_depth;
    sv.mig_period = params->mig_period;
    sv.ring_if_better = params->ring_if_better;

    // one-entry tables the kernels read this population through
    s->h_ls[0] = ls_args_for(s, false, s->d_work);
    s->h_ls[1] = ls_args_for(s, true, s->d_work + 1);
    s->h_prefix[0] = 0;
    s->h_prefix[1] = P;
    s->vsx = VsxLaunch{s->d_view, s->d_prefix, 1, n, P, params->v_storage == PSO_V_BF16, 0, s->d_work + 2};
    s->ls_iter = LsLaunch{s->d_ls, s->d_work, 1, n, (int)ls_kind(s->h_ls[0]), 0, P};
    s->ls_init = LsLaunch{s->d_ls + 1, s->d_work + 1, 1, n, (int)ls_kind(s->h_ls[1]), 0, P};
    // parts of whole swarms for the captured iterations: views and searches over their
    // particles (pointers advanced to the part's first particle and swarm; the draws
    // keyed by the swarm's index in the run, as for a part of a split run). With bf16
    // tiles (16 warps per SM in the update, a longer tail) two parts pay; with fp32
    // tiles the second search launch's per-CTA set-up costs more than the overlap gains
    // (measured at n = 64, 16 x 640 particles), so fp32 populations run as one part.
    s->nsplit = (m >= 2 && params->v_storage == PSO_V_BF16) ? kMaxSplit : 1;
    sv.ord_resets = kOrdBuckets * (1 + s->nsplit);
    StateView h_pview[kMaxSplit] = {};
    LsArgs h_pls[kMaxSplit] = {};
    int32_t h_pprefix[2 * kMaxSplit] = {};
    if (s->nsplit > 1) {
        const size_t vbytes = (size_t)sv.vstride * esz;
        for (int h = 0, fs = 0; h < s->nsplit; ++h) {
            const int cs = m / s->nsplit + (h < m % s->nsplit ? 1 : 0);  // swarms of part h
            const size_t fp = (size_t)fs * ss;
            const int cp = cs * ss;
            StateView pv = sv;
            pv.m = cs;
            pv.P = cp;
            pv.swarm_base = sv.swarm_base + fs;
            pv.V = (char*)sv.V + fp * vbytes;
            pv.X += fp * sv.ps;
            pv.Xsx += fp * sv.ps;
            pv.PL += fp * sv.ps;
            pv.costL += fp;
            pv.cost += fp;
            pv.moves += fp;
            pv.rounds += fp;
            pv.PG += (size_t)fs * sv.ps;
            pv.PG2 += (size_t)fs * sv.ps;
            pv.costG += fs;
            pv.costG2 += fs;
            pv.ord_cnt = sv.ord_cnt + kOrdBuckets * (1 + h);
            pv.ord_list = sv.ord_list + (size_t)kOrdBuckets * fp;
            pv.ord_resets = 0;
            h_pview[h] = pv;
            LsArgs a = ls_args_for(s, false, s->d_pwork + 2 * h + 1);
            a.count = cp;
            a.in = pv.Xsx;
            a.out = pv.X;
            a.cost = pv.cost;
            a.moves = pv.moves;
            a.rounds = pv.rounds;
            a.PL = pv.PL;
            a.costL = pv.costL;
            a.ord_cnt = pv.ord_cnt;
            a.ord_list = pv.ord_list;
            h_pls[h] = a;
            h_pprefix[2 * h + 1] = cp;
            s->pvsx[h] = VsxLaunch{s->d_pview + h, s->d_pprefix + 2 * h, 1, n, cp,
                                   params->v_storage == PSO_V_BF16, 0, s->d_pwork + 2 * h};
            s->pls[h] = LsLaunch{s->d_pls + h, s->d_pwork + 2 * h + 1, 1, n, (int)ls_kind(a), 0, cp};
            fs += cs;
        }
        for (int h = 0; h + 1 < s->nsplit && e == cudaSuccess; ++h) {
            e = cudaStreamCreateWithFlags(&s->aux[h], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join[h], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            pso_destroy(s);
            return status_of(e);
        }
    }
    e = cudaMemsetAsync(base, 0, off, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_view, &s->sv, sizeof(StateView), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_prefix, s->h_prefix, sizeof(s->h_prefix), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_ls, s->h_ls, sizeof(s->h_ls), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && s->nsplit > 1)
        e = cudaMemcpyAsync(s->d_pview, h_pview, sizeof(h_pview), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && s->nsplit > 1)
        e = cudaMemcpyAsync(s->d_pls, h_pls, sizeof(h_pls), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && s->nsplit > 1)
        e = cudaMemcpyAsync(s->d_pprefix, h_pprefix, sizeof(h_pprefix), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = reinit_state(s, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        pso_destroy(s);
        return status_of(e);
    }
    *out = s;
    return QAP_OK;
}

extern "C" {

int pso_footprint(int32_t n, const pso_params_t* p, size_t* bytes) {
    if (!p || !bytes || n < 2 || n > 256 || p->swarms < 1 || p->swarm_size < 1) return QAP_ERR_INVALID_ARG;
    const size_t P = (size_t)p->swarms * p->swarm_size, m = (size_t)p->swarms;
    const size_t ps = align_up(n, 16), vstride = align_up((size_t)n * n, 8);
    const size_t esz = p->v_storage == PSO_V_BF16 ? 2 : 4;
    size_t sl = 1;
    while (sl < P) sl <<= 1;
    const size_t a = 256;
    size_t t = align_up(P * vstride * esz, a) + 3 * align_up(P * ps, a) + 2 * align_up(P * 8, a) +
               2 * align_up(P * 4, a) + 2 * align_up(m * ps, a) + 2 * align_up(m * 8, a) + 4 * a +
               align_up(kResHead + ps, a) + align_up(sl * 8, a) + align_up(8 * 8, a) +
               align_up(sizeof(StateView), a) + a + align_up(2 * sizeof(LsArgs), a) + a +
               align_up(kOrdBuckets * 4 * (1 + kMaxSplit), a) + align_up(kOrdBuckets * P * 4, a) +
               align_up(kMaxSplit * sizeof(StateView), a) + align_up(kMaxSplit * sizeof(LsArgs), a) +
               2 * align_up(2 * kMaxSplit * 4, a);
    *bytes = t;
    return QAP_OK;
}

int pso_poll(pso_state_t s, int32_t* done) {
    if (!s || !done) return QAP_ERR_INVALID_ARG;
    const cudaError_t e = cudaStreamQuery(s->stream);
    if (e == cudaSuccess) {
        *done = 1;
        return QAP_OK;
    }
    if (e == cudaErrorNotReady) {
        *done = 0;
        return QAP_OK;
    }
    return status_of(e);
}

int pso_step(pso_state_t s, int32_t iterations) {
    if (!s || iterations < 0) return QAP_ERR_INVALID_ARG;
    if (iterations == 0) return QAP_OK;
    cudaError_t e = cudaSuccess;
    if (!s->g1) e = capture(s, 1, &s->g1);
    if (e == cudaSuccess && iterations >= 16 && !s->g16) e = capture(s, 16, &s->g16);
    if (e != cudaSuccess) return status_of(e);
    int left = iterations;
    while (left >= 16 && e == cudaSuccess) {
        e = cudaGraphLaunch(s->g16, s->stream);
        left -= 16;
    }
    while (left > 0 && e == cudaSuccess) {
        e = cudaGraphLaunch(s->g1, s->stream);
        --left;
    }
    return status_of(e);
}

int pso_step_timed(pso_state_t s, int32_t iterations, void* flush_buf, size_t flush_bytes,
                   float* ms_out) {
    if (!s || iterations < 0 || !ms_out) return QAP_ERR_INVALID_ARG;
    const TimedParts T{&s->vsx, &s->ls_iter, 1, s->d_view, 1, s->sv.m};
    return status_of(timed_iterations(s->stream, iterations, flush_buf, flush_bytes, T, ms_out));
}

int pso_best(pso_state_t s, int64_t* cost, int32_t* perm, int32_t* iter_found) {
    if (!s) return QAP_ERR_INVALID_ARG;
    const int n = s->sv.n;
    // counters (kCntBytes), cost (8 bytes), iteration (4), padding (4), permutation (n):
    // one copy
    cudaError_t e = cudaMemcpyAsync(s->h_res, s->sv.counters, kResHead + (size_t)n, cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return status_of(e);
    unsigned long long errs = 0;
    std::memcpy(&errs, s->h_res + 8 * CNT_ERR, 8);
    if (errs) return QAP_ERR_TIMEOUT;  // a kernel gave up a bounded wait or skipped an access
    int64_t c = 0;
    int32_t it = 0;
    std::memcpy(&c, s->h_res + kCntBytes, 8);
    std::memcpy(&it, s->h_res + kCntBytes + 8, 4);
    const uint8_t* p = s->h_res + kCntBytes + 16;
    if (cost) *cost = c;
    if (iter_found) *iter_found = it;
    if (perm)
        for (int i = 0; i < n; ++i) perm[i] = p[i];
    return QAP_OK;
}

static int stats_of_range(pso_state_t s, int32_t first, int32_t count, pso_stats_t* out) {
    cudaError_t e = launch_stats(s->sv.cost + first, count, s->stats_buf, s->stats_len, s->stats_out, s->stream);
    int64_t o[8];
    unsigned long long cnt[CNT_N];
    int64_t bc = 0;
    int32_t t = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(o, s->stats_out, sizeof(o), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, s->sv.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bc, s->sv.best_cost, 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&t, s->sv.t, 4, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return status_of(e);
    out->iteration = t;
    out->best_cost = bc;
    out->min = o[0];
    out->p5 = o[1];
    out->p25 = o[2];
    out->p50 = o[3];
    out->p75 = o[4];
    out->max = o[5];
    out->mean = mean_of_sum(o[6], o[7], count);
    out->particle_iterations = (int64_t)cnt[CNT_PIT];
    out->ls_moves = (int64_t)cnt[CNT_MOVES];
    out->ls_rounds = (int64_t)cnt[CNT_ROUNDS];
    out->delta_full = (int64_t)cnt[CNT_DELTA_FULL];
    out->delta_incr = (int64_t)cnt[CNT_DELTA_INCR];
    out->sx_ties = (int64_t)cnt[CNT_TIES];
    out->errors = (int64_t)cnt[CNT_ERR];
    return QAP_OK;
}

int pso_stats(pso_state_t s, pso_stats_t* out) {
    if (!s || !out || out->size < sizeof(pso_stats_t)) return QAP_ERR_INVALID_ARG;
    return stats_of_range(s, 0, s->sv.P, out);
}

int pso_stats_swarm(pso_state_t s, int32_t swarm, pso_stats_t* out) {
    if (!s || !out || out->size < sizeof(pso_stats_t) || swarm < 0 || swarm >= s->sv.m) return QAP_ERR_INVALID_ARG;
    return stats_of_range(s, swarm * s->sv.ss, s->sv.ss, out);
}

int pso_cost_histogram(pso_state_t s, int32_t swarm, int64_t lo, int64_t hi, int32_t bins, int64_t* counts) {
    if (!s || !counts || bins < 1 || bins > (1 << 20) || hi <= lo || swarm < -1 || swarm >= s->sv.m)
        return QAP_ERR_INVALID_ARG;
    const int first = swarm < 0 ? 0 : swarm * s->sv.ss, count = swarm < 0 ? s->sv.P : s->sv.ss;
    unsigned long long* d = nullptr;
    const size_t bytes = sizeof(unsigned long long) * (size_t)(bins + 2);
    cudaError_t e = cudaMallocAsync(&d, bytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, bytes, s->stream);
    if (e == cudaSuccess) e = launch_histogram(s->sv.cost + first, count, lo, hi, bins, d, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (d) cudaFreeAsync(d, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return status_of(e);
}

void pso_destroy(pso_state_t s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->g1) cudaGraphExecDestroy(s->g1);
    if (s->g16) cudaGraphExecDestroy(s->g16);
    for (int h = 0; h + 1 < kMaxSplit; ++h) {
        if (s->aux[h]) {
            cudaStreamSynchronize(s->aux[h]);
            cudaStreamDestroy(s->aux[h]);
        }
        if (s->ev_join[h]) cudaEventDestroy(s->ev_join[h]);
    }
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->trace.d) cudaFree(s->trace.d);
    cudaFree(s->dbase);
    if (s->h_res) cudaFreeHost(s->h_res);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

int pso_export_state(pso_state_t s, pso_host_state_t* o) {
    if (!s || !o) return QAP_ERR_INVALID_ARG;
    const StateView& sv = s->sv;
    const int n = sv.n, P = sv.P, m = sv.m, ps = sv.ps;
    const bool bf = s->prm.v_storage == PSO_V_BF16;
    const size_t esz = bf ? 2 : 4;
    std::vector<char> V((size_t)P * sv.vstride * esz);
    std::vector<uint8_t> X((size_t)P * ps), Xs((size_t)P * ps), PL((size_t)P * ps), PG((size_t)m * ps), B(ps);
    std::vector<int64_t> cL(P), c(P), cG(m);
    std::vector<int32_t> mv(P);
    int64_t bc = 0;
    int32_t bi = 0, t = 0;
    cudaStream_t st = s->stream;
    cudaError_t e = cudaMemcpyAsync(V.data(), sv.V, V.size(), cudaMemcpyDeviceToHost, st);
    auto cp = [&](void* dst, const void* src, size_t b) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, st);
    };
    cp(X.data(), sv.X, X.size());
    cp(Xs.data(), sv.Xsx, Xs.size());
    cp(PL.data(), sv.PL, PL.size());
    cp(PG.data(), sv.PG, PG.size());
    cp(B.data(), sv.best, B.size());
    cp(cL.data(), sv.costL, P * 8);
    cp(c.data(), sv.cost, P * 8);
    cp(cG.data(), sv.costG, m * 8);
    cp(mv.data(), sv.moves, P * 4);
    cp(&bc, sv.best_cost, 8);
    cp(&bi, sv.best_iter, 4);
    cp(&t, sv.t, 4);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return status_of(e);
    for (int p = 0; p < P; ++p) {
        for (int k = 0; k < n * n; ++k) {
            const size_t idx = (size_t)p * sv.vstride + k;
            float f;
            if (bf) {
                uint16_t h;
                std::memcpy(&h, V.data() + idx * 2, 2);
                f = host_from_bf16(h);
            } else {
                std::memcpy(&f, V.data() + idx * 4, 4);
            }
            if (o->V) o->V[(size_t)p * n * n + k] = f;
        }
        for (int j = 0; j < n; ++j) {
            if (o->X) o->X[(size_t)p * n + j] = X[(size_t)p * ps + j];
            if (o->X_sx) o->X_sx[(size_t)p * n + j] = Xs[(size_t)p * ps + j];
            if (o->PL) o->PL[(size_t)p * n + j] = PL[(size_t)p * ps + j];
        }
        if (o->costL) o->costL[p] = cL[p];
        if (o->cost) o->cost[p] = c[p];
        if (o->moves) o->moves[p] = mv[p];
    }
    for (int k = 0; k < m; ++k) {
        for (int j = 0; j < n; ++j)
            if (o->PG) o->PG[(size_t)k * n + j] = PG[(size_t)k * ps + j];
        if (o->costG) o->costG[k] = cG[k];
    }
    if (o->best)
        for (int j = 0; j < n; ++j) o->best[j] = B[j];
    o->best_cost = bc;
    o->best_iter = bi;
    o->t = t;
    return QAP_OK;
}

int pso_import_state(pso_state_t s, const pso_host_state_t* in) {
    if (!s || !in || !in->V || !in->X || !in->PL || !in->costL || !in->cost || !in->PG ||
        !in->costG || !in->best)
        return QAP_ERR_INVALID_ARG;
    const StateView& sv = s->sv;
    const int n = sv.n, P = sv.P, m = sv.m, ps = sv.ps;
    const bool bf = s->prm.v_storage == PSO_V_BF16;
    const size_t esz = bf ? 2 : 4;
    auto perm_ok = [n](const int32_t* p) {
        std::vector<char> seen(n, 0);
        for (int j = 0; j < n; ++j) {
            if (p[j] < 0 || p[j] >= n || seen[p[j]]) return false;
            seen[p[j]] = 1;
        }
        return true;
    };
    for (int p = 0; p < P; ++p)
        if (!perm_ok(in->X + (size_t)p * n) || !perm_ok(in->PL + (size_t)p * n)) return QAP_ERR_INVALID_ARG;
    for (int k = 0; k < m; ++k)
        if (!perm_ok(in->PG + (size_t)k * n)) return QAP_ERR_INVALID_ARG;
    if (!perm_ok(in->best) || in->t < 0) return QAP_ERR_INVALID_ARG;
    std::vector<char> V((size_t)P * sv.vstride * esz, 0);
    std::vector<uint8_t> X((size_t)P * ps, 0), PL((size_t)P * ps, 0), PG((size_t)m * ps, 0), B(ps, 0);
    for (int p = 0; p < P; ++p) {
        for (int k = 0; k < n * n; ++k) {
            const float f = in->V[(size_t)p * n * n + k];
            if (!std::isfinite(f)) return QAP_ERR_INVALID_ARG;
            const size_t idx = (size_t)p * sv.vstride + k;
            if (bf) {
                const uint16_t h = host_bf16(f);
                std::memcpy(V.data() + idx * 2, &h, 2);
            } else {
                std::memcpy(V.data() + idx * 4, &f, 4);
            }
        }
        for (int j = 0; j < n; ++j) {
            X[(size_t)p * ps + j] = (uint8_t)in->X[(size_t)p * n + j];
            PL[(size_t)p * ps + j] = (uint8_t)in->PL[(size_t)p * n + j];
        }
    }
    for (int k = 0; k < m; ++k)
        for (int j = 0; j < n; ++j) PG[(size_t)k * ps + j] = (uint8_t)in->PG[(size_t)k * n + j];
    for (int j = 0; j < n; ++j) B[j] = (uint8_t)in->best[j];
    cudaStream_t st = s->stream;
    cudaError_t e = cudaStreamSynchronize(st);
    auto cp = [&](void* dst, const void* src, size_t b) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, st);
    };
    cp(sv.V, V.data(), V.size());
    cp(sv.X, X.data(), X.size());
    cp(sv.PL, PL.data(), PL.size());
    cp(sv.PG, PG.data(), PG.size());
    cp(sv.best, B.data(), B.size());
    cp(sv.costL, in->costL, P * 8);
    cp(sv.cost, in->cost, P * 8);
    cp(sv.costG, in->costG, m * 8);
    cp(sv.best_cost, &in->best_cost, 8);
    cp(sv.best_iter, &in->best_iter, 4);
    cp(sv.t, &in->t, 4);
    // recorded statistics belong to the replaced run
    if (e == cudaSuccess && s->trace.d)
        e = cudaMemsetAsync(s->trace.d, 0, 8 * (size_t)s->trace.capacity * s->trace.len, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return status_of(e);
}

static int run_ls_hook(qap_instance_t inst, int force, const int32_t* perms, int32_t count, int32_t max_moves,
                       int32_t* perms_out, int64_t* costs, int32_t* moves, int32_t* rounds, float* kernel_ms) {
    const int n = inst->n;
    for (int c = 0; c < count; ++c) {
        std::vector<char> seen(n, 0);
        for (int j = 0; j < n; ++j) {
            const int32_t v = perms[(size_t)c * n + j];
            if (v < 0 || v >= n || seen[v]) return QAP_ERR_INVALID_ARG;
            seen[v] = 1;
        }
    }
    LsArgs a{};
    a.n = n;
    a.count = count;
    a.F = inst->dF;
    a.D = inst->dD;
    a.Dpk = inst->dDpk;
    a.max_moves = max_moves;
    a.tc_exact = inst->tc_exact;
    a.key_l = inst->key_l;
    a.sym = inst->sym_zd;
    a.exact32 = inst->exact32 && inst->narrow_ok;
    a.force = force;
    const LsKind kind = ls_kind(a);
    if (!ls_kind_serves(kind, a)) return QAP_ERR_UNSUPPORTED;
    const int ps = (int)align_up(n, 16);
    a.ps_in = a.ps_out = ps;
    std::vector<uint8_t> hp((size_t)count * ps, 0);
    for (int c = 0; c < count; ++c)
        for (int j = 0; j < n; ++j) hp[(size_t)c * ps + j] = (uint8_t)perms[(size_t)c * n + j];
    uint8_t *din = nullptr, *dout = nullptr;
    int64_t* dc = nullptr;
    int32_t *dm = nullptr, *dr = nullptr, *dw = nullptr;
    cudaError_t e = cudaMalloc(&din, hp.size());
    if (e == cudaSuccess) e = cudaMalloc(&dw, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&dout, hp.size());
    if (e == cudaSuccess) e = cudaMalloc(&dc, (size_t)count * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dm, (size_t)count * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dr, (size_t)count * 4);
    if (e == cudaSuccess) e = cudaMemcpy(din, hp.data(), hp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        a.in = din;
        a.out = dout;
        a.cost = dc;
        a.moves = dm;
        a.rounds = dr;
        a.work = dw;
        LsArgs* da = nullptr;
        e = cudaMalloc(&da, sizeof(LsArgs));
        if (e == cudaSuccess) e = cudaMemcpy(da, &a, sizeof(LsArgs), cudaMemcpyHostToDevice);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (e == cudaSuccess && kernel_ms) e = cudaEventCreate(&e0);
        if (e == cudaSuccess && kernel_ms) e = cudaEventCreate(&e1);
        if (e == cudaSuccess && kernel_ms) e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) e = launch_ls(LsLaunch{da, dw, 1, n, (int)kind, 0, count}, 0);
        if (e == cudaSuccess && kernel_ms) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess && kernel_ms) e = cudaEventElapsedTime(kernel_ms, e0, e1);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(da);
    }
    std::vector<int64_t> hc(count);
    std::vector<int32_t> hm(count), hr(count);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(hp.data(), dout, hp.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hc.data(), dc, (size_t)count * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hm.data(), dm, (size_t)count * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hr.data(), dr, (size_t)count * 4, cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    cudaFree(dc);
    cudaFree(dm);
    cudaFree(dr);
    cudaFree(dw);
    if (e != cudaSuccess) return status_of(e);
    for (int c = 0; c < count; ++c) {
        if (perms_out)
            for (int j = 0; j < n; ++j) perms_out[(size_t)c * n + j] = hp[(size_t)c * ps + j];
        if (costs) costs[c] = hc[c];
        if (moves) moves[c] = hm[c];
        if (rounds) rounds[c] = hr[c];
    }
    return QAP_OK;
}

// the search kernel a QAP_SEARCH_* choice names for this instance (-1: automatic)
static int forced_kind(const qap_instance* inst, int32_t kernel, int* out) {
    LsArgs a{};
    a.n = inst->n;
    a.tc_exact = inst->tc_exact;
    a.sym = inst->sym_zd;
    a.exact32 = inst->exact32 && inst->narrow_ok;
    a.force = -1;
    switch (kernel) {
        case QAP_SEARCH_AUTO: *out = -1; return QAP_OK;
        case QAP_SEARCH_TENSOR: {
            const LsKind k = !inst->sym_zd ? LS_GEN
                             : inst->n <= 32 ? LS_TEAM1
                             : inst->n <= 64 ? LS_TEAM2
                             : inst->n <= 128 ? LS_TEAM8 : LS_TEAM8N;
            *out = (int)k;
            return ls_kind_serves(k, a) ? QAP_OK : QAP_ERR_UNSUPPORTED;
        }
        case QAP_SEARCH_SIMT: *out = (int)LS_SIMT; return ls_kind_serves(LS_SIMT, a) ? QAP_OK : QAP_ERR_UNSUPPORTED;
        case QAP_SEARCH_INT64: {
            const LsKind k = ls_kind_serves(LS_SIMT64, a) ? LS_SIMT64 : LS_DIRECT;
            *out = (int)k;
            return QAP_OK;
        }
        case QAP_SEARCH_DIRECT: *out = (int)LS_DIRECT; return QAP_OK;
        default: return QAP_ERR_INVALID_ARG;
    }
}

int qap_eval_costs(qap_instance_t inst, const int32_t* perms, int32_t count, int64_t* out) {
    return qap_search_with(inst, QAP_SEARCH_AUTO, const_cast<int32_t*>(perms), count, -1, out, nullptr, nullptr,
                           nullptr);
}

int qap_local_search(qap_instance_t inst, int32_t* perms, int32_t count, int32_t max_moves,
                     int64_t* costs, int32_t* moves, int32_t* rounds) {
    if (max_moves < 0) return QAP_ERR_INVALID_ARG;
    return qap_search_with(inst, QAP_SEARCH_AUTO, perms, count, max_moves, costs, moves, rounds, nullptr);
}

int qap_search_with(qap_instance_t inst, int32_t kernel, int32_t* perms, int32_t count, int32_t max_moves,
                    int64_t* costs, int32_t* moves, int32_t* rounds, float* kernel_ms) {
    if (!inst || !perms || count < 0) return QAP_ERR_INVALID_ARG;
    if (max_moves < 0 && !costs) return QAP_ERR_INVALID_ARG;
    if (!inst->exact64) return QAP_ERR_OVERFLOW;
    int force = -1;
    const int st = forced_kind(inst, kernel, &force);
    if (st != QAP_OK) return st;
    if (count == 0) return QAP_OK;
    return run_ls_hook(inst, force, perms, count, max_moves, max_moves < 0 ? nullptr : perms, costs, moves,
                       rounds, kernel_ms);
}

int qap_delta_table(qap_instance_t inst, const int32_t* perm, int64_t* out) {
    if (!inst || !perm || !out) return QAP_ERR_INVALID_ARG;
    const int n = inst->n;
    std::vector<char> seen(n, 0);
    for (int j = 0; j < n; ++j) {
        if (perm[j] < 0 || perm[j] >= n || seen[perm[j]]) return QAP_ERR_INVALID_ARG;
        seen[perm[j]] = 1;
    }
    // every term is at most 2 max_f max_d in magnitude, 2 n terms
    if (4.0 * (n + 1) * (double)inst->max_f * (double)inst->max_d >= 9.0e18) return QAP_ERR_OVERFLOW;
    const size_t npairs = (size_t)n * (n - 1) / 2;
    int32_t* dp = nullptr;
    int64_t* dout = nullptr;
    cudaError_t e = cudaMalloc(&dp, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dout, npairs * 8);
    if (e == cudaSuccess) e = cudaMemcpy(dp, perm, (size_t)n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_delta_table(inst->dF, inst->dD, n, dp, dout, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, npairs * 8, cudaMemcpyDeviceToHost);
    cudaFree(dp);
    cudaFree(dout);
    return status_of(e);
}

int pso_discretize(const float* Y, const int32_t* Z, int32_t n, int32_t count, const pso_params_t* params,
                   uint64_t seed, const int32_t* swarm, const int32_t* particle, int32_t t,
                   int32_t* out_perm) {
    if (!Y || !Z || !params || !swarm || !particle || !out_perm) return QAP_ERR_INVALID_ARG;
    if (n < 2 || n > 256 || count < 0 || t < 0) return QAP_ERR_INVALID_ARG;
    if (params->sx_rule != PSO_SX_ALG1 && params->sx_rule != PSO_SX_TOPD) return QAP_ERR_INVALID_ARG;
    if (params->sx_kind == PSO_SXK_SECOND_TARGET && (params->depth < 0 || params->depth >= n))
        return QAP_ERR_INVALID_ARG;  // d < n (section 3.1); PickColumn has no depth
    if (params->tie_rule != PSO_TIE_RANDOM && params->tie_rule != PSO_TIE_FIRST) return QAP_ERR_INVALID_ARG;
    if (params->sx_kind != PSO_SXK_SECOND_TARGET && params->sx_kind != PSO_SXK_PICK_COLUMN) return QAP_ERR_INVALID_ARG;
    if (n > velocity_sx_max_n(0)) return QAP_ERR_UNSUPPORTED;
    if (count == 0) return QAP_OK;
    for (int i = 0; i < count; ++i) {
        if (swarm[i] < 0 || particle[i] < 0) return QAP_ERR_INVALID_ARG;
        std::vector<char> seen(n, 0);
        for (int j = 0; j < n; ++j) {
            const int32_t v = Z[(size_t)i * n + j];
            if (v < 0 || v >= n || seen[v]) return QAP_ERR_INVALID_ARG;
            seen[v] = 1;
        }
        for (int k = 0; k < n * n; ++k)
            if (!std::isfinite(Y[(size_t)i * n * n + k])) return QAP_ERR_INVALID_ARG;
    }
    // the velocity kernel's layout: 16-byte tiles (bulk copies) and 16-byte permutation rows
    const size_t vstride = align_up((size_t)n * n, 4);
    const size_t ps = align_up(n, 16);
    std::vector<float> hv((size_t)count * vstride, 0.0f);
    std::vector<uint8_t> hz((size_t)count * ps, 0);
    for (int i = 0; i < count; ++i) {
        std::memcpy(hv.data() + (size_t)i * vstride, Y + (size_t)i * n * n, (size_t)n * n * 4);
        for (int j = 0; j < n; ++j) hz[(size_t)i * ps + j] = (uint8_t)Z[(size_t)i * n + j];
    }
    char* base = nullptr;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = align_up(off + b, 256);
        return o;
    };
    const size_t oV = take(hv.size() * 4), oX = take(hz.size()), oS = take(hz.size()),
                 oSw = take((size_t)count * 4), oPi = take((size_t)count * 4), oT = take(4),
                 oC = take(CNT_N * 8), oView = take(sizeof(StateView)), oPre = take(8);
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) return status_of(e);
    StateView sv{};
    sv.n = n;
    sv.m = 1;
    sv.ss = 1;
    sv.P = count;
    sv.ps = (int32_t)ps;
    sv.vstride = (int64_t)vstride;
    sv.V = base + oV;
    sv.X = (uint8_t*)(base + oX);
    sv.Xsx = (uint8_t*)(base + oS);
    sv.t = (int32_t*)(base + oT);
    sv.counters = (unsigned long long*)(base + oC);
    sv.seed = seed;
    sv.sx_rule = params->sx_rule;
    sv.depth = params->depth;
    sv.tie_rule = params->tie_rule;
    sv.sx_kind = params->sx_kind;
    sv.sx_only = 1;
    sv.sx_swarm = (const int32_t*)(base + oSw);
    sv.sx_pis = (const int32_t*)(base + oPi);
    const int32_t prefix[2] = {0, count};
    auto up = [&](size_t o, const void* src, size_t b) {
        if (e == cudaSuccess) e = cudaMemcpy(base + o, src, b, cudaMemcpyHostToDevice);
    };
    up(oV, hv.data(), hv.size() * 4);
    up(oX, hz.data(), hz.size());
    up(oSw, swarm, (size_t)count * 4);
    up(oPi, particle, (size_t)count * 4);
    up(oT, &t, 4);
    up(oView, &sv, sizeof(sv));
    up(oPre, prefix, sizeof(prefix));
    if (e == cudaSuccess) e = cudaMemset(base + oC, 0, CNT_N * 8);
    if (e == cudaSuccess)
        e = launch_velocity_sx(VsxLaunch{(const StateView*)(base + oView), (const int32_t*)(base + oPre), 1, n,
                                         count, 0, 0, nullptr},
                               0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned long long cnt[CNT_N] = {};
    if (e == cudaSuccess) e = cudaMemcpy(cnt, base + oC, sizeof(cnt), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hz.data(), base + oS, hz.size(), cudaMemcpyDeviceToHost);
    cudaFree(base);
    if (e != cudaSuccess) return status_of(e);
    if (cnt[CNT_ERR]) return QAP_ERR_TIMEOUT;
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < n; ++j) out_perm[(size_t)i * n + j] = hz[(size_t)i * ps + j];
    return QAP_OK;
}

}  // extern "C"

// ------------------------------------------------ parts of a run (multi-process)
extern "C" {

int pso_swarm_bests(pso_state_t s, int64_t* costs, int32_t* perms) {
    if (!s || !costs) return QAP_ERR_INVALID_ARG;
    const StateView& sv = s->sv;
    std::vector<uint8_t> pg((size_t)sv.m * sv.ps);
    cudaError_t e = cudaMemcpyAsync(costs, sv.costG, (size_t)sv.m * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && perms)
        e = cudaMemcpyAsync(pg.data(), sv.PG, pg.size(), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return status_of(e);
    if (perms)
        for (int k = 0; k < sv.m; ++k)
            for (int j = 0; j < sv.n; ++j) perms[(size_t)k * sv.n + j] = pg[(size_t)k * sv.ps + j];
    return QAP_OK;
}

int pso_set_swarm_best(pso_state_t s, int32_t swarm, int64_t cost, const int32_t* perm) {
    if (!s || !perm || swarm < 0 || swarm >= s->sv.m) return QAP_ERR_INVALID_ARG;
    const StateView& sv = s->sv;
    std::vector<uint8_t> row(sv.ps, 0);
    std::vector<char> seen(sv.n, 0);
    for (int j = 0; j < sv.n; ++j) {
        if (perm[j] < 0 || perm[j] >= sv.n || seen[perm[j]]) return QAP_ERR_INVALID_ARG;
        seen[perm[j]] = 1;
        row[j] = (uint8_t)perm[j];
    }
    // after the queued work, then synchronously (the host buffers are locals)
    cudaError_t e = cudaMemcpyAsync(sv.PG + (size_t)swarm * sv.ps, row.data(), sv.n, cudaMemcpyHostToDevice,
                                    s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv.costG + swarm, &cost, 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return status_of(e);
}

int pso_particle(pso_state_t s, int32_t index, int64_t* cost, int32_t* perm) {
    if (!s || !cost || !perm || index < 0 || index >= s->sv.P) return QAP_ERR_INVALID_ARG;
    const StateView& sv = s->sv;
    std::vector<uint8_t> row(sv.ps);
    int64_t c = 0;
    cudaError_t e = cudaMemcpyAsync(row.data(), sv.X + (size_t)index * sv.ps, sv.ps, cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, sv.cost + index, 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return status_of(e);
    *cost = c;
    for (int j = 0; j < sv.n; ++j) perm[j] = row[j];
    return QAP_OK;
}

int qap_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag, uint32_t block,
               uint32_t* out4) {
    if (!out4 || tag > 255 || block > 0xFFFFFFu) return QAP_ERR_INVALID_ARG;
    const U4 u = draw(seed, c0, c1, c2, tag, block);
    out4[0] = u.x;
    out4[1] = u.y;
    out4[2] = u.z;
    out4[3] = u.w;
    return QAP_OK;
}

}  // extern "C"
