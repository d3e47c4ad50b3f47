"""Thin ctypes binding of ``libqap_pso.so`` (C-ABI in include/qap_pso.h).

Argument marshalling only: every step of the PSO iteration runs in the CUDA
library. Loading fails loudly if the library has not been built; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqap_pso.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_OVERFLOW, ERR_UNSUPPORTED = range(7)
SV_RAW, SV_NORM = 0, 1
SX_ALG1, SX_TOPD = 0, 1
TIE_RANDOM, TIE_FIRST = 0, 1
MIG_NONE, MIG_RANK, MIG_RING = 0, 1, 2
V_FP32, V_BF16 = 0, 1
SXK_SECOND_TARGET, SXK_PICK_COLUMN = 0, 1
SEARCH_AUTO, SEARCH_TENSOR, SEARCH_SIMT, SEARCH_INT64, SEARCH_DIRECT = range(5)

# every exported symbol of include/qap_pso.h
EXPORTS = [
    "qap_status_string", "qap_create_instance", "qap_destroy_instance", "qap_instance_info",
    "pso_params_default", "pso_init", "pso_step", "pso_step_timed", "pso_best", "pso_stats", "pso_destroy",
    "pso_export_state", "pso_import_state", "qap_eval_costs", "qap_local_search",
    "qap_cost_stats_noalloc", "pso_batch_create", "pso_batch_step", "pso_batch_step_timed",
    "pso_batch_size", "pso_batch_member", "pso_batch_destroy", "pso_footprint", "pso_poll",
    "qap_delta_table", "pso_discretize", "pso_stats_swarm", "pso_cost_histogram", "qap_search_with",
    "qap_int32_peak", "pso_trace_start", "pso_trace_record_len", "pso_trace_read", "pso_trace_stop",
    "pso_init_part", "pso_swarm_bests", "pso_set_swarm_best", "pso_particle", "qap_philox",
]
NOALLOC_MAX_COUNT = 65536


class QapError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("swarms", C.c_int32), ("swarm_size", C.c_int32),
        ("c1", C.c_float), ("c2", C.c_float), ("c3", C.c_float),
        ("sv_kind", C.c_int32), ("v_max", C.c_float),
        ("sx_rule", C.c_int32), ("depth", C.c_int32), ("tie_rule", C.c_int32),
        ("pos_uses_new_v", C.c_int32), ("ls_max_moves", C.c_int32), ("ls_at_init", C.c_int32),
        ("mig_kind", C.c_int32), ("mig_depth", C.c_int32), ("mig_period", C.c_int32),
        ("ring_if_better", C.c_int32), ("v_storage", C.c_int32), ("sx_kind", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [
        ("size", C.c_uint32), ("iteration", C.c_int32), ("best_cost", C.c_int64),
        ("min", C.c_int64), ("p5", C.c_int64), ("p25", C.c_int64), ("p50", C.c_int64),
        ("p75", C.c_int64), ("max", C.c_int64), ("mean", C.c_double),
        ("particle_iterations", C.c_int64), ("ls_moves", C.c_int64), ("ls_rounds", C.c_int64),
        ("delta_full", C.c_int64), ("delta_incr", C.c_int64), ("sx_ties", C.c_int64),
        ("errors", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "size"}


class InstanceInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("symmetric_zero_diag", C.c_int32), ("max_f", C.c_int32),
                ("max_d", C.c_int32), ("exact_int32", C.c_int32), ("exact_int64", C.c_int32)]


class HostState(C.Structure):
    _fields_ = [
        ("V", C.POINTER(C.c_float)), ("X", C.POINTER(C.c_int32)), ("X_sx", C.POINTER(C.c_int32)),
        ("PL", C.POINTER(C.c_int32)), ("costL", C.POINTER(C.c_int64)), ("cost", C.POINTER(C.c_int64)),
        ("moves", C.POINTER(C.c_int32)), ("PG", C.POINTER(C.c_int32)), ("costG", C.POINTER(C.c_int64)),
        ("best", C.POINTER(C.c_int32)), ("best_cost", C.c_int64), ("best_iter", C.c_int32),
        ("t", C.c_int32),
    ]


_lib = None


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.qap_status_string.argtypes = [C.c_int]
        L.qap_status_string.restype = C.c_char_p
        L.qap_create_instance.argtypes = [C.c_int32, vp, vp, C.POINTER(vp)]
        L.qap_destroy_instance.argtypes = [vp]
        L.qap_destroy_instance.restype = None
        L.qap_instance_info.argtypes = [vp, C.POINTER(InstanceInfo)]
        L.pso_params_default.argtypes = [C.POINTER(Params)]
        L.pso_params_default.restype = None
        L.pso_init.argtypes = [vp, C.POINTER(Params), C.c_uint64, vp, C.POINTER(vp)]
        L.pso_step.argtypes = [vp, C.c_int32]
        L.pso_step_timed.argtypes = [vp, C.c_int32, vp, C.c_size_t, C.POINTER(C.c_float)]
        L.pso_best.argtypes = [vp, C.POINTER(C.c_int64), vp, C.POINTER(C.c_int32)]
        L.pso_stats.argtypes = [vp, C.POINTER(Stats)]
        L.pso_destroy.argtypes = [vp]
        L.pso_destroy.restype = None
        L.pso_export_state.argtypes = [vp, C.POINTER(HostState)]
        L.pso_import_state.argtypes = [vp, C.POINTER(HostState)]
        L.qap_eval_costs.argtypes = [vp, vp, C.c_int32, vp]
        L.qap_local_search.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, vp, vp]
        L.qap_search_with.argtypes = [vp, C.c_int32, vp, C.c_int32, C.c_int32, vp, vp, vp, C.POINTER(C.c_float)]
        L.qap_int32_peak.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.pso_trace_start.argtypes = [vp, C.c_int32, C.c_int64, C.c_int64, C.c_int32]
        L.pso_trace_record_len.argtypes = [vp, C.POINTER(C.c_int32)]
        L.pso_trace_read.argtypes = [vp, vp, C.c_int32, C.POINTER(C.c_int32)]
        L.pso_trace_stop.argtypes = [vp]
        L.pso_init_part.argtypes = [vp, C.POINTER(Params), C.c_uint64, C.c_int32, vp, C.POINTER(vp)]
        L.pso_swarm_bests.argtypes = [vp, vp, vp]
        L.pso_set_swarm_best.argtypes = [vp, C.c_int32, C.c_int64, vp]
        L.pso_particle.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64), vp]
        L.qap_philox.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, vp]
        L.qap_cost_stats_noalloc.argtypes = [vp, C.c_int32, vp, vp, C.POINTER(C.c_double)]
        L.pso_batch_create.argtypes = [C.c_int32, vp, vp, vp, vp, C.c_int32, C.POINTER(vp)]
        L.pso_batch_step.argtypes = [vp, C.c_int32]
        L.pso_batch_step_timed.argtypes = [vp, C.c_int32, vp, C.c_size_t, C.POINTER(C.c_float)]
        L.pso_batch_size.argtypes = [vp, C.POINTER(C.c_int32)]
        L.pso_batch_member.argtypes = [vp, C.c_int32, C.POINTER(vp)]
        L.pso_batch_destroy.argtypes = [vp]
        L.pso_batch_destroy.restype = None
        L.pso_footprint.argtypes = [C.c_int32, C.POINTER(Params), C.POINTER(C.c_size_t)]
        L.pso_poll.argtypes = [vp, C.POINTER(C.c_int32)]
        L.qap_delta_table.argtypes = [vp, vp, vp]
        L.pso_stats_swarm.argtypes = [vp, C.c_int32, C.POINTER(Stats)]
        L.pso_cost_histogram.argtypes = [vp, C.c_int32, C.c_int64, C.c_int64, C.c_int32, vp]
        L.pso_discretize.argtypes = [vp, vp, C.c_int32, C.c_int32, C.POINTER(Params), C.c_uint64, vp, vp,
                                     C.c_int32, vp]
        _lib = L
    return _lib


def status_string(st):
    try:
        return lib().qap_status_string(st).decode()
    except Exception:
        return str(st)


def _check(st, what):
    if st != OK:
        raise QapError(st, what)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def default_params(**kw) -> Params:
    p = Params()
    lib().pso_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def cost_stats_noalloc(costs_dev_ptr, count, stream=None):
    """Statistics of `count` int64 costs already in device memory, computed without
    any device allocation (for callers that must not allocate; see the header).
    Returns dict(min, p5, p25, p50, p75, max, mean)."""
    out = np.zeros(6, np.int64)
    mean = C.c_double()
    st = C.c_void_p(stream) if stream else None
    _check(lib().qap_cost_stats_noalloc(C.c_void_p(costs_dev_ptr), count, st, _ptr(out),
                                        C.byref(mean)), "qap_cost_stats_noalloc")
    return dict(min=int(out[0]), p5=int(out[1]), p25=int(out[2]), p50=int(out[3]),
                p75=int(out[4]), max=int(out[5]), mean=mean.value)


def int32_peak(stream=None):
    """Measured integer throughput of the current GPU: (multiply-add lane operations/s
    counting two per multiply-add, add lane operations/s)."""
    mad, add = C.c_double(), C.c_double()
    st = C.c_void_p(stream) if stream else None
    _check(lib().qap_int32_peak(st, C.byref(mad), C.byref(add)), "qap_int32_peak")
    return mad.value, add.value


def philox(seed, c0, c1, c2, tag, block):
    """The library's Philox4x32-10 draw (host code): four uint32 words."""
    out = np.zeros(4, np.uint32)
    _check(lib().qap_philox(seed, c0, c1, c2, tag, block, _ptr(out)), "qap_philox")
    return out


def footprint(n, params):
    """Device bytes a population of size n with these parameters allocates."""
    b = C.c_size_t()
    _check(lib().pso_footprint(n, C.byref(params), C.byref(b)), "pso_footprint")
    return b.value


class Instance:
    """A QAP instance resident on the device (F, D copied at construction)."""

    def __init__(self, F, D):
        F = np.ascontiguousarray(F, np.int32)
        D = np.ascontiguousarray(D, np.int32)
        if F.shape != D.shape or F.ndim != 2 or F.shape[0] != F.shape[1]:
            raise ValueError("F and D must be square and of equal size")
        self.n = F.shape[0]
        h = C.c_void_p()
        _check(lib().qap_create_instance(self.n, _ptr(F), _ptr(D), C.byref(h)), "qap_create_instance")
        self.h = h

    def info(self):
        i = InstanceInfo()
        _check(lib().qap_instance_info(self.h, C.byref(i)), "qap_instance_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def eval_costs(self, perms):
        perms = np.ascontiguousarray(perms, np.int32).reshape(-1, self.n)
        out = np.zeros(len(perms), np.int64)
        _check(lib().qap_eval_costs(self.h, _ptr(perms), len(perms), _ptr(out)), "qap_eval_costs")
        return out

    def local_search(self, perms, max_moves=0):
        perms = np.ascontiguousarray(perms, np.int32).reshape(-1, self.n).copy()
        k = len(perms)
        costs = np.zeros(k, np.int64)
        moves = np.zeros(k, np.int32)
        rounds = np.zeros(k, np.int32)
        _check(lib().qap_local_search(self.h, _ptr(perms), k, max_moves, _ptr(costs), _ptr(moves),
                                      _ptr(rounds)), "qap_local_search")
        return perms, costs, moves, rounds

    def search_with(self, kernel, perms, max_moves=0, timed=False):
        """The goal function (max_moves < 0) or the local search on the named search
        kernel (SEARCH_*); returns (perms, costs, moves, rounds), plus the kernel's
        device milliseconds when timed."""
        perms = np.ascontiguousarray(perms, np.int32).reshape(-1, self.n).copy()
        k = len(perms)
        costs = np.zeros(k, np.int64)
        moves = np.zeros(k, np.int32)
        rounds = np.zeros(k, np.int32)
        ms = C.c_float()
        _check(lib().qap_search_with(self.h, kernel, _ptr(perms), k, max_moves, _ptr(costs), _ptr(moves),
                                     _ptr(rounds), C.byref(ms) if timed else None), "qap_search_with")
        return (perms, costs, moves, rounds, ms.value) if timed else (perms, costs, moves, rounds)

    def delta_table(self, perm):
        """Delta(r, s) of every pair r < s of `perm`, r-major (n (n - 1) / 2 int64)."""
        perm = np.ascontiguousarray(perm, np.int32).reshape(self.n)
        out = np.zeros(self.n * (self.n - 1) // 2, np.int64)
        _check(lib().qap_delta_table(self.h, _ptr(perm), _ptr(out)), "qap_delta_table")
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().qap_destroy_instance(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def discretize(Y, Z, params: Params, seed: int, swarm, particle, t: int):
    """S_x (SecondTarget) of count matrices Y (count x n x n fp32) with Z (count x n
    permutations); ties draw from the Philox stream of (particle, swarm, t)."""
    Y = np.ascontiguousarray(Y, np.float32)
    if Y.ndim == 2:
        Y = Y[None]
    count, n = Y.shape[0], Y.shape[1]
    Z = np.ascontiguousarray(Z, np.int32).reshape(count, n)
    sw = np.ascontiguousarray(np.broadcast_to(np.asarray(swarm, np.int32), (count,)))
    pa = np.ascontiguousarray(np.broadcast_to(np.asarray(particle, np.int32), (count,)))
    out = np.zeros((count, n), np.int32)
    _check(lib().pso_discretize(_ptr(Y), _ptr(Z), n, count, C.byref(params), seed, _ptr(sw), _ptr(pa), t,
                                _ptr(out)), "pso_discretize")
    return out


class Swarm:
    """Population state of one PSO run on the device."""

    def __init__(self, inst: Instance, params: Params, seed: int, stream=None, _handle=None,
                 first_swarm=None):
        """first_swarm: the state is the part of a larger run holding swarms
        first_swarm .. first_swarm + params.swarms - 1 (pso_init_part; no migration)."""
        self.inst = inst  # keeps the instance alive
        self.params = params
        self.n = inst.n
        self.P = params.swarms * params.swarm_size
        self._owned = _handle is None
        if _handle is not None:
            self.h = _handle
            return
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        if first_swarm is None:
            _check(lib().pso_init(inst.h, C.byref(params), seed, st, C.byref(h)), "pso_init")
        else:
            _check(lib().pso_init_part(inst.h, C.byref(params), seed, first_swarm, st, C.byref(h)),
                   "pso_init_part")
        self.h = h

    def swarm_bests(self):
        """(costs m int64, permutations m x n int32) of the swarm bests P^G."""
        m = self.params.swarms
        costs = np.zeros(m, np.int64)
        perms = np.zeros((m, self.n), np.int32)
        _check(lib().pso_swarm_bests(self.h, _ptr(costs), _ptr(perms)), "pso_swarm_bests")
        return costs, perms

    def set_swarm_best(self, swarm, cost, perm):
        perm = np.ascontiguousarray(perm, np.int32)
        _check(lib().pso_set_swarm_best(self.h, swarm, int(cost), _ptr(perm)), "pso_set_swarm_best")

    def particle(self, index):
        """(cost, permutation) of particle `index` (swarm-major within the state)."""
        c = C.c_int64()
        perm = np.zeros(self.n, np.int32)
        _check(lib().pso_particle(self.h, index, C.byref(c), _ptr(perm)), "pso_particle")
        return c.value, perm

    def step(self, iterations=1):
        _check(lib().pso_step(self.h, iterations), "pso_step")

    def step_timed(self, iterations=1, flush_ptr=None, flush_bytes=0):
        """Runs iterations with per-kernel device times; returns milliseconds of
        [position S_x, goal function + local search, bests + migration, span, velocity]."""
        ms = (C.c_float * 5)()
        fp = C.c_void_p(flush_ptr) if flush_ptr else None
        _check(lib().pso_step_timed(self.h, iterations, fp, flush_bytes, ms), "pso_step_timed")
        return list(ms)

    def done(self):
        """True when all work queued on this population's stream has finished."""
        d = C.c_int32()
        _check(lib().pso_poll(self.h, C.byref(d)), "pso_poll")
        return bool(d.value)

    def best(self):
        c = C.c_int64()
        it = C.c_int32()
        perm = np.zeros(self.n, np.int32)
        _check(lib().pso_best(self.h, C.byref(c), _ptr(perm), C.byref(it)), "pso_best")
        return c.value, perm, it.value

    def stats(self):
        s = Stats()
        s.size = C.sizeof(Stats)
        _check(lib().pso_stats(self.h, C.byref(s)), "pso_stats")
        return s.as_dict()

    def stats_swarm(self, swarm):
        """Statistics of one swarm's current costs (section 4.2's swarm percentiles)."""
        s = Stats()
        s.size = C.sizeof(Stats)
        _check(lib().pso_stats_swarm(self.h, swarm, C.byref(s)), "pso_stats_swarm")
        return s.as_dict()

    def cost_histogram(self, lo, hi, bins, swarm=-1):
        """Counts of current costs: [below lo, bins equal-width bins of [lo, hi), >= hi]."""
        out = np.zeros(bins + 2, np.int64)
        _check(lib().pso_cost_histogram(self.h, swarm, lo, hi, bins, _ptr(out)), "pso_cost_histogram")
        return out

    def trace_start(self, capacity, lo, hi, bins):
        """Record the statistics of every following iteration on the device."""
        _check(lib().pso_trace_start(self.h, capacity, lo, hi, bins), "pso_trace_start")

    def trace_read(self, max_records=None):
        """The recorded iterations, oldest first: a list of dicts with t, the population
        statistics, per-swarm statistics (m x 7: min, p5, p25, p50, p75, max, mean) and
        the histogram."""
        ln = C.c_int32()
        _check(lib().pso_trace_record_len(self.h, C.byref(ln)), "pso_trace_record_len")
        cap = max_records if max_records is not None else 1 << 16
        buf = np.zeros((cap, ln.value), np.int64)
        cnt = C.c_int32()
        _check(lib().pso_trace_read(self.h, _ptr(buf), cap, C.byref(cnt)), "pso_trace_read")
        m = self.params.swarms
        out = []
        for r in buf[: cnt.value]:
            def block(w, count):
                total = (int(w[7]) << 64) | (int(w[6]) & 0xFFFFFFFFFFFFFFFF)
                q, rem = int(total // count), int(total % count)
                if total < 0 and rem:  # truncated quotient, as the C side divides
                    q, rem = q + 1, rem - count
                return dict(min=int(w[0]), p5=int(w[1]), p25=int(w[2]), p50=int(w[3]), p75=int(w[4]),
                            max=int(w[5]), mean=float(q) + float(rem) / count, sum=total)
            out.append(dict(t=int(r[0]), population=block(r[1:9], self.P),
                            swarms=[block(r[9 + 8 * k: 17 + 8 * k], self.params.swarm_size) for k in range(m)],
                            histogram=r[9 + 8 * m:].copy()))
        return out

    def trace_stop(self):
        _check(lib().pso_trace_stop(self.h), "pso_trace_stop")

    def export_state(self):
        n, P, m = self.n, self.P, self.params.swarms
        a = dict(V=np.zeros((P, n, n), np.float32), X=np.zeros((P, n), np.int32),
                 X_sx=np.zeros((P, n), np.int32), PL=np.zeros((P, n), np.int32),
                 costL=np.zeros(P, np.int64), cost=np.zeros(P, np.int64),
                 moves=np.zeros(P, np.int32), PG=np.zeros((m, n), np.int32),
                 costG=np.zeros(m, np.int64), best=np.zeros(n, np.int32))
        hs = HostState()
        for k, v in a.items():
            ty = {np.float32: C.c_float, np.int32: C.c_int32, np.int64: C.c_int64}[v.dtype.type]
            setattr(hs, k, v.ctypes.data_as(C.POINTER(ty)))
        _check(lib().pso_export_state(self.h, C.byref(hs)), "pso_export_state")
        a["best_cost"], a["best_iter"], a["t"] = hs.best_cost, hs.best_iter, hs.t
        return a

    def import_state(self, a):
        hs = HostState()
        keep = {}
        for k, dt, ty in (("V", np.float32, C.c_float), ("X", np.int32, C.c_int32),
                          ("PL", np.int32, C.c_int32), ("costL", np.int64, C.c_int64),
                          ("cost", np.int64, C.c_int64), ("PG", np.int32, C.c_int32),
                          ("costG", np.int64, C.c_int64), ("best", np.int32, C.c_int32)):
            v = np.ascontiguousarray(a[k], dt)
            keep[k] = v
            setattr(hs, k, v.ctypes.data_as(C.POINTER(ty)))
        hs.best_cost, hs.best_iter, hs.t = int(a["best_cost"]), int(a["best_iter"]), int(a["t"])
        _check(lib().pso_import_state(self.h, C.byref(hs)), "pso_import_state")

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                lib().pso_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many populations (instances of uneven n) advanced by shared launches."""

    def __init__(self, instances, params, seeds, stream=None, autotune=True):
        self.instances = list(instances)
        self.params = list(params)
        k = len(self.instances)
        if len(self.params) != k or len(seeds) != k:
            raise ValueError("instances, params and seeds must have equal length")
        handles = (C.c_void_p * k)(*[i.h for i in self.instances])
        parr = (Params * k)(*self.params)
        sarr = (C.c_uint64 * k)(*[int(s) for s in seeds])
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        _check(lib().pso_batch_create(k, handles, parr, sarr, st, 1 if autotune else 0, C.byref(h)),
               "pso_batch_create")
        self.h = h
        self.members = []
        for i in range(k):
            mh = C.c_void_p()
            _check(lib().pso_batch_member(self.h, i, C.byref(mh)), "pso_batch_member")
            self.members.append(Swarm(self.instances[i], self.params[i], 0, _handle=mh))

    def step(self, iterations=1):
        _check(lib().pso_batch_step(self.h, iterations), "pso_batch_step")

    def step_timed(self, iterations=1, flush_ptr=None, flush_bytes=0):
        ms = (C.c_float * 5)()
        fp = C.c_void_p(flush_ptr) if flush_ptr else None
        _check(lib().pso_batch_step_timed(self.h, iterations, fp, flush_bytes, ms), "pso_batch_step_timed")
        return list(ms)

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            lib().pso_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
