"""ctypes front end of the plain-C CPU oracle (``oracle/*.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The oracle shares no code with the CUDA
library and this module imports nothing from the product package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["philox.c", "qap.c", "pso.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

TAG_R, TAG_TIE, TAG_INIT_X, TAG_INIT_V, TAG_MIG = 0, 1, 2, 3, 4
C_PIT, C_MOVES, C_ROUNDS, C_DELTA_FULL, C_DELTA_INCR, C_TIES = range(6)
NCOUNTERS = 6


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so with gcc (plain C11)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("swarms", C.c_int32), ("swarm_size", C.c_int32),
        ("c1", C.c_double), ("c2", C.c_double), ("c3", C.c_double),
        ("sv_kind", C.c_int32), ("v_max", C.c_double),
        ("depth", C.c_int32), ("sx_rule", C.c_int32), ("tie_rule", C.c_int32),
        ("pos_uses_new_v", C.c_int32), ("ls_max_moves", C.c_int32), ("ls_at_init", C.c_int32),
        ("mig_kind", C.c_int32), ("mig_depth", C.c_int32), ("mig_period", C.c_int32),
        ("ring_if_better", C.c_int32), ("v_storage", C.c_int32), ("sx_kind", C.c_int32),
    ]


class _State(C.Structure):
    _fields_ = [
        ("V", C.POINTER(C.c_double)), ("X", C.POINTER(C.c_int32)), ("PL", C.POINTER(C.c_int32)),
        ("costL", C.POINTER(C.c_int64)), ("cost", C.POINTER(C.c_int64)),
        ("PG", C.POINTER(C.c_int32)), ("costG", C.POINTER(C.c_int64)),
        ("best_p", C.POINTER(C.c_int32)), ("best_cost", C.POINTER(C.c_int64)),
        ("best_iter", C.POINTER(C.c_int32)), ("t", C.POINTER(C.c_int32)),
        ("counters", C.POINTER(C.c_int64)), ("moves", C.POINTER(C.c_int32)),
    ]


_I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_I64P = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_F32P = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_U32P = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_U32P, _U32P, _U32P]
            L.orc_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.c_uint32, _U32P]
            L.orc_u01.argtypes = [C.c_uint32]
            L.orc_u01.restype = C.c_double
            L.orc_below.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_below.restype = C.c_uint32
            for f in ("orc_cost", "orc_cost_eq1"):
                getattr(L, f).argtypes = [C.c_int, _I32P, _I32P, _I32P]
                getattr(L, f).restype = C.c_int64
            L.orc_delta.argtypes = [C.c_int, _I32P, _I32P, _I32P, C.c_int, C.c_int]
            L.orc_delta.restype = C.c_int64
            L.orc_local_search.argtypes = [C.c_int, _I32P, _I32P, _I32P, C.c_int,
                                           C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                           C.c_void_p, C.c_int]
            L.orc_local_search.restype = C.c_int
            L.orc_brute_force.argtypes = [C.c_int, _I32P, _I32P, _I32P]
            L.orc_brute_force.restype = C.c_int64
            L.orc_round_bf16.argtypes = [C.c_double]
            L.orc_round_bf16.restype = C.c_double
            L.orc_velocity.argtypes = [C.POINTER(Params), C.c_int, _F64P, _I32P, _I32P, _I32P,
                                       C.c_double, C.c_double, _F64P]
            L.orc_second_target.argtypes = [C.POINTER(Params), C.c_int, _F32P, _I32P, C.c_uint64,
                                            C.c_uint32, C.c_uint32, C.c_uint32, _I32P, C.c_void_p]
            L.orc_second_target.restype = C.c_int
            L.orc_pick_column.argtypes = [C.POINTER(Params), C.c_int, _F32P, C.c_uint64, C.c_uint32,
                                          C.c_uint32, C.c_uint32, _I32P, C.c_void_p]
            L.orc_pick_column.restype = C.c_int
            L.orc_particle_iteration.argtypes = [
                C.POINTER(Params), C.c_int, _I32P, _I32P, C.c_uint64, C.c_int, C.c_int, C.c_int,
                _F64P, _I32P, _I32P, _I32P, _F64P, _I32P, _I32P, C.POINTER(C.c_int64),
                C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
            for f in ("orc_init", "orc_step"):
                getattr(L, f).argtypes = [C.POINTER(Params), C.c_int, _I32P, _I32P, C.c_uint64,
                                          C.POINTER(_State)]
            L.orc_bests_and_migration.argtypes = [C.POINTER(Params), C.c_int, C.c_uint64, C.c_int,
                                                  C.POINTER(_State)]
            L.orc_stats.argtypes = [_I64P, C.c_int, _I64P, C.POINTER(C.c_double)]
            L.orc_histogram.argtypes = [_I64P, C.c_int, C.c_int64, C.c_int64, C.c_int, _I64P]
            L.orc_histogram.restype = None
            _lib = L
    return _lib


# --------------------------------------------------------------------------- params

DEFAULTS = dict(swarms=1, swarm_size=32, c1=0.8, c2=0.5, c3=0.5, sv_kind=1, v_max=1.0, depth=2,
                sx_rule=0, tie_rule=0, pos_uses_new_v=0, ls_max_moves=0, ls_at_init=0,
                mig_kind=0, mig_depth=0, mig_period=1, ring_if_better=0, v_storage=0, sx_kind=0)


def make_params(**kw) -> Params:
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    p = Params()
    for k, v in d.items():
        # coefficients are fp32 values on the device; the oracle takes them exactly
        if k in ("c1", "c2", "c3", "v_max"):
            v = float(np.float32(v))
        setattr(p, k, v)
    return p


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# --------------------------------------------------------------------------- wrappers

def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def draw(seed, c0, c1, c2, tag, block):
    out = np.zeros(4, np.uint32)
    lib().orc_draw(seed, c0, c1, c2, tag, block, out)
    return out


def u01(u):
    return lib().orc_u01(int(u))


def below(u, k):
    return lib().orc_below(int(u), int(k))


def cost(F, D, p):
    F, D = _i32(F), _i32(D)
    return lib().orc_cost(F.shape[0], F, D, _i32(p))


def cost_eq1(F, D, p):
    F, D = _i32(F), _i32(D)
    return lib().orc_cost_eq1(F.shape[0], F, D, _i32(p))


def delta(F, D, p, r, s):
    F, D = _i32(F), _i32(D)
    return lib().orc_delta(F.shape[0], F, D, _i32(p), r, s)


def local_search(F, D, p, max_moves=0, trace_cap=0):
    """Returns (perm, cost, moves, rounds, trace)."""
    F, D = _i32(F), _i32(D)
    p = _i32(p).copy()
    c, r = C.c_int64(), C.c_int64()
    tr = np.zeros(max(2 * trace_cap, 2), np.int32)
    mv = lib().orc_local_search(F.shape[0], F, D, p, max_moves, C.byref(c), C.byref(r),
                                tr.ctypes.data if trace_cap else None, trace_cap)
    return p, c.value, mv, r.value, tr[: 2 * min(mv, trace_cap)].reshape(-1, 2)


def brute_force(F, D):
    F, D = _i32(F), _i32(D)
    bp = np.zeros(F.shape[0], np.int32)
    c = lib().orc_brute_force(F.shape[0], F, D, bp)
    return c, bp


def round_bf16(x):
    return lib().orc_round_bf16(float(x))


def velocity(q: Params, V, x, pl, pg, r2, r3):
    n = len(x)
    out = np.zeros((n, n), np.float64)
    lib().orc_velocity(C.byref(q), n, np.ascontiguousarray(V, np.float64), _i32(x), _i32(pl),
                       _i32(pg), float(r2), float(r3), out)
    return out


def second_target(q: Params, Y, z, seed=0, c0=0, c1=0, c2=0, want_order=False):
    n = len(z)
    out = np.zeros(n, np.int32)
    order = np.zeros((n, 2), np.int32)
    ties = lib().orc_second_target(C.byref(q), n, np.ascontiguousarray(Y, np.float32), _i32(z),
                                   seed, c0, c1, c2, out, order.ctypes.data if want_order else None)
    if want_order:
        return out, ties, order
    return out, ties


def pick_column(q: Params, Y, seed=0, c0=0, c1=0, c2=0, want_order=False):
    n = Y.shape[0]
    out = np.zeros(n, np.int32)
    order = np.zeros((n, 2), np.int32)
    ties = lib().orc_pick_column(C.byref(q), n, np.ascontiguousarray(Y, np.float32), seed, c0, c1, c2, out,
                                 order.ctypes.data if want_order else None)
    if want_order:
        return out, ties, order
    return out, ties


def particle_iteration(q: Params, F, D, seed, t, swarm, pis, V, x, pl, pg):
    """One particle's iteration; returns dict(V_new, p_sx, p_out, cost, moves, rounds, ties)."""
    F, D = _i32(F), _i32(D)
    n = F.shape[0]
    Vn = np.zeros((n, n), np.float64)
    psx = np.zeros(n, np.int32)
    pout = np.zeros(n, np.int32)
    c, mv, rd, nt = C.c_int64(), C.c_int32(), C.c_int64(), C.c_int32()
    lib().orc_particle_iteration(C.byref(q), n, F, D, seed, t, swarm, pis,
                                 np.ascontiguousarray(V, np.float64), _i32(x), _i32(pl), _i32(pg),
                                 Vn, psx, pout, C.byref(c), C.byref(mv), C.byref(rd), C.byref(nt))
    return dict(V_new=Vn, p_sx=psx, p_out=pout, cost=c.value, moves=mv.value, rounds=rd.value,
                ties=nt.value)


class State:
    """Whole-population oracle state, as numpy arrays."""

    def __init__(self, q: Params, n: int):
        m, ss = q.swarms, q.swarm_size
        P = m * ss
        self.q, self.n = q, n
        self.V = np.zeros((P, n, n), np.float64)
        self.X = np.zeros((P, n), np.int32)
        self.PL = np.zeros((P, n), np.int32)
        self.costL = np.zeros(P, np.int64)
        self.cost = np.zeros(P, np.int64)
        self.PG = np.zeros((m, n), np.int32)
        self.costG = np.zeros(m, np.int64)
        self.best_p = np.zeros(n, np.int32)
        self.best_cost = np.zeros(1, np.int64)
        self.best_iter = np.zeros(1, np.int32)
        self.t = np.zeros(1, np.int32)
        self.counters = np.zeros(NCOUNTERS, np.int64)
        self.moves = np.zeros(P, np.int32)

    def _c(self):
        def p(a, ty):
            return a.ctypes.data_as(C.POINTER(ty))
        return _State(p(self.V, C.c_double), p(self.X, C.c_int32), p(self.PL, C.c_int32),
                      p(self.costL, C.c_int64), p(self.cost, C.c_int64), p(self.PG, C.c_int32),
                      p(self.costG, C.c_int64), p(self.best_p, C.c_int32),
                      p(self.best_cost, C.c_int64), p(self.best_iter, C.c_int32),
                      p(self.t, C.c_int32), p(self.counters, C.c_int64), p(self.moves, C.c_int32))

    def copy(self):
        o = State.__new__(State)
        o.q, o.n = self.q, self.n
        for k in ("V", "X", "PL", "costL", "cost", "PG", "costG", "best_p", "best_cost",
                  "best_iter", "t", "counters", "moves"):
            setattr(o, k, getattr(self, k).copy())
        return o


def init(q: Params, F, D, seed) -> State:
    F, D = _i32(F), _i32(D)
    s = State(q, F.shape[0])
    cs = s._c()
    lib().orc_init(C.byref(q), F.shape[0], F, D, seed, C.byref(cs))
    return s


def step(q: Params, F, D, seed, s: State, iterations: int = 1) -> State:
    F, D = _i32(F), _i32(D)
    cs = s._c()
    for _ in range(iterations):
        lib().orc_step(C.byref(q), F.shape[0], F, D, seed, C.byref(cs))
    return s


def step_parallel(q: Params, F, D, seed, s: State, iterations: int = 1, threads=None) -> State:
    """The same iterations as step(), with the particles spread over `threads` host
    threads (default: every core): each particle goes through the oracle's
    particle_iteration (its C code releases the GIL), then the end-of-iteration
    bookkeeping runs once, as in orc_step. Nothing of the arithmetic changes, so the
    result equals step()."""
    from concurrent.futures import ThreadPoolExecutor
    F, D = _i32(F), _i32(D)
    n = F.shape[0]
    ss = q.swarm_size
    P = q.swarms * ss
    npairs = n * (n - 1) // 2
    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        for _ in range(iterations):
            t = int(s.t[0])

            def one(idx):
                k, i = divmod(idx, ss)
                return particle_iteration(q, F, D, seed, t, k, i, s.V[idx], s.X[idx], s.PL[idx], s.PG[k])

            for idx, r in enumerate(ex.map(one, range(P))):
                s.V[idx] = r["V_new"]
                s.X[idx] = r["p_out"]
                s.cost[idx] = r["cost"]
                if r["cost"] < s.costL[idx]:
                    s.costL[idx] = r["cost"]
                    s.PL[idx] = r["p_out"]
                s.moves[idx] = r["moves"]
                s.counters[C_PIT] += 1
                s.counters[C_MOVES] += r["moves"]
                s.counters[C_ROUNDS] += r["rounds"]
                if r["rounds"] > 0:
                    s.counters[C_DELTA_FULL] += npairs
                    s.counters[C_DELTA_INCR] += (r["rounds"] - 1) * npairs
                s.counters[C_TIES] += r["ties"]
            bests_and_migration(q, seed, t, s)
            s.t[0] = t + 1
    return s


def bests_and_migration(q: Params, seed, t, s: State) -> State:
    cs = s._c()
    lib().orc_bests_and_migration(C.byref(q), s.n, seed, t, C.byref(cs))
    return s


def histogram(cost, lo, hi, bins):
    cost = np.ascontiguousarray(cost, np.int64)
    out = np.zeros(bins + 2, np.int64)
    lib().orc_histogram(cost, len(cost), int(lo), int(hi), int(bins), out)
    return out


def stats(cost):
    cost = np.ascontiguousarray(cost, np.int64)
    out = np.zeros(6, np.int64)
    mean = C.c_double()
    lib().orc_stats(cost, len(cost), out, C.byref(mean))
    return dict(min=int(out[0]), p5=int(out[1]), p25=int(out[2]), p50=int(out[3]),
                p75=int(out[4]), max=int(out[5]), mean=mean.value)
