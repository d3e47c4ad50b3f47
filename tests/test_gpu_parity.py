"""CUDA path against the oracle, element by element, on identical seeded inputs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W
from tests.replay import check_velocity, compare_step, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1504_05158_gb300 import qap_pso
    qap_pso.lib()
    return qap_pso


INSTANCES = {
    "n2": lambda: W.dense_uniform(2, 1),
    "n3": lambda: W.dense_uniform(3, 2),
    "tiny9": W.tiny9,
    "dense30": W.dense30,
    "n33": lambda: W.dense_uniform(33, 5),
    "grid64": W.grid64,
    "n65grid": lambda: W.grid_sparse(65, 6),
    "n97": lambda: W.dense_uniform(97, 10),
    "n100": lambda: W.dense_uniform(100, 7),
    "n128grid": lambda: W.grid_sparse(128, 8),
    "n150": lambda: W.dense_uniform(150, 9),
    "n80wide": lambda: W.dense_uniform(80, 11, 0, 400),  # entries above 255: 16-bit staging
    "n160grid": lambda: W.grid_sparse(160, 12),
}


# ------------------------------------------------------------ goal function

@pytest.mark.parametrize("name", list(INSTANCES))
def test_eval_costs_bit_exact(Q, name):
    inst = INSTANCES[name]()
    gi = Q.Instance(inst.F, inst.D)
    perms = W.random_perms(77, inst.n, 3)
    got = gi.eval_costs(perms)
    want = np.array([O.cost(inst.F, inst.D, p) for p in perms])
    assert np.array_equal(got, want)


def test_eval_costs_general_instance(Q):
    inst = W.random_asymmetric(21, 4, hi=200)
    gi = Q.Instance(inst.F, inst.D)
    assert gi.info()["symmetric_zero_diag"] == 0
    perms = W.random_perms(40, 21, 4)
    assert np.array_equal(gi.eval_costs(perms), [O.cost(inst.F, inst.D, p) for p in perms])


# ------------------------------------------------------------ local search

@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("cap", [0, 3])
def test_local_search_bit_exact(Q, name, cap):
    inst = INSTANCES[name]()
    gi = Q.Instance(inst.F, inst.D)
    count = 40 if inst.n <= 64 else 9  # the oracle's search is O(n^3) per round
    perms = W.random_perms(count, inst.n, 11)
    gp, gc, gm, gr = gi.local_search(perms, cap)
    for i, p in enumerate(perms):
        op, oc, om, orr, _ = O.local_search(inst.F, inst.D, p, cap)
        assert np.array_equal(gp[i], op) and gc[i] == oc and gm[i] == om and gr[i] == orr, i


def test_local_search_rejects_bad_input(Q):
    inst = W.dense_uniform(8, 1)
    gi = Q.Instance(inst.F, inst.D)
    with pytest.raises(Q.QapError):
        gi.local_search(np.zeros((1, 8), np.int32))  # not a permutation
    # entries so large that costs could leave int64: refused, never wrapped
    n = 64
    huge = np.full((n, n), 2**31 - 1, np.int32)
    np.fill_diagonal(huge, 0)
    gh = Q.Instance(huge, huge)
    assert gh.info()["exact_int64"] == 0
    for call in (lambda: gh.local_search(W.random_perms(1, n, 1)),
                 lambda: gh.eval_costs(W.random_perms(1, n, 1)),
                 lambda: Q.Swarm(gh, Q.default_params(), seed=1)):
        with pytest.raises(Q.QapError) as e:
            call()
        assert e.value.status == Q.ERR_OVERFLOW
    # a kernel that is not exact for the instance is refused by name
    big = W.random_asymmetric(8, 2, hi=3000)
    ga = Q.Instance(big.F, big.D)
    for k in (Q.SEARCH_TENSOR, Q.SEARCH_SIMT):
        with pytest.raises(Q.QapError) as e:
            ga.search_with(k, W.random_perms(1, 8, 1))
        assert e.value.status == Q.ERR_UNSUPPORTED


# ------------------------------------------------------------ init

@pytest.mark.parametrize("storage", [0, 1])
def test_init_bit_exact(Q, storage):
    inst = W.dense30()
    prm = Q.default_params(swarms=3, swarm_size=37, v_storage=storage, v_max=0.75)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=123)
    st = sw.export_state()
    q = oracle_params(prm)
    o = O.init(q, inst.F, inst.D, 123)
    assert np.array_equal(st["X"], o.X) and np.array_equal(st["cost"], o.cost)
    assert np.array_equal(st["V"].astype(np.float64), o.V)
    assert np.array_equal(st["PL"], o.PL) and np.array_equal(st["costL"], o.costL)
    assert np.array_equal(st["PG"], o.PG) and np.array_equal(st["costG"], o.costG)
    assert st["best_cost"] == o.best_cost[0] and np.array_equal(st["best"], o.best_p)
    assert st["t"] == 0 and st["best_iter"] == 0


# ------------------------------------------------------------ whole iterations

VARIANTS = {
    "default": dict(),
    "raw": dict(sv_kind=0, v_max=0.5),
    "topd": dict(sx_rule=1, depth=3),
    "globalmax": dict(depth=0),
    "tiefirst": dict(tie_rule=1, sv_kind=0, v_max=0.25),
    "newv": dict(pos_uses_new_v=1),
    "bf16": dict(v_storage=1),
    "nols": dict(ls_max_moves=-1),
    "lscap": dict(ls_max_moves=2, ls_at_init=1),
    "rank": dict(mig_kind=1, mig_depth=1, mig_period=1),
    "ring": dict(mig_kind=2, mig_period=2),
    "ringbetter": dict(mig_kind=2, mig_period=1, ring_if_better=1),
    "pickcol": dict(sx_kind=1),
    "pickcol_newv_first": dict(sx_kind=1, pos_uses_new_v=1, tie_rule=1),
}


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("name,m,ss", [("tiny9", 3, 11), ("dense30", 3, 21), ("grid64", 4, 13)])
def test_iterations_replay(Q, variant, name, m, ss):
    inst = INSTANCES[name]()
    kw = dict(swarms=m, swarm_size=ss)
    kw.update(VARIANTS[variant])
    prm = Q.default_params(**kw)
    seed = 1000 + m
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=seed)
    q = oracle_params(prm)
    before = sw.export_state()
    for _ in range(3):
        sw.step(1)
        after = sw.export_state()
        compare_step(q, inst.F, inst.D, seed, before, after, prm)
        before = after


@pytest.mark.parametrize("name", ["n2", "n3", "n65grid", "n80wide", "n100", "n150", "n160grid"])
def test_iterations_replay_edge_sizes(Q, name):
    inst = INSTANCES[name]()
    prm = Q.default_params(swarms=2, swarm_size=5, depth=min(2, inst.n - 1), mig_kind=1,
                           mig_depth=0)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=5)
    q = oracle_params(prm)
    before = sw.export_state()
    for _ in range(2):
        sw.step(1)
        after = sw.export_state()
        compare_step(q, inst.F, inst.D, 5, before, after, prm)
        before = after


def test_ties_from_imported_state(Q):
    # velocities in {-1, 0, 1}: most S_x steps see several equal maxima
    inst = W.dense_uniform(20, 3)
    for rule in (0, 1):
        prm = Q.default_params(swarms=2, swarm_size=9, sv_kind=0, depth=3, sx_rule=rule)
        sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=9)
        st = sw.export_state()
        rng = np.random.default_rng(rule)
        st["V"] = rng.integers(-1, 2, st["V"].shape).astype(np.float32)
        sw.import_state(st)
        before = sw.export_state()
        sw.step(1)
        after = sw.export_state()
        compare_step(oracle_params(prm), inst.F, inst.D, 9, before, after, prm)
        assert sw.stats()["sx_ties"] > 0


def test_full_size_grid64_sampled(Q):
    # the n = 64, 16 x 640 workload, with ring migration every 20 iterations
    inst = W.grid64()
    for storage in (0, 1):
        prm = Q.default_params(swarms=16, swarm_size=640, mig_kind=2, mig_period=20,
                               v_storage=storage)
        sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=64)
        q = oracle_params(prm)
        sw.step(18)
        before = sw.export_state()
        rng = np.random.default_rng(storage)
        for _ in range(3):  # iterations 19, 20 (ring), 21
            sw.step(1)
            after = sw.export_state()
            sample = np.concatenate([[0, 639, 640, 10239], rng.choice(10240, 28, replace=False)])
            compare_step(q, inst.F, inst.D, 64, before, after, prm, sample=sample)
            before = after


def _most_tied(q, before, seed, candidates, k):
    """The k candidates whose S_x (on the exported V(t) and X(t), by the oracle) has
    the most steps with several maxima."""
    from concurrent.futures import ThreadPoolExecutor
    n = before["X"].shape[1]
    ss = q.swarm_size
    t = int(before["t"])

    def ties(p):
        sw, i = divmod(int(p), ss)
        Y = (before["V"][p] + (np.arange(n)[:, None] == before["X"][p][None, :])).astype(np.float32)
        return O.second_target(q, Y, before["X"][p], seed, i, sw, t)[1]

    with ThreadPoolExecutor(max_workers=8) as ex:  # the oracle's C calls release the GIL
        tc = np.array(list(ex.map(ties, candidates)))
    order = np.argsort(-tc, kind="stable")
    return np.asarray(candidates)[order[:k]], tc


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("start", [60, 200])
def test_full_size_grid64_tie_regime(Q, storage, start):
    # the n = 64, 16 x 640 workload deep in the run, where the swarms have converged and
    # most greedy steps of S_x choose among several equal maxima: iterations start + 1 ..
    # start + 3, on the most tied particles plus a random sample, element by element
    inst = W.grid64()
    prm = Q.default_params(swarms=16, swarm_size=640, mig_kind=2, mig_period=20, v_storage=storage)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=64)
    q = oracle_params(prm)
    sw.step(start)
    before = sw.export_state()
    rng = np.random.default_rng(start + storage)
    s0 = sw.stats()
    for _ in range(3):
        cand = rng.choice(10240, 1024, replace=False)
        tied, tc = _most_tied(q, before, 64, cand, 16)
        assert tc.mean() > 20, f"expected the tie regime, mean S_x ties {tc.mean():.1f}"
        rest = np.setdiff1d(rng.choice(10240, 24, replace=False), tied)[:16]
        sample = np.concatenate([tied, rest, [0, 10239]])
        sw.step(1)
        after = sw.export_state()
        compare_step(q, inst.F, inst.D, 64, before, after, prm, sample=sample)
        before = after
    s1 = sw.stats()
    assert s1["errors"] == 0
    assert (s1["sx_ties"] - s0["sx_ties"]) / (s1["particle_iterations"] - s0["particle_iterations"]) > 20


def test_full_size_dense30_sampled(Q):
    inst = W.dense30()
    prm = Q.default_params(swarms=10, swarm_size=1000)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=30)
    before = sw.export_state()
    sw.step(1)
    after = sw.export_state()
    compare_step(oracle_params(prm), inst.F, inst.D, 30, before, after, prm,
                 sample=np.arange(0, 10000, 313))


# ------------------------------------------------------------ results and statistics

def test_stats_and_best(Q):
    inst = W.dense30()
    prm = Q.default_params(swarms=5, swarm_size=200)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=77)
    sw.step(4)
    st = sw.export_state()
    got = sw.stats()
    want = O.stats(st["cost"])
    for k in ("min", "p5", "p25", "p50", "p75", "max"):
        assert got[k] == want[k], k
    assert got["mean"] == want["mean"]
    assert got["iteration"] == 4 and got["particle_iterations"] == 4 * 1000
    assert got["errors"] == 0
    assert got["ls_rounds"] == got["ls_moves"] + 4 * 1000
    n = 30
    assert got["delta_full"] == 4 * 1000 * n * (n - 1) // 2
    assert got["delta_incr"] == got["ls_moves"] * n * (n - 1) // 2
    c, perm, it = sw.best()
    assert c == got["best_cost"] == O.cost(inst.F, inst.D, perm) and 0 <= it <= 4


def test_tiny9_reaches_optimum(Q):
    inst = W.tiny9()
    opt, _ = O.brute_force(inst.F, inst.D)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), Q.default_params(swarms=1, swarm_size=32), seed=1)
    sw.step(100)
    c, perm, _ = sw.best()
    assert c == opt == O.cost(inst.F, inst.D, perm)


def test_invalid_params(Q):
    inst = W.dense_uniform(10, 1)
    gi = Q.Instance(inst.F, inst.D)
    for bad in (dict(depth=10), dict(swarms=0), dict(v_max=0.0), dict(mig_kind=1, mig_depth=1,
                                                                       swarms=2)):
        with pytest.raises(Q.QapError) as e:
            Q.Swarm(gi, Q.default_params(**bad), seed=1)
        assert e.value.status == Q.ERR_INVALID_ARG


KERNELS = {"tensor": "SEARCH_TENSOR", "simt": "SEARCH_SIMT", "int64": "SEARCH_INT64",
           "direct": "SEARCH_DIRECT"}


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("name", ["n3", "tiny9", "dense30", "n33", "grid64", "n65grid", "n97", "n128grid",
                                  "n80wide", "n150", "n160grid"])
def test_local_search_every_kernel(Q, kernel, name):
    # every search kernel that serves the instance gives the oracle's search exactly
    inst = INSTANCES[name]()
    gi = Q.Instance(inst.F, inst.D)
    k = getattr(Q, KERNELS[kernel])
    count = 37 if kernel != "direct" or inst.n <= 64 else 6  # the direct kernel is O(n^3) per round
    perms = W.random_perms(count, inst.n, 17)
    try:
        gp, gc, gm, gr = gi.search_with(k, perms, 0)
    except Q.QapError as e:
        assert e.status == Q.ERR_UNSUPPORTED
        assert kernel == "simt" and inst.n > 150, "only the int32 SIMT search has a smaller n limit here"
        return
    for i, p in enumerate(perms):
        op, oc, om, orr, _ = O.local_search(inst.F, inst.D, p, 0)
        assert np.array_equal(gp[i], op) and gc[i] == oc and gm[i] == om and gr[i] == orr, i
    _, costs, _, _ = gi.search_with(k, perms, -1)
    assert np.array_equal(costs, [O.cost(inst.F, inst.D, p) for p in perms])
    assert np.array_equal(gi.eval_costs(perms), costs)


def _large_symmetric(n, seed, hi_f, hi_d):
    rng = np.random.default_rng(seed)
    F = np.triu(rng.integers(0, hi_f + 1, (n, n)), 1)
    D = np.triu(rng.integers(0, hi_d + 1, (n, n)), 1)
    return (F + F.T).astype(np.int32), (D + D.T).astype(np.int32)


@pytest.mark.parametrize("n,hi_f,hi_d", [(5, 10**8, 10**8), (24, 10**5, 10**5), (64, 10**5, 10**5),
                                         (64, 40, 2_000_000), (97, 3000, 70_000), (150, 10**5, 10**5),
                                         (200, 10**4, 10**5)])
def test_large_entries_exact_int64(Q, n, hi_f, hi_d):
    # entries far beyond the int32 bound: costs and swap values need int64; the search
    # is still bit-exact
    F, D = _large_symmetric(n, n + hi_d % 97, hi_f, hi_d)
    gi = Q.Instance(F, D)
    info = gi.info()
    assert info["exact_int32"] == 0 and info["exact_int64"] == 1
    count = 12 if n <= 100 else 3
    perms = W.random_perms(count, n, 8)
    assert np.array_equal(gi.eval_costs(perms), [O.cost(F, D, p) for p in perms])
    gp, gc, gm, gr = gi.local_search(perms, 0)
    for i, p in enumerate(perms):
        op, oc, om, orr, _ = O.local_search(F, D, p, 0)
        assert np.array_equal(gp[i], op) and gc[i] == oc and gm[i] == om and gr[i] == orr, i


@pytest.mark.parametrize("n,hi", [(9, 10**6), (40, 50_000), (64, 100_000)])
def test_large_entries_general_instance(Q, n, hi):
    # asymmetric with a nonzero diagonal and entries up to 10^5 or more: the direct kernel
    inst = W.random_asymmetric(n, 21, hi=hi)
    gi = Q.Instance(inst.F, inst.D)
    perms = W.random_perms(8, n, 9)
    assert np.array_equal(gi.eval_costs(perms), [O.cost(inst.F, inst.D, p) for p in perms])
    gp, gc, gm, gr = gi.local_search(perms, 0)
    for i, p in enumerate(perms):
        op, oc, om, orr, _ = O.local_search(inst.F, inst.D, p, 0)
        assert np.array_equal(gp[i], op) and gc[i] == oc and gm[i] == om and gr[i] == orr, i


@pytest.mark.parametrize("general", [False, True])
def test_large_entries_iterations_replay(Q, general):
    # whole iterations on an instance with entries up to 10^5 (int64 search inside pso_step)
    n = 40
    if general:
        inst = W.random_asymmetric(n, 5, hi=100_000)
        F, D = inst.F, inst.D
    else:
        F, D = _large_symmetric(n, 3, 100_000, 100_000)
    prm = Q.default_params(swarms=3, swarm_size=7, mig_kind=1, mig_depth=1)
    sw = Q.Swarm(Q.Instance(F, D), prm, seed=41)
    q = oracle_params(prm)
    before = sw.export_state()
    for _ in range(3):
        sw.step(1)
        after = sw.export_state()
        compare_step(q, F, D, 41, before, after, prm)
        before = after
    assert sw.stats()["errors"] == 0


def test_large_values_use_exact_simt_setup(Q):
    # entries above 2048 leave the fp16 range: the SIMT set-up takes over, still exact
    rng = np.random.default_rng(3)
    n = 24
    F = rng.integers(0, 5000, (n, n))
    F = np.triu(F, 1)
    F = (F + F.T).astype(np.int32)
    D = rng.integers(0, 40, (n, n))
    D = np.triu(D, 1)
    D = (D + D.T).astype(np.int32)
    gi = Q.Instance(F, D)
    perms = W.random_perms(20, n, 4)
    gp, gc, gm, gr = gi.local_search(perms, 0)
    for i, p in enumerate(perms):
        op, oc, om, orr, _ = O.local_search(F, D, p, 0)
        assert np.array_equal(gp[i], op) and gc[i] == oc and gm[i] == om, i


# ------------------------------------------------------------ general instances

def _diag_instance(n, seed):
    """Symmetric F and D with a nonzero diagonal (installation costs)."""
    inst = W.dense_uniform(n, seed, 0, 60)
    rng = np.random.default_rng(seed)
    F = inst.F.copy()
    D = inst.D.copy()
    F[np.arange(n), np.arange(n)] = rng.integers(0, 30, n)
    D[np.arange(n), np.arange(n)] = rng.integers(0, 30, n)
    return F, D


@pytest.mark.parametrize("n,seed,hi", [(2, 1, 20), (3, 2, 20), (9, 3, 50), (21, 4, 200), (40, 5, 99),
                                       (64, 6, 99), (97, 7, 60), (128, 8, 40)])
@pytest.mark.parametrize("cap", [0, 2])
def test_general_local_search_bit_exact(Q, n, seed, hi, cap):
    inst = W.random_asymmetric(n, seed, hi=hi)
    gi = Q.Instance(inst.F, inst.D)
    assert gi.info()["symmetric_zero_diag"] == 0
    perms = W.random_perms(12 if n <= 64 else 5, n, seed)
    gp, gc, gm, gr = gi.local_search(perms, cap)
    for i, p in enumerate(perms):
        op, oc, om, orr, _ = O.local_search(inst.F, inst.D, p, cap)
        assert np.array_equal(gp[i], op) and gc[i] == oc and gm[i] == om and gr[i] == orr, i
    assert np.array_equal(gi.eval_costs(perms), [O.cost(inst.F, inst.D, p) for p in perms])


def test_general_local_search_with_diagonal(Q):
    F, D = _diag_instance(30, 9)
    gi = Q.Instance(F, D)
    perms = W.random_perms(16, 30, 9)
    gp, gc, gm, gr = gi.local_search(perms, 0)
    for i, p in enumerate(perms):
        op, oc, om, orr, _ = O.local_search(F, D, p, 0)
        assert np.array_equal(gp[i], op) and gc[i] == oc and gm[i] == om and gr[i] == orr, i


@pytest.mark.parametrize("variant", ["default", "rank"])
def test_general_iterations_replay(Q, variant):
    inst = W.random_asymmetric(21, 4, hi=200)
    kw = dict(swarms=3, swarm_size=9)
    kw.update(VARIANTS[variant])
    prm = Q.default_params(**kw)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=77)
    q = oracle_params(prm)
    before = sw.export_state()
    for _ in range(3):
        sw.step(1)
        after = sw.export_state()
        compare_step(q, inst.F, inst.D, 77, before, after, prm)
        before = after
