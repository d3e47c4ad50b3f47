"""Single-kernel entry points against the oracle: the swap-value table of one
permutation (general O(n) formula, any instance) and the discretisation S_x alone
(Algorithm 1) on caller-formed fp32 Y."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W
from tests.golden.load import load

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1504_05158_gb300 import qap_pso
    qap_pso.lib()
    return qap_pso


DELTA_CASES = {
    "n2": lambda: W.dense_uniform(2, 1),
    "tiny9": W.tiny9,
    "asym21": lambda: W.random_asymmetric(21, 4, hi=200),
    "dense30": W.dense30,
    "grid64": W.grid64,
    "asym70": lambda: W.random_asymmetric(70, 5, hi=99),
    "n150": lambda: W.dense_uniform(150, 9),
}


@pytest.mark.parametrize("name", list(DELTA_CASES))
def test_delta_table_bit_exact(Q, name):
    inst = DELTA_CASES[name]()
    n = inst.n
    gi = Q.Instance(inst.F, inst.D)
    for p in W.random_perms(3, n, 21):
        got = gi.delta_table(p)
        want = [O.delta(inst.F, inst.D, p, r, s) for r in range(n) for s in range(r + 1, n)]
        assert np.array_equal(got, np.array(want, np.int64))


def test_delta_table_rejects_non_permutation(Q):
    inst = W.dense_uniform(6, 1)
    gi = Q.Instance(inst.F, inst.D)
    with pytest.raises(Q.QapError) as e:
        gi.delta_table(np.zeros(6, np.int32))
    assert e.value.status == Q.ERR_INVALID_ARG


def _ys(count, n, seed, quantised):
    """Y = X(t) + V with V in [-1, 1): continuous, or on a grid of 1/8 (many ties)."""
    rng = np.random.default_rng(seed)
    Z = W.random_perms(count, n, seed + 1)
    V = rng.uniform(-1.0, 1.0, (count, n, n)).astype(np.float32)
    if quantised:
        V = (np.round(V * 8.0) / 8.0).astype(np.float32)
    Y = V.copy()
    for i in range(count):
        Y[i, Z[i], np.arange(n)] += np.float32(1.0)
    return Y, Z


@pytest.mark.parametrize("n", [2, 3, 9, 33, 64, 100, 150])
@pytest.mark.parametrize("rule,depth,tie", [(0, 2, 0), (1, 2, 0), (0, 0, 0), (1, 1, 1), (0, 3, 1)])
@pytest.mark.parametrize("quantised", [False, True])
def test_discretize_matches_oracle(Q, n, rule, depth, tie, quantised):
    depth = min(depth, n - 1)
    count = 12
    Y, Z = _ys(count, n, 100 + n, quantised)
    seed = 0xBEEF0000 + n
    swarm = np.arange(count, dtype=np.int32) % 3
    particle = np.arange(count, dtype=np.int32) * 7
    t = 11
    g = Q.default_params(sx_rule=rule, depth=depth, tie_rule=tie)
    q = O.make_params(sx_rule=rule, depth=depth, tie_rule=tie)
    got = Q.discretize(Y, Z, g, seed, swarm, particle, t)
    for i in range(count):
        want, _ = O.second_target(q, Y[i], Z[i], seed, int(particle[i]), int(swarm[i]), t)
        assert np.array_equal(got[i], want), i
        assert sorted(got[i]) == list(range(n))


def _ys_converged(count, n, seed):
    """Y of a converged swarm under Norm: V is -0.5 at the X(t) cell and +0.5 at one
    other row of each column, tiny (or zero) elsewhere, so every X(t) cell of Y equals
    0.5 exactly, as do the largest plain values: most greedy steps see many maxima."""
    rng = np.random.default_rng(seed)
    Z = W.random_perms(count, n, seed + 1)
    V = (rng.uniform(-1.0, 1.0, (count, n, n)) * 1e-20).astype(np.float32)
    V[rng.random((count, n, n)) < 0.3] = 0.0
    for i in range(count):
        for j in range(n):
            V[i, Z[i, j], j] = -0.5
            if n > 1:
                r = int(rng.integers(0, n - 1))
                V[i, r if r < Z[i, j] else r + 1, j] = 0.5
    Y = V.copy()
    for i in range(count):
        Y[i, Z[i], np.arange(n)] += np.float32(1.0)
    return Y, Z


@pytest.mark.parametrize("n", [2, 9, 33, 64, 100])
@pytest.mark.parametrize("kind,rule,depth,tie", [(0, 0, 2, 0), (0, 1, 2, 0), (0, 0, 0, 1), (1, 0, 0, 0)])
def test_discretize_converged_pattern(Q, n, kind, rule, depth, tie):
    depth = min(depth, n - 1)
    count = 12
    Y, Z = _ys_converged(count, n, 300 + n)
    assert np.all(Y[0, Z[0], np.arange(n)] == np.float32(0.5))
    seed = 0xC0DE0000 + n
    swarm = np.arange(count, dtype=np.int32) % 4
    particle = np.arange(count, dtype=np.int32) * 5
    t = 77
    g = Q.default_params(sx_kind=kind, sx_rule=rule, depth=depth, tie_rule=tie)
    q = O.make_params(sx_kind=kind, sx_rule=rule, depth=depth, tie_rule=tie)
    got = Q.discretize(Y, Z, g, seed, swarm, particle, t)
    for i in range(count):
        if kind == 1:
            want, _ = O.pick_column(q, Y[i], seed, int(particle[i]), int(swarm[i]), t)
        else:
            want, _ = O.second_target(q, Y[i], Z[i], seed, int(particle[i]), int(swarm[i]), t)
        assert np.array_equal(got[i], want), i
        assert sorted(got[i]) == list(range(n))


def test_discretize_worked_example(Q):
    # the 3 x 3 example of section 3.1 (GlobalMax keeps the stuck particle; the
    # SecondTarget pictures of Eq. 6 under the top-d reading)
    g = load("sx_worked_example.txt")
    Y = g["XplusV"].astype(np.float32)
    z = g["z"].astype(np.int32)
    for rule in (0, 1):
        got = Q.discretize(Y, z, Q.default_params(depth=0, sx_rule=rule), 1, 0, 0, 0)[0]
        assert np.array_equal(got, g["globalmax"])
    got = Q.discretize(Y, z, Q.default_params(depth=1, sx_rule=1), 1, 0, 0, 0)[0]
    assert np.array_equal(got, g["d1_perm"])
    got = Q.discretize(Y, z, Q.default_params(depth=2, sx_rule=1, tie_rule=1), 1, 0, 0, 0)[0]
    assert np.array_equal(got, g["d2b_perm"])
    seeds = np.arange(40)
    outs = [tuple(Q.discretize(Y, z, Q.default_params(depth=2, sx_rule=1), int(sd), 0, 0, 0)[0])
            for sd in seeds]
    assert set(outs) == {tuple(g["d2a_perm"]), tuple(g["d2b_perm"])}


def test_discretize_rejects_bad_input(Q):
    g = Q.default_params(depth=2)
    Y = np.zeros((1, 4, 4), np.float32)
    with pytest.raises(Q.QapError):
        Q.discretize(Y, np.zeros(4, np.int32), g, 1, 0, 0, 0)  # Z not a permutation
    Y[0, 1, 1] = np.nan
    with pytest.raises(Q.QapError):
        Q.discretize(Y, np.arange(4, dtype=np.int32), g, 1, 0, 0, 0)
    with pytest.raises(Q.QapError):
        Q.discretize(np.zeros((1, 4, 4), np.float32), np.arange(4, dtype=np.int32),
                     Q.default_params(depth=4), 1, 0, 0, 0)  # depth >= n


@pytest.mark.parametrize("n", [2, 3, 9, 33, 64, 100, 150])
@pytest.mark.parametrize("tie", [0, 1])
@pytest.mark.parametrize("quantised", [False, True])
def test_discretize_pick_column_matches_oracle(Q, n, tie, quantised):
    count = 12
    Y, Z = _ys(count, n, 300 + n, quantised)
    seed = 0xC0FFEE + n
    swarm = np.arange(count, dtype=np.int32) % 4
    particle = np.arange(count, dtype=np.int32) * 3
    t = 5
    g = Q.default_params(sx_kind=1, tie_rule=tie)
    q = O.make_params(sx_kind=1, tie_rule=tie)
    got = Q.discretize(Y, Z, g, seed, swarm, particle, t)
    for i in range(count):
        want, _ = O.pick_column(q, Y[i], seed, int(particle[i]), int(swarm[i]), t)
        assert np.array_equal(got[i], want), i


def test_invalid_sx_kind(Q):
    with pytest.raises(Q.QapError) as e:
        Q.discretize(np.zeros((1, 4, 4), np.float32), np.arange(4, dtype=np.int32), Q.default_params(sx_kind=2),
                     1, 0, 0, 0)
    assert e.value.status == Q.ERR_INVALID_ARG


def test_swarm_stats_and_histogram(Q):
    inst = W.grid64()
    gi = Q.Instance(inst.F, inst.D)
    sw = Q.Swarm(gi, Q.default_params(swarms=5, swarm_size=37, mig_kind=2, mig_period=3), seed=8)
    for it in range(4):
        sw.step(1)
        st = sw.export_state()
        cost = st["cost"]
        for k in (0, 2, 4):
            got = sw.stats_swarm(k)
            want = O.stats(cost[k * 37:(k + 1) * 37])
            keys = ("min", "p5", "p25", "p50", "p75", "max")
            assert [got[x] for x in keys] == [want[x] for x in keys]
            assert got["mean"] == want["mean"]
        lo, hi = int(cost.min()) + 17, int(cost.max()) - 5
        for bins, swarm in ((1, -1), (7, -1), (50, 3)):
            sel = cost if swarm < 0 else cost[swarm * 37:(swarm + 1) * 37]
            assert np.array_equal(sw.cost_histogram(lo, hi, bins, swarm), O.histogram(sel, lo, hi, bins))
    with pytest.raises(Q.QapError):
        sw.stats_swarm(5)
    with pytest.raises(Q.QapError):
        sw.cost_histogram(10, 10, 4)
