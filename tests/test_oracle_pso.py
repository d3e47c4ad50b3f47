"""Pins of the oracle's PSO parts: Philox, velocity (Eq. 4, S_v), S_x
(SecondTarget, Algorithm 1 / Eq. 6), initialisation, bests and migration
(Algorithm 2, ring) and statistics, each against something other than itself."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W
from tests.golden.load import load


# ------------------------------------------------------------------ Philox

def _triton_philox(ctrs, keys):
    """Philox4x32-10 from Triton's library implementation, run by its CPU interpreter."""
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    import triton.language as tl
    import torch

    @triton.jit
    def kern(o0, o1, o2, o3, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i),
                               tl.load(c3p + i))
        tl.store(o0 + i, a)
        tl.store(o1 + i, b)
        tl.store(o2 + i, c)
        tl.store(o3 + i, d)

    out = np.zeros((len(ctrs), 4), np.uint32)
    for row, (ctr, key) in enumerate(zip(ctrs, keys)):
        cs = [torch.tensor([int(np.int32(np.uint32(c)))] * 2, dtype=torch.int32) for c in ctr]
        os_ = [torch.zeros(2, dtype=torch.int32) for _ in range(4)]
        seed = int(key[0]) | (int(key[1]) << 32)
        kern[(1,)](*os_, *cs, seed, N=2)
        out[row] = [np.uint32(o.numpy()[0].view(np.uint32)) for o in os_]
    return out


def test_philox_matches_library_implementation():
    rng = np.random.default_rng(0)
    ctrs = rng.integers(0, 2**32, size=(12, 4), dtype=np.uint64).astype(np.uint32)
    keys = rng.integers(0, 2**32, size=(12, 2), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    keys[0] = 0
    ctrs[1] = 0xFFFFFFFF
    keys[1] = 0xFFFFFFFF
    ref = _triton_philox(ctrs, keys)
    for c, k, r in zip(ctrs, keys, ref):
        assert np.array_equal(O.philox(c, k), r)


def test_draw_counter_layout():
    seed = 0x1234_5678_9ABC_DEF0
    got = O.draw(seed, 7, 3, 11, 2, 5)
    want = O.philox([7, 3, 11, (2 << 24) | 5], [0x9ABCDEF0, 0x12345678])
    assert np.array_equal(got, want)


def test_u01_and_below_uniform():
    us = np.concatenate([O.draw(99, i, 0, 0, 0, 0) for i in range(4000)])
    x = np.array([O.u01(u) for u in us])
    assert x.min() >= 0.0 and x.max() < 1.0
    hist, _ = np.histogram(x, bins=16, range=(0, 1))
    exp = len(x) / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 40.0  # 15 dof, p ~ 5e-4
    k = np.array([O.below(u, 7) for u in us])
    assert k.min() == 0 and k.max() == 6
    hist = np.bincount(k, minlength=7)
    exp = len(k) / 7
    assert ((hist - exp) ** 2 / exp).sum() < 30.0
    assert O.u01(0xFFFFFFFF) == (2**24 - 1) / 2**24
    assert O.below(0xFFFFFFFF, 5) == 4 and O.below(0, 5) == 0


# ------------------------------------------------------------------ velocity

def _mats(n, p):
    M = np.zeros((n, n))
    M[p, np.arange(n)] = 1.0
    return M


def test_velocity_closed_form_raw():
    n = 6
    rng = np.random.default_rng(1)
    V = rng.uniform(-3, 3, (n, n))
    x, pl, pg = (W.random_perms(3, n, 4))
    q = O.make_params(c1=0.5, c2=0.75, c3=0.25, sv_kind=0, v_max=1.0, v_storage=0)
    r2, r3 = 0.5, 0.25
    got = O.velocity(q, V, x, pl, pg, r2, r3)
    X, L, G = _mats(n, x), _mats(n, pl), _mats(n, pg)
    want = np.clip(0.5 * V + 0.75 * 0.5 * (L - X) + 0.25 * 0.25 * (G - X), -1, 1)
    want = want.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want)


def test_velocity_norm_zero_inertia():
    # V = 0, P^L = X: column j holds +b at P^G's row and -b at X's row, so Norm gives
    # +1/2 and -1/2 there; columns where P^G agrees with X stay all zero.
    n = 7
    x = np.arange(n, dtype=np.int32)
    pg = x.copy()
    pg[[1, 4]] = pg[[4, 1]]
    q = O.make_params(c1=0.8, c2=0.5, c3=0.5, sv_kind=1, v_max=1.0)
    got = O.velocity(q, np.zeros((n, n)), x, x, pg, 0.3, 0.6)
    want = np.zeros((n, n))
    for j in (1, 4):
        want[pg[j], j] = 0.5
        want[x[j], j] = -0.5
    assert np.array_equal(got, want)


def test_velocity_norm_invariants_and_storage():
    n = 20
    rng = np.random.default_rng(2)
    x, pl, pg = W.random_perms(3, n, 9)
    for storage in (0, 1):
        q = O.make_params(c1=0.8, c2=0.5, c3=0.5, sv_kind=1, v_max=1.0, v_storage=storage)
        V = rng.uniform(-1, 1, (n, n))
        got = O.velocity(q, V, x, pl, pg, 0.9, 0.1)
        colsum = np.abs(got).sum(axis=0)
        tol = 1e-6 if storage == 0 else n * 2.0**-8
        assert np.all(np.abs(colsum - 1.0) <= tol)
        if storage == 1:
            import torch
            t = torch.tensor(got, dtype=torch.float32)
            assert torch.equal(t, t.to(torch.bfloat16).to(torch.float32))
        else:
            assert np.array_equal(got, got.astype(np.float32).astype(np.float64))


def test_round_bf16_matches_library_on_fp32_values():
    import torch
    rng = np.random.default_rng(3)
    vals = np.concatenate([
        rng.standard_normal(2000).astype(np.float32),
        (rng.standard_normal(200) * 1e-39).astype(np.float32),  # fp32 subnormals
        np.array([1.0 + 2**-8, 1.0 + 3 * 2**-8, -(1.0 + 2**-8), 2**-126 * (1 + 2**-8)],
                 np.float32)])  # exact halfway cases
    ref = torch.tensor(vals).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.round_bf16(float(v)) for v in vals])
    assert np.array_equal(got, ref)


def test_round_bf16_fp64_is_nearest():
    # the result lies on the bf16 grid and no grid neighbour is closer to the input
    rng = np.random.default_rng(4)
    for v in rng.standard_normal(500) * 3.0:
        r = O.round_bf16(v)
        bits = np.array([r], np.float32).view(np.uint32)[0]
        assert bits & 0xFFFF == 0
        for nb_bits in (bits + 0x10000, bits - 0x10000):
            nb = float(np.array([nb_bits], np.uint32).view(np.float32)[0])
            assert abs(r - v) <= abs(nb - v)


# ------------------------------------------------------------------ S_x

def _example():
    g = load("sx_worked_example.txt")
    Y = g["XplusV"].astype(np.float32)
    z = g["z"].astype(np.int32)
    return g, Y, z


def test_sx_worked_example_globalmax():
    g, Y, z = _example()
    assert np.array_equal((g["X"] + g["V"]), g["XplusV"])
    for rule in (0, 1):
        q = O.make_params(depth=0, sx_rule=rule)
        p, ties = O.second_target(q, Y, z)
        assert np.array_equal(p, g["globalmax"]) and ties == 0


def test_sx_worked_example_topd_reading():
    g, Y, z = _example()
    q = O.make_params(depth=1, sx_rule=1)
    p, ties, order = O.second_target(q, Y, z, want_order=True)
    assert np.array_equal(order, g["d1_picks"]) and np.array_equal(p, g["d1_perm"])
    q = O.make_params(depth=2, sx_rule=1, tie_rule=0)
    seen = set()
    for seed in range(40):
        p, ties, order = O.second_target(q, Y, z, seed=seed, want_order=True)
        assert ties == 1
        if np.array_equal(order, g["d2a_picks"]):
            assert np.array_equal(p, g["d2a_perm"])
            seen.add("a")
        else:
            assert np.array_equal(order, g["d2b_picks"]) and np.array_equal(p, g["d2b_perm"])
            seen.add("b")
    assert seen == {"a", "b"}
    # with the deterministic tie rule the first element of M in column-major order is taken
    q = O.make_params(depth=2, sx_rule=1, tie_rule=1)
    _, _, order = O.second_target(q, Y, z, want_order=True)
    assert np.array_equal(order, g["d2b_picks"])


def test_sx_worked_example_algorithm1_reading():
    g, Y, z = _example()
    # Algorithm 1 as printed ignores every Z-one in the first d steps: with d = 2 the
    # only candidates of value 4 not in Z give the second picture of Eq. 6.
    q = O.make_params(depth=2, sx_rule=0)
    p, ties, order = O.second_target(q, Y, z, want_order=True)
    assert np.array_equal(order, g["d2b_picks"]) and ties == 0
    # with d = 1 it picks 4 at (2,2) first and ends at the identity (not Eq. 6's d = 1
    # picture): the two readings differ here, which is why both are kept.
    q = O.make_params(depth=1, sx_rule=0)
    p, _, order = O.second_target(q, Y, z, want_order=True)
    assert np.array_equal(order, [[1, 1], [0, 0], [2, 2]])
    assert np.array_equal(p, [0, 1, 2])


def greedy_sorted(Y, z, depth, rule):
    """SecondTarget with the first-element tie rule as a greedy pass over all cells
    sorted by (value descending, column, row): each step takes the first cell whose
    row and column are free (and, in the first `depth` steps, not excluded)."""
    n = len(z)
    cells = sorted((-float(Y[r, c]), c, r) for r in range(n) for c in range(n))
    if depth == 0:
        excl = set()
    elif rule == 0:
        excl = {(int(z[c]), c) for c in range(n)}
    else:
        zs = sorted((-float(Y[z[c], c]), c) for c in range(n))[:depth]
        excl = {(int(z[c]), c) for _, c in zs}
    rows, cols = set(), set()
    p = np.full(n, -1, np.int32)
    for step in range(n):
        for _, c, r in cells:
            if r in rows or c in cols or (step < depth and (r, c) in excl):
                continue
            p[c] = r
            rows.add(r)
            cols.add(c)
            break
    return p


@pytest.mark.parametrize("n", [5, 9, 16])
@pytest.mark.parametrize("depth,rule", [(0, 0), (2, 0), (2, 1), (4, 0), (4, 1)])
def test_sx_matches_sorted_greedy(n, depth, rule):
    rng = np.random.default_rng(n * 10 + depth + rule)
    for trial in range(6):
        if trial % 2:
            Y = rng.integers(-2, 3, (n, n)).astype(np.float32)  # many ties
        else:
            Y = rng.standard_normal((n, n)).astype(np.float32)
        z = W.random_perms(1, n, trial)[0]
        q = O.make_params(depth=depth, sx_rule=rule, tie_rule=1)
        p, _ = O.second_target(q, Y, z)
        assert np.array_equal(np.sort(p), np.arange(n))
        assert np.array_equal(p, greedy_sorted(Y, z, depth, rule))


def test_sx_random_ties_uniform():
    n = 3
    Y = np.zeros((n, n), np.float32)
    q = O.make_params(depth=0, tie_rule=0)
    first = np.zeros(9, np.int64)
    for c0 in range(1800):
        _, ties, order = O.second_target(q, Y, np.arange(n, dtype=np.int32), seed=5, c0=c0,
                                         want_order=True)
        assert ties == 2  # 9 then 4 then 1 candidates
        r, c = order[0]
        first[c * n + r] += 1
    exp = 1800 / 9
    assert ((first - exp) ** 2 / exp).sum() < 30.0


# ------------------------------------------------------------------ init

def test_init_fisher_yates_uniform_and_v0_range():
    inst = W.dense_uniform(3, 1)
    q = O.make_params(swarms=4, swarm_size=600, v_max=0.5)
    s = O.init(q, inst.F, inst.D, 17)
    keys = [tuple(p) for p in s.X]
    for p in keys:
        assert sorted(p) == [0, 1, 2]
    from collections import Counter
    cnt = Counter(keys)
    assert len(cnt) == 6
    exp = len(keys) / 6
    assert sum((v - exp) ** 2 / exp for v in cnt.values()) < 25.0
    assert s.V.min() >= -0.5 and s.V.max() < 0.5
    assert np.array_equal(s.PL, s.X) and np.array_equal(s.costL, s.cost)
    for k in range(4):
        sw = s.cost[k * 600:(k + 1) * 600]
        assert s.costG[k] == sw.min()
        assert np.array_equal(s.PG[k], s.X[k * 600 + int(np.argmin(sw))])
    assert s.best_cost[0] == s.cost.min() and s.best_iter[0] == 0


# ------------------------------------------------------------------ bests, migration

def _fake_state(m, ss, n, seed):
    q = O.make_params(swarms=m, swarm_size=ss)
    s = O.State(q, n)
    rng = np.random.default_rng(seed)
    s.X[:] = W.random_perms(m * ss, n, seed)
    s.cost[:] = rng.integers(100, 1000, m * ss)
    s.costG[:] = rng.integers(50, 2000, m)
    s.PG[:] = W.random_perms(m, n, seed + 1)
    s.best_cost[0] = 10**9
    return s


def test_swarm_bests_strict_and_lowest_index():
    m, ss, n = 3, 5, 6
    s = _fake_state(m, ss, n, 1)
    s.cost[:] = 500
    s.cost[7] = 100
    s.cost[8] = 100  # tie in swarm 1 -> particle 7 (lower index) wins
    s.costG[:] = [500, 200, 40]
    pg0 = s.PG.copy()
    q = O.make_params(swarms=m, swarm_size=ss, mig_kind=0)
    O.bests_and_migration(q, 0, 4, s)
    assert np.array_equal(s.PG[0], pg0[0]) and s.costG[0] == 500  # equal is not better
    assert np.array_equal(s.PG[1], s.X[7]) and s.costG[1] == 100
    assert np.array_equal(s.PG[2], pg0[2]) and s.costG[2] == 40
    assert s.best_cost[0] == 100 and np.array_equal(s.best_p, s.X[7]) and s.best_iter[0] == 5


def test_rank_migration_algorithm2():
    m, ss, n, d = 9, 7, 5, 4
    s = _fake_state(m, ss, n, 2)
    s.cost[:] = 10**6  # no swarm best changes
    q = O.make_params(swarms=m, swarm_size=ss, mig_kind=1, mig_depth=d, mig_period=1)
    before_c, before_p = s.costG.copy(), s.PG.copy()
    order = sorted(range(m), key=lambda k: (before_c[k], k))
    O.bests_and_migration(q, 77, 3, s)
    for k in range(d):
        donor, target = order[k], order[m - 1 - k]
        j = O.below(O.draw(77, k, 0, 3, O.TAG_MIG, 0)[0], ss)
        assert np.array_equal(s.PG[target], s.X[donor * ss + j])
        assert s.costG[target] == s.cost[donor * ss + j]  # accepted although worse
        assert np.array_equal(s.PG[donor], before_p[donor])
    for k in order[d:m - d]:
        assert np.array_equal(s.PG[k], before_p[k]) and s.costG[k] == before_c[k]


def test_ring_migration_and_period():
    m, ss, n = 5, 3, 4
    s = _fake_state(m, ss, n, 3)
    s.cost[:] = 10**6
    q = O.make_params(swarms=m, swarm_size=ss, mig_kind=2, mig_period=20)
    c0, p0 = s.costG.copy(), s.PG.copy()
    O.bests_and_migration(q, 1, 17, s)  # iteration 18 of 20: nothing moves
    assert np.array_equal(s.PG, p0)
    O.bests_and_migration(q, 1, 19, s)  # 20th iteration: ring shift
    for k in range(m):
        assert np.array_equal(s.PG[(k + 1) % m], p0[k]) and s.costG[(k + 1) % m] == c0[k]
    s2 = _fake_state(m, ss, n, 3)
    s2.cost[:] = 10**6
    q2 = O.make_params(swarms=m, swarm_size=ss, mig_kind=2, mig_period=20, ring_if_better=1)
    O.bests_and_migration(q2, 1, 19, s2)
    for k in range(m):
        dst = (k + 1) % m
        assert s2.costG[dst] == (c0[k] if c0[k] < c0[dst] else c0[dst])


# ------------------------------------------------------------------ stats

def test_stats_nearest_rank():
    rng = np.random.default_rng(5)
    for P in (1, 2, 7, 50, 1000):
        c = rng.integers(0, 10**9, P)
        st = O.stats(c)
        for key, q in (("p5", 0.05), ("p25", 0.25), ("p50", 0.5), ("p75", 0.75)):
            assert st[key] == int(np.percentile(c, q * 100, method="inverted_cdf"))
        assert st["min"] == c.min() and st["max"] == c.max()
        assert abs(st["mean"] - c.mean()) <= 1e-9 * abs(c.mean())


def test_stats_mean_exact_for_huge_costs():
    # costs near the int64 limit: their sum leaves int64, yet the mean is the exact
    # rational sum / P to within one rounding of a double
    from fractions import Fraction
    rng = np.random.default_rng(11)
    for P in (1, 3, 64, 1001):
        c = rng.integers(2**62, 2**63 - 1, P, dtype=np.int64)
        exact = Fraction(sum(int(x) for x in c), P)
        got = O.stats(c)["mean"]
        assert abs(Fraction(got) - exact) <= exact * Fraction(1, 2**52)
    c = np.array([-7, 2, 0], np.int64)  # a negative total: remainder of the truncated quotient
    assert abs(Fraction(O.stats(c)["mean"]) - Fraction(-5, 3)) <= Fraction(5, 3) * Fraction(1, 2**52)


# ------------------------------------------------------------------ whole runs

def test_tiny9_reaches_brute_force_optimum():
    inst = W.tiny9()
    opt, _ = O.brute_force(inst.F, inst.D)
    q = O.make_params(swarms=1, swarm_size=32, ls_max_moves=0)
    s = O.init(q, inst.F, inst.D, 1)
    O.step(q, inst.F, inst.D, 1, s, 100)
    assert s.best_cost[0] == opt
    assert s.t[0] == 100
    assert s.counters[O.C_PIT] == 3200
    # best never above the cost of its own permutation
    assert O.cost(inst.F, inst.D, s.best_p) == s.best_cost[0]


def test_step_bookkeeping_invariants():
    inst = W.dense_uniform(12, 3)
    q = O.make_params(swarms=3, swarm_size=8, ls_max_moves=0, mig_kind=1, mig_depth=1)
    s = O.init(q, inst.F, inst.D, 9)
    hist_min = s.costL.copy()
    for _ in range(5):
        O.step(q, inst.F, inst.D, 9, s)
        hist_min = np.minimum(hist_min, s.cost)
        assert np.array_equal(s.costL, hist_min)
        for i in range(24):
            assert O.cost(inst.F, inst.D, s.X[i]) == s.cost[i]
            assert O.cost(inst.F, inst.D, s.PL[i]) == s.costL[i]
        for k in range(3):
            assert O.cost(inst.F, inst.D, s.PG[k]) == s.costG[k]
        assert s.best_cost[0] <= hist_min.min()


# ------------------------------------------------------------ PickColumn (section 3.1)

def test_pick_column_is_a_greedy_over_columns():
    # every pick is a largest element of its column among the rows still free
    rng = np.random.default_rng(11)
    for n in (1, 2, 5, 9, 13):
        for rep in range(6):
            Y = rng.normal(size=(n, n)).astype(np.float32)
            if rep % 2:
                Y = np.round(Y * 2) / 2  # many equal values
            q = O.make_params(sx_kind=1, tie_rule=rep % 2)
            p, ties, order = O.pick_column(q, Y, seed=rep, c0=rep, want_order=True)
            assert sorted(p) == list(range(n))
            assert sorted(order[:, 1]) == list(range(n))  # every column once
            free = np.ones(n, bool)
            for r, c in order:
                assert free[r] and Y[r, c] == Y[free, c].max()
                free[r] = False
            assert all(p[c] == r for r, c in order)


def test_pick_column_distinct_column_maxima_is_argmax():
    # maxima of the columns in distinct rows: the result is the column-wise argmax,
    # whatever the order of the columns
    rng = np.random.default_rng(12)
    for n in (3, 8, 20):
        perm = rng.permutation(n)
        Y = (rng.random((n, n)) * 0.5).astype(np.float32)
        Y[perm, np.arange(n)] += 1.0
        for seed in range(5):
            p, ties = O.pick_column(O.make_params(sx_kind=1), Y, seed=seed)
            assert np.array_equal(p, perm) and ties == 0


def test_pick_column_all_equal_first_rule():
    # all values equal and the first element taken: the k-th column of the order gets
    # the k-th row
    n = 7
    Y = np.zeros((n, n), np.float32)
    p, ties, order = O.pick_column(O.make_params(sx_kind=1, tie_rule=1), Y, seed=3, want_order=True)
    assert ties == n - 1
    assert np.array_equal(order[:, 0], np.arange(n))


def test_pick_column_order_uniform():
    # the column order is a uniform permutation (Fisher-Yates from Philox)
    n = 3
    Y = np.eye(n, dtype=np.float32) * 0  # all equal, first rule: the order shows in the rows
    counts = {}
    for seed in range(1200):
        _, _, order = O.pick_column(O.make_params(sx_kind=1, tie_rule=1), Y, seed=seed, want_order=True)
        key = tuple(order[:, 1])
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 6
    chi2 = sum((c - 200) ** 2 / 200 for c in counts.values())
    assert chi2 < 20.5  # 5 degrees of freedom, p ~ 0.001


def test_pick_column_random_ties_uniform():
    n = 2
    Y = np.zeros((n, n), np.float32)
    first_rows = [O.pick_column(O.make_params(sx_kind=1), Y, seed=s, want_order=True)[2][0, 0]
                  for s in range(800)]
    frac = np.mean(first_rows)
    assert 0.42 < frac < 0.58


def test_histogram_by_brute_force():
    # the bins against exact rational edges computed with Python integers
    from fractions import Fraction
    rng = np.random.default_rng(21)
    for _ in range(20):
        P = int(rng.integers(1, 200))
        cost = rng.integers(-50, 1000, P).astype(np.int64)
        lo = int(rng.integers(-60, 300))
        hi = lo + int(rng.integers(1, 900))
        bins = int(rng.integers(1, 40))
        got = O.histogram(cost, lo, hi, bins)
        want = np.zeros(bins + 2, np.int64)
        for c in cost.tolist():
            if c < lo:
                want[0] += 1
            elif c >= hi:
                want[-1] += 1
            else:
                w = Fraction(hi - lo, bins)
                b = 0
                while not (lo + b * w <= c < lo + (b + 1) * w):
                    b += 1
                want[1 + b] += 1
        assert np.array_equal(got, want) and got.sum() == P


def test_parallel_step_equals_step():
    # the all-cores form of the oracle's iteration (the CPU baseline) is the same
    # computation: identical state after a few iterations, with migration
    inst = W.dense_uniform(12, 4)
    q = O.make_params(swarms=4, swarm_size=9, mig_kind=1, mig_depth=1)
    a = O.init(q, inst.F, inst.D, 31)
    b = a.copy()
    O.step(q, inst.F, inst.D, 31, a, 4)
    O.step_parallel(q, inst.F, inst.D, 31, b, 4, threads=4)
    for k in ("V", "X", "PL", "costL", "cost", "PG", "costG", "best_p", "best_cost", "best_iter", "t",
              "counters", "moves"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
