"""Helpers that compare the CUDA path with the oracle on identical inputs."""
import numpy as np

from oracle import oracle as O

V_RTOL = 1e-5        # elementwise relative bound on fp32 velocities against the fp64 oracle
V_FLOOR = 2.0 ** -10  # below this magnitude the bound is absolute: 1e-5 * 2^-10


def oracle_params(prm):
    d = prm.as_dict()
    return O.make_params(**{k: v for k, v in d.items() if k in O.DEFAULTS})


def oracle_state_from(q, n, st):
    """An oracle State holding the exported GPU state (V exact in fp64)."""
    s = O.State(q, n)
    s.V[:] = st["V"].astype(np.float64)
    s.X[:] = st["X"]
    s.PL[:] = st["PL"]
    s.costL[:] = st["costL"]
    s.cost[:] = st["cost"]
    s.PG[:] = st["PG"]
    s.costG[:] = st["costG"]
    s.best_p[:] = st["best"]
    s.best_cost[0] = st["best_cost"]
    s.best_iter[0] = st["best_iter"]
    s.t[0] = st["t"]
    return s


def bf16_ulp(x):
    x = np.maximum(np.abs(x), 2.0**-126)
    return 2.0 ** (np.floor(np.log2(x)) - 7)


def check_velocity(got, want, bf16, what=""):
    """Elementwise: |g - o| <= 1e-5 max(|o|, 2^-10) for every element (fp32 storage);
    bf16 storage adds one bf16 ulp of the larger magnitude (the oracle rounds its fp64
    value to bf16 once, the device its fp32 value once, and the two roundings may
    fall on either side of a bf16 rounding boundary)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want)
    allowed = V_RTOL * np.maximum(np.abs(want), V_FLOOR)
    if bf16:
        allowed = allowed + bf16_ulp(np.maximum(np.abs(got), np.abs(want)))
    bad = err > allowed
    if bad.any():
        i = np.unravel_index(np.argmax(err / allowed), err.shape)
        raise AssertionError(f"{what}: velocity mismatch at {i}: got {got[i]!r}, want {want[i]!r}, "
                             f"err {err[i]:.3g} > allowed {allowed[i]:.3g}")


def compare_step(q, F, D, seed, before, after, prm, sample=None):
    """Checks one GPU iteration (before -> after) against the oracle.

    With sample=None the whole population goes through the oracle's step; otherwise
    only the listed particles are recomputed and the bookkeeping is checked on the
    device's own (already verified) positions and costs."""
    n = F.shape[0]
    bf16 = prm.v_storage == 1
    ss = prm.swarm_size
    if sample is None and not prm.pos_uses_new_v:
        s = oracle_state_from(q, n, before)
        O.step(q, F, D, seed, s)
        assert np.array_equal(s.X, after["X"]), "positions differ"
        assert np.array_equal(s.cost, after["cost"]), "costs differ"
        assert np.array_equal(s.moves, after["moves"]), "local-search moves differ"
        assert np.array_equal(s.PL, after["PL"]) and np.array_equal(s.costL, after["costL"])
        assert np.array_equal(s.PG, after["PG"]) and np.array_equal(s.costG, after["costG"])
        assert s.best_cost[0] == after["best_cost"] and np.array_equal(s.best_p, after["best"])
        assert s.best_iter[0] == after["best_iter"] and s.t[0] == after["t"]
        for p in range(len(s.X)):
            check_velocity(after["V"][p], s.V[p], bf16, f"particle {p}")
        return
    idx = range(len(before["X"])) if sample is None else sample
    t = int(before["t"])
    for p in idx:
        k, i = divmod(int(p), ss)
        r = O.particle_iteration(q, F, D, seed, t, k, i, before["V"][p].astype(np.float64),
                                 before["X"][p], before["PL"][p], before["PG"][k])
        check_velocity(after["V"][p], r["V_new"], bf16, f"particle {p}")
        if prm.pos_uses_new_v:
            # S_x on the device's own V(t+1): decisions on identical fp32 inputs
            Y = (after["V"][p].astype(np.float32) + (np.arange(n)[:, None] == before["X"][p][None, :]))
            Y = Y.astype(np.float32)
            if q.sx_kind == 1:
                psx, _ = O.pick_column(q, Y, seed, i, k, t)
            else:
                psx, _ = O.second_target(q, Y, before["X"][p], seed, i, k, t)
            assert np.array_equal(psx, after["X_sx"][p]), f"S_x differs at particle {p}"
            pls, c, mv, _, _ = O.local_search(F, D, psx, q.ls_max_moves) if q.ls_max_moves >= 0 \
                else (psx, O.cost(F, D, psx), 0, 0, None)
            assert np.array_equal(pls, after["X"][p]) and c == after["cost"][p] and mv == after["moves"][p]
        else:
            assert np.array_equal(r["p_sx"], after["X_sx"][p]), f"S_x differs at particle {p}"
            assert np.array_equal(r["p_out"], after["X"][p]), f"position differs at particle {p}"
            assert r["cost"] == after["cost"][p] and r["moves"] == after["moves"][p]
    # bookkeeping on the device's positions and costs
    s = oracle_state_from(q, n, before)
    s.X[:] = after["X"]
    s.cost[:] = after["cost"]
    better = s.cost < s.costL
    s.PL[better] = s.X[better]
    s.costL[better] = s.cost[better]
    O.bests_and_migration(q, seed, t, s)
    assert np.array_equal(s.PL, after["PL"]) and np.array_equal(s.costL, after["costL"])
    assert np.array_equal(s.PG, after["PG"]) and np.array_equal(s.costG, after["costG"])
    assert s.best_cost[0] == after["best_cost"] and np.array_equal(s.best_p, after["best"])
    assert s.best_iter[0] == after["best_iter"] and t + 1 == after["t"]
