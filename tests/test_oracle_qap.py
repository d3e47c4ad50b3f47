"""Pins of the oracle's goal function, swap-move values, local search and brute
force against definitions that do not go through the oracle's own code."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W
from tests.golden.load import load


def perm_matrix(p):
    """x_ki = 1 iff k = p(i) (Eq. 2)."""
    n = len(p)
    X = np.zeros((n, n), np.int64)
    X[p, np.arange(n)] = 1
    return X


def cost_trace_form(F, D, p):
    """f(p) = tr(F^T X^T D X): Eq. 1 as a product of matrices (numpy int64 matmul)."""
    X = perm_matrix(p)
    return int(np.trace(F.astype(np.int64).T @ X.T @ D.astype(np.int64) @ X))


def test_cost_golden_hand_example():
    g = load("cost_3x3_asym.txt")
    assert O.cost(g["F"], g["D"], g["p"]) == g["cost"]
    assert O.cost_eq1(g["F"], g["D"], g["p"]) == g["cost"]
    assert cost_trace_form(g["F"], g["D"], g["p"]) == g["cost"]


@pytest.mark.parametrize("n,seed", [(2, 1), (5, 2), (7, 3), (12, 4)])
def test_cost_matches_eq1_and_trace_form(n, seed):
    inst = W.random_asymmetric(n, seed)
    for p in W.random_perms(6, n, seed):
        c = O.cost(inst.F, inst.D, p)
        assert c == cost_trace_form(inst.F, inst.D, p)
        if n <= 7:
            assert c == O.cost_eq1(inst.F, inst.D, p)


def test_cost_symmetric_transpose_and_identity():
    inst = W.dense30()
    for p in W.random_perms(4, 30, 7):
        assert O.cost(inst.F, inst.D, p) == O.cost(inst.F.T.copy(), inst.D.T.copy(), p)
    ident = np.arange(30, dtype=np.int32)
    assert O.cost(inst.F, inst.D, ident) == int((inst.F.astype(np.int64) * inst.D).sum())


@pytest.mark.parametrize("n,seed,sym", [(4, 11, False), (9, 12, False), (16, 13, False),
                                        (30, 14, True), (17, 15, True)])
def test_delta_equals_recomputed_cost(n, seed, sym):
    inst = W.dense_uniform(n, seed) if sym else W.random_asymmetric(n, seed)
    for p in W.random_perms(3, n, seed):
        base = cost_trace_form(inst.F, inst.D, p)
        for r in range(n):
            for s in range(r + 1, n):
                q = p.copy()
                q[r], q[s] = q[s], q[r]
                assert O.delta(inst.F, inst.D, p, r, s) == cost_trace_form(inst.F, inst.D, q) - base


def neighbourhood_costs(F, D, p):
    """Costs of every swap neighbour, by recomputation (numpy)."""
    n = len(p)
    out = {}
    for r in range(n):
        for s in range(r + 1, n):
            q = p.copy()
            q[r], q[s] = q[s], q[r]
            out[(r, s)] = cost_trace_form(F, D, q)
    return out


@pytest.mark.parametrize("n,seed,sym", [(8, 21, True), (10, 22, False), (12, 23, True)])
def test_local_search_is_best_improvement(n, seed, sym):
    inst = W.dense_uniform(n, seed) if sym else W.random_asymmetric(n, seed)
    p0 = W.random_perms(1, n, seed)[0]
    p_final, c_final, moves, rounds, trace = O.local_search(inst.F, inst.D, p0, 0, trace_cap=1000)
    # replay: every move is the lowest (r-major first) of the recomputed neighbour costs
    p = p0.copy()
    for r, s in trace:
        nb = neighbourhood_costs(inst.F, inst.D, p)
        best = min(nb.values())
        first = min(k for k, v in nb.items() if v == best)
        assert (r, s) == first
        assert best < cost_trace_form(inst.F, inst.D, p)
        p[r], p[s] = p[s], p[r]
    assert np.array_equal(p, p_final)
    assert c_final == cost_trace_form(inst.F, inst.D, p_final)
    # the result is a swap local optimum
    nb = neighbourhood_costs(inst.F, inst.D, p_final)
    assert min(nb.values()) >= c_final
    assert rounds == moves + 1


def test_local_search_cap():
    inst = W.dense_uniform(20, 5)
    p0 = W.random_perms(1, 20, 5)[0]
    _, _, full_moves, _, full_trace = O.local_search(inst.F, inst.D, p0, 0, trace_cap=500)
    assert full_moves > 3
    p3, c3, m3, r3, t3 = O.local_search(inst.F, inst.D, p0, 3, trace_cap=10)
    assert m3 == 3 and r3 == 3
    assert np.array_equal(t3, full_trace[:3])
    assert c3 == O.cost(inst.F, inst.D, p3)


def brute_force_numpy(F, D):
    n = F.shape[0]
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.int64)
    Fl, Dl = F.astype(np.int64), D.astype(np.int64)
    costs = np.zeros(len(perms), np.int64)
    for i in range(n):
        for j in range(n):
            if Fl[i, j]:
                costs += Fl[i, j] * Dl[perms[:, i], perms[:, j]]
    k = int(np.argmin(costs))
    return int(costs[k]), perms[k]


@pytest.mark.parametrize("n,seed", [(5, 1), (7, 2)])
def test_brute_force_matches_enumeration(n, seed):
    inst = W.random_asymmetric(n, seed)
    c, p = O.brute_force(inst.F, inst.D)
    c2, p2 = brute_force_numpy(inst.F, inst.D)
    assert c == c2 and np.array_equal(p, p2)


def test_brute_force_tiny9_and_local_search_bound():
    inst = W.tiny9()
    c, p = O.brute_force(inst.F, inst.D)
    c2, _ = brute_force_numpy(inst.F, inst.D)
    assert c == c2
    for q in W.random_perms(20, 9, 3):
        _, cl, _, _, _ = O.local_search(inst.F, inst.D, q, 0)
        assert cl >= c
