"""Whole runs: a checkpoint round trip (k iterations, export, import into a fresh
population, k more) equals 2 k iterations straight; and the distribution of final
best costs over 32 seeds agrees between the CUDA path (fp32 and bf16 storage of V)
and the oracle. Rounding in the velocity can flip a discrete choice of S_x, so whole
runs are compared by their distributions, not run by run."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W
from tests.replay import oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1504_05158_gb300 import qap_pso
    qap_pso.lib()
    return qap_pso


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("variant", [dict(mig_kind=2, mig_period=3), dict(mig_kind=1, mig_depth=1, mig_period=2)])
def test_checkpoint_round_trip(Q, storage, variant):
    inst = W.grid_sparse(40, 12)
    prm = Q.default_params(swarms=4, swarm_size=30, v_storage=storage, **variant)
    gi = Q.Instance(inst.F, inst.D)
    a = Q.Swarm(gi, prm, seed=55)
    a.step(7)
    ckpt = a.export_state()
    a.step(7)  # straight: 14 iterations
    b = Q.Swarm(gi, prm, seed=55)  # a fresh population of the same run (same seed)
    b.step(3)  # whatever it did before is overwritten
    b.import_state(ckpt)
    b.step(7)
    sa, sb = a.export_state(), b.export_state()
    for k in ("V", "X", "X_sx", "PL", "costL", "cost", "moves", "PG", "costG", "best"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["best_cost"] == sb["best_cost"] and sa["best_iter"] == sb["best_iter"] and sa["t"] == sb["t"] == 14
    assert a.best()[0] == b.best()[0]


def _ks(x, y):
    """Two-sample Kolmogorov-Smirnov statistic."""
    x, y = np.sort(x), np.sort(y)
    grid = np.concatenate([x, y])
    fx = np.searchsorted(x, grid, side="right") / len(x)
    fy = np.searchsorted(y, grid, side="right") / len(y)
    return np.abs(fx - fy).max()


def test_final_cost_distribution_32_seeds(Q):
    inst = W.dense_uniform(20, 44)
    seeds = list(range(300, 332))
    iters = 25
    kw = dict(swarms=2, swarm_size=12, mig_kind=2, mig_period=5)
    finals = {}
    for name, storage in (("fp32", 0), ("bf16", 1)):
        prm = Q.default_params(v_storage=storage, **kw)
        gi = Q.Instance(inst.F, inst.D)
        out = []
        for sd in seeds:
            sw = Q.Swarm(gi, prm, seed=sd)
            sw.step(iters)
            out.append(sw.best()[0])
            sw.close()
        finals[name] = np.array(out, np.float64)
    q = oracle_params(Q.default_params(**kw))
    orc = []
    for sd in seeds:
        s = O.init(q, inst.F, inst.D, sd)
        O.step_parallel(q, inst.F, inst.D, sd, s, iters)
        orc.append(int(s.best_cost[0]))
    orc = np.array(orc, np.float64)
    same = int((finals["fp32"] == orc).sum())
    # fp32 against the fp64 oracle: the same distribution (5 % critical value of the KS
    # statistic for two samples of 32 is about 0.34) and the same mean within 1 %
    assert _ks(finals["fp32"], orc) <= 0.34, (same, finals["fp32"], orc)
    assert abs(finals["fp32"].mean() / orc.mean() - 1.0) <= 0.01, (same, finals["fp32"], orc)
    # bf16 storage of V: final quality within 2 % of fp32 at this small scale
    assert abs(finals["bf16"].mean() / finals["fp32"].mean() - 1.0) <= 0.02
    assert _ks(finals["bf16"], finals["fp32"]) <= 0.5
