"""Batches of populations with uneven n: each member is bit-identical to the same
population run alone, and one batch iteration replays through the oracle."""
import numpy as np
import pytest

from paper_1504_05158_gb300 import workloads as W
from tests.replay import compare_step, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1504_05158_gb300 import qap_pso
    qap_pso.lib()
    return qap_pso


def _members():
    # n = 9, 24 (one-warp teams), 40, 64 (two-warp teams), 70, 100 (SIMT set-up)
    insts = [W.tiny9(), W.dense_uniform(24, 2), W.grid_sparse(40, 3), W.grid64(),
             W.dense_uniform(70, 5), W.grid_sparse(100, 6)]
    return insts


def _params(Q, i, storage):
    return Q.default_params(swarms=2 + i % 3, swarm_size=11 + 5 * i, mig_kind=2 - i % 3,
                            mig_depth=0, mig_period=3, v_storage=storage)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_members_equal_individual_runs(Q, storage, autotune):
    insts = _members()
    ginsts = [Q.Instance(i.F, i.D) for i in insts]
    params = [_params(Q, i, storage) for i in range(len(insts))]
    seeds = [100 + i for i in range(len(insts))]
    batch = Q.Batch(ginsts, params, seeds, autotune=autotune)
    batch.step(5)
    for i, gi in enumerate(ginsts):
        solo = Q.Swarm(gi, params[i], seed=seeds[i])
        solo.step(5)
        a, b = batch.members[i].export_state(), solo.export_state()
        for k in ("X", "X_sx", "PL", "costL", "cost", "moves", "PG", "costG", "best"):
            assert np.array_equal(a[k], b[k]), (i, k)
        assert np.array_equal(a["V"], b["V"]), i
        assert (a["best_cost"], a["best_iter"], a["t"]) == (b["best_cost"], b["best_iter"], b["t"])
        sa, sb = batch.members[i].stats(), solo.stats()
        assert sa == sb, i
        solo.close()
    batch.close()


def test_batch_iteration_replays_through_oracle(Q):
    insts = _members()
    ginsts = [Q.Instance(i.F, i.D) for i in insts]
    params = [_params(Q, i, 0) for i in range(len(insts))]
    seeds = [7 + i for i in range(len(insts))]
    batch = Q.Batch(ginsts, params, seeds, autotune=False)
    batch.step(2)
    before = [m.export_state() for m in batch.members]
    batch.step(1)
    for i, m in enumerate(batch.members):
        after = m.export_state()
        P = len(after["X"])
        sample = None if P <= 40 else np.array([0, P - 1, P // 2, 3, 17])
        compare_step(oracle_params(params[i]), insts[i].F, insts[i].D, seeds[i], before[i], after,
                     params[i], sample=sample)
    batch.close()


def test_batch_rejects_mixed_storage(Q):
    a = Q.Instance(W.tiny9().F, W.tiny9().D)
    with pytest.raises(Q.QapError) as e:
        Q.Batch([a, a], [Q.default_params(v_storage=0), Q.default_params(v_storage=1)], [1, 2])
    assert e.value.status == Q.ERR_INVALID_ARG
