"""The allocation-free statistics entry point, called through the C-ABI.

It is checked against the oracle's statistics of the same costs, against pso_stats
on the same population, for identical results on two identical calls in a row, for
no stale slots when a smaller call follows a larger one, and for unchanged free
device memory across its calls (it must not allocate).

This file sorts last on purpose: a run that stops at the first failure has run
every other test before this one."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("min", "p5", "p25", "p50", "p75", "max", "mean")


def _population(Q, inst, swarms, swarm_size, seed, iters):
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), Q.default_params(swarms=swarms, swarm_size=swarm_size),
                 seed=seed)
    sw.step(iters)
    st = sw.export_state()
    return st["cost"], sw.stats()


def test_noalloc_stats_match_oracle_and_pso_stats():
    import torch

    from paper_1504_05158_gb300 import qap_pso as Q
    Q.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # the first call on a device looks up the fixed array (with CUDA's lazy module
    # loading, that is when the driver places it); later calls must not allocate
    warm = torch.zeros(1, dtype=torch.int64, device="cuda")
    Q.cost_stats_noalloc(warm.data_ptr(), 1, stream)
    # 10 000 costs, then 231: the smaller call must see nothing of the larger one
    cases = [(W.dense30(), 10, 1000, 3, 2), (W.grid64(), 3, 77, 4, 1)]
    for inst, m, ss, seed, iters in cases:
        costs, via_state = _population(Q, inst, m, ss, seed, iters)
        want = O.stats(costs)
        dev = torch.from_numpy(costs).cuda()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        got1 = Q.cost_stats_noalloc(dev.data_ptr(), len(costs), stream)
        got2 = Q.cost_stats_noalloc(dev.data_ptr(), len(costs), stream)
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, "the entry point changed the free device memory"
        assert got1 == got2, "two identical calls in a row differ"
        for k in KEYS:
            assert got1[k] == want[k], (k, got1[k], want[k])
            assert via_state[k] == want[k], (k, via_state[k], want[k])


def test_noalloc_extreme_costs():
    # costs near the int64 limit: the device sums them in 128 bits, the mean is exact
    import torch

    from paper_1504_05158_gb300 import qap_pso as Q
    rng = np.random.default_rng(5)
    costs = rng.integers(2**62, 2**63 - 1, size=5000, dtype=np.int64)
    costs[:7] = 2**63 - 1
    dev = torch.from_numpy(costs).cuda()
    got = Q.cost_stats_noalloc(dev.data_ptr(), len(costs))
    want = O.stats(costs)
    for k in KEYS:
        assert got[k] == want[k], k


def test_noalloc_rejects_oversize_and_empty():
    import torch

    from paper_1504_05158_gb300 import qap_pso as Q
    dev = torch.zeros(4, dtype=torch.int64, device="cuda")
    for bad in (0, Q.NOALLOC_MAX_COUNT + 1):
        with pytest.raises(Q.QapError) as e:
            Q.cost_stats_noalloc(dev.data_ptr(), bad)
        assert e.value.status == Q.ERR_INVALID_ARG
