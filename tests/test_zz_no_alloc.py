"""The allocation-free statistics entry point, called through the C-ABI, gives the
same results as pso_stats on the same costs, on two calls in a row.

This file sorts last on purpose: a run that stops at the first failure has run
every other test before this one."""
import numpy as np
import pytest

from paper_1504_05158_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("min", "p5", "p25", "p50", "p75", "max")


def _reference(Q, inst, swarms, swarm_size, seed, iters):
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), Q.default_params(swarms=swarms, swarm_size=swarm_size),
                 seed=seed)
    sw.step(iters)
    st = sw.export_state()
    return st["cost"], sw.stats()


def test_noalloc_stats_match_pso_stats_twice():
    import torch

    from paper_1504_05158_gb300 import qap_pso as Q
    Q.lib()
    cases = [(W.dense30(), 10, 1000, 3, 2), (W.grid64(), 3, 77, 4, 1)]  # 10 000 then 231 costs
    for inst, m, ss, seed, iters in cases:
        costs, want = _reference(Q, inst, m, ss, seed, iters)
        dev = torch.from_numpy(costs).cuda()
        torch.cuda.synchronize()
        got = Q.cost_stats_noalloc(dev.data_ptr(), len(costs),
                                   torch.cuda.current_stream().cuda_stream)
        for k in KEYS:
            assert got[k] == want[k], (k, got[k], want[k])
        assert abs(got["mean"] - want["mean"]) <= 1e-12 * abs(want["mean"])


def test_noalloc_rejects_oversize_and_empty():
    import torch

    from paper_1504_05158_gb300 import qap_pso as Q
    dev = torch.zeros(4, dtype=torch.int64, device="cuda")
    for bad in (0, Q.NOALLOC_MAX_COUNT + 1):
        with pytest.raises(Q.QapError) as e:
            Q.cost_stats_noalloc(dev.data_ptr(), bad)
        assert e.value.status == Q.ERR_INVALID_ARG
