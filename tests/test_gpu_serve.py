"""The serving loop on the GPU: every result served in the mix equals the same
request solved alone; memory stays within the budget; requests overlap."""
import numpy as np
import pytest

from paper_1504_05158_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_served_results_equal_solo_runs():
    from paper_1504_05158_gb300 import qap_pso as Q
    from paper_1504_05158_gb300 import serve as S
    rng = np.random.default_rng(0)
    jobs = []
    for i in range(14):
        n = int(rng.choice([9, 24, 33, 64]))
        inst = W.dense_uniform(n, 40 + i) if i % 2 else W.grid_sparse(n, 40 + i)
        p = Q.default_params(swarms=int(rng.integers(2, 5)), swarm_size=int(rng.integers(16, 64)),
                             mig_kind=2, mig_period=3, v_storage=i % 2)
        jobs.append(S.Job(i, 0.002 * i, inst.F, inst.D, p, 1000 + i, int(rng.integers(5, 25))))
    budget = 4 * max(S.Server(1).footprint(j) for j in jobs)
    srv = S.Server(budget_bytes=budget, chunk=4)
    rep = srv.run(jobs)
    assert len(rep.results) == len(jobs)
    assert rep.peak_bytes <= budget and rep.peak_slots > 1
    for r, j in zip(rep.results, jobs):
        solo = Q.Swarm(Q.Instance(j.F, j.D), j.params, seed=j.seed)
        solo.step(j.iterations)
        c, perm, it = solo.best()
        assert (c, it) == (r.best_cost, r.best_iter) and np.array_equal(perm, r.best_perm), r.rid
        solo.close()


def test_footprint_matches_allocation():
    import torch
    from paper_1504_05158_gb300 import qap_pso as Q
    inst = W.grid64()
    gi = Q.Instance(inst.F, inst.D)
    p = Q.default_params(swarms=8, swarm_size=512)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sw = Q.Swarm(gi, p, seed=1)
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    fp = Q.footprint(64, p)
    assert fp <= used + (2 << 20) and used <= fp + (4 << 20), (fp, used)
    sw.close()
