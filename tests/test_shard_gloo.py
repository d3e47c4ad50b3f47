"""A run split by whole swarms over two processes (gloo on CPU): with the exchange of
the sharded driver, every swarm best, migration choice, position, velocity and the
global best equal those of the unsplit run of the oracle, bit for bit.

The parts here are computed by the oracle (test infrastructure standing in for the
CUDA parts, which need a GPU); the exchange and its bookkeeping are the product's
(paper_1504_05158_gb300.shard)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W

CASES = {
    "ring": dict(mig_kind=2, mig_period=2),
    "ring_if_better": dict(mig_kind=2, mig_period=1, ring_if_better=1),
    "rank": dict(mig_kind=1, mig_depth=2, mig_period=1),
    "rank_period3": dict(mig_kind=1, mig_depth=1, mig_period=3),
}
M, SS, N, SEED, ITERS = 5, 6, 12, 77, 7


class OraclePart:
    """Swarms [first, first + count) of an oracle run, iterated with the whole run's
    draws (swarm index first + k) and no migration."""

    def __init__(self, q_full, F, D, seed, first, count):
        self.F, self.D, self.seed, self.first, self.count = F, D, seed, first, count
        self.ss = q_full.swarm_size
        kw = {k: getattr(q_full, k) for k, _ in O.Params._fields_}
        kw.update(swarms=count, mig_kind=0)
        self.q = O.make_params(**kw)
        full = O.init(q_full, F, D, seed)
        a, b = first * self.ss, (first + count) * self.ss
        s = O.State(self.q, F.shape[0])
        s.V[:], s.X[:], s.PL[:] = full.V[a:b], full.X[a:b], full.PL[a:b]
        s.costL[:], s.cost[:] = full.costL[a:b], full.cost[a:b]
        s.PG[:], s.costG[:] = full.PG[first:first + count], full.costG[first:first + count]
        gi = int(np.argmin(s.cost))  # the part's best at initialisation (lowest index on ties)
        s.best_p[:], s.best_cost[0], s.best_iter[0] = s.X[gi], s.cost[gi], 0
        self.s = s

    def step(self, k):
        s, q = self.s, self.q
        for _ in range(k):
            t = int(s.t[0])
            for idx in range(self.count * self.ss):
                kk, i = divmod(idx, self.ss)
                r = O.particle_iteration(q, self.F, self.D, self.seed, t, self.first + kk, i, s.V[idx], s.X[idx],
                                         s.PL[idx], s.PG[kk])
                s.V[idx], s.X[idx], s.cost[idx] = r["V_new"], r["p_out"], r["cost"]
                if r["cost"] < s.costL[idx]:
                    s.costL[idx], s.PL[idx] = r["cost"], r["p_out"]
            O.bests_and_migration(q, self.seed, t, s)
            s.t[0] = t + 1

    def swarm_bests(self):
        return self.s.costG.copy(), self.s.PG.copy()

    def set_swarm_best(self, k, cost, perm):
        self.s.costG[k] = cost
        self.s.PG[k] = perm

    def particle(self, index):
        return int(self.s.cost[index]), self.s.X[index].copy()

    def best(self):
        return int(self.s.best_cost[0]), self.s.best_p.copy(), int(self.s.best_iter[0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, q_out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1504_05158_gb300 import qap_pso as Q
    from paper_1504_05158_gb300 import shard as S
    inst = W.dense_uniform(N, 3)
    qf = O.make_params(swarms=M, swarm_size=SS, **CASES[case])
    prm = Q.default_params(swarms=M, swarm_size=SS, **CASES[case])
    first, count = S.partition(M, world)[rank]
    part = OraclePart(qf, inst.F, inst.D, SEED, first, count)
    run = S.ShardedRun(part, prm, M, SEED, S.TorchComm())
    run.step(ITERS)
    best = run.best()
    s = part.s
    q_out.put((rank, first, count, s.X.copy(), s.V.copy(), s.PL.copy(), s.costL.copy(), s.cost.copy(),
               s.PG.copy(), s.costG.copy(), best))
    dist.destroy_process_group()


@pytest.mark.parametrize("case", list(CASES))
def test_two_ranks_equal_unsplit_oracle(case):
    inst = W.dense_uniform(N, 3)
    q = O.make_params(swarms=M, swarm_size=SS, **CASES[case])
    ref = O.init(q, inst.F, inst.D, SEED)
    O.step(q, inst.F, inst.D, SEED, ref, ITERS)
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    qo = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, qo)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((qo.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, first, count, X, V, PL, costL, cost, PG, costG, best in got:
        a, b = first * SS, (first + count) * SS
        assert np.array_equal(X, ref.X[a:b]) and np.array_equal(cost, ref.cost[a:b]), rank
        assert np.array_equal(V, ref.V[a:b]), rank
        assert np.array_equal(PL, ref.PL[a:b]) and np.array_equal(costL, ref.costL[a:b]), rank
        assert np.array_equal(PG, ref.PG[first:first + count]), (rank, "P^G")
        assert np.array_equal(costG, ref.costG[first:first + count]), (rank, "P^G cost")
        c, perm, it = best
        assert c == ref.best_cost[0] and it == ref.best_iter[0] and np.array_equal(perm, ref.best_p), rank


def test_partition():
    from paper_1504_05158_gb300 import shard as S
    assert S.partition(5, 2) == [(0, 3), (3, 2)]
    assert S.partition(16, 4) == [(0, 4), (4, 4), (8, 4), (12, 4)]
    assert S.partition(3, 3) == [(0, 1), (1, 1), (2, 1)]
    with pytest.raises(ValueError):
        S.partition(2, 3)
