"""A run split by whole swarms into CUDA parts (pso_init_part) that migrate through
the sharded driver equals the unsplit CUDA run bit for bit: positions, velocities,
local and swarm bests, migration choices and the global best.

The parts run on the one GPU of the test in two host threads, each with its own
stream; an in-process communicator stands in for the process group (the exchange
itself is covered over gloo by test_shard_gloo). No kernel waits for another part:
the parts meet only on the host."""
import queue
import threading
from collections import defaultdict

import numpy as np
import pytest

from paper_1504_05158_gb300 import workloads as W

pytestmark = pytest.mark.gpu


class Hub:
    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world)
        self.slots = [None] * world
        self.lock = threading.Lock()
        self.mail = defaultdict(queue.Queue)


class ThreadComm:
    """The communicator interface of shard.ShardedRun for ranks that are threads."""

    def __init__(self, hub, rank):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def allgather(self, a):
        h = self.hub
        h.barrier.wait()
        h.slots[self.rank] = np.array(a, np.int64)
        h.barrier.wait()
        out = np.stack(h.slots)
        h.barrier.wait()
        return out

    def exchange(self, sends, recvs):
        for a, dst, tag in sends:
            self.hub.mail[(self.rank, dst, tag)].put(np.array(a, np.int64))
        return [self.hub.mail[(src, self.rank, tag)].get(timeout=60) for _, src, tag in recvs]

    def bcast(self, a, src):
        h = self.hub
        h.barrier.wait()
        if self.rank == src:
            h.slots[0] = np.array(a, np.int64)
        h.barrier.wait()
        out = h.slots[0].copy()
        h.barrier.wait()
        return out


CASES = {
    "ring": dict(mig_kind=2, mig_period=2),
    "ring_if_better": dict(mig_kind=2, mig_period=1, ring_if_better=1),
    "rank": dict(mig_kind=1, mig_depth=2, mig_period=1),
    "rank_bf16": dict(mig_kind=1, mig_depth=1, mig_period=2, v_storage=1),
}


@pytest.mark.parametrize("case", list(CASES))
def test_parts_equal_unsplit_gpu_run(case):
    import torch

    from paper_1504_05158_gb300 import qap_pso as Q
    from paper_1504_05158_gb300 import shard as S
    inst = W.dense30()
    m, ss, seed, iters, world = 5, 24, 91, 9, 2
    prm = Q.default_params(swarms=m, swarm_size=ss, **CASES[case])
    gi = Q.Instance(inst.F, inst.D)
    whole = Q.Swarm(gi, prm, seed=seed)
    whole.step(iters)
    ref = whole.export_state()
    ref_best = whole.best()

    hub = Hub(world)
    results, errors = {}, []

    def rank_main(rank):
        try:
            first, count = S.partition(m, world)[rank]
            kw = {k: getattr(prm, k) for k, _ in prm._fields_}
            kw.update(swarms=count)
            stream = torch.cuda.Stream()
            part = Q.Swarm(gi, Q.default_params(**kw), seed=seed, stream=stream.cuda_stream, first_swarm=first)
            run = S.ShardedRun(part, prm, m, seed, ThreadComm(hub, rank))
            run.step(iters)
            results[rank] = (first, count, part.export_state(), run.best())
            part.close()
        except Exception as e:  # reported by the main thread
            errors.append(repr(e))
            hub.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for rank, (first, count, st, best) in results.items():
        a, b = first * ss, (first + count) * ss
        for key in ("X", "X_sx", "PL", "costL", "cost", "moves", "V"):
            assert np.array_equal(st[key], ref[key][a:b]), (rank, key)
        assert np.array_equal(st["PG"], ref["PG"][first:first + count]), (rank, "PG")
        assert np.array_equal(st["costG"], ref["costG"][first:first + count]), (rank, "costG")
        assert st["t"] == ref["t"] == iters
        c, perm, it = best
        assert c == ref_best[0] and it == ref_best[2] and np.array_equal(perm, ref_best[1]), rank
