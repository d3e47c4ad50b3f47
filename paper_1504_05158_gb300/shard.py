"""One multi-swarm PSO run split by whole swarms over several processes, one GPU each.

The swarms of a run are independent within an iteration; they meet only in the
migration step (section 3.2), which moves one permutation per migrating swarm. So
each process holds a part of the run (pso_init_part: swarms [first, first + count),
every random draw keyed by the swarm's index in the whole run, no migration on the
device) and the processes exchange, at every migration event, the m swarm-best
costs (an allgather of m int64) and the migrating permutations (point to point, n
ints each):

  ring (every mig_period iterations): swarm k's best replaces swarm k + 1's (mod m),
    all from a snapshot, optionally only if strictly better; inside a part the shift
    is local, across a boundary one permutation goes to the next process;
  Algorithm 2 (rank): the swarms ordered by (P^G cost, index); for k < d the k-th
    worst swarm's P^G becomes the current position of particle j of the k-th best
    swarm, j from Philox tag 4 with counter (k, 0, t), accepted even if worse; the
    donor's process sends it to the target's.

The global best is the minimum of the parts' bests by (cost, iteration found, part),
which is the unsplit run's rule (lowest particle index on equal cost and iteration).
Results equal those of the unsplit run exactly.

Host logic only: every iteration runs in the CUDA library. The communicator is
torch.distributed (gloo over host memory: the messages are a few kilobytes) or any
object with the same five methods.
"""
from __future__ import annotations

import numpy as np

from . import qap_pso as Q

TAG_MIG = 4


def partition(m: int, world: int):
    """Contiguous (first swarm, count) of each rank; counts differ by at most one."""
    if world < 1 or m < world:
        raise ValueError("need at least one swarm per rank")
    base, extra = divmod(m, world)
    parts, first = [], 0
    for r in range(world):
        cnt = base + (1 if r < extra else 0)
        parts.append((first, cnt))
        first += cnt
    return parts


class TorchComm:
    """The exchange over a torch.distributed process group (int64 host tensors for
    gloo, device tensors for nccl)."""

    def __init__(self, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"

    def _t(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, np.int64)).to(self.device)

    def allgather(self, a):
        """(world, len(a)) int64: every rank's a (equal lengths)."""
        t = self._t(a)
        out = [self.torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        return np.stack([o.cpu().numpy() for o in out])

    def exchange(self, sends, recvs):
        """Posts every (array, dst, tag) send, then every (length, src, tag) receive;
        returns the received arrays in the order of recvs."""
        reqs, bufs = [], []
        for a, dst, tag in sends:
            t = self._t(a)
            bufs.append(t)
            reqs.append(self.dist.isend(t, dst, group=self.group, tag=tag))
        outs = []
        for ln, src, tag in recvs:
            t = self.torch.empty(ln, dtype=self.torch.int64, device=self.device)
            outs.append(t)
            reqs.append(self.dist.irecv(t, src, group=self.group, tag=tag))
        for r in reqs:
            r.wait()
        return [o.cpu().numpy() for o in outs]

    def bcast(self, a, src):
        t = self._t(a)
        self.dist.broadcast(t, src, group=self.group)
        return t.cpu().numpy()


class ShardedRun:
    """This rank's part of a run of `swarms_total` swarms (each `params.swarm_size`
    particles): `pop` holds the rank's swarms (a qap_pso.Swarm created with
    first_swarm, or any object with step, swarm_bests, set_swarm_best, particle and
    best), `params` are the run's parameters (their migration settings are applied
    here), `comm` the communicator."""

    def __init__(self, pop, params, swarms_total: int, seed: int, comm, t0: int = 0):
        self.pop, self.prm, self.m, self.seed, self.comm = pop, params, swarms_total, seed, comm
        self.parts = partition(swarms_total, comm.world)
        self.first, self.count = self.parts[comm.rank]
        self.ss = params.swarm_size
        self.t = t0

    def owner(self, g):
        for r, (f, c) in enumerate(self.parts):
            if f <= g < f + c:
                return r
        raise IndexError(g)

    def step(self, iterations: int = 1):
        """`iterations` iterations of the whole run (each rank calls it alike)."""
        period = max(1, self.prm.mig_period)
        for _ in range(iterations):
            self.pop.step(1)
            t = self.t
            self.t += 1
            if self.prm.mig_kind != Q.MIG_NONE and (t + 1) % period == 0:
                self._migrate(t)

    def _global_costs(self):
        costs, perms = self.pop.swarm_bests()
        width = max(c for _, c in self.parts)
        pad = np.full(width, np.iinfo(np.int64).max, np.int64)
        pad[: self.count] = costs
        rows = self.comm.allgather(pad)
        G = np.concatenate([rows[r, :c] for r, (_, c) in enumerate(self.parts)])
        return G, costs, perms

    def _migrate(self, t):
        G, costs, perms = self._global_costs()  # the snapshot every rank works from
        rank, world, m, n = self.comm.rank, self.comm.world, self.m, perms.shape[1]
        if self.prm.mig_kind == Q.MIG_RING:
            # the source of this part's first swarm is the previous part's last swarm
            sends, recvs = [], []
            if world > 1:
                sends.append((perms[self.count - 1], (rank + 1) % world, 1))
                recvs.append((n, (rank - 1) % world, 1))
            got = self.comm.exchange(sends, recvs)
            prev = got[0] if world > 1 else perms[self.count - 1]
            for k in range(self.count):
                g = self.first + k
                src = (g - 1) % m
                if self.prm.ring_if_better and not (G[src] < G[g]):
                    continue
                p = perms[k - 1] if k > 0 else prev
                self.pop.set_swarm_best(k, G[src], p)
        elif self.prm.mig_kind == Q.MIG_RANK and self.prm.mig_depth > 0:
            order = sorted(range(m), key=lambda k: (G[k], k))
            sends, recvs, local = [], [], []
            for k in range(self.prm.mig_depth):
                donor, target = order[k], order[m - 1 - k]
                j = int((int(Q.philox(self.seed, k, 0, t, TAG_MIG, 0)[0]) * self.ss) >> 32)
                dr, tr = self.owner(donor), self.owner(target)
                if dr == rank:
                    c, p = self.pop.particle((donor - self.first) * self.ss + j)
                    msg = np.concatenate([[c], p]).astype(np.int64)
                    if tr == rank:
                        local.append((target, msg))
                    else:
                        sends.append((msg, tr, 100 + k))
                elif tr == rank:
                    recvs.append((n + 1, dr, 100 + k))
                    local.append((target, None))
            got = iter(self.comm.exchange(sends, recvs))
            for target, msg in local:
                if msg is None:
                    msg = next(got)
                self.pop.set_swarm_best(target - self.first, int(msg[0]), msg[1:].astype(np.int32))

    def best(self):
        """(cost, permutation, iteration found) of the whole run, on every rank."""
        c, p, it = self.pop.best()
        rows = self.comm.allgather(np.array([c, it, self.comm.rank], np.int64))
        win = min(range(len(rows)), key=lambda r: (rows[r, 0], rows[r, 1], rows[r, 2]))
        perm = self.comm.bcast(np.asarray(p, np.int64), win)
        return int(rows[win, 0]), perm.astype(np.int32), int(rows[win, 1])
