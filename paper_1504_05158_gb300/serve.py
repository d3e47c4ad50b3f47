"""Continuous-batching serving loop for PSO solves.

Requests (a QAP instance, PSO parameters, a seed and an iteration budget) arrive
over time. A request is admitted as a slot as soon as its device footprint fits
the memory budget (first come, first served); every slot keeps its population on
the device, on its own CUDA stream, so work of different requests overlaps on the
GPU. The loop feeds chunks of iterations to the oldest slots first, up to a number
of particles with work in flight (enough to fill the GPU; more would only share it
out and delay every result), and retires a slot when its budget is spent, reading
back the best solution and freeing its memory. Latency is measured from arrival to
the read-back of the result.

Host logic only: all of the iteration runs in the CUDA library.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from . import qap_pso as Q


@dataclass
class Job:
    rid: int
    arrival_s: float
    F: object
    D: object
    params: object  # qap_pso.Params
    seed: int
    iterations: int


@dataclass
class Result:
    rid: int
    n: int
    particles: int
    iterations: int
    best_cost: int
    best_perm: object
    best_iter: int
    arrival_s: float
    admit_s: float
    done_s: float
    error: str | None = None  # set when the device reported a failure: no result

    @property
    def latency_s(self):
        return self.done_s - self.arrival_s


@dataclass
class _Slot:
    job: Job
    inst: Q.Instance
    swarm: Q.Swarm
    bytes: int
    queued: int = 0
    admit_s: float = 0.0
    idle: bool = True


@dataclass
class ServeReport:
    results: list = field(default_factory=list)
    makespan_s: float = 0.0
    peak_bytes: int = 0
    peak_slots: int = 0
    peak_inflight: int = 0

    def latencies(self):
        return sorted(r.latency_s for r in self.results)

    def percentile(self, q):
        lat = self.latencies()
        if not lat:
            return None
        k = max(0, min(len(lat) - 1, int(-(-q * len(lat) // 1)) - 1))  # nearest rank
        return lat[k]

    def particle_iterations(self):
        return sum(r.particles * r.iterations for r in self.results if r.error is None)

    def failed(self):
        return [r for r in self.results if r.error is not None]

    def summary(self):
        return {"requests": len(self.results), "failed": len(self.failed()), "makespan_s": self.makespan_s,
                "p50_s": self.percentile(0.5), "p99_s": self.percentile(0.99),
                "particle_iterations_per_s": self.particle_iterations() / max(self.makespan_s, 1e-9),
                "peak_bytes": self.peak_bytes, "peak_slots": self.peak_slots,
                "peak_inflight_particles": self.peak_inflight}


class Server:
    """Admits jobs under `budget_bytes` of device memory. `chunk` iterations are
    queued per slot at a time; slots receive work oldest first while fewer than
    `inflight_particles` particles have work in flight (the oldest waiting slot
    always may start, so a request larger than the limit still runs)."""

    def __init__(self, budget_bytes: int, chunk: int = 1 << 20, max_slots: int = 512,
                 inflight_particles: int = 1 << 62, clock=time.perf_counter):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.max_slots = int(max_slots)
        self.inflight = int(inflight_particles)
        self.clock = clock

    def footprint(self, job: Job) -> int:
        n = int(job.F.shape[0])
        return Q.footprint(n, job.params) + 2 * n * n * 4  # population + instance copy

    def run(self, jobs, realtime: bool = True) -> ServeReport:
        """Serves `jobs` (sorted by arrival). With realtime=False every job counts as
        arrived at once (throughput at saturation)."""
        pending = sorted(jobs, key=lambda j: j.arrival_s)
        for j in pending:
            if self.footprint(j) > self.budget:
                raise ValueError(f"request {j.rid} alone exceeds the memory budget")
        rep = ServeReport()
        active: list[_Slot] = []
        used = 0
        t0 = self.clock()
        head = 0
        while head < len(pending) or active:
            now = self.clock() - t0
            # admission, first come first served, while memory and slots allow
            while head < len(pending) and (not realtime or pending[head].arrival_s <= now):
                job = pending[head]
                need = self.footprint(job)
                if used + need > self.budget or len(active) >= self.max_slots:
                    break
                inst = Q.Instance(job.F, job.D)
                sw = Q.Swarm(inst, job.params, seed=job.seed)
                active.append(_Slot(job, inst, sw, need, 0, self.clock() - t0))
                used += need
                head += 1
            rep.peak_bytes = max(rep.peak_bytes, used)
            rep.peak_slots = max(rep.peak_slots, len(active))
            # supply the oldest slots with work, up to the in-flight particle limit
            busy = 0
            submitted = False
            idle = []
            for s in active:
                s.idle = s.swarm.done()
                if not s.idle:
                    busy += s.swarm.P
            for s in active:
                if s.idle and s.queued < s.job.iterations and (busy == 0 or busy + s.swarm.P <= self.inflight):
                    k = min(self.chunk, s.job.iterations - s.queued)
                    s.swarm.step(k)
                    s.queued += k
                    s.idle = False
                    busy += s.swarm.P
                    submitted = True
            rep.peak_inflight = max(rep.peak_inflight, busy)
            # retire finished slots
            still = []
            for s in active:
                if s.queued >= s.job.iterations and s.idle:
                    # a kernel that gave up a bounded wait makes best() fail: the
                    # request fails instead of returning a possibly incomplete result
                    try:
                        cost, perm, it = s.swarm.best()
                        err = None
                    except Q.QapError as e:
                        cost, perm, it, err = None, None, -1, str(e)
                    rep.results.append(Result(s.job.rid, s.swarm.n, s.swarm.P, s.job.iterations, cost,
                                              perm, it, s.job.arrival_s if realtime else 0.0,
                                              s.admit_s, self.clock() - t0, err))
                    s.swarm.close()
                    s.inst.close()
                    used -= s.bytes
                else:
                    still.append(s)
            retired = len(still) < len(active)
            active = still
            if active and not submitted and not retired:
                time.sleep(0.0002)
            elif not active and head < len(pending) and realtime:
                time.sleep(max(0.0, min(0.01, pending[head].arrival_s - (self.clock() - t0))))
        rep.makespan_s = self.clock() - t0
        rep.results.sort(key=lambda r: r.rid)
        return rep


def jobs_from_stream(requests, params_fn=None):
    """Jobs from workloads.serving_stream requests (dense-uniform or grid instances,
    particles split into 8..32 swarms, fixed iteration budget)."""
    out = []
    for i, r in enumerate(requests):
        p = params_fn(r) if params_fn else Q.default_params(swarms=r.swarms, swarm_size=r.swarm_size)
        out.append(Job(i, r.arrival_s, r.instance.F, r.instance.D, p, r.seed, r.iterations))
    return out
