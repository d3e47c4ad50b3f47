"""Host logic of the serving loop against a fake backend (no GPU): admission
under the memory budget, first come first served, overlap, latency accounting."""
import numpy as np
import pytest

from paper_1504_05158_gb300 import serve as S


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


class FakeSwarm:
    live = 0
    max_live = 0

    def __init__(self, inst, params, seed):
        self.n = inst.n
        self.P = params.swarms * params.swarm_size
        self.seed = seed
        self.pending = 0
        FakeSwarm.live += 1
        FakeSwarm.max_live = max(FakeSwarm.max_live, FakeSwarm.live)

    running = 0
    max_running = 0

    def done(self):
        if self.pending:
            self.pending -= 1  # one poll per queued chunk
            if not self.pending:
                FakeSwarm.running -= 1
            return False
        return True

    def step(self, k):
        if not self.pending:
            FakeSwarm.running += 1
            FakeSwarm.max_running = max(FakeSwarm.max_running, FakeSwarm.running)
        self.pending += 1

    def best(self):
        return int(self.seed) * 10, np.arange(self.n), 1

    def close(self):
        FakeSwarm.live -= 1


class FakeInstance:
    def __init__(self, F, D):
        self.n = F.shape[0]

    def close(self):
        pass


class P:
    def __init__(self, swarms, swarm_size):
        self.swarms, self.swarm_size = swarms, swarm_size


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(S.Q, "Instance", FakeInstance)
    monkeypatch.setattr(S.Q, "Swarm", FakeSwarm)
    monkeypatch.setattr(S.Q, "footprint", lambda n, p: 1000 * p.swarms * p.swarm_size)
    FakeSwarm.live = FakeSwarm.max_live = 0
    FakeSwarm.running = FakeSwarm.max_running = 0


def _jobs(k):
    z = np.zeros((4, 4), np.int32)
    return [S.Job(i, 0.0001 * i, z, z, P(2, 5), 100 + i, 30) for i in range(k)]


def test_budget_never_exceeded_and_all_served(fake):
    jobs = _jobs(12)
    per = 1000 * 10 + 2 * 16 * 4
    srv = S.Server(budget_bytes=3 * per, chunk=10, clock=FakeClock())
    rep = srv.run(jobs)
    assert [r.rid for r in rep.results] == list(range(12))
    assert rep.peak_bytes <= 3 * per
    assert FakeSwarm.max_live == 3 and rep.peak_slots == 3  # overlap up to the budget
    assert all(r.best_cost == 10 * (100 + r.rid) for r in rep.results)
    assert all(r.done_s >= r.admit_s >= r.arrival_s for r in rep.results)


def test_first_come_first_served(fake):
    jobs = _jobs(6)
    srv = S.Server(budget_bytes=1000 * 10 + 200, chunk=10, clock=FakeClock())
    rep = srv.run(jobs)
    admits = [r.admit_s for r in sorted(rep.results, key=lambda r: r.rid)]
    assert admits == sorted(admits)
    assert FakeSwarm.max_live == 1


def test_inflight_limit_serves_oldest_first(fake):
    # memory admits all 8 jobs at once, but only two jobs' particles may have work in
    # flight: at most two run, and results come back in arrival order
    jobs = _jobs(8)
    srv = S.Server(budget_bytes=10 ** 9, chunk=10, inflight_particles=20, clock=FakeClock())
    rep = srv.run(jobs)
    assert FakeSwarm.max_live == 8 and FakeSwarm.max_running == 2
    assert rep.peak_inflight == 20
    done = [r.done_s for r in rep.results]
    assert done == sorted(done)


def test_inflight_limit_below_one_job_still_runs(fake):
    jobs = _jobs(3)
    srv = S.Server(budget_bytes=10 ** 9, chunk=10, inflight_particles=1, clock=FakeClock())
    rep = srv.run(jobs)
    assert len(rep.results) == 3 and FakeSwarm.max_running == 1


def test_oversized_request_rejected(fake):
    jobs = _jobs(1)
    with pytest.raises(ValueError):
        S.Server(budget_bytes=10).run(jobs)


def test_report_percentiles():
    rep = S.ServeReport()
    for i in range(100):
        rep.results.append(S.Result(i, 4, 10, 30, 0, None, 0, 0.0, 0.0, float(i + 1)))
    rep.makespan_s = 10.0
    s = rep.summary()
    assert s["p50_s"] == 50.0 and s["p99_s"] == 99.0
    assert s["particle_iterations_per_s"] == 100 * 10 * 30 / 10.0


def test_device_failure_fails_the_request(fake, monkeypatch):
    # a population whose kernels reported an error (pso_best returns a status) fails
    # its request; the others complete and the memory is returned
    def best(self):
        if self.seed == 3:
            raise S.Q.QapError(S.Q.ERR_TIMEOUT, "pso_best")
        return int(self.seed) * 10, np.arange(self.n), 1
    monkeypatch.setattr(FakeSwarm, "best", best)
    monkeypatch.setattr(S.Q, "status_string", lambda st: "device wait timed out")
    F = np.zeros((8, 8), np.int32)
    jobs = [S.Job(i, 0.0, F, F, P(2, 4), seed=i, iterations=3) for i in range(6)]
    rep = S.Server(budget_bytes=10**9, clock=FakeClock()).run(jobs, realtime=False)
    assert len(rep.results) == 6
    bad = rep.failed()
    assert [r.rid for r in bad] == [3] and bad[0].best_cost is None and "timed out" in bad[0].error
    assert all(r.best_cost == r.rid * 10 for r in rep.results if r.rid != 3)
    assert rep.summary()["failed"] == 1
    assert FakeSwarm.live == 0
