"""Per-iteration statistics recorded on the device (section 4.2: percentile ranks of
the population and of every swarm, and the cost histogram), compared record by
record with the oracle's statistics of the exported costs of each iteration."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_05158_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("min", "p5", "p25", "p50", "p75", "max", "mean")


@pytest.fixture(scope="module")
def Q():
    from paper_1504_05158_gb300 import qap_pso
    qap_pso.lib()
    return qap_pso


def _check_record(rec, costs, ss, lo, hi, bins):
    want = O.stats(costs)
    for k in KEYS:
        assert rec["population"][k] == want[k], (k, rec["population"][k], want[k])
    assert rec["population"]["sum"] == int(costs.astype(object).sum())
    for k, sw in enumerate(rec["swarms"]):
        ws = O.stats(costs[k * ss:(k + 1) * ss])
        for key in KEYS:
            assert sw[key] == ws[key], (k, key)
    assert np.array_equal(rec["histogram"], O.histogram(costs, lo, hi, bins))


@pytest.mark.parametrize("name,m,ss,bins", [("dense30", 5, 60, 17), ("grid64", 4, 333, 64),
                                            ("tiny9", 3, 9, 5)])
def test_trace_each_iteration(Q, name, m, ss, bins):
    inst = {"dense30": W.dense30, "grid64": W.grid64, "tiny9": W.tiny9}[name]()
    prm = Q.default_params(swarms=m, swarm_size=ss, mig_kind=2, mig_period=2)
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), prm, seed=3)
    c0 = sw.export_state()["cost"]
    lo, hi = int(c0.min()) // 2, int(c0.max()) - 1  # some costs fall outside [lo, hi)
    sw.trace_start(capacity=4, lo=lo, hi=hi, bins=bins)
    costs = []
    for _ in range(6):
        sw.step(1)
        costs.append(sw.export_state()["cost"])
    recs = sw.trace_read()
    assert [r["t"] for r in recs] == [3, 4, 5, 6]  # the ring keeps the last four
    for rec, c in zip(recs, costs[2:]):
        _check_record(rec, c, ss, lo, hi, bins)
    # many iterations in one call (graph replays of 16 and 1): one record each
    sw.step(21)
    recs = sw.trace_read()
    assert [r["t"] for r in recs] == [24, 25, 26, 27]
    _check_record(recs[-1], sw.export_state()["cost"], ss, lo, hi, bins)
    assert len(sw.trace_read(max_records=2)) == 2
    sw.trace_stop()
    sw.step(2)
    assert sw.stats()["iteration"] == 29 and sw.stats()["errors"] == 0


def test_trace_wide_range_and_large_swarms(Q):
    # costs spread over many orders (entries up to 10^5: radix selection needs several
    # passes) and swarms of 3000 particles (a 4096-entry sort in shared memory)
    rng = np.random.default_rng(8)
    n = 20
    F = np.triu(rng.integers(0, 100_000, (n, n)), 1)
    D = np.triu(rng.integers(0, 100_000, (n, n)), 1)
    F, D = (F + F.T).astype(np.int32), (D + D.T).astype(np.int32)
    prm = Q.default_params(swarms=3, swarm_size=3000, ls_max_moves=2)
    sw = Q.Swarm(Q.Instance(F, D), prm, seed=4)
    sw.trace_start(capacity=2, lo=0, hi=2**40, bins=1000)
    sw.step(2)
    recs = sw.trace_read()
    c = sw.export_state()["cost"]
    assert recs[-1]["t"] == 2
    _check_record(recs[-1], c, 3000, 0, 2**40, 1000)


def test_trace_rejects_bad_arguments(Q):
    inst = W.tiny9()
    sw = Q.Swarm(Q.Instance(inst.F, inst.D), Q.default_params(), seed=1)
    for bad in (dict(capacity=0, lo=0, hi=10, bins=3), dict(capacity=2, lo=5, hi=5, bins=3),
                dict(capacity=2, lo=0, hi=10, bins=0)):
        with pytest.raises(Q.QapError) as e:
            sw.trace_start(**bad)
        assert e.value.status == Q.ERR_INVALID_ARG
