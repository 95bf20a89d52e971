"""The serving loop: scheduling on the host with a fake executor (CPU), and
on the GPU the same result for every request alone and in the mix."""
import time

import numpy as np
import pytest

from paper_2308_01999_gb300 import inputs as gen
from paper_2308_01999_gb300 import serving


class FakeExecutor:
    """Sleeps instead of computing; records the memory in use at every start."""

    def __init__(self, fail_rid=None):
        self.fail_rid = fail_rid
        self.live = 0
        self.max_live = 0
        self.batches = []

    def alloc(self, req):
        return None

    def _work(self, reqs, dt):
        self.live += sum(r.state_bytes for r in reqs)
        self.max_live = max(self.max_live, self.live)
        time.sleep(dt)
        self.live -= sum(r.state_bytes for r in reqs)

    def run_large(self, req, state):
        if req.rid == self.fail_rid:
            raise RuntimeError("injected failure")
        self._work([req], 0.01)
        return np.full(req.n, float(req.rid))

    def run_batch(self, reqs, states):
        self.batches.append([r.rid for r in reqs])
        self._work(reqs, 0.005)
        return [np.full(r.n, float(r.rid)) for r in reqs]


def _trace(count, rate, seed=4):
    return serving.make_requests(gen.serving_trace(count=count, rate=rate, nmin=12, nmax=30, seed=seed))


def test_scheduler_completes_everything_within_the_budget():
    reqs = _trace(60, 2000.0)
    budget = 20 << 30
    ex = FakeExecutor()
    eng = serving.ServingEngine(ex, hbm_budget=budget, large_workers=3)
    out = eng.run(reqs)
    assert all(r.error is None and r.result is not None for r in out)
    assert all(np.all(r.result == r.rid) for r in out)          # results routed to their request
    assert eng.peak_bytes <= budget and ex.max_live <= budget
    assert all(r.t_admit >= r.arrival - 1e-9 and r.t_done >= r.t_admit for r in out)
    # small requests that waited together went out in one batch
    assert any(len(b) > 1 for b in ex.batches)
    st = serving.latency_stats(out)
    assert st["completed"] == 60 and st["p99_s"] >= st["p50_s"]


def test_scheduler_reports_failures_and_oversized_requests():
    reqs = _trace(30, 1000.0)
    big = max(reqs, key=lambda r: r.n)
    ex = FakeExecutor(fail_rid=big.rid)
    eng = serving.ServingEngine(ex, hbm_budget=(8 << big.n) + (1 << 20), small_max_qubits=20, large_workers=2)
    out = eng.run(reqs)
    failed = [r for r in out if r.error is not None]
    assert big.rid in [r.rid for r in failed]
    assert all(r.result is not None for r in out if r.error is None)
    tiny = serving.ServingEngine(FakeExecutor(), hbm_budget=1 << 20).run(_trace(5, 100.0, seed=7))
    assert all(r.error == "state larger than the HBM budget" for r in tiny if r.state_bytes > (1 << 20))


def test_serial_engine_orders_and_waits():
    reqs = _trace(8, 400.0)
    out = serving.serial_engine(lambda r: np.zeros(r.n), reqs)
    for a, b in zip(out, out[1:]):
        assert b.t_admit >= a.t_done - 1e-9 and b.t_admit >= b.arrival - 1e-9


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    import torch
    from oracle import oracle as orc
    ex = serving.GpuExecutor(fusion_width=4)
    trace = gen.serving_trace(count=14, rate=500.0, nmin=12, nmax=22, dmin=3, dmax=8, seed=11)
    mix = serving.ServingEngine(ex, hbm_budget=8 << 30, small_max_qubits=16, large_workers=3).run(
        serving.make_requests(trace))
    assert all(r.error is None for r in mix)
    for r in mix:
        alone = serving.ServingEngine(ex, hbm_budget=8 << 30, small_max_qubits=16, large_workers=3).run(
            [serving.Request(r.rid, 0.0, r.n, r.depth, r.seed)])[0]
        assert alone.error is None
        assert np.max(np.abs(alone.result - r.result)) <= 1e-6, r.rid
        if r.n <= 16:
            ref = orc.expect_z_all(orc.run_circuit(r.gates(), r.n))
            assert np.max(np.abs(r.result - ref)) <= 1e-6
    torch.cuda.synchronize()
