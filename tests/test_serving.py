"""The serving loop: scheduling on the host with a fake executor (CPU), and
on the GPU the same result for every request alone and in the mix."""
import time

import numpy as np
import pytest

from paper_2308_01999_gb300 import inputs as gen
from paper_2308_01999_gb300 import serving


class FakeExecutor:
    """Sleeps instead of computing; keeps the state memory as a byte budget and
    records the memory in use at every start."""

    def __init__(self, budget, fail_rid=None):
        self.capacity = budget
        self.fail_rid = fail_rid
        self.held = 0
        self.live = 0
        self.max_live = 0
        self.batches = []
        self.concurrent_batches = 0
        self.max_concurrent_batches = 0
        self._blocks = {}

    def alloc(self, req):
        if self.held + req.state_bytes > self.capacity:
            return None
        self.held += req.state_bytes
        blk = object()
        self._blocks[id(blk)] = (blk, req.state_bytes)
        return blk

    def free(self, blk):
        _, nbytes = self._blocks.pop(id(blk))
        self.held -= nbytes

    def _work(self, reqs, dt):
        self.live += sum(r.state_bytes for r in reqs)
        self.max_live = max(self.max_live, self.live)
        time.sleep(dt)
        self.live -= sum(r.state_bytes for r in reqs)

    def run_large(self, req, blk):
        assert id(blk) in self._blocks
        if req.rid == self.fail_rid:
            raise RuntimeError("injected failure")
        self._work([req], 0.01)
        return np.full(req.n, float(req.rid))

    def run_batch(self, reqs, blks):
        assert all(id(b) in self._blocks for b in blks) and len(blks) == len(reqs)
        self.batches.append([r.rid for r in reqs])
        self.concurrent_batches += 1
        self.max_concurrent_batches = max(self.max_concurrent_batches, self.concurrent_batches)
        self._work(reqs, 0.02)
        self.concurrent_batches -= 1
        return [np.full(r.n, float(r.rid)) for r in reqs]


def _trace(count, rate, seed=4):
    return serving.make_requests(gen.serving_trace(count=count, rate=rate, nmin=12, nmax=30, seed=seed))


def test_scheduler_completes_everything_within_the_budget():
    reqs = _trace(60, 2000.0)
    budget = 20 << 30
    ex = FakeExecutor(budget)
    eng = serving.ServingEngine(ex, large_workers=3, batch_slots=2)
    out = eng.run(reqs)
    assert all(r.error is None and r.result is not None for r in out)
    assert all(np.all(r.result == r.rid) for r in out)          # results routed to their request
    assert eng.peak_bytes <= budget and ex.max_live <= budget
    assert ex.held == 0                                           # every block returned
    assert all(r.t_admit >= r.arrival - 1e-9 and r.t_done >= r.t_admit for r in out)
    # small requests that waited together went out in one batch
    assert any(len(b) > 1 for b in ex.batches)
    st = serving.latency_stats(out)
    assert st["completed"] == 60 and st["p99_s"] >= st["p50_s"]


def test_scheduler_reports_failures_and_oversized_requests():
    reqs = _trace(30, 1000.0)
    big = max(reqs, key=lambda r: r.n)
    ex = FakeExecutor((8 << big.n) + (1 << 20), fail_rid=big.rid)
    eng = serving.ServingEngine(ex, small_max_qubits=20, large_workers=2)
    out = eng.run(reqs)
    failed = [r for r in out if r.error is not None]
    assert big.rid in [r.rid for r in failed]
    assert all(r.result is not None for r in out if r.error is None)
    assert ex.held == 0
    tiny = serving.ServingEngine(FakeExecutor(1 << 20)).run(_trace(5, 100.0, seed=7))
    assert all(r.error == "state larger than the HBM budget" for r in tiny if r.state_bytes > (1 << 20))


def test_small_requests_start_in_a_free_batch_slot():
    """Small requests that arrive while a batch runs start in the second slot
    instead of waiting for the first batch to finish."""
    reqs = serving.make_requests([(0.0, 12, 5, 1), (0.002, 13, 5, 2), (0.004, 14, 5, 3), (0.006, 12, 5, 4)])
    ex = FakeExecutor(1 << 30)
    eng = serving.ServingEngine(ex, batch_slots=2)
    out = eng.run(reqs)
    assert all(r.error is None for r in out)
    assert ex.max_concurrent_batches == 2
    first = out[0]
    assert any(r.t_admit < first.t_done for r in out[1:])


def test_small_requests_pass_a_large_request_waiting_for_memory():
    reqs = serving.make_requests([(0.0, 24, 5, 1), (0.001, 24, 5, 2), (0.002, 12, 5, 3)])
    ex = FakeExecutor((8 << 24) + (8 << 12))
    out = serving.ServingEngine(ex, small_max_qubits=20).run(reqs)
    assert all(r.error is None for r in out)
    assert out[2].t_admit < out[1].t_admit          # the small one did not wait behind the second large one


def test_medium_requests_go_to_batches_of_their_own():
    reqs = serving.make_requests([(0.0, 12, 5, 1), (0.0, 22, 5, 2), (0.001, 13, 5, 3), (0.001, 24, 5, 4),
                                  (0.002, 28, 5, 5)])
    ex = FakeExecutor(1 << 34)
    out = serving.ServingEngine(ex, small_max_qubits=20, batch_max_qubits=26).run(reqs)
    assert all(r.error is None for r in out)
    by_rid = {r.rid: r.n for r in out}
    for b in ex.batches:
        sizes = [by_rid[i] for i in b]
        assert all(n <= 20 for n in sizes) or all(20 < n <= 26 for n in sizes), sizes
    assert any(all(by_rid[i] > 20 for i in b) for b in ex.batches)
    assert all(by_rid[i] <= 26 for b in ex.batches for i in b)       # the 28-qubit one ran alone


def test_serial_engine_orders_and_waits():
    reqs = _trace(8, 400.0)
    out = serving.serial_engine(lambda r: np.zeros(r.n), reqs)
    for a, b in zip(out, out[1:]):
        assert b.t_admit >= a.t_done - 1e-9 and b.t_admit >= b.arrival - 1e-9


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    """Every request of a mixed trace (small states batched in shared memory,
    medium ones batched and split over the GPU, concurrent large ones) gives the
    same <Z_q> alone and in the mix, and matches the complex128 oracle, for
    every request size in the trace (12-22 qubits)."""
    import torch
    from oracle import oracle as orc
    orc.set_threads(0)
    ex = serving.GpuExecutor(hbm_budget=8 << 30, fusion_width=4, batch_widths=(2, 4), plain_max_qubits=22)
    trace = gen.serving_trace(count=14, rate=500.0, nmin=12, nmax=22, dmin=3, dmax=8, seed=11)
    mix = serving.ServingEngine(ex, small_max_qubits=14, batch_max_qubits=18, large_workers=3,
                                batch_slots=2).run(serving.make_requests(trace))
    assert all(r.error is None for r in mix)
    assert ex.bytes_in_use() == 0
    for r in mix:
        alone = serving.ServingEngine(ex, small_max_qubits=14, batch_max_qubits=18, large_workers=3).run(
            [serving.Request(r.rid, 0.0, r.n, r.depth, r.seed)])[0]
        assert alone.error is None
        assert np.max(np.abs(alone.result - r.result)) <= 1e-6, r.rid
        ref = orc.expect_z_all(orc.run_circuit(r.gates(), r.n))
        assert np.max(np.abs(r.result - ref)) <= 1e-6, (r.rid, r.n)
        plain = ex.run_plain(r)
        assert np.max(np.abs(plain - ref)) <= 1e-6, (r.rid, r.n)
    torch.cuda.synchronize()
    ex.close()
