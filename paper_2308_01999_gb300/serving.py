"""Continuous-batching serving loop for state-vector circuits.

Requests (random circuits of 12-30 qubits) arrive over time. Each is admitted
when its state vector (2^n x 8 bytes, complex64) fits in the free HBM budget,
keeps that state resident on the device until it finishes, and returns <Z_q>
for every qubit (FP64). Admitted work overlaps on the GPU:

* small requests (n <= small_max_qubits) that are admitted while the previous
  batch runs are gathered into the next batch: one persistent launch of the
  batched engine (``sv.Batch``) advances all of them;
* every large request runs on its own CUDA stream (a pool of worker threads,
  one stream each) as one fused call (``sv_apply_fused``, native precision)
  followed by its expectation values.

So requests that arrive while others are on the GPU are admitted as memory
and workers free up, and their kernels run concurrently with the ones already
in flight. A request's result does not depend on what else is in the mix: the
batched kernel gives every state its own CTA and fixed-order reductions, and a
large request's kernels touch only its own state.

The scheduler is host code; every computation runs in libsv.so. The executor
is pluggable so that the scheduling logic can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Callable, Optional

import numpy as np

from . import inputs as gen

__all__ = ["Request", "ServingEngine", "GpuExecutor", "serial_engine", "latency_stats", "make_requests"]


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the trace
    n: int
    depth: int
    seed: int
    t_admit: float = float("nan")
    t_done: float = float("nan")
    result: Optional[np.ndarray] = None
    error: Optional[str] = None

    @property
    def state_bytes(self) -> int:
        return 8 << self.n

    def gates(self):
        return gen.circuit_config1(self.n, self.depth, self.seed)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def make_requests(trace) -> list:
    """Requests from ``inputs.serving_trace`` tuples (arrival, n, depth, seed)."""
    return [Request(i, a, n, d, s) for i, (a, n, d, s) in enumerate(trace)]


def latency_stats(reqs) -> dict:
    done = [r for r in reqs if r.error is None and r.t_done == r.t_done]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    span = max(r.t_done for r in done) - min(r.arrival for r in reqs) if done else float("nan")
    return {"completed": len(done), "failed": sum(r.error is not None for r in reqs),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "circuits_per_s": len(done) / span if span > 0 else float("nan"),
            "makespan_s": span}


class GpuExecutor:
    """Runs requests on the GPU through libsv.so."""

    def __init__(self, device: int = 0, fusion_width: int = 4, batch_width: int = 2):
        import torch

        from . import sv
        self.torch, self.sv = torch, sv
        self.device = torch.device("cuda", device)
        self.fusion_width = fusion_width
        self.batch_width = batch_width
        self._local = threading.local()

    def _stream(self):
        s = getattr(self._local, "stream", None)
        if s is None:
            s = self.torch.cuda.Stream(self.device)
            self._local.stream = s
        return s

    def alloc(self, req: Request):
        return self.torch.empty(1 << req.n, dtype=self.torch.complex64, device=self.device)

    def run_large(self, req: Request, state) -> np.ndarray:
        torch, sv = self.torch, self.sv
        stream = self._stream()
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            s = sv.StateVector(state, stream)
            try:
                s.set_basis_state(0)
                s.apply_fused(req.gates(), self.fusion_width, sv.SV_PREC_NATIVE)
                return s.expectation_z_all()
            finally:
                s.close()

    def run_plain(self, req: Request) -> np.ndarray:
        """The plain engine: one launch per gate, unfused, then the expectations."""
        torch, sv = self.torch, self.sv
        stream = self._stream()
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            state = self.alloc(req)
            s = sv.StateVector(state, stream)
            try:
                s.set_basis_state(0)
                s.apply_circuit(req.gates())
                return s.expectation_z_all()
            finally:
                s.close()

    def run_batch(self, reqs, states) -> list:
        torch, sv = self.torch, self.sv
        stream = self._stream()
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            items = [(r.n, r.gates(), 3 * np.eye(r.n, dtype=np.int32)) for r in reqs]   # row q: Z on qubit q
            b = sv.Batch(stream)
            try:
                b.compile(items, fusion_width=self.batch_width)
                total = sum(1 << r.n for r in reqs)
                buf = states if states is not None and states.numel() >= total else \
                    torch.empty(total, dtype=torch.complex64, device=self.device)
                b.launch(buf)
                return [np.asarray(v) for v in b.results()]
            finally:
                b.close()


class ServingEngine:
    """Admission by free memory, continuous batching of small requests, one
    stream per large request. ``run(requests)`` replays arrival times in real
    time and returns the requests with t_admit / t_done / result filled in."""

    def __init__(self, executor, hbm_budget: int, small_max_qubits: int = 20, large_workers: int = 4,
                 clock: Callable[[], float] = time.perf_counter, poll_s: float = 0.0005):
        self.ex = executor
        self.budget = int(hbm_budget)
        self.small_max = small_max_qubits
        self.workers = large_workers
        self.clock = clock
        self.poll = poll_s
        self.peak_bytes = 0
        self.occupancy = []          # (t, bytes in use) samples

    def run(self, requests) -> list:
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = collections.deque(reqs)
        waiting = collections.deque()
        used = 0
        small_q = []
        inflight = {}                # future -> (kind, [requests], bytes)
        pool = cf.ThreadPoolExecutor(max_workers=self.workers + 1)
        batch_busy = False
        large_busy = 0
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        try:
            while pending or waiting or small_q or inflight:
                t = now()
                while pending and pending[0].arrival <= t:
                    waiting.append(pending.popleft())
                # admission in arrival order, while the state fits the budget
                while waiting:
                    r = waiting[0]
                    if r.state_bytes > self.budget:
                        waiting.popleft()
                        r.error = "state larger than the HBM budget"
                        r.t_done = now()
                        continue
                    if used + r.state_bytes > self.budget:
                        break
                    if r.n > self.small_max and large_busy >= self.workers:
                        break
                    waiting.popleft()
                    used += r.state_bytes
                    r.t_admit = now()
                    if r.n <= self.small_max:
                        small_q.append(r)
                    else:
                        st = self.ex.alloc(r)
                        fut = pool.submit(self.ex.run_large, r, st)
                        inflight[fut] = ("large", [r], r.state_bytes, st)
                        large_busy += 1
                self.peak_bytes = max(self.peak_bytes, used)
                self.occupancy.append((now(), used))
                # the next batch takes every small request admitted so far
                if small_q and not batch_busy:
                    batch = small_q
                    small_q = []
                    fut = pool.submit(self.ex.run_batch, batch, None)
                    inflight[fut] = ("batch", batch, sum(r.state_bytes for r in batch), None)
                    batch_busy = True
                done = [f for f in inflight if f.done()]
                for f in done:
                    kind, rs, nbytes, _st = inflight.pop(f)
                    tdone = now()
                    try:
                        res = f.result()
                        if kind == "large":
                            rs[0].result = res
                        else:
                            for r, v in zip(rs, res):
                                r.result = v
                    except Exception as e:  # a failed request is reported, the others go on
                        for r in rs:
                            r.error = f"{type(e).__name__}: {e}"
                    for r in rs:
                        r.t_done = tdone
                    used -= nbytes
                    if kind == "batch":
                        batch_busy = False
                    else:
                        large_busy -= 1
                if not done:
                    if pending and not inflight and not waiting and not small_q:
                        time.sleep(max(0.0, min(pending[0].arrival - now(), 0.01)))
                    else:
                        time.sleep(self.poll)
        finally:
            pool.shutdown(wait=True)
        return reqs


def serial_engine(executor_run_one, requests, clock=time.perf_counter) -> list:
    """One request at a time in arrival order (the plain engine): waits for each
    arrival, runs it to completion, then takes the next."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    for r in reqs:
        wait = r.arrival - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        r.t_admit = clock() - t0
        try:
            r.result = executor_run_one(r)
        except Exception as e:
            r.error = f"{type(e).__name__}: {e}"
        r.t_done = clock() - t0
    return reqs
