"""Continuous-batching serving loop for state-vector circuits.

Requests (random circuits of 12-30 qubits) arrive over time. Each is admitted
when its state vector (2^n x 8 bytes, complex64) finds a block in the HBM
arena, keeps that block -- its state stays resident on the device -- until it
finishes, and returns <Z_q> for every qubit (FP64). Admitted work overlaps on
the GPU:

* small requests (n <= small_max_qubits) are gathered into batches: one
  persistent launch of the batched engine (``sv.Batch``) advances all the
  states of a batch, their gate layers applied together. Up to
  ``batch_slots`` batches are in flight at once, so requests that arrive
  while a batch runs start in the next free slot instead of waiting for that
  batch to drain;
* medium requests (up to batch_max_qubits, at most 26) go to batches of their
  own: the batched engine splits each of their passes over all CTAs, so
  resident states of 21-26 qubits also advance together, layer by layer, in
  one launch;
* every large request runs on a worker's CUDA stream as one fused call
  (``sv_apply_fused``, native precision) followed by its expectation values;
  several large requests run concurrently on different streams.

Nothing is allocated per request: the executor allocates one arena of device
memory once and places states in it with the library's buddy pool
(``sv_pool_*``, so admission asks exactly whether a state fits, fragmentation
included); each call borrows a pooled resource set -- a stream, a handle
rebound to the request's state with ``sv_set_state``, and a batched engine
whose device program buffer is reused. A request's result does not depend on what else is in the
mix: the batched kernel gives every state its own CTA and fixed-order
reductions, and a large request's kernels touch only its own state.

The scheduler is host code; every computation runs in libsv.so. The executor
is pluggable so that the scheduling logic can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import contextlib
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
    """Runs requests on the GPU through libsv.so without allocating per request.

    hbm_budget bytes of device memory are allocated once as the state arena
    (a block of 2^n complex64 amplitudes per admitted request, placed by the
    native buddy pool). Each call borrows a worker resource set -- a CUDA
    stream, a handle and a batched engine -- from a free list; sets are created
    only when more calls run at once than ever before, and reused afterwards. The
    plain engines (``run_plain``, ``run_fused_serial``: one request at a time)
    use one preallocated buffer of the largest state instead of the arena.
    The batched engine's fusion and window widths come from the autotuner
    (``autotune.BatchTuner``) unless given."""

    MIN_BLOCK = 1 << 12

    def __init__(self, hbm_budget: int, device: int = 0, fusion_width: int = 4, batch_widths=None,
                 tuner=None, plain_max_qubits: int = 30):
        import torch

        from . import sv
        self.torch, self.sv = torch, sv
        self.device = torch.device("cuda", device)
        self.fusion_width = fusion_width
        self.batch_widths = batch_widths
        self.tuner = tuner
        self.arena = torch.empty(int(hbm_budget), dtype=torch.uint8, device=self.device)
        self.base = self.arena.data_ptr()
        self.pool = sv.StatePool(self.base, int(hbm_budget), self.MIN_BLOCK)
        self.capacity = self.pool.stats()["capacity"]
        self.plain_max_qubits = plain_max_qubits
        self._plain_buf = None
        self._workers = []
        self._free = []
        self._lock = threading.Lock()

    # ---- state memory ----
    def alloc(self, req: Request):
        """Device address of a block for the request's state, or None if none fits now."""
        return self.pool.alloc(req.state_bytes)

    def free(self, ptr):
        if ptr is not None:
            self.pool.free(ptr)

    def bytes_in_use(self) -> int:
        return self.pool.stats()["in_use"]

    # ---- worker resources: a stream, a handle and a batched engine ----
    @contextlib.contextmanager
    def _worker(self):
        """Borrow a resource set from the free list (created on first need; at
        most as many exist as calls ever ran at once) and return it afterwards."""
        with self._lock:
            w = self._free.pop() if self._free else None
        if w is None:
            torch, sv = self.torch, self.sv
            with torch.cuda.device(self.device):
                stream = torch.cuda.Stream(self.device)
                h = sv.sv_create(1, sv.SV_C64, self.base, stream.cuda_stream)
                w = {"stream": stream, "handle": h, "batch": sv.Batch(stream)}
            with self._lock:
                self._workers.append(w)
        try:
            yield w
        finally:
            with self._lock:
                self._free.append(w)

    def _z_all(self, h, n):
        return self.sv.sv_expectation_pauli(h, np.full((n, 1), 3, np.int32), np.arange(n, dtype=np.int32)[:, None])

    def run_large(self, req: Request, ptr) -> np.ndarray:
        """One fused call on the request's state in the arena, then <Z_q> for all q."""
        torch, sv = self.torch, self.sv
        with self._worker() as w, torch.cuda.device(self.device), torch.cuda.stream(w["stream"]):
            h = w["handle"]
            sv.sv_set_state(h, req.n, sv.SV_C64, ptr)
            sv.sv_set_basis_state(h, 0)
            sv.sv_apply_fused(h, req.gates(), self.fusion_width, sv.SV_PREC_NATIVE)
            return self._z_all(h, req.n)

    def run_batch(self, reqs, ptrs) -> list:
        """One persistent launch over the requests' states, each at its arena block."""
        torch, sv = self.torch, self.sv
        with self._worker() as w, torch.cuda.device(self.device), torch.cuda.stream(w["stream"]):
            items = [(r.n, r.gates(), 3 * np.eye(r.n, dtype=np.int32)) for r in reqs]   # row q: Z on qubit q
            offsets = [(p - self.base) // 8 for p in ptrs]
            b = w["batch"]
            if self.batch_widths is not None:
                b.compile(items, *self.batch_widths, state_offsets=offsets)
            else:
                b.compile(items, state_offsets=offsets, tuner=self.tuner, autotune=self.tuner is None)
            b.launch(self.base)
            return [np.asarray(v).copy() for v in b.results()]

    def _plain_state(self, req: Request):
        if req.n > self.plain_max_qubits:
            raise ValueError("request larger than the plain engine's buffer")
        if self._plain_buf is None:
            self._plain_buf = self.torch.empty(8 << self.plain_max_qubits, dtype=self.torch.uint8,
                                               device=self.device)
        return self._plain_buf.data_ptr()

    def run_plain(self, req: Request) -> np.ndarray:
        """The plain engine: one request at a time, one launch per gate (unfused)."""
        torch, sv = self.torch, self.sv
        with self._worker() as w, torch.cuda.device(self.device), torch.cuda.stream(w["stream"]):
            h = w["handle"]
            sv.sv_set_state(h, req.n, sv.SV_C64, self._plain_state(req))
            sv.sv_set_basis_state(h, 0)
            for g in req.gates():
                sv.sv_apply_matrix(h, g.targets, g.matrix, g.controls, g.control_values or None)
            return self._z_all(h, req.n)

    def run_fused_serial(self, req: Request) -> np.ndarray:
        """One request at a time with the same fusion as run_large: separates the
        gain of fusion from the gain of batching and overlap."""
        torch, sv = self.torch, self.sv
        with self._worker() as w, torch.cuda.device(self.device), torch.cuda.stream(w["stream"]):
            h = w["handle"]
            sv.sv_set_state(h, req.n, sv.SV_C64, self._plain_state(req))
            sv.sv_set_basis_state(h, 0)
            sv.sv_apply_fused(h, req.gates(), self.fusion_width, sv.SV_PREC_NATIVE)
            return self._z_all(h, req.n)

    def close(self):
        self.torch.cuda.synchronize(self.device)
        with self._lock:
            for w in self._workers:
                w["batch"].close()
                self.sv.sv_destroy(w["handle"])
            self._workers.clear()
        self.pool.close()


class ServingEngine:
    """Admission into the executor's state memory, continuous batching, one
    stream per large request. Requests of at most ``small_max_qubits`` qubits
    go to small batches; with ``batch_max_qubits`` above that, requests up to
    it go to separate medium batches (their states are split over the whole
    GPU inside the batched launch, so their gate layers run together with the
    other states'), and only larger ones run as single fused calls. Each batch
    class has ``batch_slots`` batches in flight at most; a free slot takes every
    request of its class admitted so far. ``run(requests)`` replays arrival
    times in real time and returns the requests with t_admit / t_done / result
    filled in."""

    def __init__(self, executor, small_max_qubits: int = 20, large_workers: int = 4, batch_slots: int = 2,
                 batch_max_qubits: Optional[int] = None,
                 clock: Callable[[], float] = time.perf_counter, poll_s: float = 0.0005):
        self.ex = executor
        self.small_max = small_max_qubits
        self.batch_max = max(small_max_qubits, batch_max_qubits or small_max_qubits)
        self.workers = large_workers
        self.batch_slots = batch_slots
        self.clock = clock
        self.poll = poll_s
        self.peak_bytes = 0
        self.occupancy = []          # (t, bytes of admitted states) samples
        self.batch_sizes = []

    def _cls(self, r) -> int:
        """0: small batch, 1: medium batch, 2: large (single fused call)."""
        return 0 if r.n <= self.small_max else (1 if r.n <= self.batch_max else 2)

    def run(self, requests) -> list:
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = collections.deque(reqs)
        waiting = collections.deque()
        used = 0
        queued = ([], [])            # admitted requests of each batch class not yet in a batch: (request, block)
        inflight = {}                # future -> (kind, [requests], [blocks], bytes)
        pool = cf.ThreadPoolExecutor(max_workers=self.workers + 2 * self.batch_slots)
        batches = [0, 0]
        large_busy = 0
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        cap = self.ex.capacity
        try:
            while pending or waiting or queued[0] or queued[1] or inflight:
                t = now()
                while pending and pending[0].arrival <= t:
                    waiting.append(pending.popleft())
                # admission in arrival order while blocks are found; batched requests
                # may pass a large one that waits for memory or a worker
                blocked_large = False
                for r in list(waiting):
                    c = self._cls(r)
                    if r.state_bytes > cap:
                        waiting.remove(r)
                        r.error = "state larger than the HBM budget"
                        r.t_done = now()
                        continue
                    if blocked_large and c == 2:
                        continue
                    if c == 2 and large_busy >= self.workers:
                        blocked_large = True
                        continue
                    blk = self.ex.alloc(r)
                    if blk is None:
                        if c < 2:
                            break
                        blocked_large = True
                        continue
                    waiting.remove(r)
                    used += r.state_bytes
                    r.t_admit = now()
                    if c < 2:
                        queued[c].append((r, blk))
                    else:
                        fut = pool.submit(self.ex.run_large, r, blk)
                        inflight[fut] = ("large", [r], [blk], r.state_bytes)
                        large_busy += 1
                self.peak_bytes = max(self.peak_bytes, used)
                self.occupancy.append((now(), used))
                # a free batch slot of a class takes every request of that class admitted so far
                for c in (0, 1):
                    if queued[c] and batches[c] < self.batch_slots:
                        rs = [r for r, _ in queued[c]]
                        blks = [b for _, b in queued[c]]
                        queued[c].clear()
                        fut = pool.submit(self.ex.run_batch, rs, blks)
                        inflight[fut] = (c, rs, blks, sum(r.state_bytes for r in rs))
                        self.batch_sizes.append(len(rs))
                        batches[c] += 1
                done = [f for f in inflight if f.done()]
                for f in done:
                    kind, rs, blks, nbytes = inflight.pop(f)
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
                    for b in blks:
                        self.ex.free(b)
                    used -= nbytes
                    if kind == "large":
                        large_busy -= 1
                    else:
                        batches[kind] -= 1
                if not done:
                    if pending and not inflight and not waiting and not queued[0] and not queued[1]:
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
