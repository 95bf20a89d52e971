"""Autotuner of the batched engine's compile options.

The batched engine (``sv.Batch``) has four knobs that trade host-side fusion
against on-chip work: the gate-fusion width (blocks of 1-4 qubits, Sec. II-B),
the register-window width (runs of small ops applied to 2^w amplitudes held in
registers, 0 = off), the keep-permutations fusion rule (blocks of CNOTs and
other permutations take no dense gate, so they stay register exchanges) and
the tile size (local qubits of a pass over a state held in shared memory).
Which combination is fastest depends on the workload's
qubit counts and circuit depth, so the tuner measures it: it compiles a
stratified sample of the batch (every k-th state in order of qubit count, so
the sample keeps the workload's size mix) with each candidate, times one
launch of each on the device, keeps the fastest, and caches the choice under
a coarse workload signature (qubit range and gates per qubit), so batches of
the same kind of work reuse it without timing again.

The timer is pluggable: ``gpu_timer`` runs the real kernel; tests pass a fake.
"""
from __future__ import annotations

import math
import threading
from typing import Callable, Dict, Optional, Sequence, Tuple

import numpy as np

__all__ = ["CANDIDATES", "signature", "stratified_sample", "BatchTuner", "gpu_timer", "default_tuner"]

# (fusion width, window width, keep permutations, tile qubits)
CANDIDATES: Tuple[Tuple[int, int, int, int], ...] = (
    (1, 4, 0, 14), (2, 4, 0, 14), (2, 4, 1, 14), (3, 4, 0, 14), (3, 4, 1, 14), (4, 4, 0, 14),
    (1, 3, 0, 14), (2, 3, 0, 14), (2, 3, 1, 14), (1, 0, 0, 14), (2, 0, 0, 14), (2, 4, 0, 13), (2, 3, 0, 12))


def signature(ns: Sequence[int], gate_counts: Sequence[int]) -> tuple:
    """Coarse key of a batch: smallest and largest qubit count and the rounded
    log2 of the mean number of gates per qubit."""
    if not ns:
        return (0, 0, 0)
    gpq = float(np.mean([g / max(1, n) for n, g in zip(ns, gate_counts)]))
    return (int(min(ns)), int(max(ns)), int(round(math.log2(max(gpq, 1.0)))))


def stratified_sample(ns: Sequence[int], k: int) -> list:
    """Indices of about k states, every (len / k)-th in order of qubit count
    (ties in input order), so that the sample keeps the size distribution."""
    m = len(ns)
    if k >= m:
        return list(range(m))
    order = sorted(range(m), key=lambda i: (ns[i], i))
    step = m / k
    return sorted(order[int(j * step)] for j in range(k))


class BatchTuner:
    """Chooses (fusion width, window width, keep permutations, tile qubits) for
    a batch by timing candidates.

    timer(packed_sample, fusion_width, window_qubits, keep_permutations,
    tile_qubits) -> seconds (or any monotone cost). ``choose`` returns the
    cached choice for the batch's signature, timing the candidates on a
    stratified sample the first time."""

    def __init__(self, timer: Callable, candidates: Sequence[Tuple[int, int, int, int]] = CANDIDATES,
                 sample: int = 1024):
        self.timer = timer
        self.candidates = tuple(candidates)
        self.sample = int(sample)
        self.cache: Dict[tuple, Tuple[int, int, int, int]] = {}
        self.timings: Dict[tuple, Dict[Tuple[int, int, int, int], float]] = {}
        self._lock = threading.Lock()

    def choose(self, packed) -> Tuple[int, int, int, int]:
        from . import sv
        sig = signature(packed.ns, packed.gate_counts)
        with self._lock:
            if sig in self.cache:
                return self.cache[sig]
        idx = stratified_sample(packed.ns, self.sample)
        sub = _subset(packed, idx)
        times = {}
        for cand in self.candidates:
            try:
                times[cand] = float(self.timer(sub, *cand))
            except sv.SvError:
                continue          # an option the compiler rejects for this work
        if not times:
            raise RuntimeError("no autotuner candidate compiled")
        best = min(times, key=lambda c: (times[c], self.candidates.index(c)))
        with self._lock:
            self.cache[sig] = best
            self.timings[sig] = times
        return best


def _subset(packed, idx):
    """The states `idx` of a PackedBatch, laid out back to back. Their gate
    records are copied as they are: the matrix pointers still point into the
    original batch's matrix buffer, which the subset keeps alive."""
    from . import sv
    items = np.zeros(len(idx), dtype=sv.ITEM_DTYPE)
    recs, pls, ns, counts = [], [], [], []
    g0 = p0 = o0 = a0 = 0
    for j, i in enumerate(idx):
        it = packed.items[i]
        n, gb, ng = int(it["n_qubits"]), int(it["gate_begin"]), int(it["n_gates"])
        pb, nstr = int(it["pauli_begin"]), int(it["n_strings"])
        items[j] = (n, g0, ng, p0, nstr, o0, a0)
        recs.append(packed.gate_rec[gb:gb + ng])
        pls.append(packed.paulis[pb:pb + nstr * n])
        ns.append(n)
        counts.append(ng)
        g0 += ng
        p0 += nstr * n
        o0 += nstr
        a0 += 1 << n
    rec = np.concatenate(recs) if recs else np.zeros(0, dtype=sv.GATE_DTYPE)
    pl = np.concatenate(pls) if pls else np.zeros(0, np.int32)
    return sv.PackedBatch(items, rec, packed.matrices, pl, o0, a0, ns, counts)


def gpu_timer(stream=None, reps: int = 2) -> Callable:
    """Timer that compiles the sample, launches it once to warm up and then
    `reps` times between CUDA events on `stream`; returns seconds per launch."""
    import torch

    from . import sv
    state = {"buf": None}

    def timer(packed, fusion_width, window_qubits, keep_permutations=0, tile_qubits=sv.SV_BATCH_TILE_QUBITS):
        st = stream or torch.cuda.current_stream()
        b = sv.Batch(st)
        try:
            b.compile(packed, fusion_width, window_qubits, bool(keep_permutations), tile_qubits)
            buf = state["buf"]
            if buf is None or buf.numel() < b.state_amps:
                buf = state["buf"] = torch.empty(max(1, b.state_amps), dtype=torch.complex64, device="cuda")
            b.launch(buf)
            b.results()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                b.launch(buf)
            e1.record(st)
            b.results()
            return e0.elapsed_time(e1) / reps / 1e3
        finally:
            b.close()

    return timer


_default: Optional[BatchTuner] = None
_default_lock = threading.Lock()


def default_tuner(stream=None) -> BatchTuner:
    """The process-wide tuner with a GPU timer (its cache is shared)."""
    global _default
    with _default_lock:
        if _default is None:
            _default = BatchTuner(gpu_timer(stream))
        return _default
