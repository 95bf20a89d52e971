"""Benchmark: unfused gate application on a 28-qubit complex64 state.

Workload (the paper's headline measurement is utilised HBM bandwidth of gate
application, Sec. II-B): a 28-qubit random circuit of depth 40 -- per layer a
Haar SU(2) on every qubit, then CZ / CNOT / CRZ on 14 random disjoint pairs --
applied one gate per launch to a 2 GiB complex64 state resident in HBM, then
<Z_q> for every qubit, 8 random Pauli strings and one parity measurement.
One step = that whole pass (1680 gate launches + the reductions).

value = algorithmic bytes moved per step / step time (GB/s): a dense one-qubit
gate reads and writes every amplitude (16 B per amplitude); CNOT and CRZ touch
the half where the control is 1; CZ the quarter where both bits are 1; each
reduction pass reads the state once. The state (2 GiB) is larger than L2
(129 MB), so no flush is needed between iterations.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the path does not shard:
one state per GPU); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2308_01999_gb300 import inputs as gen  # noqa: E402

N_QUBITS = 28
DEPTH = 40
AMP_BYTES = 8
METRIC = "gate-apply HBM GB/s (28-qubit complex64 random circuit, unfused, one gate per launch)"
UNIT = "GB/s"
def workload_name():
    return (f"{N_QUBITS}-qubit random circuit, complex64 state ({(8 << N_QUBITS) / 2**30:g} GiB) resident in HBM, "
            f"depth 40: Haar SU(2) on all qubits + CZ/CNOT/CRZ on {N_QUBITS // 2} random disjoint pairs per layer, "
            f"one gate per launch, then <Z_q> for all {N_QUBITS} qubits, 8 random Pauli strings and a 2-qubit "
            "parity measurement")
FRACTION = {"su2": 1.0, "cnot": 0.5, "crz": 0.5, "cz": 0.25}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload():
    gates = gen.circuit_config1(N_QUBITS, DEPTH, seed=1)
    paulis, sites = gen.random_pauli_strings(N_QUBITS, 8, gen.rng_for(101))
    return gates, paulis, sites


def gate_bytes(g):
    return FRACTION[g.name] * 2 * AMP_BYTES * (1 << N_QUBITS)


def reduction_passes(paulis):
    """Passes over the state: <Z_q> (x = 0, 8 strings per pass), the Pauli strings
    grouped by their X/Y mask (8 per pass), and one parity pass."""
    zpasses = (N_QUBITS + 7) // 8
    xs = {}
    for p in paulis:
        x = 0
        for q, c in enumerate(p):
            if c in (1, 2):
                x |= 1 << q
        xs[x] = xs.get(x, 0) + 1
    return zpasses + sum((c + 7) // 8 for c in xs.values()) + 1


def step_bytes(gates, paulis):
    return sum(gate_bytes(g) for g in gates) + reduction_passes(paulis) * AMP_BYTES * (1 << N_QUBITS)


class Clocks:
    """nvidia-smi sampling during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.dev = device_id
        self.proc = None
        self.path = os.path.join("/tmp", f"sv_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        load = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id(torch, dev) -> str:
    """nvidia-smi's name for the device (its UUID, independent of CUDA_VISIBLE_DEVICES)."""
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return "0"


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(vals, device=None):
    """Element-wise maximum of `vals` over all ranks (identity without a process
    group); the step time of a replica job is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_throughput(bytes_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job GB/s of `world` independent replicas, timed by the slowest rank."""
    return world * bytes_per_rank / (max_ms * 1e-3) / 1e9


def cpu_baseline(gates, budget_s: float = 12.0):
    """The CPU oracle (complex128, OpenMP) on the first gates of the same circuit
    at the same size, until `budget_s` of CPU work; value in the metric's unit
    (the complex64 workload's algorithmic bytes for those gates / time)."""
    from oracle import oracle as orc
    cores = orc.set_threads(0)
    psi = orc.zero_state(N_QUBITS)
    done, moved = 0, 0.0
    t0 = time.perf_counter()
    while done < len(gates) and (done < 3 or time.perf_counter() - t0 < budget_s):
        orc.apply(psi, gates[done])
        moved += gate_bytes(gates[done])
        done += 1
    dt = time.perf_counter() - t0
    return {"value": moved / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} of {len(gates)} gates of the same 28-qubit circuit, complex128 oracle "
                      f"({cores} OpenMP threads), {dt:.1f} s; GB/s counts the complex64 workload's bytes"}


def line_config(world: int, n_gates: int, nbytes: float) -> dict:
    """The workload's `config` object, the same on both arms of the bench."""
    return {"workload": workload_name(), "n_qubits": N_QUBITS, "depth": DEPTH, "gates_per_step": n_gates,
            "state_bytes": AMP_BYTES << N_QUBITS, "bytes_per_step": nbytes,
            "l2": f"no flush: the {(8 << N_QUBITS) / 2**30:g} GiB state exceeds the 129 MB L2",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle as it stands, timed on the host cores on the same workload,
    each step a bounded sample (a fixed slice of the circuit's gates)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import oracle as orc
    gates, paulis, _ = workload()
    config = line_config(world, len(gates), step_bytes(gates, paulis))
    cores = orc.set_threads(0)
    psi = orc.zero_state(N_QUBITS)
    per_step = 4
    pos = 0

    def one_step():
        nonlocal pos
        moved = 0.0
        for _ in range(per_step):
            g = gates[pos % len(gates)]
            orc.apply(psi, g)
            moved += gate_bytes(g)
            pos += 1
        return moved

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    moved = sum(one_step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    value = moved / dt / 1e9
    sample = (f"each step {per_step} consecutive gates of the {N_QUBITS}-qubit circuit's {len(gates)} (the "
              f"config's step), complex128 oracle, {cores} OpenMP threads; GB/s counts the complex64 "
              "workload's bytes of the gates applied")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import torch

    from paper_2308_01999_gb300 import sv

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gates, paulis, sites = workload()
    nbytes = step_bytes(gates, paulis)
    n_gates = len(gates)
    stream = torch.cuda.Stream(dev)
    psi = torch.zeros(1 << N_QUBITS, dtype=torch.complex64, device=dev)
    s = sv.StateVector(psi, stream)
    zp = np.full((N_QUBITS, 1), 3, np.int32)
    zs = np.arange(N_QUBITS, dtype=np.int32)[:, None]

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    su2_idx = [i for i, g in enumerate(gates) if g.name == "su2"]
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_gates)]
          for _ in range(args.steps)]

    def one_step(step_events=None, st=None):
        st = st or s
        for i, g in enumerate(gates):
            if step_events is not None:
                step_events[i][0].record(stream)
            st.apply_gate(g)
            if step_events is not None:
                step_events[i][1].record(stream)
        z = st.expectation_z_all()
        e = st.expectation_pauli(paulis, sites)
        p = st.measure_probs([0, N_QUBITS - 1])
        return z, e, p

    with torch.cuda.stream(stream):
        s.set_basis_state(0)
        for _ in range(args.warmup):
            one_step()
        torch.cuda.synchronize()
        clocks = Clocks(gpu_id(torch, dev))
        launches0 = s.launches()
        per_gate_ms = {i: 0.0 for i in range(n_gates)}
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            one_step(ev[k])
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        for k in range(args.steps):
            for i in range(n_gates):
                per_gate_ms[i] += ev[k][i][0].elapsed_time(ev[k][i][1])
        ms = t0.elapsed_time(t1) / args.steps
        launches = (s.launches() - launches0) // max(1, args.steps) * args.steps

        # end to end through the C ABI with host buffers: every step copies a full
        # initial state in from pinned host memory, runs the circuit and the
        # reductions, and copies the final state out. Two device states alternate
        # on two streams, so that step k+1's input copy and step k's output copy
        # (sv_copy_*_async) run while the other state computes. All `steps` steps
        # are timed, three times over; the median is the value, the others the spread.
        h_in = torch.zeros(1 << N_QUBITS, dtype=torch.complex64, pin_memory=True)
        h_in[0] = 1
        h_out = [torch.empty(1 << N_QUBITS, dtype=torch.complex64, pin_memory=True) for _ in range(2)]
        stream2 = torch.cuda.Stream(dev)
        psi2 = torch.empty_like(psi)
        s2 = sv.StateVector(psi2, stream2)
        pair = [s, s2]
        e_steps = max(2, args.steps)
        e2e_runs = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            barrier()
            e0.record(stream)
            stream2.wait_event(e0)
            sv.sv_copy_from_host_async(pair[0].handle, h_in.data_ptr())
            for k in range(e_steps):
                cur, nxt = pair[k % 2], pair[(k + 1) % 2]
                if k + 1 < e_steps:
                    sv.sv_copy_from_host_async(nxt.handle, h_in.data_ptr())
                one_step(st=cur)
                sv.sv_copy_to_host_async(cur.handle, h_out[k % 2].data_ptr())
            stream.wait_stream(stream2)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            e2e_runs.append(e0.elapsed_time(e1) / e_steps)
        s2.close()
        del psi2
        e2e_ms = statistics.median(e2e_runs)

    ms, e2e_ms = max_over_ranks([ms, e2e_ms], dev)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peak, peak_kind = load_peaks()
    su2_ms = [per_gate_ms[i] / args.steps for i in su2_idx]
    su2_bytes = 2 * AMP_BYTES * (1 << N_QUBITS)
    avg_su2 = sum(su2_ms) / len(su2_ms)
    achieved = su2_bytes / (avg_su2 * 1e-3) / 1e9
    per_q = {}
    for i in su2_idx:
        q = gates[i].targets[0]
        per_q.setdefault(q, []).append(per_gate_ms[i] / args.steps)
    per_target = {str(q): round(su2_bytes / (np.mean(v) * 1e-3) / 1e9, 1) for q, v in sorted(per_q.items())}
    per_kind = {}
    for kind in ("cz", "cnot", "crz"):
        idx = [i for i, g in enumerate(gates) if g.name == kind]
        if idx:
            t = np.mean([per_gate_ms[i] / args.steps for i in idx])
            per_kind[kind] = round(gate_bytes(gates[idx[0]]) / (t * 1e-3) / 1e9, 1)
    gates_ms = sum(per_gate_ms.values()) / args.steps
    value = job_throughput(nbytes, world, ms)
    cpu = cpu_baseline(gates) if world == 1 and not args.no_cpu_baseline else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile) and N_QUBITS == 28:
        with open(tfile) as f:
            traffic = json.load(f).get("k_dense_1q_per_launch_bytes")
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": line_config(world, n_gates, nbytes),
        "gates_per_s": round(world * n_gates / (gates_ms * 1e-3), 1),
        "gate_time_ms_per_step": round(gates_ms, 3),
        "roofline": {"bound": "hbm", "kernel": "k_dense (1-qubit dense, SU(2))", "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "frac_of_8tbs": round(achieved / 8000.0, 4), "traffic": traffic,
                     "algorithmic_bytes_per_launch": su2_bytes, "avg_launch_ms": round(avg_su2, 4)},
        "per_target_gbs": per_target, "per_kind_gbs": per_kind,
        "gpu_launches": int(launches),
        "e2e": {"value": round(job_throughput(nbytes, world, e2e_ms), 1), "unit": UNIT,
                "h2d_bytes_per_step": AMP_BYTES << N_QUBITS, "d2h_bytes_per_step": AMP_BYTES << N_QUBITS,
                "ms_per_step": round(e2e_ms, 3), "steps": e_steps, "runs": len(e2e_runs),
                "spread_gbs": [round(job_throughput(nbytes, world, max(e2e_runs)), 1),
                               round(job_throughput(nbytes, world, min(e2e_runs)), 1)],
                "copies": "full state in and out each step; two device states alternate so the copies "
                          "overlap the other state's gates; every step timed, three runs, median value"},
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    s.close()
    del s, psi
    torch.cuda.empty_cache()
    if world == 1 and not args.main_only:
        # the 30-qubit size of the bandwidth target, the bandwidth by number of
        # targets (complex64, 20 random sets per width), the 32-qubit fused
        # circuit and the other two parts of the headline metric, on the same
        # GPU after the 28-qubit step (rank 0 at N = 1 only, like the CPU baseline)
        line["n30"] = n30_section(args)
        line["e1"] = e1_section(20, 0)
        line["fused32"] = fused32_section(args)
        line["batch"] = batch_section(args)
        line["serve"] = serve_section(args)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_fused(args):
    """The 32-qubit brick-wall circuit (40 layers of Haar SU(2) + CZ wall, 1900
    gates) on a 32 GiB complex64 state: greedy fusion to 5- and 6-qubit blocks
    applied on the tensor cores (TF32, split BF16) or on CUDA cores (native),
    against the unfused complex64 run, with errors measured against an unfused
    complex128 run of the same circuit (64 GiB). Per-block kernel times come
    from CUDA events around each block's launch on the handle's stream."""
    import torch

    from paper_2308_01999_gb300 import sv

    n = args.fused_qubits
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    gates = gen.circuit_config2(n, 40, seed=2)
    stream = torch.cuda.Stream(dev)
    state_bytes = 2 * AMP_BYTES * (1 << n)          # read + write of the c64 state
    peak_hbm, _ = load_peaks()
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        bf16_peak = float(json.load(f)["bf16_tflops"])
    tf32_peak = bf16_peak * 1.1 / 2.25              # nominal dense TF32 : BF16 ratio
    out = {"workload": f"{n}-qubit brick wall, 40 layers, {len(gates)} gates, complex64", "n_qubits": n}

    def event_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    ref = None
    with torch.cuda.stream(stream):
        if not args.no_ref:
            ref = torch.empty(1 << n, dtype=torch.complex128, device=dev)
            r = sv.StateVector(ref, stream)
            r.set_basis_state(0)
            e0, e1 = event_pair()
            e0.record(stream)
            r.apply_circuit(gates)
            e1.record(stream)
            torch.cuda.synchronize()
            out["c128_unfused_s"] = round(e0.elapsed_time(e1) / 1e3, 3)
            ref_z = r.expectation_z_all()
            r.close()
        psi = torch.empty(1 << n, dtype=torch.complex64, device=dev)
        s = sv.StateVector(psi, stream)

        def errors():
            if ref is None:
                return {}
            num, den, mx = 0.0, 0.0, 0.0
            chunk = 1 << 27
            for a in range(0, 1 << n, chunk):
                d = psi[a:a + chunk].to(torch.complex128) - ref[a:a + chunk]
                num += float(torch.sum(torch.abs(d) ** 2))
                den += float(torch.sum(torch.abs(ref[a:a + chunk]) ** 2))
                mx = max(mx, float(torch.max(torch.abs(d))))
            z = s.expectation_z_all()
            return {"rel_l2": num ** 0.5 / den ** 0.5, "max_abs": mx, "max_abs_z": float(np.max(np.abs(z - ref_z)))}

        s.set_basis_state(0)
        e0, e1 = event_pair()
        e0.record(stream)
        s.apply_circuit(gates)
        e1.record(stream)
        torch.cuda.synchronize()
        out["unfused_c64"] = {"s": round(e0.elapsed_time(e1) / 1e3, 3), "launches": len(gates), **errors()}

        precs = {"tf32": sv.SV_PREC_TF32, "bf16": sv.SV_PREC_SPLIT_BF16, "native": sv.SV_PREC_NATIVE}
        for w in [int(x) for x in args.widths.split(",")]:
            plan = sv.sv_fuse_plan(gates, n, w)
            blocks = [gen.Gate(tuple(t), m) for t, m in plan]
            for prec_name in args.precs.split(","):
                prec = precs[prec_name]
                s.set_basis_state(0)
                torch.cuda.synchronize()
                evs = [event_pair() for _ in blocks]
                t0, t1 = event_pair()
                t0.record(stream)
                for b, (a, z) in zip(blocks, evs):
                    a.record(stream)
                    s.apply_fused([b], 6, prec)
                    z.record(stream)
                t1.record(stream)
                torch.cuda.synchronize()
                s.check()
                per = [a.elapsed_time(z) for a, z in evs]
                big = [ms for b, ms in zip(blocks, per) if b.k >= 5]
                rec = {"blocks": len(blocks), "blocks_5_6": len(big), "s": round(t0.elapsed_time(t1) / 1e3, 3),
                       "kernel_s": round(sum(per) / 1e3, 3)}
                if big:
                    avg = sum(big) / len(big)
                    rec["avg_block_ms"] = round(avg, 3)
                    rec["block_gbs"] = round(state_bytes / (avg * 1e-3) / 1e9, 1)
                    rec["hbm_frac"] = round(state_bytes / (avg * 1e-3) / 1e9 / peak_hbm, 4)
                    if prec_name != "native":
                        flop = 2 * 128 * 128 * (1 << (n - 6)) * (3 if prec_name == "bf16" else 1)
                        rec["tensor_tflops"] = round(flop / (avg * 1e-3) / 1e12, 1)
                        pk = bf16_peak if prec_name == "bf16" else tf32_peak
                        rec["tensor_frac"] = round(flop / (avg * 1e-3) / 1e12 / pk, 4)
                if big and prec_name != "native":
                    # per-block time by the lowest and the highest target qubit
                    by_lo, by_hi = {}, {}
                    for blk, ms in zip(blocks, per):
                        if blk.k >= 5:
                            by_lo.setdefault(min(blk.targets), []).append(ms)
                            by_hi.setdefault(max(blk.targets), []).append(ms)
                    rec["ms_by_lowest_target"] = {str(q): round(float(np.mean(v)), 2) for q, v in sorted(by_lo.items())}
                    rec["ms_by_highest_target"] = {str(q): round(float(np.mean(v)), 2) for q, v in sorted(by_hi.items())}
                rec.update(errors())
                # the same circuit as one sv_apply_fused call: host fusion, qubit
                # relabelling (tensor-core precisions) and every block
                s.set_basis_state(0)
                torch.cuda.synchronize()
                c0, c1 = event_pair()
                h0 = time.perf_counter()
                c0.record(stream)
                s.apply_fused(gates, w, prec)
                c1.record(stream)
                torch.cuda.synchronize()
                rec["one_call_s"] = round(c0.elapsed_time(c1) / 1e3, 3)
                rec["one_call_wall_s"] = round(time.perf_counter() - h0, 3)
                out[f"w{w}_{prec_name}"] = rec
                print(json.dumps({f"w{w}_{prec_name}": rec}), file=sys.stderr, flush=True)
        s.close()
    out["peaks"] = {"hbm_gbs": peak_hbm, "bf16_tflops": bf16_peak, "tf32_tflops_from_nominal_ratio": round(tf32_peak, 1)}
    print(json.dumps(out))


def fused32_section(args, n: int = 32) -> dict:
    """The 32-qubit fused brick wall (40 layers of Haar SU(2) + CZ wall, 1900
    gates, 32 GiB complex64 state) in the default line: the unfused complex64
    run (one gate per launch), then one sv_apply_fused call at width 6 in TF32
    and one in split BF16 (host fusion, relabelling choice and every block,
    5-6-qubit blocks on the tensor cores), each timed with CUDA events on the
    handle's stream. Errors of the fused runs are measured against the
    unfused complex64 state (whose own distance to a complex128 run of the
    circuit is ~2e-6, far below the tensor-core errors)."""
    import torch

    from paper_2308_01999_gb300 import sv

    dev = torch.device("cuda", 0)
    torch.cuda.empty_cache()
    gates = gen.circuit_config2(n, 40, seed=2)
    stream = torch.cuda.Stream(dev)
    out = {"workload": f"{n}-qubit brick wall, 40 layers of Haar SU(2) + CZ, {len(gates)} gates, complex64 "
                       "(32 GiB); fused width 6 on the tensor cores vs unfused"}

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    with torch.cuda.stream(stream):
        ref = torch.empty(1 << n, dtype=torch.complex64, device=dev)
        r = sv.StateVector(ref, stream)
        r.set_basis_state(0)
        out["unfused_c64_s"] = round(timed(lambda: r.apply_circuit(gates)), 3)
        ref_z = r.expectation_z_all()
        r.close()
        psi = torch.empty(1 << n, dtype=torch.complex64, device=dev)
        s = sv.StateVector(psi, stream)
        for name, prec in (("tf32", sv.SV_PREC_TF32), ("bf16", sv.SV_PREC_SPLIT_BF16)):
            s.set_basis_state(0)
            torch.cuda.synchronize()
            sec = timed(lambda: s.apply_fused(gates, 6, prec))
            s.check()
            num = den = mx = 0.0
            chunk = 1 << 28
            for a in range(0, 1 << n, chunk):
                d = psi[a:a + chunk] - ref[a:a + chunk]
                num += float(torch.sum(torch.abs(d).double() ** 2))
                den += float(torch.sum(torch.abs(ref[a:a + chunk]).double() ** 2))
                mx = max(mx, float(torch.max(torch.abs(d))))
            z = s.expectation_z_all()
            out[name] = {"one_call_s": round(sec, 3), "speedup_vs_unfused": round(out["unfused_c64_s"] / sec, 2),
                         "rel_l2_vs_unfused_c64": num ** 0.5 / den ** 0.5, "max_abs_vs_unfused_c64": mx,
                         "max_abs_z_vs_unfused_c64": float(np.max(np.abs(z - ref_z)))}
        s.close()
    del psi, ref
    torch.cuda.empty_cache()
    out["blocks"] = len(sv.sv_fuse_plan(gates, n, 6))
    return out


def run_e1(args):
    print(json.dumps(e1_section(args.e1_sets, args.e1_sets_c128)))


def e1_section(sets_c64: int, sets_c128: int) -> dict:
    """Gate-application bandwidth by number of targets (the paper's Sec. II-B
    experiment): for k = 1..6, `sets_c64` random target sets (sorted, seeded)
    with a random dense 2^k x 2^k matrix each, one sv_apply_matrix launch per
    set on a 33-qubit complex64 state (64 GiB) and `sets_c128` sets on a
    32-qubit complex128 state (64 GiB; none: skipped), each launch timed with CUDA events on
    the handle's stream (the state is 500 times L2, so no launch finds its
    input in cache). Algorithmic bytes per launch: one read and one write of
    the state. Per k: median, 10th/90th percentile, min and max GB/s, and the
    median as a fraction of the measured copy peak."""
    import torch

    from paper_2308_01999_gb300 import sv

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    peak, kind = load_peaks()
    out = {"workload": "random dense k-qubit gates, k = 1..6, one launch each", "peak_gbs": peak, "peak_kind": kind}
    torch.cuda.empty_cache()
    for name, n, dtype, sets in (("c64_33q", 33, torch.complex64, sets_c64),
                                 ("c128_32q", 32, torch.complex128, sets_c128)):
        if sets <= 0:
            continue
        rng = gen.rng_for(2308 + n)
        nbytes = 2 * (1 << n) * (8 if dtype == torch.complex64 else 16)
        rec = {}
        with torch.cuda.stream(stream):
            psi = torch.empty(1 << n, dtype=dtype, device=dev)
            s = sv.StateVector(psi, stream)
            s.set_basis_state(0)
            for k in range(1, 7):
                cases = [(sorted(int(q) for q in rng.choice(n, k, replace=False)), gen.random_gate_dense(rng, k))
                         for _ in range(sets)]
                s.apply(cases[0][0], cases[0][1])          # first launch of this width: set-up
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in cases]
                for (t, m), (a, b) in zip(cases, ev):
                    a.record(stream)
                    s.apply(t, m)
                    b.record(stream)
                torch.cuda.synchronize()
                gbs = np.array([nbytes / (a.elapsed_time(b) * 1e-3) / 1e9 for a, b in ev])
                rec[str(k)] = {"sets": sets, "median_gbs": round(float(np.median(gbs)), 1),
                               "p10_gbs": round(float(np.percentile(gbs, 10)), 1),
                               "p90_gbs": round(float(np.percentile(gbs, 90)), 1),
                               "min_gbs": round(float(gbs.min()), 1), "max_gbs": round(float(gbs.max()), 1),
                               "median_frac_of_peak": round(float(np.median(gbs)) / peak, 4)}
                print(json.dumps({name: {str(k): rec[str(k)]}}), file=sys.stderr, flush=True)
            rec["norm_minus_1"] = float(s.norm2() - 1.0)
            s.close()
        del psi
        torch.cuda.empty_cache()
        out[name] = rec
    return out


def n30_section(args, n: int = 30) -> dict:
    """The size of the >= 80 %-of-HBM target: one dense one-qubit SU(2) gate
    per launch on every target qubit of a 30-qubit complex64 state (8 GiB,
    60 times L2, so no launch finds its input in cache), two rounds over the
    30 targets, the second timed launch by launch with CUDA events on the
    launching stream. Algorithmic bytes per launch: one read and one write of
    the state. The norm after the 60 gates checks that they were applied."""
    import torch

    from paper_2308_01999_gb300 import sv

    dev = torch.device("cuda", 0)
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream(dev)
    rng = gen.rng_for(30)
    mats = [gen.haar_su2(rng) for _ in range(2 * n)]
    nbytes = 2 * AMP_BYTES * (1 << n)
    peak, kind = load_peaks()
    with torch.cuda.stream(stream):
        psi = torch.empty(1 << n, dtype=torch.complex64, device=dev)
        s = sv.StateVector(psi, stream)
        s.set_basis_state(0)
        for q in range(n):
            s.apply([q], mats[q])
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        clocks = Clocks(gpu_id(torch, dev))
        torch.cuda.synchronize()
        clocks.start()
        for q in range(n):
            ev[q][0].record(stream)
            s.apply([q], mats[n + q])
            ev[q][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        norm = s.norm2()
        s.close()
    ms = [a.elapsed_time(b) for a, b in ev]
    gbs = [nbytes / (t * 1e-3) / 1e9 for t in ms]
    total = n * nbytes / (sum(ms) * 1e-3) / 1e9
    del psi
    torch.cuda.empty_cache()
    return {"workload": f"{n}-qubit complex64 state (8 GiB), dense one-qubit SU(2) gate on each of the {n} target "
                        "qubits, one launch each",
            "gate_gbs": round(total, 1), "frac_of_8tbs": round(total / 8000.0, 4),
            "frac_of_peak": round(total / peak, 4), "peak_gbs": peak, "peak_kind": kind,
            "per_target_gbs_min": round(min(gbs), 1), "per_target_gbs_max": round(max(gbs), 1),
            "ms_per_gate": round(sum(ms) / n, 4), "norm_minus_1": float(norm - 1.0), "clocks": clk}


def batch_section(args) -> dict:
    """Many small states in one persistent launch: 4096 independent states with
    qubit counts uniform on 10..20, each a hardware-efficient ansatz of 6 layers
    (RY, RZ per qubit, CNOT ladder) followed by 8 random Pauli strings reduced in
    FP64. The product autotuner (``autotune.BatchTuner``) picks the fusion and
    window widths on a stratified sample; the full batch is then timed with its
    choice. On a sample of the same states, for comparison: the plain engine
    (one state at a time, one launch per gate, then the expectation call), the
    same with the batch's fusion (one fused call per state), and the plain
    launches replayed from one CUDA graph per state. None of the comparison
    engines allocates per state: one handle is rebound to each state
    (sv_set_state) inside one preallocated buffer."""
    import torch

    from paper_2308_01999_gb300 import autotune, sv

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t_gen = time.perf_counter()
    work = gen.batched_ansatz_workload(count=args.batch_states, seed=3)
    states = [(n, gates, paulis) for n, gates, paulis, _ in work]
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream(dev)
    out = {"workload": f"{len(states)} states, qubits uniform 10..20, 6-layer ansatz, 8 Pauli strings each, "
                       "complex64 states, FP64 expectation sums",
           "states": len(states), "gates": sum(len(g) for _, g, _ in states)}
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        packed = sv.pack_batch(states)
        out["pack_s"] = round(time.perf_counter() - t0, 2)
        b = sv.Batch(stream)
        t0 = time.perf_counter()
        if args.batch_widths:
            # fixed widths, no tuning (profiling captures of one configuration)
            parts = [int(x) for x in args.batch_widths.split(",")]
            fw, win = parts[0], parts[1]
            keep = parts[2] if len(parts) > 2 else 0
            tile = parts[3] if len(parts) > 3 else sv.SV_BATCH_TILE_QUBITS
            info = b.compile(packed, fw, win, bool(keep), tile)
            out["autotune"] = {"fixed": {"fusion_width": fw, "window_qubits": win, "keep_permutations": keep,
                                         "tile_qubits": tile}}
        else:
            tuner = autotune.BatchTuner(autotune.gpu_timer(stream), sample=args.tune_sample)
            info = b.compile(packed, tuner=tuner)            # the product path: tuned, then compiled
            sig = autotune.signature(packed.ns, packed.gate_counts)
            out["autotune"] = {"sample_states": min(args.tune_sample, len(states)), "signature": list(sig),
                               "choice": {"fusion_width": b.choice[0], "window_qubits": b.choice[1],
                                          "keep_permutations": b.choice[2], "tile_qubits": b.choice[3]},
                               "sample_ms": {f"fusion{fw}_window{win}" + ("_keepperm" if kp else "") +
                                             f"_tile{tile}": round(t * 1e3, 3)
                                             for (fw, win, kp, tile), t in tuner.timings[sig].items()}}
        out["tune_and_compile_s"] = round(time.perf_counter() - t0, 2)
        out["ops"], out["stages"] = info["ops"], info["stages"]
        buf = torch.empty(b.state_amps, dtype=torch.complex64, device=dev)
        for _ in range(2):
            b.launch(buf)
        res_batched = b.results()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.launch(buf)
        e1.record(stream)
        b.results()
        ms = e0.elapsed_time(e1) / reps
        out["batched_ms"] = round(ms, 3)
        out["batched_states_per_s"] = round(len(states) / (ms * 1e-3), 1)
        b.close()
        del buf
        torch.cuda.empty_cache()

        # comparison engines on a sample, one handle rebound to each state
        sample_idx = autotune.stratified_sample(packed.ns, args.plain_sample)
        sample = [states[i] for i in sample_idx]
        offs, a0 = [], 0
        for n, _, _ in sample:
            offs.append(a0)
            a0 += 1 << n
        arena = torch.empty(a0, dtype=torch.complex64, device=dev)
        h = sv.sv_create(1, sv.SV_C64, arena.data_ptr(), stream.cuda_stream)

        def sites(n, p):
            return np.tile(np.arange(n, dtype=np.int32), (p.shape[0], 1))

        def run_engine(fused):
            res = []
            for (n, gates, paulis), o in zip(sample, offs):
                sv.sv_set_state(h, n, sv.SV_C64, arena.data_ptr() + 8 * o)
                sv.sv_set_basis_state(h, 0)
                if fused:
                    sv.sv_apply_fused(h, gates, b.choice[0], sv.SV_PREC_NATIVE)
                else:
                    for g in gates:
                        sv.sv_apply_matrix(h, g.targets, g.matrix, g.controls, g.control_values or None)
                res.append(sv.sv_expectation_pauli(h, paulis, sites(n, paulis)))
            return res

        run_engine(False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_plain = run_engine(False)
        torch.cuda.synchronize()
        dt_plain = time.perf_counter() - t0
        t0 = time.perf_counter()
        run_engine(True)
        torch.cuda.synchronize()
        dt_fused = time.perf_counter() - t0
        # the plain launches captured once per state in a CUDA graph and replayed
        graphs = []
        for (n, gates, paulis), o in zip(sample, offs):
            sv.sv_set_state(h, n, sv.SV_C64, arena.data_ptr() + 8 * o)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                sv.sv_set_basis_state(h, 0)
                for gt in gates:
                    sv.sv_apply_matrix(h, gt.targets, gt.matrix, gt.controls, gt.control_values or None)
            graphs.append(g)
        for g in graphs[:2]:
            g.replay()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g, (n, gates, paulis), o in zip(graphs, sample, offs):
            g.replay()
            sv.sv_set_state(h, n, sv.SV_C64, arena.data_ptr() + 8 * o)
            sv.sv_expectation_pauli(h, paulis, sites(n, paulis))
        torch.cuda.synchronize()
        dt_graph = time.perf_counter() - t0
        del graphs
        sv.sv_destroy(h)
        del arena
        torch.cuda.empty_cache()
    diff = max(float(np.max(np.abs(res_batched[i] - r))) for i, r in zip(sample_idx, res_plain))
    m = len(sample)
    out["sample_states"] = m
    out["plain_states_per_s"] = round(m / dt_plain, 1)
    out["fused_serial_states_per_s"] = round(m / dt_fused, 1)
    out["graph_states_per_s"] = round(m / dt_graph, 1)
    out["speedup_vs_plain"] = round(out["batched_states_per_s"] / out["plain_states_per_s"], 1)
    out["speedup_vs_fused_serial"] = round(out["batched_states_per_s"] / out["fused_serial_states_per_s"], 1)
    out["speedup_vs_graph"] = round(out["batched_states_per_s"] / out["graph_states_per_s"], 1)
    out["max_abs_diff_batched_vs_plain"] = diff
    # algorithmic FP32 work: per layer and qubit one 2x2 complex product (RY and RZ
    # multiplied together) at 16 flop per amplitude; CNOTs move amplitudes only
    flop = sum(6 * n * 16 * (1 << n) for n, _, _ in states)
    out["fp32_flop"] = flop
    out["batched_tflops"] = round(flop / (ms * 1e-3) / 1e12, 2)
    # FP32 ALU roofline: 128 FP32 lanes per SM, one FMA (2 flop) each per clock,
    # at the maximum SM clock
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = 2070.0
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as f:
            sm_mhz = float(json.load(f).get("sm_max_mhz", sm_mhz))
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    out["roofline"] = {"bound": "alu", "kernel": "k_batch", "achieved": out["batched_tflops"],
                       "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                       "frac": round(out["batched_tflops"] / fp32_peak, 3), "traffic": None,
                       "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz"}
    out["generation_s"] = round(t_gen, 1)
    return out


def serve_section(args) -> dict:
    """Serving trace: Poisson arrivals of random circuits (12..30 qubits, depth
    10..60, the gate mix of the 28-qubit circuit, complex64), each returning
    <Z_q> for all its qubits. The continuous-batching engine (admission into a
    pooled HBM arena, batched small states in concurrent batch slots, one stream
    per large request, fused native gates) against two serial engines on the
    same trace: the plain one (one request at a time, one launch per gate) and
    one with the same fusion (so the gains of fusion and of batching separate);
    then all three again at 0.7x the plain engine's measured capacity, so that
    latency reflects service rather than backlog."""
    import torch

    from paper_2308_01999_gb300 import autotune, serving, sv

    torch.cuda.set_device(0)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(0.8 * (free - (9 << 30)), args.serve_budget_gb * (1 << 30)))
    ex = serving.GpuExecutor(budget, fusion_width=4)
    # the batched engine's widths: tuned once on a sample of small requests of
    # the trace's kind (12..20 qubits, depth 10..60); the choice serves every batch
    tune_reqs = serving.make_requests(gen.serving_trace(count=96, rate=1000.0, nmin=12, nmax=20, seed=98))
    tuner = autotune.BatchTuner(autotune.gpu_timer(torch.cuda.Stream()), sample=96)
    packed = sv.pack_batch([(r.n, r.gates(), 3 * np.eye(r.n, dtype=np.int32)) for r in tune_reqs])
    ex.batch_widths = tuner.choose(packed)
    # warm-up of every path (library load, first launches, worker resources)
    warm = serving.make_requests(gen.serving_trace(count=8, rate=1000.0, nmin=12, nmax=24, dmin=3, dmax=5, seed=99))
    serving.ServingEngine(ex).run(warm)
    for r in warm[:2]:
        ex.run_plain(r)
        ex.run_fused_serial(r)
    torch.cuda.synchronize()

    def served(trace, batch_max):
        eng = serving.ServingEngine(ex, small_max_qubits=20, batch_max_qubits=batch_max, large_workers=4,
                                    batch_slots=2)
        mix = eng.run(serving.make_requests(trace))
        occ = eng.occupancy
        tw = 0.0
        for (t_a, b_a), (t_b, _) in zip(occ, occ[1:]):
            tw += b_a * (t_b - t_a)
        span = occ[-1][0] - occ[0][0] if len(occ) > 1 else 1.0
        rec = {k: round(v, 4) for k, v in serving.latency_stats(mix).items()}
        rec.update({"hbm_peak_gib": round(eng.peak_bytes / (1 << 30), 2),
                    "hbm_mean_gib": round(tw / span / (1 << 30), 2), "batches": len(eng.batch_sizes),
                    "mean_batch_size": round(float(np.mean(eng.batch_sizes)), 2) if eng.batch_sizes else 0})
        return mix, rec

    def one(rate, count, seed):
        trace = gen.serving_trace(count=count, rate=rate, seed=seed)
        mix, rec = served(trace, args.serve_batch_max)
        alt = 26 if args.serve_batch_max != 26 else 20
        mix_alt, rec_alt = served(trace, alt)
        plain = serving.serial_engine(ex.run_plain, serving.make_requests(trace))
        fused = serving.serial_engine(ex.run_fused_serial, serving.make_requests(trace))
        diffs = [float(np.max(np.abs(a.result - b.result))) for m in (mix, mix_alt) for a, b in zip(m, plain)
                 if a.result is not None and b.result is not None]
        service = [r.t_done - r.t_admit for r in plain if r.error is None]
        return {"requests": count, "rate_per_s": round(rate, 3),
                "served": rec, f"served_batches_to_{alt}_qubits": rec_alt,
                "plain": {k: round(v, 4) for k, v in serving.latency_stats(plain).items()},
                "fused_serial": {k: round(v, 4) for k, v in serving.latency_stats(fused).items()},
                "max_abs_diff_vs_plain": max(diffs) if diffs else None,
                "plain_capacity_per_s": round(len(service) / sum(service), 3) if service else None}

    out = {"workload": "serving trace, Poisson arrivals, qubits 12..30, depth 10..60, complex64, <Z_q> for all q",
           "hbm_budget_gib": round(budget / (1 << 30), 1),
           "served_config": {"small_batches_to_qubits": 20, "medium_batches_to_qubits": args.serve_batch_max,
                             "larger": "one fused call each (native, width 4), 4 concurrent streams",
                             "batch_slots_per_class": 2},
           "batch_widths": {"fusion_width": ex.batch_widths[0], "window_qubits": ex.batch_widths[1],
                            "keep_permutations": ex.batch_widths[2], "tile_qubits": ex.batch_widths[3]},
           "sample_note": (f"{args.serve_requests} requests of the 10000-request trace at the offered rate: "
                           "the offered load is far above one GPU's capacity, so the trace is a backlog drain "
                           "whose length only scales the makespan, and 10000 requests would hold the GPU for "
                           "about half an hour per engine")}
    hot = one(args.serve_rate, args.serve_requests, 4)
    out["at_offered_rate"] = hot
    print(json.dumps({"at_offered_rate": hot}), file=sys.stderr, flush=True)
    cap = hot["plain_capacity_per_s"] or 1.0
    out["at_0.7x_plain_capacity"] = one(0.7 * cap, args.serve_low_requests, 5)
    ex.close()
    del ex
    torch.cuda.empty_cache()
    return out


GATE_CASES = ("1:0 1:3 2:0,1 2:3,9 2:1,5 3:0,1,2 3:0,1,5 3:3,9,14 3:20,22,24 3:0,4,9 3:1,9,12 "
              "4:0,1,2,3 4:0,1,2,7 4:0,1,4,6 4:0,3,6,9 4:1,2,3,4 4:1,3,5,7 4:2,3,4,5 4:3,9,14,20 4:20,22,24,26")


def gate_table(args) -> dict:
    """Dense gates by width and target set: single launches of a random dense
    2^k x 2^k matrix on a complex64 state ("k:t0,t1,..."), or one 6-qubit block
    on the tensor cores ("tf32:..." / "bf16:..." with six targets), CUDA events
    around each call on the handle's stream, L2 flushed (a 256 MiB write)
    before each, median of the timed calls; GB/s counts one read and one write
    of every amplitude."""
    import torch

    from paper_2308_01999_gb300 import sv

    n = args.qubits
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    psi = torch.zeros(1 << n, dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    rng = gen.rng_for(5)
    out = {"n_qubits": n, "state_bytes": 8 << n, "cases": {}}
    with torch.cuda.stream(stream):
        s = sv.StateVector(psi, stream)
        s.set_basis_state(0)
        precs = {"tf32": sv.SV_PREC_TF32, "bf16": sv.SV_PREC_SPLIT_BF16}
        for case in args.gate_cases.split():
            k, ts = case.split(":")
            t = [int(x) for x in ts.split(",")]
            assert max(t) < n and (k in precs and len(t) == 6 or k not in precs and len(t) == int(k))
            m = gen.random_gate_dense(rng, len(t))
            if k in precs:      # one 6-qubit block on the tensor cores
                g = gen.Gate(tuple(t), m)
                run = lambda: s.apply_fused([g], 6, precs[k])  # noqa: E731
            else:
                run = lambda: s.apply(t, m)  # noqa: E731
            for _ in range(2):
                run()
            times = []
            for _ in range(args.gate_reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = float(np.median(times))
            out["cases"][case] = {"ms": round(ms, 4), "gbs": round(16 * (1 << n) / (ms * 1e-3) / 1e9, 1),
                                  "fp32_tflops": round(8 * (1 << len(t)) * (1 << n) / (ms * 1e-3) / 1e12, 1)}
            if k in precs:
                out["cases"][case].pop("fp32_tflops")
        s.close()
    return out


def run_gate_table(args):
    print(json.dumps(gate_table(args)))


def _oracle_states_worker(args):
    """One process of the per-state CPU baseline: the oracle, single-threaded,
    on a slice of the batched workload (ansatz circuit, then the 8 strings)."""
    lo, hi, count = args
    from oracle import oracle as orc
    orc.set_threads(1)
    work = gen.batched_ansatz_workload(count=count, seed=3)
    t0 = time.perf_counter()
    for n, gates, paulis, sites in work[lo:hi]:
        psi = orc.run_circuit(gates, n)
        for p_, s_ in zip(paulis, sites):
            orc.expect_pauli(psi, p_, s_)
    return time.perf_counter() - t0


def cpu_plan(args) -> dict:
    """The CPU-baseline plan: the oracle as it stands (complex128, plain loops,
    OpenMP over amplitude groups) timed on this host's cores, with one thread
    and with all of them, on the 16-qubit parity circuit (whole), the 28-qubit
    benchmark circuit (all threads: whole; one thread: its first layer) and the
    4096-state batched workload (all threads: one single-threaded process per
    core, states dealt round robin; one thread: a stratified sample of 128
    states, scaled by their share of the total amplitude work). Host memory is
    reported so that the 64 GiB complex128 run of the 32-qubit brick wall can
    be judged against it."""
    import multiprocessing as mp

    from oracle import oracle as orc

    cores = len(os.sched_getaffinity(0))
    out = {"host_cores": cores, "kind": "oracle"}
    try:
        with open("/proc/meminfo") as f:
            kb = {ln.split(":")[0]: int(ln.split()[1]) for ln in f if ln.split()[0].endswith(":")}
        out["host_mem_gib"] = round(kb["MemTotal"] / 2**20, 1)
        out["host_mem_available_gib"] = round(kb.get("MemAvailable", 0) / 2**20, 1)
    except (OSError, KeyError, ValueError):
        out["host_mem_gib"] = None
    out["c128_32q_state_fits_host"] = bool(out.get("host_mem_available_gib") and
                                           out["host_mem_available_gib"] > 80)
    # 16-qubit parity circuit
    gates0 = gen.circuit_config0(0)
    rec = {}
    for th in (1, cores):
        orc.set_threads(th)
        t0 = time.perf_counter()
        psi = orc.run_circuit(gates0, 16)
        orc.expect_z_all(psi)
        rec[f"threads_{th}_s"] = round(time.perf_counter() - t0, 3)
    out["circuit16"] = {"gates": len(gates0), **rec}
    # 28-qubit benchmark circuit
    gates1 = gen.circuit_config1()
    orc.set_threads(cores)
    t0 = time.perf_counter()
    orc.run_circuit(gates1, 28)
    dt_all = time.perf_counter() - t0
    orc.set_threads(1)
    layer = gates1[:42]
    t0 = time.perf_counter()
    orc.run_circuit(layer, 28)
    dt_one = time.perf_counter() - t0
    out["circuit28"] = {"gates": len(gates1), f"threads_{cores}_s": round(dt_all, 2),
                        f"threads_{cores}_gates_per_s": round(len(gates1) / dt_all, 2),
                        "threads_1_sample": "first layer (42 gates)", "threads_1_sample_s": round(dt_one, 2),
                        "threads_1_gates_per_s": round(len(layer) / dt_one, 3),
                        "threads_1_est_s": round(dt_one * len(gates1) / len(layer), 1)}
    # 4096-state batched workload
    count = args.batch_states
    work = gen.batched_ansatz_workload(count=count, seed=3)
    ns = [n for n, _, _, _ in work]
    from paper_2308_01999_gb300 import autotune
    idx = autotune.stratified_sample(ns, 128)
    orc.set_threads(1)
    t0 = time.perf_counter()
    for i in idx:
        n, gates, paulis, sites = work[i]
        psi = orc.run_circuit(gates, n)
        for p_, s_ in zip(paulis, sites):
            orc.expect_pauli(psi, p_, s_)
    dt_s = time.perf_counter() - t0
    share = sum(len(work[i][1]) * (1 << work[i][0]) for i in idx) / sum(len(g) * (1 << n) for n, g, _, _ in work)
    ctx = mp.get_context("spawn")
    step = (count + cores - 1) // cores
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_states_worker, [(lo, min(count, lo + step), count) for lo in range(0, count, step)])
    dt_p = time.perf_counter() - t0
    out["batch4096"] = {"states": count, f"processes_{cores}_s": round(dt_p, 1),
                        f"processes_{cores}_states_per_s": round(count / dt_p, 1),
                        "threads_1_sample": "128 states, stratified by qubit count",
                        "threads_1_sample_s": round(dt_s, 2),
                        "threads_1_est_s": round(dt_s / share, 1),
                        "threads_1_states_per_s": round(count / (dt_s / share), 2)}
    return out


def run_cpu_plan(args):
    print(json.dumps(cpu_plan(args)))


def run_batch(args):
    print(json.dumps(batch_section(args)))


def run_serve(args):
    print(json.dumps(serve_section(args)))


def run_n30(args):
    print(json.dumps(n30_section(args)))


def run_fused_brief(args):
    print(json.dumps(fused32_section(args)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--qubits", type=int, default=28,
                    help="state size; 28 is the benchmark workload, smaller sizes are for profiling captures")
    ap.add_argument("--workload", choices=("circuit28", "fused32", "fused32-brief", "batch", "serve", "n30",
                                           "e1", "cpu-plan", "gates"),
                    default="circuit28",
                    help="fused32: the 32-qubit fused brick-wall study (tensor cores, errors vs complex128)")
    ap.add_argument("--fused-qubits", type=int, default=32)
    ap.add_argument("--no-ref", action="store_true", help="fused32 without the complex128 reference run")
    ap.add_argument("--widths", default="5,6", help="fused32: fusion widths")
    ap.add_argument("--batch-states", type=int, default=4096, help="batch: number of states")
    ap.add_argument("--plain-sample", type=int, default=256, help="batch: states run through the plain engine")
    ap.add_argument("--tune-sample", type=int, default=1024, help="batch: states the autotuner times")
    ap.add_argument("--batch-widths", default="", help="batch: 'fusion,window[,keep_permutations[,tile_qubits]]' instead of the autotuner")
    ap.add_argument("--gate-cases", default=GATE_CASES, help="gates: 'k:t0,t1,..' cases, space separated")
    ap.add_argument("--gate-reps", type=int, default=5, help="gates: timed launches per case")
    ap.add_argument("--e1-sets", type=int, default=100, help="e1: random target sets per width, complex64")
    ap.add_argument("--e1-sets-c128", type=int, default=20, help="e1: random target sets per width, complex128")
    ap.add_argument("--main-only", action="store_true",
                    help="only the 28-qubit line, without its batch and serve sections")
    ap.add_argument("--serve-requests", type=int, default=120, help="serve: requests of the offered-rate trace")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serve: offered arrival rate (1/s)")
    ap.add_argument("--serve-low-requests", type=int, default=40, help="serve: requests of the 0.7x-capacity trace")
    ap.add_argument("--serve-budget-gb", type=float, default=200.0, help="serve: HBM budget for resident states")
    ap.add_argument("--serve-batch-max", type=int, default=20,
                    help="serve: largest request (qubits) that goes to a batch; larger ones run as fused calls")
    ap.add_argument("--precs", default="tf32,bf16,native", help="fused32: precisions")
    args = ap.parse_args()
    global N_QUBITS
    N_QUBITS = args.qubits
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "fused32":
        run_fused(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "n30":
        run_n30(args)
    elif args.workload == "e1":
        run_e1(args)
    elif args.workload == "fused32-brief":
        run_fused_brief(args)
    elif args.workload == "cpu-plan":
        run_cpu_plan(args)
    elif args.workload == "gates":
        run_gate_table(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
