"""The N > 1 path of bench.py on CPU: replicas timed by their slowest rank
(gloo, world size 2), and the reference arm under torchrun printing exactly
one line from rank 0. The path itself does not shard (one state per GPU), so
the only cross-rank steps are the barrier and this maximum."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    vals = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 5.0])
    dist.barrier()
    q.put((rank, vals, bench.job_throughput(4e9, world, vals[0])))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, vals, thr in got:
        assert vals == [2.0, 10.0, 5.0]
        assert abs(thr - 2 * 4e9 / 2e-3 / 1e9) < 1e-6


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--qubits", "10", "--steps", "2", "--warmup", "1", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the same `config` object as the GPU arm's line for this workload and world size
    sys.path.insert(0, ROOT)
    import bench
    bench.N_QUBITS = 10
    gates, paulis, _ = bench.workload()
    assert d["config"] == json.loads(json.dumps(bench.line_config(2, len(gates), bench.step_bytes(gates, paulis))))
