"""The largest states one GPU holds: 34 qubits in complex64 and 33 in
complex128 (128 GiB each). Amplitude indices above 2^32 must survive every
kernel's index arithmetic; the checks use closed forms that hold at any size,
since no complex128 copy of the state fits on the host.

Circuit, with t = n - 1 the top qubit: Haar SU(2) gates on qubits 0, 1, 5, 31,
32 and t from |0...0> (a product state: amplitude i is the product of
U_q[bit q of i][0], zero wherever another bit is set), then CNOT(t -> 2),
CZ(32, 0) and CRZ(1 -> t): the CNOT maps index i to i ^ (bit t of i) << 2, the
other two multiply amplitude i by a phase of its bits. Sampled amplitudes and
all n <Z_q> are compared with that
closed form (1e-5 / 1e-6 in complex64, 1e-12 in complex128). Then, in complex64,
two 6-qubit dense blocks, each followed by its inverse, run
on the tensor cores in split BF16 (one through the raw-operand kernel, lowest
target 3; one with qubit 0 a target): <Z_q> and the norm must come back
within the per-block error bound of the split-BF16 operands (the derivation is
in test_gpu_tc.py: sqrt(128) * (3 * 2^-18 + 384 * 2^-24) relative L2 per block).
"""
import math

import numpy as np
import pytest

from paper_2308_01999_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

PER_BLOCK_BF16 = math.sqrt(128) * (3 * 2.0 ** -18 + 384 * 2.0 ** -24)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return torch, sv


@pytest.mark.parametrize("name,N", [("c64", 34), ("c128", 33)])
def test_max_size_closed_forms_and_tensor_core_echo(env, name, N):
    torch, sv = env
    amp_bytes = 8 if name == "c64" else 16
    amp_tol, z_tol = (1e-5, 1e-6) if name == "c64" else (1e-12, 1e-12)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < (1 << N) * amp_bytes + (4 << 30):
        pytest.skip(f"needs {((1 << N) * amp_bytes >> 30) + 4} GiB of free device memory, {free >> 30} GiB free")
    rng = gen.rng_for(N)
    top = N - 1
    us = {q: gen.haar_su2(rng) for q in (0, 1, 5, 31, 32, top)}
    theta = 1.1
    rz = gen.gate_rz(theta)
    psi = torch.zeros(1 << N, dtype=torch.complex64 if name == "c64" else torch.complex128, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    for q, u in us.items():
        s.apply_gate(gen.Gate((q,), u))
    s.apply_gate(gen.cnot(top, 2))
    s.apply_gate(gen.cz(32, 0))
    s.apply_gate(gen.crz(1, top, theta))
    s.check()

    def closed_form(idx):
        i = idx.astype(np.uint64)
        bit = lambda x, q: ((x >> np.uint64(q)) & np.uint64(1)).astype(np.int64)
        j = i ^ (np.uint64(bit(i, top)) << np.uint64(2))         # before the CNOT
        amp = np.ones(len(i), dtype=np.complex128)
        mask = np.uint64(sum(1 << q for q in us))
        for q, u in us.items():
            amp *= u[bit(j, q), 0]
        amp[(j & ~mask) != 0] = 0
        amp *= np.where((bit(i, 32) == 1) & (bit(i, 0) == 1), -1.0, 1.0)
        amp *= np.where(bit(i, 1) == 1, rz[bit(i, top), bit(i, top)], 1.0)
        return amp

    # in the support: free bits on the Haar qubits, bit 2 = the top bit; outside: one other bit set
    m = 4096
    idx = np.zeros(m, dtype=np.int64)
    for q in us:
        idx |= rng.integers(0, 2, size=m).astype(np.int64) << q
    idx |= ((idx >> top) & 1) << 2
    outside = idx[:512] | (np.int64(1) << rng.choice([3, 4, 6, 7, 13, 20, 30], size=512).astype(np.int64))
    idx = np.concatenate([idx, outside, np.array([0, (1 << N) - 1, (1 << top) | (1 << 32) | 7], np.int64)])
    got = psi[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    want = closed_form(idx)
    err = float(np.max(np.abs(got - want)))
    assert err <= amp_tol, f"{N}q {name} sampled amplitudes: max|d| = {err:.3e}"
    assert np.all(got[m:m + 512] == 0), "amplitudes outside the product-state support must stay exactly 0"

    zq = np.ones(N)
    for q, u in us.items():
        zq[q] = abs(u[0, 0]) ** 2 - abs(u[1, 0]) ** 2
    zq[2] = zq[top]                                              # bit 2 copies the top bit
    z = s.expectation_z_all()
    assert np.max(np.abs(z - zq)) <= z_tol, f"{N}q {name} <Z_q>: max|d| = {np.max(np.abs(z - zq)):.3e}"
    if name == "c128":
        print(f"[max size] {N}q {name}: sampled max|d| {err:.3e}, max|d<Z>| {np.max(np.abs(z - zq)):.3e}")
        s.close()
        del psi
        torch.cuda.empty_cache()
        return

    # tensor-core blocks and their inverses, each its own fused call
    for targets in ((3, 9, 17, 26, 32, 33), (0, 2, 12, 20, 31, 33)):
        g = gen.random_gate_dense(rng, 6)
        assert s.apply_fused([gen.Gate(targets, g)], 6, sv.SV_PREC_SPLIT_BF16) == 1
        assert s.apply_fused([gen.Gate(targets, g.conj().T)], 6, sv.SV_PREC_SPLIT_BF16) == 1
    s.check()
    rel = 4 * PER_BLOCK_BF16                  # relative L2 error bound after 4 blocks
    z = s.expectation_z_all()
    zerr = float(np.max(np.abs(z - zq)))
    norm = s.norm2()
    print(f"[max size] {N}q {name}: sampled max|d| {err:.3e}; after 4 BF16 blocks max|d<Z>| {zerr:.3e}, "
          f"|norm - 1| {abs(norm - 1):.3e}, bound {2 * rel + rel * rel:.3e}")
    assert zerr <= 2 * rel + rel * rel
    assert abs(norm - 1) <= 2 * rel + rel * rel
    s.close()
    del psi
    torch.cuda.empty_cache()
