"""The largest state one GPU holds in complex64: 34 qubits, 2^34 amplitudes
(128 GiB). Amplitude indices above 2^32 must survive every kernel's index
arithmetic; the checks use closed forms that hold at any size, since no
complex128 copy of the state fits on the host.

Circuit: Haar SU(2) gates on qubits 0, 1, 5, 31, 32, 33 from |0...0> (a product
state: amplitude i is the product of U_q[bit q of i][0], zero wherever another
bit is set), then CNOT(33 -> 2), CZ(32, 0) and CRZ(1 -> 33): the CNOT maps
index i to i ^ (bit 33 of i) << 2, the other two multiply amplitude i by a
phase of its bits. Sampled amplitudes and all 34 <Z_q> are compared with that
closed form. Then two 6-qubit dense blocks, each followed by its inverse, run
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

N = 34
PER_BLOCK_BF16 = math.sqrt(128) * (3 * 2.0 ** -18 + 384 * 2.0 ** -24)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return torch, sv


def test_max_size_34q_closed_forms_and_tensor_core_echo(env):
    torch, sv = env
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < (1 << N) * 8 + (4 << 30):
        pytest.skip(f"needs {((1 << N) * 8 >> 30) + 4} GiB of free device memory, {free >> 30} GiB free")
    rng = gen.rng_for(34)
    us = {q: gen.haar_su2(rng) for q in (0, 1, 5, 31, 32, 33)}
    theta = 1.1
    rz = gen.gate_rz(theta)
    psi = torch.zeros(1 << N, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    for q, u in us.items():
        s.apply_gate(gen.Gate((q,), u))
    s.apply_gate(gen.cnot(33, 2))
    s.apply_gate(gen.cz(32, 0))
    s.apply_gate(gen.crz(1, 33, theta))
    s.check()

    def closed_form(idx):
        i = idx.astype(np.uint64)
        bit = lambda x, q: ((x >> np.uint64(q)) & np.uint64(1)).astype(np.int64)
        j = i ^ (np.uint64(bit(i, 33)) << np.uint64(2))          # before the CNOT
        amp = np.ones(len(i), dtype=np.complex128)
        mask = np.uint64(sum(1 << q for q in us))
        for q, u in us.items():
            amp *= u[bit(j, q), 0]
        amp[(j & ~mask) != 0] = 0
        amp *= np.where((bit(i, 32) == 1) & (bit(i, 0) == 1), -1.0, 1.0)
        amp *= np.where(bit(i, 1) == 1, rz[bit(i, 33), bit(i, 33)], 1.0)
        return amp

    # in the support: free bits on the Haar qubits, bit 2 = bit 33; outside: one other bit set
    m = 4096
    idx = np.zeros(m, dtype=np.int64)
    for q in us:
        idx |= rng.integers(0, 2, size=m).astype(np.int64) << q
    idx |= ((idx >> 33) & 1) << 2
    outside = idx[:512] | (np.int64(1) << rng.choice([3, 4, 6, 7, 13, 20, 30], size=512).astype(np.int64))
    idx = np.concatenate([idx, outside, np.array([0, (1 << N) - 1, (1 << 33) | (1 << 32) | 7], np.int64)])
    got = psi[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    want = closed_form(idx)
    err = float(np.max(np.abs(got - want)))
    assert err <= 1e-5, f"34q sampled amplitudes: max|d| = {err:.3e}"
    assert np.all(got[m:m + 512] == 0), "amplitudes outside the product-state support must stay exactly 0"

    zq = np.ones(N)
    for q, u in us.items():
        zq[q] = abs(u[0, 0]) ** 2 - abs(u[1, 0]) ** 2
    zq[2] = zq[33]                                               # bit 2 copies bit 33
    z = s.expectation_z_all()
    assert np.max(np.abs(z - zq)) <= 1e-6, f"34q <Z_q>: max|d| = {np.max(np.abs(z - zq)):.3e}"

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
    print(f"[max size] 34q: sampled max|d| {err:.3e}; after 4 BF16 blocks max|d<Z>| {zerr:.3e}, "
          f"|norm - 1| {abs(norm - 1):.3e}, bound {2 * rel + rel * rel:.3e}")
    assert zerr <= 2 * rel + rel * rel
    assert abs(norm - 1) <= 2 * rel + rel * rel
    s.close()
    del psi
    torch.cuda.empty_cache()
