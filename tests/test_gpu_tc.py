"""Tensor-core fused gates (tcgen05, TF32 and split-BF16) against the FP64 oracle.

No exactness is expected: the stated error bounds follow from the operand
rounding. With u the unit roundoff of the operand format (TF32: 2^-11;
split BF16: hi + lo carries 2^-17 of each operand, the dropped lo*lo term
2^-18) and FP32 accumulation over K = 128 terms, every output of one 64x64
gate has |error| <= c * sum_k |A_mk x_k| with c = 2u + 128 * 2^-24 (TF32) or
c = 3 * 2^-18 + 384 * 2^-24 (split BF16); for a unitary gate that sum is at
most sqrt(128) times the group's norm, so one gate changes the relative L2
error by at most sqrt(128) * c and G gates by G times that. The tests assert
these worst-case bounds and print the measured errors. The TF32 kernel for
lowest targets >= 2 (both precisions) contracts over the 64 members in two FP32
sums of 64 terms (real and imaginary parts of G; split BF16: three products per
term) joined by one addition, inside the same bounds.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

C_TF32 = 2 * 2.0 ** -11 + 128 * 2.0 ** -24
C_BF16 = 3 * 2.0 ** -18 + 384 * 2.0 ** -24
PER_GATE = {"tf32": math.sqrt(128) * C_TF32, "bf16": math.sqrt(128) * C_BF16}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return torch, sv


def prec_code(sv, name):
    return sv.SV_PREC_TF32 if name == "tf32" else sv.SV_PREC_SPLIT_BF16


def rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("name", ["tf32", "bf16"])
@pytest.mark.parametrize("n,targets", [(12, (2, 3, 5, 7, 8, 11)), (13, (0, 1, 2, 3, 4, 5)),
                                       (10, (4, 5, 6, 7, 8, 9)), (14, (1, 4, 6, 9, 12, 13)),
                                       (8, (0, 2, 3, 5, 6, 7)), (6, (0, 1, 2, 3, 4, 5)),
                                       # lowest target >= 2: one ragged tile (8 or 32 columns),
                                       # several tiles, far and contiguous targets
                                       (9, (3, 4, 5, 6, 7, 8)), (11, (3, 5, 6, 8, 9, 10)),
                                       (16, (5, 9, 10, 12, 14, 15)), (20, (3, 8, 12, 16, 18, 19)),
                                       (17, (11, 12, 13, 14, 15, 16)),
                                       # 7 qubits, qubit 0 free: a single pair of columns
                                       (7, (1, 2, 3, 4, 5, 6))])
def test_single_six_qubit_gate(env, name, n, targets):
    torch, sv = env
    rng = gen.rng_for(n * 100 + targets[0])
    g = gen.Gate(tuple(targets), gen.random_gate_dense(rng, 6))
    init = gen.random_state(n, n + 3)
    ref = init.copy()
    orc.apply(ref, g)
    psi = torch.from_numpy(init).to(torch.complex64).cuda()
    s = sv.StateVector(psi)
    nf = s.apply_fused([g], 6, prec_code(sv, name))
    assert nf == 1
    s.check()
    got = psi.cpu().numpy().astype(np.complex128)
    err = rel_l2(got, ref)
    print(f"[tc] {name} n={n} targets={targets}: rel L2 {err:.3e}, max|d| {np.max(np.abs(got - ref)):.3e}, "
          f"bound {PER_GATE[name]:.3e}")
    assert err <= PER_GATE[name] + 2.0 ** -22


@pytest.mark.parametrize("name", ["tf32", "bf16"])
@pytest.mark.parametrize("width", [5, 6])
def test_fused_brick_wall(env, name, width):
    torch, sv = env
    n = 15
    gates = gen.circuit_config2(n=n, layers=12, seed=12)
    ref = orc.run_circuit(gates, n)
    psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    nf = s.apply_fused(gates, width, prec_code(sv, name))
    s.check()
    got = psi.cpu().numpy().astype(np.complex128)
    err = rel_l2(got, ref)
    z = s.expectation_z_all()
    zerr = float(np.max(np.abs(z - orc.expect_z_all(ref))))
    print(f"[tc] {name} brick wall n={n} w={width}: {nf} blocks, rel L2 {err:.3e}, max|d| "
          f"{np.max(np.abs(got - ref)):.3e}, max|d<Z>| {zerr:.3e}, bound {nf * PER_GATE[name]:.3e}")
    assert err <= nf * PER_GATE[name]
    assert abs(s.norm2() - 1) <= 2 * nf * PER_GATE[name]


def test_native_and_tensor_core_agree_on_structure(env):
    """A fused block that is diagonal or controlled takes the exact kernels, so
    TF32 requests on such blocks reproduce the native result exactly."""
    torch, sv = env
    n = 12
    gates = [gen.cz(a, a + 1) for a in range(0, n - 1)]
    psi = torch.from_numpy(gen.random_state(n, 4)).to(torch.complex64).cuda()
    ref = psi.clone()
    s = sv.StateVector(psi)
    s.apply_fused(gates, 6, sv.SV_PREC_TF32)
    r = sv.StateVector(ref)
    r.apply_circuit(gates)
    assert torch.equal(psi, ref)


@pytest.mark.parametrize("name", ["tf32", "bf16"])
def test_low_targets_relabelled_by_index_bit_swaps(env, name):
    """Wide blocks whose lowest target is below qubit 2 run after a qubit
    relabelling (two extra index-bit-swap passes) when enough of them gain from
    it; the result is unchanged."""
    torch, sv = env
    n = 24
    rng = gen.rng_for(91)
    gates = []
    for layer in range(72):
        for q in range(7):
            gates.append(gen.Gate((q,), gen.haar_su2(rng)))
        for a in range(layer % 2, 6, 2):
            gates.append(gen.cz(a, a + 1))
    gates.append(gen.Gate((13,), gen.haar_su2(rng)))
    ref = orc.run_circuit(gates, n)
    psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    l0 = s.launches()
    nf = s.apply_fused(gates, 6, prec_code(sv, name))
    s.check()
    assert s.launches() - l0 == nf + 2      # the blocks plus the two swap passes
    got = psi.cpu().numpy().astype(np.complex128)
    err = rel_l2(got, ref)
    print(f"[tc] {name} low targets relabelled n={n}: {nf} blocks, rel L2 {err:.3e}")
    assert err <= nf * PER_GATE[name]


@pytest.mark.parametrize("name", ["tf32", "bf16"])
def test_full_size_32q_fused_echo(env, name):
    """The 32-qubit brick wall (1900 gates, 32 GiB state) fused on the tensor
    cores, then its inverse fused the same way, returns |0...0>: amplitude 0
    comes back to 1 and the norm stays 1 within the per-block bound above --
    a check at the full size, where no complex128 oracle fits on the host."""
    torch, sv = env
    n = 32
    gates = gen.circuit_config2()
    inverse = [gen.Gate(g.targets, g.matrix.conj().T, g.controls, g.control_values) for g in reversed(gates)]
    psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    nf = s.apply_fused(gates, 6, prec_code(sv, name))
    nb = s.apply_fused(inverse, 6, prec_code(sv, name))
    s.check()
    a0 = complex(psi[0].item())
    norm = s.norm2()
    bound = (nf + nb) * PER_GATE[name]
    print(f"[tc] {name} 32q echo: {nf} + {nb} blocks, |a0 - 1| {abs(a0 - 1):.3e}, |norm - 1| {abs(norm - 1):.3e}, "
          f"bound {bound:.3e}")
    assert abs(a0 - 1) <= bound
    assert abs(norm - 1) <= 2 * bound
    s.close()
    del psi
    torch.cuda.empty_cache()
