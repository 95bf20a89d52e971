"""Tensor-core fused gates (tcgen05, TF32 and split-BF16) against the FP64 oracle.

No exactness is expected. The bounds come from the statistical rounding model
in ``tests/tc_error_model.py``: per fused block the relative L2 error has RMS
at most sigma (TF32 3.99e-4, split BF16 8.84e-6, from the operand rounding and
the FP32 accumulation), errors of different blocks add in quadrature, and the
tests allow twice the model -- both on the relative L2 error and, element by
element, on the largest amplitude error (a Gaussian tail over the state's
support, measured by its inverse participation ratio).
Expectation values and the norm then follow exactly: |<Z>' - <Z>| and
|<psi'|psi'> - 1| are at most 2 e + e^2 for a relative L2 error e of a unit
state. Every test prints the measured errors beside its bounds.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen
from tests.tc_error_model import l2_bound, max_abs_bound

pytestmark = pytest.mark.gpu


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


def wide_blocks(sv, gates, n, width):
    """Blocks of 5-6 qubits in the fusion plan: the ones the tensor cores apply."""
    return sum(1 for t, _ in sv.sv_fuse_plan(gates, n, width) if len(t) >= 5)


def check_state(name, got, ref, blocks, what):
    err = rel_l2(got, ref)
    mx = float(np.max(np.abs(got - ref)))
    b2, bm = l2_bound(name, blocks), max_abs_bound(name, blocks, ref)
    print(f"[tc] {name} {what}: {blocks} tensor-core blocks, rel L2 {err:.3e} (bound {b2:.3e}, "
          f"{err / b2:.2f}), max|d| {mx:.3e} (bound {bm:.3e}, {mx / bm:.2f})")
    assert err <= b2, f"{what}: relative L2 error {err:.3e} > {b2:.3e}"
    assert mx <= bm, f"{what}: max |d amplitude| {mx:.3e} > {bm:.3e}"
    return err


@pytest.mark.parametrize("name", ["tf32", "bf16"])
@pytest.mark.parametrize("n,targets", [(12, (2, 3, 5, 7, 8, 11)), (13, (0, 1, 2, 3, 4, 5)),
                                       (10, (4, 5, 6, 7, 8, 9)), (14, (1, 4, 6, 9, 12, 13)),
                                       (8, (0, 2, 3, 5, 6, 7)), (6, (0, 1, 2, 3, 4, 5)),
                                       # lowest target >= 2: one ragged tile (8 or 32 columns),
                                       # several tiles, far and contiguous targets
                                       (9, (3, 4, 5, 6, 7, 8)), (11, (3, 5, 6, 8, 9, 10)),
                                       (16, (5, 9, 10, 12, 14, 15)), (20, (3, 8, 12, 16, 18, 19)),
                                       (17, (11, 12, 13, 14, 15, 16)),
                                       # qubit 0 a target at 18 qubits, qubit 1 lowest at 19
                                       (18, (0, 2, 7, 11, 15, 17)), (19, (1, 2, 3, 9, 13, 18)),
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
    # the operand the kernel starts from is the complex64 copy of init; its own
    # rounding (2^-24) is far below either precision's and is left in
    check_state(name, psi.cpu().numpy().astype(np.complex128), ref, 1, f"n={n} targets={targets}")


@pytest.mark.parametrize("name", ["tf32", "bf16"])
@pytest.mark.parametrize("n,layers,width", [(15, 12, 5), (15, 12, 6), (20, 8, 6), (18, 10, 5)])
def test_fused_brick_wall(env, name, n, layers, width):
    torch, sv = env
    gates = gen.circuit_config2(n=n, layers=layers, seed=12)
    ref = orc.run_circuit(gates, n)
    psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    s.apply_fused(gates, width, prec_code(sv, name))
    s.check()
    blocks = wide_blocks(sv, gates, n, width)
    err = check_state(name, psi.cpu().numpy().astype(np.complex128), ref, blocks,
                      f"brick wall n={n} layers={layers} w={width}")
    b2 = l2_bound(name, blocks)
    zerr = float(np.max(np.abs(s.expectation_z_all() - orc.expect_z_all(ref))))
    print(f"[tc] {name}   max|d<Z>| {zerr:.3e}, |norm - 1| {abs(s.norm2() - 1):.3e} "
          f"(bound {2 * b2 + b2 * b2:.3e}; measured L2 gives {2 * err + err * err:.3e})")
    assert zerr <= 2 * b2 + b2 * b2
    assert abs(s.norm2() - 1) <= 2 * b2 + b2 * b2


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
    check_state(name, psi.cpu().numpy().astype(np.complex128), ref, wide_blocks(sv, gates, n, 6),
                f"low targets relabelled n={n}")


@pytest.mark.parametrize("name", ["tf32", "bf16"])
def test_full_size_32q_fused_echo(env, name):
    """The 32-qubit brick wall (1900 gates, 32 GiB state) fused on the tensor
    cores, then its inverse fused the same way, returns |0...0>: the distance
    ||psi - e_0|| (a relative L2 error, the state has unit norm) stays within
    the error model's bound for both halves' blocks -- a check at the full
    size, where no complex128 oracle fits on the host."""
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
    blocks = wide_blocks(sv, gates, n, 6) + wide_blocks(sv, inverse, n, 6)
    norm = s.norm2()
    a0 = complex(psi[0].item())
    psi[0] = 0
    rest = s.norm2()                      # sum over i > 0 of |psi_i|^2, in FP64
    dist = (abs(a0 - 1) ** 2 + rest) ** 0.5
    bound = l2_bound(name, blocks)
    print(f"[tc] {name} 32q echo: {nf} + {nb} blocks ({blocks} on tensor cores), ||psi - e0|| {dist:.3e} "
          f"(bound {bound:.3e}, {dist / bound:.2f}), |a0 - 1| {abs(a0 - 1):.3e}, |norm - 1| {abs(norm - 1):.3e}")
    assert bound < 0.02
    assert dist <= bound
    assert abs(norm - 1) <= 2 * bound + bound * bound
    s.close()
    del psi
    torch.cuda.empty_cache()
