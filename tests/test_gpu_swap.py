"""Index-bit swap (Table I) against the oracle applying SWAP gates."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return torch, sv


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("pairs", [[(0, 5)], [(1, 9), (3, 4)], [(2, 11), (0, 7), (5, 6), (8, 10)], [(10, 11)]])
def test_swap_index_bits_equals_swap_gates(env, dtype, pairs):
    torch, sv = env
    n = 12
    init = gen.random_state(n, 17)
    ref = init.copy()
    for a, b in pairs:
        orc.apply_gate(ref, [a, b], gen.gate_swap())
    dt = torch.complex64 if dtype == "c64" else torch.complex128
    psi = torch.from_numpy(init).to(dt).cuda()
    s = sv.StateVector(psi)
    s.swap_index_bits(pairs)
    got = psi.cpu().numpy().astype(np.complex128)
    # a permutation moves amplitudes without arithmetic: equal to the stored values
    want = ref.astype(np.complex64).astype(np.complex128) if dtype == "c64" else ref
    assert np.array_equal(got, want)
    s.swap_index_bits(pairs)
    assert np.array_equal(psi.cpu().numpy().astype(np.complex128),
                          init.astype(np.complex64).astype(np.complex128) if dtype == "c64" else init)


def test_swap_index_bits_rejects_bad_pairs(env):
    torch, sv = env
    psi = torch.zeros(1 << 6, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    for bad in ([(0, 0)], [(0, 6)], [(1, 2), (2, 3)], [(-1, 2)]):
        with pytest.raises(sv.SvError) as ei:
            s.swap_index_bits(bad)
        assert ei.value.code == 1
