"""The allocation-free expectation entry point, called through the C ABI.

sv_expectation_pauli_noalloc serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or they cannot afford the
allocation's latency and device synchronisation): it takes no handle and keeps
its scratch in a fixed device array inside the library. Its results must equal
those of the handle-based sv_expectation_pauli on the same state, call after
call (the shared scratch keeps the previous call's contents).

This file is collected last on purpose, and passes both alone in a fresh
process and after the other GPU tests.
"""
import numpy as np
import pytest

from paper_2308_01999_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-6}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return torch, sv


@pytest.mark.parametrize("name", ["c64", "c128"])
def test_noalloc_matches_handle_entry_point_twice(env, name):
    torch, sv = env
    n = 18
    dt = torch.complex64 if name == "c64" else torch.complex128
    code = sv.SV_C64 if name == "c64" else sv.SV_C128
    psi = torch.from_numpy(gen.random_state(n, 31)).to(dt).cuda()
    stream = torch.cuda.current_stream()
    s = sv.StateVector(psi, stream)
    rng = gen.rng_for(32)
    paulis, sites = gen.random_pauli_strings(n, 20, rng)
    zs = np.full((n, 1), 3, np.int32)
    zq = np.arange(n, dtype=np.int32)[:, None]
    for p, q in ((paulis, sites), (zs, zq)):
        want = s.expectation_pauli(p, q)
        for _ in range(2):   # two calls in a row share the static scratch
            got = sv.sv_expectation_pauli_noalloc(n, code, psi.data_ptr(), stream.cuda_stream, p, q)
            bound = TOL[name] * np.maximum(1.0, np.abs(want))
            assert np.all(np.abs(got - want) <= bound), (got, want)
    s.close()


def test_noalloc_rejects_too_many_strings(env):
    torch, sv = env
    psi = torch.zeros(1 << 4, dtype=torch.complex64, device="cuda")
    p = np.zeros((4097, 1), np.int32)
    q = np.zeros((4097, 1), np.int32)
    with pytest.raises(sv.SvError) as ei:
        sv.sv_expectation_pauli_noalloc(4, sv.SV_C64, psi.data_ptr(), 0, p, q)
    assert ei.value.code == 3
    with pytest.raises(sv.SvError) as ei:
        sv.sv_expectation_pauli_noalloc(4, sv.SV_C64, psi.data_ptr(), 0, np.array([[1]]), np.array([[4]]))
    assert ei.value.code == 1
