"""Device-side failure detection without a GPU fault: a bounded wait that
nothing completes gives up after its clock budget, records SV_ERR_TIMEOUT in
the handle's status word, and the context stays usable afterwards."""
import numpy as np
import pytest

from paper_2308_01999_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import torch
    from paper_2308_01999_gb300 import sv
    psi = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    assert s.launches() == 0
    assert sv.sv_check_bounded_wait(s.handle, 2_000_000) == 5      # ~1 ms of clock, then SV_ERR_TIMEOUT
    assert sv.sv_check_device_status(s.handle) == 0                # the flag was cleared
    s.set_basis_state(0)
    s.apply([0], gen.gate_h())
    torch.cuda.synchronize()
    v = psi.cpu().numpy()
    assert np.allclose(v[:2], [2 ** -0.5, 2 ** -0.5]) and s.norm2() == pytest.approx(1.0, abs=1e-6)
    assert sv.sv_check_bounded_wait(s.handle, 10) == 1             # budget out of range


def test_batch_wait_for_another_cta_times_out_and_context_survives():
    """In the batched engine a CTA that takes a pass of a state above 14 qubits
    waits (bounded) for the previous pass, which other CTAs run. The diagnostic
    flag makes every such wait one pass longer than will ever finish: the wait
    gives up, the launch stops early, sv_batch_results reports SV_ERR_TIMEOUT,
    and the next launch of the same program runs normally."""
    import torch
    from paper_2308_01999_gb300 import sv
    n = 16
    gates = gen.ansatz_circuit(n, 2, gen.rng_for(3))
    paulis = 3 * np.eye(n, dtype=np.int32)[:2]
    b = sv.Batch(torch.cuda.current_stream())
    b.compile([(n, gates, paulis)], fusion_width=2)
    buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
    b.launch(buf, flags=sv.SV_BATCH_CHECK_WAIT)
    with pytest.raises(sv.SvError) as ei:
        b.results()
    assert ei.value.code == 5
    b.launch(buf)
    good = b.results()[0]
    psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    s.apply_circuit(gates)
    want = s.expectation_pauli(paulis, np.tile(np.arange(n, dtype=np.int32), (2, 1)))
    assert np.all(np.abs(good - want) <= 1e-6)
    b.close()
    s.close()
