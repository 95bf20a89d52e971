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
