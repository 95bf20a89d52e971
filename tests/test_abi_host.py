"""CPU-only checks of libsv.so: it loads, exports every entry point that
include/sv.h declares, and its host-side fusion pass (Sec. II-B) composes
blocks that reproduce the unfused circuit under the oracle. No GPU call."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sv():
    from paper_2308_01999_gb300 import _build
    _build.build()
    from paper_2308_01999_gb300 import sv as mod
    mod.lib()
    return mod


def header_functions():
    text = open(os.path.join(ROOT, "include", "sv.h")).read()
    return sorted(set(re.findall(r"^SV_API\s+[^()]*?\b(sv_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_entry_point(sv):
    declared = header_functions()
    assert len(declared) >= 18
    L = sv.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(sv.EXPORTED) == declared


def test_binding_constants_match_the_header(sv):
    """Every #define of include/sv.h that the binding restates has the same value."""
    text = open(os.path.join(ROOT, "include", "sv.h")).read()
    defines = {k: int(v) for k, v in re.findall(r"^#define\s+(SV_\w+)\s+(\d+)\b", text, flags=re.M)}
    shared = [k for k in defines if hasattr(sv, k)]
    assert {"SV_BATCH_MAX_QUBITS", "SV_BATCH_TILE_QUBITS", "SV_BATCH_KEEP_STATES", "SV_BATCH_CHECK_WAIT"} <= set(shared)
    for k in shared:
        assert getattr(sv, k) == defines[k], k


def test_status_strings(sv):
    assert sv.sv_status_string(0) == "SV_OK"
    assert sv.sv_status_string(1) == "SV_ERR_INVALID_ARGUMENT"
    assert sv.sv_status_string(5) == "SV_ERR_TIMEOUT"
    assert sv.sv_status_string(99) == "SV_ERR_UNKNOWN"


def _apply_plan(plan, n):
    psi = orc.zero_state(n)
    for targets, m in plan:
        orc.apply_gate(psi, list(targets), m)
    return psi


@pytest.mark.parametrize("width", [1, 2, 3, 4, 5, 6])
def test_fusion_plan_reproduces_unfused_circuit(sv, width):
    n = 9
    gates = gen.layered_random_circuit(n, 6, seed=40 + width, kinds=("cz", "cnot", "crz"))
    ref = orc.run_circuit(gates, n)
    plan = sv.sv_fuse_plan(gates, n, width)
    assert all(len(t) <= max(width, 2) for t, _ in plan)
    if width >= 4:
        assert len(plan) < len(gates) / 3
    got = _apply_plan(plan, n)
    np.testing.assert_allclose(got, ref, atol=1e-12, rtol=0)


def test_fusion_of_brick_wall_and_controls(sv):
    n = 10
    gates = gen.circuit_config2(n=n, layers=8, seed=5)
    rng = gen.rng_for(6)
    # add multi-qubit and multi-control gates, incl. control value 0
    for _ in range(10):
        qs = [int(x) for x in rng.choice(n, 4, replace=False)]
        gates.append(gen.Gate((qs[0], qs[1]), gen.random_gate_dense(rng, 2), (qs[2], qs[3]), (0, 1)))
    ref = orc.run_circuit(gates, n)
    for w in (3, 5, 6):
        plan = sv.sv_fuse_plan(gates, n, w)
        np.testing.assert_allclose(_apply_plan(plan, n), ref, atol=1e-12, rtol=0)


def test_fusion_rejects_bad_gates(sv):
    bad = [gen.Gate((0, 0), np.eye(4))]
    with pytest.raises(sv.SvError):
        sv.sv_fuse_plan(bad, 3, 2)
    with pytest.raises(sv.SvError):
        sv.sv_fuse_plan([gen.Gate((3,), np.eye(2))], 3, 2)
    with pytest.raises(sv.SvError):
        sv.sv_fuse_plan([gen.Gate((0,), np.eye(2))], 3, 7)


@pytest.mark.parametrize("width,dwidth", [(2, 4), (3, 6), (4, 5), (6, 6)])
def test_diagonal_fusion_plan_reproduces_circuit(sv, width, dwidth):
    n = 10
    gates = gen.qaoa_circuit(n, 2, seed=width + dwidth)
    ref = orc.run_circuit(gates, n)
    plan = sv.sv_fuse_plan(gates, n, width, max_fused_diagonal_qubits=dwidth)
    plain = sv.sv_fuse_plan(gates, n, width)
    np.testing.assert_allclose(_apply_plan(plan, n), ref, atol=1e-12, rtol=0)
    diag = [m for _, m in plan if np.count_nonzero(m - np.diag(np.diag(m))) == 0 and m.shape[0] > 2]
    assert diag and max(m.shape[0] for m in diag) <= (1 << dwidth)
    assert max(len(t) for t, _ in plain) <= width
