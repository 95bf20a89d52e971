"""GPU parity: libsv.so (through its C ABI) against the CPU oracle, element by
element on the same seeded inputs.

Tolerances (stated by the build's target): max |d amplitude| <= 1e-12 for
complex128 and <= 1e-5 for complex64; expectation values and probabilities
within 1e-6 * max(1, |ref|) for complex64 and 1e-12 for complex128.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

AMP_TOL = {"c128": 1e-12, "c64": 1e-5}
EXP_TOL = {"c128": 1e-12, "c64": 1e-6}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return torch, sv


def tdtype(torch, name):
    return torch.complex128 if name == "c128" else torch.complex64


def make_state(env, n, name, init=None):
    torch, sv = env
    if init is None:
        psi = torch.zeros(1 << n, dtype=tdtype(torch, name), device="cuda")
        s = sv.StateVector(psi)
        s.set_basis_state(0)
    else:
        psi = torch.from_numpy(init.astype(np.complex128)).to(tdtype(torch, name)).cuda()
        s = sv.StateVector(psi)
    return psi, s


def host(psi):
    return psi.cpu().numpy().astype(np.complex128)


def assert_amps(got, ref, name, what=""):
    err = np.max(np.abs(got - ref)) if ref.size else 0.0
    assert err <= AMP_TOL[name], f"{what} max|d amp| = {err:.3e} > {AMP_TOL[name]}"


def assert_exp(got, ref, name, what=""):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    bound = EXP_TOL[name] * np.maximum(1.0, np.abs(ref))
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{what} expectation mismatch: {got[bad]} vs {ref[bad]}"


NAMES = ["c128", "c64"]


@pytest.mark.parametrize("name", NAMES)
def test_config0_circuit_amplitudes_and_z(env, name):
    n = 16
    gates = gen.circuit_config0(0)
    ref = orc.run_circuit(gates, n)
    psi, s = make_state(env, n, name)
    s.apply_circuit(gates)
    assert_amps(host(psi), ref, name, "config0")
    z = s.expectation_z_all()
    assert_exp(z, orc.expect_z_all(ref), name, "<Z_q>")
    assert abs(s.norm2() - 1) <= EXP_TOL[name]


@pytest.mark.parametrize("name", NAMES)
def test_one_qubit_gate_on_every_position(env, name):
    n = 13
    rng = gen.rng_for(21)
    init = gen.random_state(n, 21)
    ref = init.copy()
    psi, s = make_state(env, n, name, init)
    for q in range(n):
        u = gen.haar_su2(rng)
        s.apply([q], u)
        orc.apply_gate(ref, [q], u)
    assert_amps(host(psi), ref, name, "1q sweep")


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_dense_gates_random_targets_and_controls(env, name, k):
    n = 11
    rng = gen.rng_for(100 + k)
    init = gen.random_state(n, 100 + k)
    ref = init.copy()
    psi, s = make_state(env, n, name, init)
    for it in range(8):
        c = int(rng.integers(0, min(3, n - k) + 1))
        qs = [int(x) for x in rng.choice(n, k + c, replace=False)]
        if it == 0:
            qs = list(range(k + c))            # lowest bits: target (or control) on bit 0
        elif it == 1:
            qs = list(range(n - k - c, n))     # highest bits
        t, ctl = qs[:k], qs[k:]
        cv = [int(v) for v in rng.integers(0, 2, size=c)]
        m = gen.random_gate_dense(rng, k)
        adj = bool(it % 3 == 2)
        s.apply(t, m, ctl, cv, adjoint=adj)
        orc.apply_gate(ref, t, m.conj().T if adj else m, ctl, cv)
    assert_amps(host(psi), ref, name, f"k={k}")


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("n", [3, 4, 5, 6, 9, 10, 14, 17])
def test_dense_gates_on_low_target_runs(env, name, n):
    """Dense 2- to 4-qubit gates with qubit 1 among the targets (staged through
    shared memory by warps for complex64, when every control lies above the
    staged block), with and without controls (high and low), targets given in
    any order, on states from fewer groups than a warp holds to many blocks."""
    rng = gen.rng_for(300 + n)
    init = gen.random_state(n, 300 + n)
    ref = init.copy()
    psi, s = make_state(env, n, name, init)
    cases = [(0, 1, 2), (0, 1, 2, 3), (0, 1, 5), (0, 1, 2, 7), (0, 1, 4, 6), (2, 0, 1), (3, 1, 0, 2),
             (1, 2, 3, 4), (1, 5), (1, 2), (0, 1), (1, 9, 12), (4, 1, 8, 13), (1, 3, 5, 7)]
    for it, t in enumerate(cases):
        if max(t) >= n:
            continue
        free = [q for q in range(n) if q not in t]
        c = min(len(free), it % 3, max(0, n - len(t) - 1))
        ctl = [int(x) for x in rng.choice(free, c, replace=False)] if c else []
        cv = [int(v) for v in rng.integers(0, 2, size=c)]
        m = gen.random_gate_dense(rng, len(t))
        adj = bool(it % 2)
        s.apply(list(t), m, ctl, cv, adjoint=adj)
        orc.apply_gate(ref, list(t), m.conj().T if adj else m, ctl, cv)
    assert_amps(host(psi), ref, name, f"low runs n={n}")


@pytest.mark.parametrize("name", NAMES)
def test_structured_gates(env, name):
    """Diagonal, generalized-permutation and control-revealing dense matrices
    (exercises the structure analysis), incl. bit-0 controls and targets."""
    n = 10
    rng = gen.rng_for(7)
    init = gen.random_state(n, 7)
    ref = init.copy()
    psi, s = make_state(env, n, name, init)
    ops = []
    for a, b in [(0, 1), (1, 0), (5, 9), (9, 2), (3, 0)]:
        ops.append(gen.dense_form(gen.cz(a, b)))
        ops.append(gen.dense_form(gen.cnot(a, b)))
        ops.append(gen.dense_form(gen.crz(a, b, float(rng.uniform(0, 6.28)))))
        ops.append(gen.cz(a, b))
        ops.append(gen.cnot(a, b))
        ops.append(gen.crz(a, b, 1.1))
    for k in range(1, 7):
        qs = [int(x) for x in rng.choice(n, k + 1, replace=False)]
        d = np.exp(1j * rng.uniform(0, 6.28, size=1 << k))
        ops.append(gen.Gate(tuple(qs[:k]), np.diag(d), (qs[k],), (int(rng.integers(0, 2)),)))
        ops.append(gen.Gate(tuple(qs[:k]), np.diag(d)))
        perm = rng.permutation(1 << k)
        pm = np.zeros((1 << k, 1 << k), dtype=np.complex128)
        pm[np.arange(1 << k), perm] = np.exp(1j * rng.uniform(0, 6.28, size=1 << k))
        ops.append(gen.Gate(tuple(qs[:k]), pm, (qs[k],), (1,)))
        ops.append(gen.Gate(tuple(qs[:k]), pm))
    ops.append(gen.Gate((4,), gen.gate_phase(0.3)))
    ops.append(gen.Gate((0,), gen.gate_phase(-0.7), (1, 2), (1, 0)))
    ops.append(gen.Gate((2, 7), np.eye(4)))
    ops.append(gen.Gate((0, 5), gen.gate_swap()))
    ops.append(gen.Gate((0,), gen.gate_y(), (3,), (0,)))
    for g in ops:
        s.apply_gate(g)
        orc.apply(ref, g)
    assert_amps(host(psi), ref, name, "structured")


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("n,k,c", [(1, 1, 0), (2, 2, 0), (2, 1, 1), (3, 2, 1), (6, 6, 0), (7, 6, 1), (7, 6, 0),
                                   (8, 5, 3), (5, 4, 1), (4, 3, 0)])
def test_edge_sizes(env, name, n, k, c):
    rng = gen.rng_for(1000 + 10 * n + k + c)
    init = gen.random_state(n, n + k + c)
    ref = init.copy()
    psi, s = make_state(env, n, name, init)
    for _ in range(4):
        qs = [int(x) for x in rng.choice(n, k + c, replace=False)]
        m = gen.random_gate_dense(rng, k)
        cv = [int(v) for v in rng.integers(0, 2, size=c)]
        s.apply(qs[:k], m, qs[k:], cv)
        orc.apply_gate(ref, qs[:k], m, qs[k:], cv)
    assert_amps(host(psi), ref, name, f"n={n} k={k} c={c}")


@pytest.mark.parametrize("name", NAMES)
def test_pauli_expectations(env, name):
    n = 12
    rng = gen.rng_for(55)
    init = gen.random_state(n, 55)
    psi, s = make_state(env, n, name, init)
    paulis, sites = gen.random_pauli_strings(n, 40, rng)
    extra = np.zeros((8, n), dtype=np.int32)
    extra[1, 0] = 1                 # X on qubit 0 only (partner in the same 16-byte unit)
    extra[2, :] = 2                 # all Y
    extra[3, :] = 3                 # all Z
    extra[4, 1] = 2                 # Y on qubit 1
    extra[5, [0, 5, 11]] = [2, 1, 3]
    extra[6, n - 1] = 1
    extra[7, [0, 1]] = [1, 1]
    paulis = np.vstack([paulis, extra])
    sites = np.tile(np.arange(n, dtype=np.int32), (paulis.shape[0], 1))
    got = s.expectation_pauli(paulis, sites)
    ref_state = host(psi)   # the state as stored in this precision
    want = np.array([orc.expect_pauli(ref_state, p, q).real for p, q in zip(paulis, sites)])
    assert_exp(got, want, name, "pauli")
    # a subset of sites, in shuffled order
    sub = np.array([[7, 2, 9]], dtype=np.int32)
    ps = np.array([[2, 1, 3]], dtype=np.int32)
    assert_exp(s.expectation_pauli(ps, sub), [orc.expect_pauli(ref_state, ps[0], sub[0]).real], name, "subset")
    # the empty string is the norm
    e = s.expectation_pauli(np.zeros((1, 0), np.int32), np.zeros((1, 0), np.int32))
    assert abs(e[0] - orc.norm2(ref_state)) <= EXP_TOL[name]


@pytest.mark.parametrize("name", NAMES)
def test_measurement_probabilities_and_collapse(env, name):
    n = 14
    psi, s = make_state(env, n, name)
    s.apply_circuit(gen.ghz_circuit(n))
    p0, p1 = s.measure_probs([5])
    assert abs(p0 - 0.5) <= EXP_TOL[name] and abs(p1 - 0.5) <= EXP_TOL[name]
    p0, p1 = s.measure_probs([2, 9])
    assert abs(p0 - 1) <= EXP_TOL[name] and p1 <= EXP_TOL[name]
    out = s.measure([3], 0.75, collapse=True)
    assert out == 1
    v = host(psi)
    assert abs(abs(v[-1]) - 1) <= AMP_TOL[name] and np.max(np.abs(v[:-1])) <= AMP_TOL[name]
    # random state: probabilities, measurement outcome and collapse vs the oracle
    init = gen.random_state(n, 77)
    psi, s = make_state(env, n, name, init)
    ref = host(psi)
    rng = gen.rng_for(78)
    for m in (1, 2, 5):
        qs = [int(x) for x in rng.choice(n, m, replace=False)]
        p0, p1 = s.measure_probs(qs)
        w0, w1 = orc.parity_probs(ref, qs)
        assert_exp([p0, p1], [w0, w1], name, "probs")
    qs = [1, 6, 13]
    r = 0.37
    out = s.measure(qs, r, collapse=True)
    want = orc.measure(ref, qs, r, collapse=True)
    assert out == want
    assert_amps(host(psi), ref, name, "collapse")
    assert abs(s.norm2() - 1) <= EXP_TOL[name]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("width", [2, 3, 4, 5, 6])
def test_fused_native_matches_unfused_oracle(env, name, width):
    n = 13
    gates = gen.circuit_config2(n=n, layers=10, seed=9) + gen.circuit_config1(n=n, depth=3, seed=10)
    ref = orc.run_circuit(gates, n)
    psi, s = make_state(env, n, name)
    nf = s.apply_fused(gates, width)
    assert nf < len(gates)
    assert_amps(host(psi), ref, name, f"fused w={width}")


def test_full_size_28q_whole_circuit(env):
    """The 28-qubit complex64 benchmark circuit, all 40 layers (1680 gates), in
    the launch configuration the benchmark times (one launch per gate), then
    the benchmark's reductions: every amplitude is compared with the complex128
    oracle run of the same circuit, and <Z_q>, the eight random Pauli strings
    (X and Y sites included, so the compensated single-precision pair sums run
    over 2^27 pairs per string) and the parity probabilities are compared with
    the oracle both on the oracle's own state (end to end) and on the GPU's
    final state (the reduction alone)."""
    orc.set_threads(0)
    n = 28
    gates = gen.circuit_config1()
    assert len(gates) == 1680
    psi, s = make_state(env, n, "c64")
    s.apply_circuit(gates)
    z_gpu = s.expectation_z_all()
    paulis, sites = gen.random_pauli_strings(n, 8, gen.rng_for(101))    # the benchmark's strings
    assert all(any(c in (1, 2) for c in p) for p in paulis)
    e_gpu = s.expectation_pauli(paulis, sites)
    pr_gpu = s.measure_probs([0, n - 1])
    got = psi.cpu().numpy()
    s.close()
    ref = orc.run_circuit(gates, n)
    err = 0.0
    chunk = 1 << 24
    for a in range(0, 1 << n, chunk):
        err = max(err, float(np.max(np.abs(got[a:a + chunk].astype(np.complex128) - ref[a:a + chunk]))))
    print(f"[28q] whole circuit: max|d amp| {err:.3e}")
    assert err <= AMP_TOL["c64"], err
    zq = (0, 13, n - 1)
    assert_exp(z_gpu[list(zq)], [orc.expect_pauli(ref, [3], [q]).real for q in zq], "c64", "28q <Z>")
    want = np.array([orc.expect_pauli(ref, p, q).real for p, q in zip(paulis, sites)])
    assert_exp(e_gpu, want, "c64", "28q Pauli strings, oracle state")
    assert_exp(pr_gpu, orc.parity_probs(ref, [0, n - 1]), "c64", "28q parity probabilities")
    del ref
    mine = got.astype(np.complex128)
    del got
    own = np.array([orc.expect_pauli(mine, p, q).real for p, q in zip(paulis, sites)])
    print(f"[28q] Pauli strings: max|d| vs oracle state {np.max(np.abs(e_gpu - want)):.3e}, "
          f"vs the GPU's own state {np.max(np.abs(e_gpu - own)):.3e}")
    assert_exp(e_gpu, own, "c64", "28q Pauli strings, GPU state")


def test_full_size_28q_echo(env):
    """The whole 28-qubit depth-40 circuit followed by its inverse returns |0...0>:
    a property that holds at any size (norm preserved, amplitude 0 back to 1)."""
    n = 28
    gates = gen.circuit_config1()
    psi, s = make_state(env, n, "c64")
    s.apply_circuit(gates)
    assert abs(s.norm2() - 1) < 1e-4
    for g in reversed(gates):
        s.apply_gate(g, adjoint=True)
    a0 = complex(psi[0].item())
    assert abs(a0 - 1) < 1e-4, a0
    assert abs(s.norm2() - 1) < 1e-4


@pytest.mark.parametrize("name", NAMES)
def test_reductions_are_deterministic(env, name):
    n = 20
    init = gen.random_state(n, 5)
    psi, s = make_state(env, n, name, init)
    paulis, sites = gen.random_pauli_strings(n, 12, gen.rng_for(6))
    a = s.expectation_pauli(paulis, sites)
    b = s.expectation_pauli(paulis, sites)
    assert np.array_equal(a, b)
    assert s.measure_probs([3, 17]) == s.measure_probs([3, 17])
    ref = host(psi)
    want = np.array([orc.expect_pauli(ref, p, q).real for p, q in zip(paulis, sites)])
    assert_exp(a, want, name, "n=20")


def test_invalid_arguments_are_rejected(env):
    torch, sv = env
    psi, s = make_state(env, 5, "c64")
    bad = [
        lambda: s.apply([5], np.eye(2)),
        lambda: s.apply([1, 1], np.eye(4)),
        lambda: s.apply([0], np.eye(2), [0]),
        lambda: s.apply([0], np.eye(2), [1], [2]),
        lambda: s.expectation_pauli(np.array([[1, 1]]), np.array([[2, 2]])),
        lambda: s.expectation_pauli(np.array([[4]]), np.array([[0]])),
        lambda: s.measure_probs([]),
        lambda: s.collapse([0], 0, 0.0),
        lambda: s.measure([0], 1.0),
    ]
    for f in bad:
        with pytest.raises(sv.SvError) as ei:
            f()
        assert ei.value.code == 1
    big = gen.Gate(tuple(range(5)), gen.random_gate_dense(gen.rng_for(1), 5))
    psi2, s2 = make_state(env, 6, "c128")
    with pytest.raises(sv.SvError) as ei:
        s2.apply_fused([big], 5, sv.SV_PREC_TF32)
    assert ei.value.code == 2
    n0 = s.launches()
    s.apply([0], gen.gate_h())
    assert s.launches() == n0 + 1
    s.check()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("n", [3, 4, 11, 12, 13, 21, 24])
def test_z_expectations_of_every_qubit_in_one_pass(env, name, n):
    """Strings of identities and single Z (the <Z_q> request) take the one-pass
    kernel; compare with the oracle, in any order, with repeats and the norm."""
    init = gen.random_state(n, 500 + n)
    psi, s = make_state(env, n, name, init)
    ref = host(psi)
    z = s.expectation_z_all()
    assert_exp(z, orc.expect_z_all(ref), name, f"<Z> n={n}")
    order = [n - 1, 0, n // 2, 0]
    paulis = np.zeros((len(order) + 1, n), np.int32)
    for r, q in enumerate(order):
        paulis[r, q] = 3
    sites = np.tile(np.arange(n, dtype=np.int32), (paulis.shape[0], 1))
    got = s.expectation_pauli(paulis, sites)
    want = [orc.expect_pauli(ref, p, q).real for p, q in zip(paulis, sites)]
    assert_exp(got, want, name, "mixed single-Z strings")


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("width,dwidth", [(2, 4), (3, 6), (4, 6)])
def test_dense_and_diagonal_fusion(env, name, width, dwidth):
    """Diagonal gates fused into diagonal blocks of up to dwidth qubits, the
    rest into dense blocks of up to width qubits (QAOA-style circuit)."""
    n = 13
    gates = gen.qaoa_circuit(n, 3, seed=width * 10 + dwidth)
    ref = orc.run_circuit(gates, n)
    psi, s = make_state(env, n, name)
    nf = s.apply_fused(gates, width, max_fused_diagonal_qubits=dwidth)
    assert nf < len(gates)
    assert_amps(host(psi), ref, name, f"fused w={width} diag={dwidth}")


def test_async_host_copies_round_trip(env):
    """sv_copy_from_host_async / sv_copy_to_host_async enqueue on the handle's
    stream: a state copied in, a gate applied and the result copied out equal the
    synchronous path, and the calls return before the stream has finished."""
    torch, sv = env
    n = 20
    init = gen.random_state(n, 77).astype(np.complex64)
    h_in = torch.from_numpy(init.copy()).pin_memory()
    h_out = torch.empty(1 << n, dtype=torch.complex64).pin_memory()
    stream = torch.cuda.Stream()
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi, stream)
    g = gen.Gate((3,), gen.haar_su2(gen.rng_for(78)))
    sv.sv_copy_from_host_async(s.handle, h_in.data_ptr())
    s.apply_gate(g)
    sv.sv_copy_to_host_async(s.handle, h_out.data_ptr())
    stream.synchronize()
    ref = init.astype(np.complex128)
    orc.apply(ref, g)
    assert np.max(np.abs(h_out.numpy().astype(np.complex128) - ref)) <= 1e-6
    sync_out = np.empty(1 << n, dtype=np.complex64)
    sv.sv_copy_to_host(s.handle, sync_out.ctypes.data)
    assert np.array_equal(sync_out, h_out.numpy())
    s.close()


@pytest.mark.parametrize("name", NAMES)
def test_empty_inputs_launch_nothing(env, name):
    """No gates, no strings, no samples: every call succeeds, launches no
    kernel and leaves the state as it was."""
    torch, sv = env
    n = 9
    psi, s = make_state(env, n, name, gen.random_state(n, 99))
    before = psi.clone()
    l0 = s.launches()
    s.apply_circuit([])
    assert s.apply_fused([], 6) == 0
    if name == "c64":
        assert s.apply_fused([], 6, sv.SV_PREC_SPLIT_BF16) == 0
    assert s.expectation_pauli(np.zeros((0, n), np.int32), np.zeros((0, n), np.int32)).shape == (0,)
    assert len(s.sample(np.zeros(0))) == 0
    assert s.launches() == l0
    assert torch.equal(psi, before)
