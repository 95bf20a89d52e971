"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test compares the C oracle with something fixed by the mathematics:
closed forms (GHZ, the QFT of a basis state, product states), textbook
identities (sequential one-qubit gates equal their Kronecker product; a
controlled gate equals its block-diagonal operator), brute-force 2^n x 2^n
operators built with numpy.kron, an independent numpy tensor contraction,
and invariants (unitarity, the U then U^dagger echo, p_even + p_odd = norm).
A transposed matrix, a reversed target order, a wrong control value, a lost
conjugate or a wrong Y sign each fails at least one of them (see
test_oracle_mutations.py, which plants those mistakes in a copy of the oracle).
"""
import numpy as np
import pytest

from oracle import np_ref
from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen


def _rand_qubits(rng, n, m):
    return [int(x) for x in rng.choice(n, size=m, replace=False)]


@pytest.mark.parametrize("seed", range(12))
def test_apply_matches_numpy_tensor_contraction(seed):
    rng = gen.rng_for(100 + seed)
    n = 7
    psi = gen.random_state(n, seed)
    ref = psi.copy()
    for _ in range(6):
        k = int(rng.integers(1, 5))
        c = int(rng.integers(0, min(3, n - k) + 1))
        qs = _rand_qubits(rng, n, k + c)
        t, ctl = qs[:k], qs[k:]
        cv = [int(v) for v in rng.integers(0, 2, size=c)]
        m = gen.random_gate_dense(rng, k)
        orc.apply_gate(psi, t, m, ctl, cv)
        ref = np_ref.apply_gate_np(ref, n, t, m, ctl, cv)
    np.testing.assert_allclose(psi, ref, atol=1e-13, rtol=0)


@pytest.mark.parametrize("n,lo,k", [(6, 0, 1), (6, 3, 2), (7, 1, 3), (8, 2, 4), (8, 0, 6), (8, 5, 3)])
def test_contiguous_gate_equals_kron_operator(n, lo, k):
    rng = gen.rng_for(7 * n + lo + k)
    m = gen.random_gate_dense(rng, k)
    psi = gen.random_state(n, n + lo)
    want = np_ref.kron_operator_contiguous(n, lo, m) @ psi
    orc.apply_gate(psi, list(range(lo, lo + k)), m)
    np.testing.assert_allclose(psi, want, atol=1e-13, rtol=0)


def test_target_order_sequential_equals_kron():
    # A on q0 then B on q1 equals kron(B, A) on targets [q0, q1]: the matrix's
    # more significant index bit belongs to targets[1].
    rng = gen.rng_for(5)
    n = 6
    for q0, q1 in [(0, 1), (4, 1), (2, 5), (5, 0)]:
        A, B = gen.haar_su2(rng), gen.haar_su2(rng)
        psi = gen.random_state(n, q0 * 10 + q1)
        seq = psi.copy()
        orc.apply_gate(seq, [q0], A)
        orc.apply_gate(seq, [q1], B)
        orc.apply_gate(psi, [q0, q1], np.kron(B, A))
        np.testing.assert_allclose(psi, seq, atol=1e-14, rtol=0)


@pytest.mark.parametrize("cval", [0, 1])
def test_controlled_gate_equals_block_operator(cval):
    rng = gen.rng_for(11 + cval)
    n = 5
    for c, t in [(0, 1), (3, 1), (4, 0), (1, 4)]:
        U = gen.haar_su2(rng)
        blk = np.zeros((4, 4), dtype=np.complex128)
        eye = np.eye(2)
        # targets [t, c]: index bit 1 is the control
        blk[:2, :2] = U if cval == 0 else eye
        blk[2:, 2:] = U if cval == 1 else eye
        psi = gen.random_state(n, c + 7 * t)
        ref = psi.copy()
        orc.apply_gate(psi, [t], U, [c], [cval])
        orc.apply_gate(ref, [t, c], blk)
        np.testing.assert_allclose(psi, ref, atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [2, 3, 4, 7])
def test_ghz_closed_form(n):
    psi = orc.run_circuit(gen.ghz_circuit(n), n)
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = want[-1] = 1 / np.sqrt(2)
    np.testing.assert_allclose(psi, want, atol=1e-15, rtol=0)
    for q in range(n):
        assert abs(orc.expect_pauli(psi, [3], [q])) < 1e-15
    for a in range(n):
        for b in range(a + 1, n):
            assert abs(orc.expect_pauli(psi, [3, 3], [a, b]) - 1) < 1e-14
    assert abs(orc.expect_pauli(psi, [1] * n, list(range(n))) - 1) < 1e-14
    # Y^n|0..0> = i^n |1..1>, Y^n|1..1> = (-i)^n |0..0>  =>  <Y^n> = Re(i^n)
    assert abs(orc.expect_pauli(psi, [2] * n, list(range(n))) - (1j ** n).real) < 1e-14
    # one Y and the rest X: <.> = Re(i * (-1)^0 ...) -> (i - i)/2 = 0 for n >= 2
    assert abs(orc.expect_pauli(psi, [2] + [1] * (n - 1), list(range(n)))) < 1e-14


@pytest.mark.parametrize("n", [3, 5, 8])
def test_qft_of_basis_state_closed_form(n):
    N = 1 << n
    for x in [0, 1, N - 1, (5 * N) // 7]:
        psi = np.zeros(N, dtype=np.complex128)
        psi[x] = 1
        orc.run_circuit(gen.qft_circuit(n), n, psi)
        y = np.arange(N)
        want = np.exp(2j * np.pi * ((x * y) % N) / N) / np.sqrt(N)
        np.testing.assert_allclose(psi, want, atol=1e-13, rtol=0)
        np.testing.assert_allclose(np.abs(psi), 1 / np.sqrt(N), atol=1e-13)


def test_unitarity_and_echo():
    n = 9
    rng = gen.rng_for(3)
    psi0 = gen.random_state(n, 3)
    psi = psi0.copy()
    gates = []
    for _ in range(25):
        k = int(rng.integers(1, 4))
        c = int(rng.integers(0, 3))
        qs = _rand_qubits(rng, n, k + c)
        g = gen.Gate(tuple(qs[:k]), gen.random_gate_dense(rng, k), tuple(qs[k:]),
                     tuple(int(v) for v in rng.integers(0, 2, size=c)))
        gates.append(g)
        orc.apply(psi, g)
        assert abs(orc.norm2(psi) - 1) < 1e-13
    for g in reversed(gates):
        orc.apply_gate(psi, g.targets, g.matrix.conj().T, g.controls, g.control_values)
    np.testing.assert_allclose(psi, psi0, atol=1e-13, rtol=0)


def test_product_state_expectations():
    # |psi> = (x)_q U_q|0>: <Z_q> = |a|^2 - |b|^2, <X_q> = 2 Re(conj(a) b),
    # <Y_q> = 2 Im(conj(a) b) with (a, b) the first column of U_q; a Pauli
    # string's value is the product over its sites.
    n = 6
    rng = gen.rng_for(17)
    us = [gen.haar_su2(rng) for _ in range(n)]
    psi = orc.zero_state(n)
    for q, u in enumerate(us):
        orc.apply_gate(psi, [q], u)
    single = []
    for u in us:
        a, b = u[0, 0], u[1, 0]
        single.append({0: 1.0, 1: 2 * (np.conj(a) * b).real, 2: 2 * (np.conj(a) * b).imag,
                       3: abs(a) ** 2 - abs(b) ** 2})
    for q in range(n):
        for p in (1, 2, 3):
            assert abs(orc.expect_pauli(psi, [p], [q]) - single[q][p]) < 1e-14
    paulis, sites = gen.random_pauli_strings(n, 20, rng)
    for ps, ss in zip(paulis, sites):
        want = np.prod([single[s][p] for p, s in zip(ps, ss)])
        got = orc.expect_pauli(psi, ps, ss)
        assert abs(got - want) < 1e-13
        assert abs(got.imag) < 1e-15


@pytest.mark.parametrize("n", [1, 3, 6, 8])
def test_pauli_expectation_equals_explicit_operator(n):
    rng = gen.rng_for(40 + n)
    psi = gen.random_state(n, 40 + n)
    paulis, sites = gen.random_pauli_strings(n, 16, rng)
    for ps, ss in zip(paulis, sites):
        P = np_ref.pauli_operator(n, ps, ss)
        want = np.vdot(psi, P @ psi)
        got = orc.expect_pauli(psi, ps, ss)
        assert abs(got - want) < 1e-13
        assert abs(got.imag) < 1e-14
    # subset of sites, in a shuffled order
    sub = [int(x) for x in rng.permutation(n)[: max(1, n // 2)]]
    ps = [int(x) for x in rng.integers(1, 4, size=len(sub))]
    want = np.vdot(psi, np_ref.pauli_operator(n, ps, sub) @ psi)
    assert abs(orc.expect_pauli(psi, ps, sub) - want) < 1e-13


def test_identity_string_is_the_norm():
    psi = gen.random_state(7, 2) * 1.5
    assert abs(orc.expect_pauli(psi, [0] * 7, list(range(7))) - orc.norm2(psi)) < 1e-13
    assert abs(orc.expect_pauli(psi, [], []) - 2.25) < 1e-13
    assert abs(orc.norm2(psi) - 2.25) < 1e-13


def test_measurement_ghz_and_collapse():
    n = 5
    psi = orc.run_circuit(gen.ghz_circuit(n), n)
    p0, p1 = orc.parity_probs(psi, [2])
    assert abs(p0 - 0.5) < 1e-15 and abs(p1 - 0.5) < 1e-15
    p0, p1 = orc.parity_probs(psi, [1, 3])
    assert abs(p0 - 1) < 1e-15 and abs(p1) < 1e-15
    # outcome 0 iff randnum < p_even / norm
    assert orc.measure(psi.copy(), [2], 0.4999, False) == 0
    assert orc.measure(psi.copy(), [2], 0.5, False) == 1
    c = psi.copy()
    out = orc.measure(c, [2], 0.9, True)
    assert out == 1
    want = np.zeros(1 << n, dtype=np.complex128)
    want[-1] = 1
    np.testing.assert_allclose(c, want, atol=1e-15)
    # after the collapse every qubit is determined
    for q in range(n):
        assert orc.parity_probs(c, [q]) == (0.0, 1.0)


def test_measurement_probabilities_sum_to_norm():
    rng = gen.rng_for(8)
    n = 8
    psi = gen.random_state(n, 8)
    for m in range(1, n + 1):
        qs = _rand_qubits(rng, n, m)
        p0, p1 = orc.parity_probs(psi, qs)
        assert abs(p0 + p1 - 1) < 1e-13
        # p_even - p_odd = <Z...Z> on the same qubits
        assert abs((p0 - p1) - orc.expect_pauli(psi, [3] * m, qs)) < 1e-13
        c = psi.copy()
        out = orc.measure(c, qs, float(rng.uniform()), True)
        assert abs(orc.norm2(c) - 1) < 1e-13
        assert orc.parity_probs(c, qs)[out] == pytest.approx(1.0, abs=1e-13)


def test_oracle_rejects_bad_arguments():
    psi = orc.zero_state(4)
    with pytest.raises(ValueError):
        orc.apply_gate(psi, [4], np.eye(2))
    with pytest.raises(ValueError):
        orc.apply_gate(psi, [1], np.eye(2), [1])
    with pytest.raises(ValueError):
        orc.apply_gate(psi, [0, 0], np.eye(4))
    with pytest.raises(ValueError):
        orc.expect_pauli(psi, [1, 1], [2, 2])


@pytest.mark.parametrize("n", [1, 3, 5])
def test_pauli_rotation_equals_matrix_exponential(n):
    import scipy.linalg
    rng = gen.rng_for(60 + n)
    paulis, sites = gen.random_pauli_strings(n, 6, rng)
    for ps, ss in zip(paulis, sites):
        theta = float(rng.uniform(-3, 3))
        psi = gen.random_state(n, 61 + n)
        want = scipy.linalg.expm(1j * theta * np_ref.pauli_operator(n, ps, ss)) @ psi
        orc.pauli_rotation(psi, ps, ss, theta)
        np.testing.assert_allclose(psi, want, atol=1e-13, rtol=0)


def test_pauli_rotation_closed_forms():
    # exp(i t Z) = diag(e^{it}, e^{-it}); exp(i t X) = [[cos t, i sin t], [i sin t, cos t]];
    # t = pi/2 gives i P; rotations about the same string add their angles
    t = 0.37
    psi = gen.random_state(3, 9)
    ref = psi.copy()
    orc.pauli_rotation(psi, [3], [1], t)
    orc.apply_gate(ref, [1], np.diag([np.exp(1j * t), np.exp(-1j * t)]))
    np.testing.assert_allclose(psi, ref, atol=1e-15)
    psi = gen.random_state(3, 10)
    ref = psi.copy()
    orc.pauli_rotation(psi, [1], [2], t)
    orc.apply_gate(ref, [2], np.array([[np.cos(t), 1j * np.sin(t)], [1j * np.sin(t), np.cos(t)]]))
    np.testing.assert_allclose(psi, ref, atol=1e-15)
    psi = gen.random_state(4, 11)
    ref = psi.copy()
    orc.pauli_rotation(psi, [2, 1, 3], [0, 2, 3], np.pi / 2)
    np.testing.assert_allclose(psi, 1j * (np_ref.pauli_operator(4, [2, 1, 3], [0, 2, 3]) @ ref), atol=1e-14)
    a = gen.random_state(4, 12)
    b = a.copy()
    orc.pauli_rotation(a, [2, 3], [1, 3], 0.4)
    orc.pauli_rotation(a, [2, 3], [1, 3], 0.9)
    orc.pauli_rotation(b, [2, 3], [1, 3], 1.3)
    np.testing.assert_allclose(a, b, atol=1e-14)


def test_sampler_closed_forms_and_frequencies():
    n = 5
    basis = np.zeros(1 << n, dtype=np.complex128)
    basis[13] = 1
    assert (orc.sample(basis, [0.0, 0.3, 0.999]) == 13).all()
    ghz = orc.run_circuit(gen.ghz_circuit(n), n)
    assert list(orc.sample(ghz, [0.1, 0.49, 0.51, 0.9])) == [0, 0, 31, 31]
    # the draw inverts the cumulative probability relative to the norm
    assert list(orc.sample(2.0 * ghz, [0.1, 0.49, 0.51, 0.9])) == [0, 0, 31, 31]
    uni = orc.run_circuit([gen.Gate((q,), gen.gate_h()) for q in range(n)], n)
    r = np.array([0.0, 0.2, 0.5, 0.77, 0.999])
    assert list(orc.sample(uni, r)) == list(np.floor(r * 32 + 1e-9).astype(int))
    # frequencies of many uniform draws follow |psi_i|^2 (chi-square at the 0.1 % level)
    psi = gen.random_state(4, 3)
    p = np.abs(psi) ** 2
    draws = orc.sample(psi, gen.rng_for(4).uniform(size=40000))
    counts = np.bincount(draws, minlength=16)
    chi2 = np.sum((counts - 40000 * p) ** 2 / (40000 * p))
    assert chi2 < 37.7   # chi-square, 15 degrees of freedom, p = 0.001
