"""The seeded generators: determinism, shapes of the benchmark circuits, and
the Haar property of the SU(2) draw."""
import numpy as np

from paper_2308_01999_gb300 import inputs as gen


def test_haar_su2_is_special_unitary_and_haar():
    rng = gen.rng_for(0)
    us = [gen.haar_su2(rng) for _ in range(4000)]
    for u in us[:50]:
        np.testing.assert_allclose(u @ u.conj().T, np.eye(2), atol=1e-14)
        assert abs(np.linalg.det(u) - 1) < 1e-14
    # Haar on SU(2): |U_00|^2 is uniform on [0, 1] (Kolmogorov-Smirnov distance)
    x = np.sort([abs(u[0, 0]) ** 2 for u in us])
    ks = np.max(np.abs(x - (np.arange(1, len(x) + 1) / len(x))))
    assert ks < 1.63 / np.sqrt(len(x))  # 1 % level


def test_random_unitary_is_unitary():
    rng = gen.rng_for(1)
    for k in range(1, 7):
        m = gen.random_gate_dense(rng, k)
        np.testing.assert_allclose(m @ m.conj().T, np.eye(1 << k), atol=1e-12)


def test_circuits_are_deterministic_and_sized():
    a, b = gen.circuit_config0(), gen.circuit_config0()
    assert len(a) == 300
    assert all(np.array_equal(x.matrix, y.matrix) and x.qubits == y.qubits for x, y in zip(a, b))
    c1 = gen.circuit_config1()
    assert len(c1) == 40 * (28 + 14)
    assert {g.name for g in c1} == {"su2", "cz", "cnot", "crz"}
    c2 = gen.circuit_config2()
    assert len(c2) == 1900
    assert sum(g.name == "cz" for g in c2) == 20 * 16 + 20 * 15
    # pairs within a layer are disjoint
    for layer in range(40):
        two = c1[layer * 42 + 28:(layer + 1) * 42]
        qs = [q for g in two for q in g.qubits]
        assert len(qs) == len(set(qs)) == 28


def test_dense_form_block_structure():
    g = gen.crz(3, 1, 0.7)
    d = gen.dense_form(g)
    assert d.targets == (1, 3) and d.controls == ()
    np.testing.assert_array_equal(d.matrix[:2, :2], np.eye(2))
    np.testing.assert_array_equal(d.matrix[2:, 2:], gen.gate_rz(0.7))


def test_pauli_strings_and_ansatz():
    rng = gen.rng_for(3)
    p, s = gen.random_pauli_strings(12, 8, rng)
    assert p.shape == (8, 12) and p.min() >= 0 and p.max() <= 3
    assert (s == np.arange(12)).all()
    w = gen.batched_ansatz_workload(count=20)
    assert all(10 <= n <= 20 and len(gates) == 6 * (3 * n - 1) for n, gates, _, _ in w)
    tr = gen.serving_trace(count=100)
    assert all(12 <= n <= 30 and 10 <= d <= 60 for _, n, d, _ in tr)
    assert all(tr[i][0] < tr[i + 1][0] for i in range(99))
