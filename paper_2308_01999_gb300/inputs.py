"""Seeded synthetic inputs: gate lists, states and Pauli strings.

This module is shared by the tests, the benchmark and the CPU oracle's
callers. It holds no simulation arithmetic: it only draws random numbers and
writes down the definitions of the standard gates (their 2x2 / 4x4 matrices)
that make up a circuit. Applying a gate, reducing an expectation value or
fusing gates happens elsewhere (the CUDA path in ``csrc/``, the oracle in
``oracle/``), and the two never import each other.

Conventions (the paper fixes only that each index bit of the state vector is
one qubit, Sec. II-C):

* qubit ``q`` is bit ``q`` of the amplitude index (little-endian);
* a gate matrix is a row-major complex128 ``2^k x 2^k`` array whose row and
  column index bit ``j`` belongs to ``targets[j]``;
* a controlled gate acts with ``matrix`` on the subspace where every control
  qubit equals its control value (1 unless stated), and as the identity
  elsewhere.

Every generator takes an explicit seed and uses ``numpy.random.Generator``
with the PCG64 bit generator, so a circuit is a pure function of its seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

__all__ = [
    "Gate", "rng_for", "haar_su2", "gate_h", "gate_x", "gate_y", "gate_z",
    "gate_rz", "gate_ry", "gate_phase", "gate_swap", "cz", "cnot", "crz",
    "dense_form", "random_state", "random_pauli_strings", "layered_random_circuit",
    "circuit_config0", "circuit_config1", "circuit_config2", "ansatz_circuit",
    "batched_ansatz_workload", "ghz_circuit", "qft_circuit", "random_gate_dense",
    "serving_trace", "gate_rx", "gate_zz", "qaoa_circuit", "PAULI_I", "PAULI_X", "PAULI_Y", "PAULI_Z",
]

PAULI_I, PAULI_X, PAULI_Y, PAULI_Z = 0, 1, 2, 3


@dataclass(frozen=True)
class Gate:
    """One gate of a circuit.

    ``targets``: the k target qubits; bit j of the matrix row/column index
    belongs to ``targets[j]``. ``matrix``: complex128, shape (2^k, 2^k).
    ``controls``/``control_values``: control qubits and the value each must
    hold (an empty ``control_values`` means all ones).
    """

    targets: tuple
    matrix: np.ndarray
    controls: tuple = ()
    control_values: tuple = ()
    name: str = field(default="", compare=False)

    @property
    def k(self) -> int:
        return len(self.targets)

    @property
    def qubits(self) -> tuple:
        return tuple(self.targets) + tuple(self.controls)

    def cvals(self) -> tuple:
        return tuple(self.control_values) if self.control_values else (1,) * len(self.controls)


def rng_for(seed: int) -> np.random.Generator:
    """The one random source of every generator here: PCG64 seeded by ``seed``."""
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# gate definitions (textbook matrices)
# ----------------------------------------------------------------------------

def haar_su2(rng: np.random.Generator) -> np.ndarray:
    """A Haar-random SU(2) matrix.

    SU(2) is the unit 3-sphere: four i.i.d. standard normals, normalised, give
    a uniform point (a0, a1, a2, a3) on S^3 (Muller's method), and
    U = [[a, -conj(b)], [b, conj(a)]] with a = a0 + i a3, b = a2 + i a1 is
    then Haar-distributed on SU(2).
    """
    v = rng.standard_normal(4)
    v = v / np.linalg.norm(v)
    a = complex(v[0], v[3])
    b = complex(v[2], v[1])
    return np.array([[a, -np.conj(b)], [b, np.conj(a)]], dtype=np.complex128)


def gate_h() -> np.ndarray:
    return np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def gate_x() -> np.ndarray:
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def gate_y() -> np.ndarray:
    return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)


def gate_z() -> np.ndarray:
    return np.array([[1, 0], [0, -1]], dtype=np.complex128)


def gate_rz(theta: float) -> np.ndarray:
    """RZ(theta) = diag(e^{-i theta/2}, e^{+i theta/2})."""
    return np.array([[np.exp(-0.5j * theta), 0], [0, np.exp(0.5j * theta)]], dtype=np.complex128)


def gate_ry(theta: float) -> np.ndarray:
    """RY(theta) = [[cos theta/2, -sin theta/2], [sin theta/2, cos theta/2]]."""
    c, s = np.cos(0.5 * theta), np.sin(0.5 * theta)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def gate_phase(phi: float) -> np.ndarray:
    """P(phi) = diag(1, e^{i phi})."""
    return np.array([[1, 0], [0, np.exp(1j * phi)]], dtype=np.complex128)


def gate_swap() -> np.ndarray:
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[3, 3] = 1
    m[1, 2] = m[2, 1] = 1
    return m


def cz(a: int, b: int) -> Gate:
    """Controlled-Z with control ``a`` and target ``b`` (the gate is symmetric)."""
    return Gate((b,), gate_z(), (a,), (), "cz")


def cnot(c: int, t: int) -> Gate:
    """CNOT with control ``c`` (the first qubit of the pair) and target ``t``."""
    return Gate((t,), gate_x(), (c,), (), "cnot")


def crz(c: int, t: int, theta: float) -> Gate:
    """Controlled RZ(theta), control ``c``, target ``t``."""
    return Gate((t,), gate_rz(theta), (c,), (), "crz")


def dense_form(g: Gate) -> Gate:
    """The same operator written as an uncontrolled gate on controls+targets.

    The new target list is ``targets + controls``; the matrix is the block
    operator that applies ``g.matrix`` where the controls hold their values
    and the identity elsewhere. Used to hand the library a 4x4 CZ/CNOT/CRZ
    instead of a controlled 2x2, which exercises its structure detection.
    """
    k, c = g.k, len(g.controls)
    d = 1 << (k + c)
    kt = 1 << k
    cv = g.cvals()
    want = sum(v << i for i, v in enumerate(cv))
    m = np.zeros((d, d), dtype=np.complex128)
    for hi in range(1 << c):
        blk = g.matrix if hi == want else np.eye(kt, dtype=np.complex128)
        m[hi * kt:(hi + 1) * kt, hi * kt:(hi + 1) * kt] = blk
    return Gate(tuple(g.targets) + tuple(g.controls), m, (), (), g.name + "_dense")


def random_gate_dense(rng: np.random.Generator, k: int) -> np.ndarray:
    """A Haar-random 2^k x 2^k unitary (QR of a complex Ginibre matrix, with the
    phases of R's diagonal moved into Q, after Mezzadri)."""
    d = 1 << k
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return (q * ph[None, :]).astype(np.complex128)


# ----------------------------------------------------------------------------
# states and observables
# ----------------------------------------------------------------------------

def random_state(n: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """A random unit vector of 2^n amplitudes (complex normal, normalised)."""
    rng = rng_for(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def random_pauli_strings(n: int, count: int, rng: np.random.Generator):
    """``count`` strings of ``n`` sites, each site uniform over {I, X, Y, Z}.

    Returns (paulis, sites), int32 arrays of shape (count, n): ``paulis[s, i]``
    acts on qubit ``sites[s, i] = i``.
    """
    paulis = rng.integers(0, 4, size=(count, n)).astype(np.int32)
    sites = np.tile(np.arange(n, dtype=np.int32), (count, 1))
    return paulis, sites


# ----------------------------------------------------------------------------
# circuit families
# ----------------------------------------------------------------------------

def layered_random_circuit(n: int, layers: int, seed: int, kinds: Sequence[str],
                           max_gates: int | None = None) -> list:
    """Alternating layers: a Haar SU(2) on every qubit, then a two-qubit gate on
    each of floor(n/2) random disjoint pairs (a random permutation of the
    qubits taken two at a time; the first of a pair is the control). The kind
    of each two-qubit gate is uniform over ``kinds`` ('cz', 'cnot', 'crz'); a
    CRZ angle is uniform on [0, 2 pi)."""
    rng = rng_for(seed)
    gates: list = []
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate((q,), haar_su2(rng), (), (), "su2"))
        perm = rng.permutation(n)
        for p in range(n // 2):
            a, b = int(perm[2 * p]), int(perm[2 * p + 1])
            kind = kinds[int(rng.integers(0, len(kinds)))]
            if kind == "cz":
                gates.append(cz(a, b))
            elif kind == "cnot":
                gates.append(cnot(a, b))
            elif kind == "crz":
                gates.append(crz(a, b, float(rng.uniform(0.0, 2.0 * np.pi))))
            else:
                raise ValueError(kind)
        if max_gates is not None and len(gates) >= max_gates:
            break
    if max_gates is not None:
        gates = gates[:max_gates]
    return gates


def circuit_config0(seed: int = 0) -> list:
    """16 qubits, 300 gates: SU(2) layers alternating with CZ/CNOT pair layers."""
    return layered_random_circuit(16, 1000, seed, ("cz", "cnot"), max_gates=300)


def circuit_config1(n: int = 28, depth: int = 40, seed: int = 1) -> list:
    """28 qubits, depth 40: SU(2) on all qubits then CZ/CNOT/CRZ on disjoint pairs."""
    return layered_random_circuit(n, depth, seed, ("cz", "cnot", "crz"))


def circuit_config2(n: int = 32, layers: int = 40, seed: int = 2) -> list:
    """Brick wall: each layer is a Haar SU(2) on every qubit followed by CZ on
    pairs (0,1),(2,3),... in even layers and (1,2),(3,4),... in odd layers."""
    rng = rng_for(seed)
    gates: list = []
    for layer in range(layers):
        for q in range(n):
            gates.append(Gate((q,), haar_su2(rng), (), (), "su2"))
        start = layer % 2
        for a in range(start, n - 1, 2):
            gates.append(cz(a, a + 1))
    return gates


def ansatz_circuit(n: int, layers: int, rng: np.random.Generator) -> list:
    """Hardware-efficient ansatz: per layer RY(theta_q) then RZ(phi_q) on every
    qubit, then CNOT(q, q+1) for q = 0..n-2 in order; angles U[0, 2 pi)."""
    gates: list = []
    for _ in range(layers):
        for q in range(n):
            th = float(rng.uniform(0.0, 2.0 * np.pi))
            ph = float(rng.uniform(0.0, 2.0 * np.pi))
            gates.append(Gate((q,), gate_ry(th), (), (), "ry"))
            gates.append(Gate((q,), gate_rz(ph), (), (), "rz"))
        for q in range(n - 1):
            gates.append(cnot(q, q + 1))
    return gates


def batched_ansatz_workload(count: int = 4096, nmin: int = 10, nmax: int = 20,
                            layers: int = 6, strings: int = 8, seed: int = 3):
    """Many independent ansatz states with qubit counts uniform on [nmin, nmax],
    each with ``strings`` random Pauli strings. Yields (n, gates, paulis, sites)."""
    rng = rng_for(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        gates = ansatz_circuit(n, layers, rng)
        paulis, sites = random_pauli_strings(n, strings, rng)
        out.append((n, gates, paulis, sites))
    return out


def gate_rx(theta: float) -> np.ndarray:
    """RX(theta) = [[cos theta/2, -i sin theta/2], [-i sin theta/2, cos theta/2]]."""
    c, s = np.cos(0.5 * theta), np.sin(0.5 * theta)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def gate_zz(theta: float) -> np.ndarray:
    """exp(-i theta/2 Z(x)Z) on two targets: diag(e^{-i t/2}, e^{i t/2}, e^{i t/2}, e^{-i t/2})."""
    a, b = np.exp(-0.5j * theta), np.exp(0.5j * theta)
    return np.diag([a, b, b, a]).astype(np.complex128)


def qaoa_circuit(n: int, p: int, seed: int, edges_per_qubit: int = 3) -> list:
    """QAOA-style circuit on a random graph: H on every qubit, then p rounds of
    ZZ(gamma) on each edge (diagonal two-qubit gates) and RX(beta) on every
    qubit; angles uniform on [0, 2 pi)."""
    rng = rng_for(seed)
    edges = set()
    while len(edges) < (n * edges_per_qubit) // 2:
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    gates = [Gate((q,), gate_h(), (), (), "h") for q in range(n)]
    for _ in range(p):
        gamma, beta = rng.uniform(0, 2 * np.pi, size=2)
        for a, b in edges:
            gates.append(Gate((a, b), gate_zz(float(gamma)), (), (), "zz"))
        for q in range(n):
            gates.append(Gate((q,), gate_rx(float(beta)), (), (), "rx"))
    return gates


def ghz_circuit(n: int) -> list:
    """H on qubit 0, then CNOT(q, q+1) for q = 0..n-2."""
    gates = [Gate((0,), gate_h(), (), (), "h")]
    for q in range(n - 1):
        gates.append(cnot(q, q + 1))
    return gates


def qft_circuit(n: int) -> list:
    """The textbook quantum Fourier transform on n qubits (qubit n-1 is the
    most significant bit): for j = n-1 down to 0, H on j then, for each lower
    qubit m, a phase e^{2 pi i / 2^(j-m+1)} controlled by m on target j;
    finally the qubit order is reversed with SWAPs. Maps |x> to
    2^{-n/2} sum_y e^{2 pi i x y / 2^n} |y>."""
    gates: list = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate((j,), gate_h(), (), (), "h"))
        for m in range(j - 1, -1, -1):
            phi = 2.0 * np.pi / float(1 << (j - m + 1))
            gates.append(Gate((j,), gate_phase(phi), (m,), (), "cp"))
    for q in range(n // 2):
        gates.append(Gate((q, n - 1 - q), gate_swap(), (), (), "swap"))
    return gates


def serving_trace(count: int = 10000, rate: float = 200.0, nmin: int = 12, nmax: int = 30,
                  dmin: int = 10, dmax: int = 60, seed: int = 4):
    """Poisson arrivals (exponential gaps with mean 1/rate) of random circuits:
    qubits uniform on [nmin, nmax], depth uniform on [dmin, dmax], gate mix of
    the 28-qubit benchmark circuit. Returns a list of (arrival_s, n, depth, circuit_seed);
    the circuit itself is ``circuit_config1(n, depth, circuit_seed)``."""
    rng = rng_for(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.integers(nmin, nmax + 1))
        d = int(rng.integers(dmin, dmax + 1))
        s = int(rng.integers(0, 2**31 - 1))
        out.append((t, n, d, s))
    return out
