"""ctypes front end of the C oracle (TEST INFRASTRUCTURE ONLY).

Thin marshalling over ``sv_oracle.c``: numpy complex128 arrays in, the same
arrays updated in place or plain numbers out. Every computation happens in the
C file, which follows the paper's definitions (exact state-vector simulation,
Sec. II; gate application, measurement and Pauli expectation, Table I).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build_oracle import build

_lib = None
_I = C.POINTER(C.c_int)
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.orc_threads.argtypes = [C.c_int]
        L.orc_threads.restype = C.c_int
        L.orc_apply.argtypes = [_D, C.c_int, _I, C.c_int, _I, _I, C.c_int, _D]
        L.orc_apply.restype = C.c_int
        L.orc_expect_pauli.argtypes = [_D, C.c_int, _I, _I, C.c_int, _D]
        L.orc_expect_pauli.restype = C.c_int
        L.orc_parity_probs.argtypes = [_D, C.c_int, _I, C.c_int, _D]
        L.orc_parity_probs.restype = C.c_int
        L.orc_collapse.argtypes = [_D, C.c_int, _I, C.c_int, C.c_int, C.c_double]
        L.orc_collapse.restype = C.c_int
        L.orc_norm2.argtypes = [_D, C.c_int]
        L.orc_norm2.restype = C.c_double
        L.orc_pauli_rotation.argtypes = [_D, C.c_int, _I, _I, C.c_int, C.c_double]
        L.orc_pauli_rotation.restype = C.c_int
        L.orc_sample.argtypes = [_D, C.c_int, _D, C.c_int, C.POINTER(C.c_int64)]
        L.orc_sample.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (<= 0 keeps it); returns the count in use."""
    return int(lib().orc_threads(int(n)))


def _ints(xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.int32).reshape(-1))
    return a, (a.ctypes.data_as(_I) if a.size else None)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _nqubits(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.dtype != np.complex128 or (1 << n) != psi.size or not psi.flags.c_contiguous:
        raise ValueError("psi must be a contiguous complex128 vector of 2^n amplitudes")
    return n


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_gate(psi: np.ndarray, targets, matrix, controls=(), control_values=()) -> np.ndarray:
    """psi <- G psi in place (see ``orc_apply``)."""
    n = _nqubits(psi)
    t, tp = _ints(targets)
    c, cp = _ints(controls)
    cv, cvp = _ints(control_values)
    m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
    if m.shape != (1 << t.size, 1 << t.size):
        raise ValueError("matrix shape does not match the target count")
    rc = lib().orc_apply(_dptr(psi), n, tp, int(t.size), cp, cvp if cv.size else None,
                         int(c.size), _dptr(m))
    if rc != 0:
        raise ValueError(f"oracle rejected the gate (code {rc})")
    return psi


def apply(psi: np.ndarray, gate) -> np.ndarray:
    """Apply one ``inputs.Gate``-like object (targets, matrix, controls, control_values)."""
    return apply_gate(psi, gate.targets, gate.matrix, gate.controls, gate.control_values)


def run_circuit(gates, n: int, psi: np.ndarray | None = None) -> np.ndarray:
    psi = zero_state(n) if psi is None else psi
    for g in gates:
        apply(psi, g)
    return psi


def expect_pauli(psi: np.ndarray, paulis, sites) -> complex:
    """<psi| P |psi> for one Pauli string (codes 0=I, 1=X, 2=Y, 3=Z on ``sites``)."""
    n = _nqubits(psi)
    p, pp = _ints(paulis)
    s, sp = _ints(sites)
    out = np.zeros(2)
    rc = lib().orc_expect_pauli(_dptr(psi), n, pp, sp, int(p.size), _dptr(out))
    if rc != 0:
        raise ValueError(f"oracle rejected the Pauli string (code {rc})")
    return complex(out[0], out[1])


def expect_z_all(psi: np.ndarray) -> np.ndarray:
    """<Z_q> for every qubit q."""
    n = _nqubits(psi)
    return np.array([expect_pauli(psi, [3], [q]).real for q in range(n)])


def parity_probs(psi: np.ndarray, qubits) -> tuple:
    n = _nqubits(psi)
    q, qp = _ints(qubits)
    out = np.zeros(2)
    rc = lib().orc_parity_probs(_dptr(psi), n, qp, int(q.size), _dptr(out))
    if rc != 0:
        raise ValueError(f"oracle rejected the measurement (code {rc})")
    return float(out[0]), float(out[1])


def measure(psi: np.ndarray, qubits, randnum: float, collapse: bool) -> int:
    """Z-product-basis measurement: outcome 0 iff randnum < p_even / (p_even + p_odd);
    with ``collapse`` the state keeps the outcome's branch, renormalised."""
    p0, p1 = parity_probs(psi, qubits)
    outcome = 0 if randnum < p0 / (p0 + p1) else 1
    if collapse:
        n = _nqubits(psi)
        q, qp = _ints(qubits)
        rc = lib().orc_collapse(_dptr(psi), n, qp, int(q.size), outcome, p0 if outcome == 0 else p1)
        if rc != 0:
            raise ValueError(f"oracle rejected the collapse (code {rc})")
    return outcome


def norm2(psi: np.ndarray) -> float:
    return float(lib().orc_norm2(_dptr(psi), _nqubits(psi)))


def pauli_rotation(psi: np.ndarray, paulis, sites, theta: float) -> np.ndarray:
    """psi <- exp(i theta P) psi in place."""
    n = _nqubits(psi)
    p, pp = _ints(paulis)
    s, sp = _ints(sites)
    rc = lib().orc_pauli_rotation(_dptr(psi), n, pp, sp, int(p.size), float(theta))
    if rc != 0:
        raise ValueError(f"oracle rejected the rotation (code {rc})")
    return psi


def sample(psi: np.ndarray, randnums) -> np.ndarray:
    """Basis indices drawn by inverting the cumulative probabilities at randnums."""
    n = _nqubits(psi)
    r = np.ascontiguousarray(np.asarray(randnums, dtype=np.float64))
    out = np.zeros(r.size, dtype=np.int64)
    rc = lib().orc_sample(_dptr(psi), n, r.ctypes.data_as(_D), int(r.size),
                          out.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc != 0:
        raise ValueError(f"oracle rejected the sampling (code {rc})")
    return out
