"""A second, independent CPU formulation in numpy (TEST INFRASTRUCTURE ONLY).

Where ``sv_oracle.c`` loops over amplitude groups, this file treats the state
as a rank-n tensor of shape [2]*n (axis n-1-q is qubit q, because C order puts
the most significant index bit first) and contracts each gate over its qubit
axes with ``numpy.tensordot``. A controlled gate becomes the full block operator
on controls+targets. It also builds explicit 2^n x 2^n operators with
``numpy.kron`` for brute-force checks at small n. Used only to pin the C oracle.
"""
from __future__ import annotations

import numpy as np


def _axis(n: int, q: int) -> int:
    return n - 1 - q


def controlled_block(matrix: np.ndarray, k: int, cvals) -> np.ndarray:
    """Operator on (targets, controls) -- index bits 0..k-1 targets, then controls --
    equal to ``matrix`` where every control holds its value, identity elsewhere."""
    c = len(cvals)
    kt = 1 << k
    want = sum(int(v) << i for i, v in enumerate(cvals))
    full = np.eye(1 << (k + c), dtype=np.complex128)
    full[want * kt:(want + 1) * kt, want * kt:(want + 1) * kt] = matrix
    return full


def apply_gate_np(psi: np.ndarray, n: int, targets, matrix, controls=(), control_values=()):
    """Return G psi, computed by tensor contraction."""
    targets = list(targets)
    controls = list(controls)
    cvals = list(control_values) if control_values else [1] * len(controls)
    qubits = targets + controls
    m = len(qubits)
    op = controlled_block(np.asarray(matrix, dtype=np.complex128), len(targets), cvals)
    # op index bit j <-> qubits[j]; as a tensor with axes (out bits msb..lsb, in bits msb..lsb)
    opt = op.reshape([2] * (2 * m))
    # tensor axis a of the first half is bit (m-1-a) i.e. qubit qubits[m-1-a]
    in_axes_op = list(range(m, 2 * m))
    st = psi.reshape([2] * n)
    st_axes = [_axis(n, qubits[m - 1 - a]) for a in range(m)]
    res = np.tensordot(opt, st, axes=(in_axes_op, st_axes))
    # res axes: m output bits (same order as st_axes) followed by the untouched state axes
    rest = [ax for ax in range(n) if ax not in st_axes]
    order = st_axes + rest
    inv = np.argsort(order)
    return np.ascontiguousarray(np.transpose(res, inv)).reshape(-1)


PAULI = {
    0: np.eye(2, dtype=np.complex128),
    1: np.array([[0, 1], [1, 0]], dtype=np.complex128),
    2: np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    3: np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def pauli_operator(n: int, paulis, sites) -> np.ndarray:
    """The explicit 2^n x 2^n operator of a Pauli string (kron, qubit n-1 leftmost)."""
    per = {int(s): int(p) for p, s in zip(paulis, sites)}
    op = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        op = np.kron(op, PAULI[per.get(q, 0)])
    return op


def kron_operator_contiguous(n: int, lo: int, matrix: np.ndarray) -> np.ndarray:
    """The 2^n operator of a k-qubit gate on targets lo, lo+1, ..., lo+k-1 (in that
    order): I_{2^(n-lo-k)} (x) M (x) I_{2^lo}."""
    k = int(np.log2(matrix.shape[0]))
    return np.kron(np.eye(1 << (n - lo - k)), np.kron(matrix, np.eye(1 << lo)))
