"""Mutation check of the oracle's pins.

Each case copies ``oracle/sv_oracle.c`` to a temporary directory, plants one
plausible mistake in the copy (a transposed matrix, a reversed target order, a
lost conjugate, a wrong Y sign, a dropped term, ...), compiles it, points the
oracle's front end at the mutant and runs the pins of test_oracle.py. The
mutant must fail at least one pin. The real oracle is never modified.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from oracle import oracle as orc
from tests import test_oracle as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "sv_oracle.c")

MUTATIONS = [
    ("transposed matrix", "acc += M[j * D + l] * in[l];", "acc += M[l * D + j] * in[l];"),
    ("reversed target order", "if ((j >> t) & 1u) off |= 1ull << targets[t];",
     "if ((j >> t) & 1u) off |= 1ull << targets[k - 1 - t];"),
    ("control value ignored", "if (control_values == NULL || control_values[t] != 0)", "if (1)"),
    ("controls ignored", "if ((base & cmask) != cwant) continue;", ";"),
    ("lost conjugate", "acc += conj(psi[i]) * phi[i];", "acc += psi[i] * phi[i];"),
    ("wrong Y sign", "case 2: m[0] = 0; m[1] = -I; m[2] = I;", "case 2: m[0] = 0; m[1] = I; m[2] = -I;"),
    ("dropped matvec term", "for (uint64_t l = 0; l < D; ++l) acc += M", "for (uint64_t l = 1; l < D; ++l) acc += M"),
    ("collapse without sqrt", "const double scale = 1.0 / sqrt(prob);", "const double scale = 1.0 / prob;"),
    ("parity from one qubit", "for (int t = 0; t < m; ++t) p ^= (int)((i >> qubits[t]) & 1u);",
     "p = (int)((i >> qubits[0]) & 1u);"),
    ("rotation sign", "psi[i] = c * psi[i] + I * sn * phi[i];", "psi[i] = c * psi[i] - I * sn * phi[i];"),
    ("rotation without cosine", "psi[i] = c * psi[i] + I * sn * phi[i];", "psi[i] = psi[i] + I * sn * phi[i];"),
    ("sampler boundary", "if (cum[mid] > target) hi = mid;", "if (cum[mid] >= target) hi = mid;"),
    ("sampler unscaled target", "const double target = randnums[t] * acc;", "const double target = randnums[t];"),
]


def _pin_calls():
    calls = []
    for s in range(4):
        calls.append(("apply_vs_numpy", lambda s=s: pins.test_apply_matches_numpy_tensor_contraction(s)))
    for args in [(6, 3, 2), (8, 0, 6)]:
        calls.append(("kron", lambda a=args: pins.test_contiguous_gate_equals_kron_operator(*a)))
    calls.append(("target_order", pins.test_target_order_sequential_equals_kron))
    for cv in (0, 1):
        calls.append(("controlled", lambda cv=cv: pins.test_controlled_gate_equals_block_operator(cv)))
    for n in (2, 3, 4):
        calls.append(("ghz", lambda n=n: pins.test_ghz_closed_form(n)))
    calls.append(("qft", lambda: pins.test_qft_of_basis_state_closed_form(5)))
    calls.append(("echo", pins.test_unitarity_and_echo))
    calls.append(("product", pins.test_product_state_expectations))
    calls.append(("pauli_explicit", lambda: pins.test_pauli_expectation_equals_explicit_operator(6)))
    calls.append(("identity", pins.test_identity_string_is_the_norm))
    calls.append(("measure_ghz", pins.test_measurement_ghz_and_collapse))
    calls.append(("measure_sum", pins.test_measurement_probabilities_sum_to_norm))
    calls.append(("rotation_expm", lambda: pins.test_pauli_rotation_equals_matrix_exponential(3)))
    calls.append(("rotation_closed", pins.test_pauli_rotation_closed_forms))
    calls.append(("sampler", pins.test_sampler_closed_forms_and_frequencies))
    return calls


def _build_mutant(tmp, before, after):
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation anchor not found exactly once: {before!r}"
    path = os.path.join(tmp, "mut.c")
    with open(path, "w") as f:
        f.write(src.replace(before, after))
    so = os.path.join(tmp, "libmut.so")
    subprocess.run(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-ffp-contract=off", path,
                    "-o", so, "-lm"], check=True, capture_output=True)
    return so


@pytest.mark.parametrize("name,before,after", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_every_planted_mistake_fails_a_pin(name, before, after):
    real = orc.lib()
    tmp = tempfile.mkdtemp(prefix="orcmut")
    try:
        so = _build_mutant(tmp, before, after)
        mut = ctypes.CDLL(so)
        for fn in ("orc_threads", "orc_apply", "orc_expect_pauli", "orc_parity_probs",
                   "orc_collapse", "orc_norm2", "orc_pauli_rotation", "orc_sample"):
            src_fn, dst_fn = getattr(real, fn), getattr(mut, fn)
            dst_fn.argtypes, dst_fn.restype = src_fn.argtypes, src_fn.restype
        orc._lib = mut
        failed = []
        for label, call in _pin_calls():
            try:
                call()
            except (AssertionError, ValueError):
                failed.append(label)
        assert failed, f"mutation '{name}' passed every pin"
    finally:
        orc._lib = real
        shutil.rmtree(tmp, ignore_errors=True)


def test_real_oracle_passes_the_same_pins():
    for label, call in _pin_calls():
        call()
