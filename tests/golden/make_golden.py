"""Write tests/golden/config0_oracle.json from the CPU oracle only.

The 16-qubit, 300-gate random circuit (seed 0: Haar SU(2) layers alternating
with CZ/CNOT on random disjoint pairs, from |0...0>) is run through the oracle;
the file keeps its norm, <Z_q> for every qubit and 32 amplitudes at fixed
indices. test_golden.py re-runs the oracle against it, so a later change of
the oracle's arithmetic shows up as a diff of this file.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc  # noqa: E402
from paper_2308_01999_gb300 import inputs as gen  # noqa: E402

INDICES = [(i * 2654435761) % (1 << 16) for i in range(32)]


def compute():
    psi = orc.run_circuit(gen.circuit_config0(0), 16)
    return {
        "circuit": "16 qubits, 300 gates, seed 0 (SU(2) layers + CZ/CNOT on random disjoint pairs)",
        "norm2": orc.norm2(psi),
        "z": [float(v) for v in orc.expect_z_all(psi)],
        "indices": INDICES,
        "amps_re": [float(psi[i].real) for i in INDICES],
        "amps_im": [float(psi[i].imag) for i in INDICES],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "config0_oracle.json"), "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
