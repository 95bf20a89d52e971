"""The oracle reproduces its committed output for the 16-qubit circuit."""
import json
import os

import numpy as np

from tests.golden import make_golden


def test_oracle_matches_committed_golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "config0_oracle.json")) as f:
        want = json.load(f)
    got = make_golden.compute()
    assert got["indices"] == want["indices"]
    assert abs(got["norm2"] - 1) < 1e-12 and abs(want["norm2"] - 1) < 1e-12
    np.testing.assert_allclose(got["z"], want["z"], atol=1e-13, rtol=0)
    np.testing.assert_allclose(got["amps_re"], want["amps_re"], atol=1e-15, rtol=0)
    np.testing.assert_allclose(got["amps_im"], want["amps_im"], atol=1e-15, rtol=0)
