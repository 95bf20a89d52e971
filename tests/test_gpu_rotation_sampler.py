"""Pauli rotation and the sampler (Table I) against the oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen

pytestmark = pytest.mark.gpu
AMP_TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return torch, sv


def state(env, n, name, seed):
    torch, sv = env
    init = gen.random_state(n, seed)
    dt = torch.complex64 if name == "c64" else torch.complex128
    psi = torch.from_numpy(init).to(dt).cuda()
    return psi, sv.StateVector(psi)


@pytest.mark.parametrize("name", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 11])
def test_pauli_rotation_matches_oracle(env, name, n):
    rng = gen.rng_for(300 + n)
    psi, s = state(env, n, name, 300 + n)
    ref = psi.cpu().numpy().astype(np.complex128)
    strings = [list(r) for r in gen.random_pauli_strings(n, 10, rng)[0]]
    strings += [[1] + [0] * (n - 1), [3] * n, [2] * n, [0] * n]
    for ps in strings:
        theta = float(rng.uniform(-3.2, 3.2))
        s.pauli_rotation(theta, ps, list(range(n)))
        orc.pauli_rotation(ref, ps, list(range(n)), theta)
    got = psi.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= AMP_TOL[name]


def _valid_draws(psi, r, idx, eps):
    p = np.abs(psi) ** 2
    cum = np.cumsum(p)
    t = r * cum[-1]
    before = np.where(idx > 0, cum[np.maximum(idx - 1, 0)], 0.0)
    return np.all(p[idx] > 0) and np.all(before <= t + eps) and np.all(t <= cum[idx] + eps)


@pytest.mark.parametrize("name", ["c64", "c128"])
@pytest.mark.parametrize("n", [3, 10, 17])
def test_sampler_draws_are_valid_and_match_oracle(env, name, n):
    psi, s = state(env, n, name, 400 + n)
    host = psi.cpu().numpy().astype(np.complex128)
    r = gen.rng_for(401).uniform(size=3000)
    got = s.sample(r)
    want = orc.sample(host, r)
    eps = 1e-6 if name == "c64" else 1e-12
    assert _valid_draws(host, r, got, eps)
    # away from a boundary the draw is unique
    assert np.mean(got == want) > 0.999


def test_sampler_ghz_and_frequencies(env):
    torch, sv = env
    n = 20
    psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    s = sv.StateVector(psi)
    s.set_basis_state(0)
    s.apply_circuit(gen.ghz_circuit(n))
    out = s.sample([0.1, 0.4999, 0.5001, 0.99])
    assert list(out) == [0, 0, (1 << n) - 1, (1 << n) - 1]
    psi2, s2 = state(env, 5, "c64", 9)
    p = np.abs(psi2.cpu().numpy().astype(np.complex128)) ** 2
    draws = s2.sample(gen.rng_for(10).uniform(size=50000))
    counts = np.bincount(draws, minlength=32)
    chi2 = np.sum((counts - 50000 * p) ** 2 / (50000 * p))
    assert chi2 < 61.1     # chi-square, 31 degrees of freedom, p = 0.001
