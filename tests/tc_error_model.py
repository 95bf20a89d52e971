"""Statistical error model of fused gates on the tensor cores (test infrastructure).

A fused block applies a 2^k x 2^k unitary G (k = 5 or 6, a 5-qubit block
padded with an identity qubit) to every column x of the state (the 64 members
of one amplitude group). The tensor-core kernels round both operands before the
product and accumulate in FP32:

* round-to-nearest of a real v to a format with p explicit mantissa bits gives
  v (1 + d); the absolute error is spread evenly over +-half an ulp, so
  E[d^2] <= e_p = 2^(-2p) / 12 (equality when v's mantissa is 1);
* TF32 (p = 10): every real part of G and of x is rounded once, so the output
  error is dG x + G dx. Summed over the outputs of a column,
  E||dG x||^2 = sum_k |x_k|^2 sum_m E|dG_mk|^2 <= e_10 ||x||^2 (each column of
  G has unit norm) and ||G dx||^2 = ||dx||^2 <= e_10 ||x||^2 (G is unitary);
  the two are independent, so E||err||^2 <= 2 e_10 ||x||^2;
* split BF16 (p = 7): v = hi + lo + r with hi = bf16(v), lo = bf16(v - hi), so
  E[r^2] <= e_7^2 v^2; of the four products the kernel drops lo*lo, with
  E|lo_G lo_x|^2 <= e_7^2 |G_mk x_k|^2 per term. Three independent terms (G's
  residual, x's residual, the dropped product) give E||err||^2 <= 3 e_7^2 ||x||^2;
* FP32 accumulation of K products (K = 128 real terms, 384 for three BF16
  products) and the FP32 store of the result add at most (K + 1) 2^-48 / 3.

Per block the relative L2 error therefore has RMS at most
    sigma_TF32 = sqrt(2 e_10 + 129 * 2^-48 / 3)          = 3.99e-4
    sigma_BF16 = sqrt(3 e_7^2 + 385 * 2^-48 / 3)        = 8.84e-6.
The rounding errors of different blocks are independent and every later block
is unitary, so after B blocks the error's RMS is at most sqrt(B) sigma
(errors add in quadrature, not linearly). For an echo (the circuit, then its
inverse with adjoint matrices) the first-order errors of a block and of its
adjoint combine into the Hermitian part of G^dagger dG, whose norm is that of
two independent errors, so the same sqrt(B) sigma holds with B counting both
halves.

The relative L2 error is an average over many independent roundings and
concentrates tightly around its RMS; the tests allow L2_SAFETY = 2 times the
model. An amplitude's error comes from the roundings inside its own groups,
so the error spreads over the state's support, not over all 2^n amplitudes:
with N_eff = ||psi||^4 / sum_i |psi_i|^4 (the inverse participation ratio:
M for a state spread evenly over M amplitudes, 2^n / 2 for a random state),
an amplitude's error is a complex Gaussian with E|err_i|^2 at most about
B sigma^2 ||psi||^2 / N_eff, and the largest of 2^n such errors stays below
sqrt(n ln 2 + 14) times that RMS except with probability about 1e-6; the
element-wise bound takes L2_SAFETY times that.
"""
import math

E10 = 2.0 ** -20 / 12          # TF32: 10 explicit mantissa bits
E7 = 2.0 ** -14 / 12           # BF16: 7 explicit mantissa bits
SIGMA = {
    "tf32": math.sqrt(2 * E10 + 129 * 2.0 ** -48 / 3),
    "bf16": math.sqrt(3 * E7 * E7 + 385 * 2.0 ** -48 / 3),
}
L2_SAFETY = 2.0


def l2_bound(prec: str, blocks: int) -> float:
    """Bound on the relative L2 error after `blocks` fused blocks in `prec`."""
    return L2_SAFETY * math.sqrt(max(1, blocks)) * SIGMA[prec]


def max_abs_bound(prec: str, blocks: int, ref) -> float:
    """Bound on max_i |err_i| after `blocks` fused blocks, for the exact result
    `ref` (a complex vector of 2^n amplitudes)."""
    import numpy as np
    ref = np.asarray(ref)
    n = int(ref.size).bit_length() - 1
    p = np.abs(ref) ** 2
    norm2 = float(p.sum())
    n_eff = norm2 * norm2 / float((p * p).sum())
    rms = math.sqrt(max(1, blocks)) * SIGMA[prec] * math.sqrt(norm2 / n_eff)
    return L2_SAFETY * rms * math.sqrt(n * math.log(2.0) + 14.0)
