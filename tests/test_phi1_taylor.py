"""The Taylor form of step a4 that the batched path evaluates (degree 16,
Paterson-Stockmeyer with blocks of four, scaling and squaring above
theta_16 = 0.977), checked on the CPU in FP64 against the oracle's phi1
(SciPy expm of the augmented matrix):

  * the truncation bound that defines theta_16: sum_{k > 16} theta^k/(k+1)!
    <= 2^-53 at theta = 0.977, and not at 1.0;
  * the Paterson-Stockmeyer grouping equals the plain Taylor sum;
  * below theta_16 the polynomial matches phi1 to FP64 rounding, and with
    s squarings by phi1(2Y) = (e^Y + I) phi1(Y) / 2, e^Y = I + Y phi1(Y), the
    result matches phi1 of the unscaled matrix to ~s u ||X||.
"""
import math

import numpy as np
import pytest

import oracle

THETA = 0.977


def taylor_ps(X):
    m = X.shape[0]
    I = np.eye(m)
    c = [1.0 / math.factorial(k + 1) for k in range(17)]
    X2 = X @ X
    X3 = X2 @ X
    X4 = X2 @ X2
    P = [I, X, X2, X3]
    F = sum(c[12 + i] * P[i] for i in range(4)) + c[16] * X4
    for j in (2, 1, 0):
        F = sum(c[4 * j + i] * P[i] for i in range(4)) + X4 @ F
    return F


def test_theta_is_the_truncation_bound():
    tail = lambda x: sum(x ** k / math.factorial(k + 1) for k in range(17, 60))
    assert tail(THETA) <= 2.0 ** -53
    assert tail(1.0) > 2.0 ** -53


def test_paterson_stockmeyer_equals_the_taylor_sum():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((12, 12))
    X *= 0.5 / np.abs(X).sum(0).max()
    plain = sum(np.linalg.matrix_power(X, k) / math.factorial(k + 1) for k in range(17))
    np.testing.assert_allclose(taylor_ps(X), plain, rtol=0, atol=1e-15)


@pytest.mark.parametrize("norm,m", [(0.1, 20), (0.5, 40), (0.97, 40), (3.0, 30), (40.0, 25)])
def test_scaled_taylor_matches_phi1(norm, m):
    rng = np.random.default_rng(int(norm * 100) + m)
    X = rng.standard_normal((m, m))
    X *= norm / np.abs(X).sum(0).max()
    s = 0 if norm <= THETA else math.ceil(math.log2(norm / THETA))
    Y = X / 2.0 ** s
    F = taylor_ps(Y)
    for _ in range(s):
        E = np.eye(m) + Y @ F
        F = 0.5 * (E @ F + F)
        Y = 2.0 * Y
    ref = oracle.phi1(X)
    assert oracle.rel_frobenius(F, ref) <= 2e-15 * max(1.0, s * norm)
