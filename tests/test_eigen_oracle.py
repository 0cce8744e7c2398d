"""The oracle's kernel eigenvalues (Sec. 3.3, App. E: eigenvalues of
exp(lambda W_hat) from the low-rank factors) pinned against what fixes them
independently of the m x m route:

  * brute force: the dense N x N matrix exp(lambda A B^T) (SciPy expm) and its
    symmetric eigenvalues (LAPACK eigvalsh), for N > m and N < m;
  * lambda = 0 gives N ones;
  * det exp(X) = exp(tr X): the eigenvalues' log-sum equals lambda tr W_hat,
    and tr W_hat = N sum_j 2 r_j / m in closed form (cos^2 + sin^2 = 1 per
    frequency);
  * largest=True is the descending order of the same multiset.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _cloud(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


@pytest.mark.parametrize("n,m", [(60, 16), (12, 32), (32, 32)])
def test_matches_dense_spectrum(n, m):
    X = _cloud(n, n)
    eps, lam, seed = 0.4, -0.3 * m / n, 7
    omega = oracle.sample_frequencies(m, eps, seed)
    r = oracle.weights(omega, eps)
    A, B = oracle.factors(X, omega, r)
    K = scipy.linalg.expm(lam * (A @ B.T))
    dense = np.sort(np.linalg.eigvalsh(0.5 * (K + K.T)))
    got = oracle.rfd_kernel_eigenvalues(X, eps, lam, m, seed)
    assert got.shape == (n,)
    np.testing.assert_allclose(got, dense, rtol=1e-9, atol=1e-11)
    top = oracle.rfd_kernel_eigenvalues(X, eps, lam, m, seed, k=5, largest=True)
    np.testing.assert_allclose(top, dense[::-1][:5], rtol=1e-9, atol=1e-11)


def test_lambda_zero_gives_ones():
    X = _cloud(50, 1)
    np.testing.assert_array_equal(oracle.rfd_kernel_eigenvalues(X, 0.2, 0.0, 16, 3), np.ones(50))


@pytest.mark.parametrize("n,m", [(200, 24), (2048, 64)])
def test_log_determinant_is_lambda_trace(n, m):
    X = _cloud(n, 2)
    eps, lam, seed = 0.1, -0.1 * m / n, 0
    kappa = oracle.rfd_kernel_eigenvalues(X, eps, lam, m, seed)
    r = oracle.weights(oracle.sample_frequencies(m, eps, seed), eps)
    trace = n * np.sum(2.0 * r / m)
    assert abs(np.sum(np.log(kappa)) - lam * trace) <= 1e-9 * max(1.0, abs(lam * trace))


def test_k_smallest_is_prefix_and_order():
    X = _cloud(300, 3)
    full = oracle.rfd_kernel_eigenvalues(X, 0.15, -0.1 * 32 / 300, 32, 5)
    assert np.all(np.diff(full) >= 0)
    np.testing.assert_array_equal(oracle.rfd_kernel_eigenvalues(X, 0.15, -0.1 * 32 / 300, 32, 5, k=32), full[:32])
    desc = oracle.rfd_kernel_eigenvalues(X, 0.15, -0.1 * 32 / 300, 32, 5, largest=True)
    np.testing.assert_array_equal(desc, full[::-1])
