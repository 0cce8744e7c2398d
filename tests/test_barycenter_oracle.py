"""The oracle's entropic Wasserstein barycenter (App. C, Algorithm
wass_barycenter): pins independent of the paper's meshes (which are not here).

  * lambda = 0 makes the kernel the identity; the iteration then settles after
    one pass on the weighted geometric mean prod_i (mu^i)^alpha_i (closed form).
  * The low-rank kernel action equals the dense exp(lambda W_hat) formed by an
    eigendecomposition (the same algorithm through a different operator route).
  * Permuting the inputs together with their weights leaves the result unchanged.
  * A single input with weight 1 and the identity kernel is returned unchanged.
"""
import numpy as np

import oracle
import synth


def _setup(n_sub=None):
    spec = synth.config_single("small", None)
    pts, _ = synth.make_cloud(spec)
    pts = np.asarray(pts, dtype=np.float64)
    if n_sub:
        pts = pts[:n_sub]
    n = pts.shape[0]

    def bump(c, s=0.3):
        d = np.linalg.norm(pts - pts[c], axis=1)
        b = np.exp(-(d / s) ** 2) + 1e-3
        return b / b.sum()

    mus = np.stack([bump(0), bump(n // 4), bump(3 * n // 4)], axis=1)
    return spec, pts, mus, np.full(n, 1.0 / n)


def test_lambda_zero_gives_the_weighted_geometric_mean():
    spec, pts, mus, area = _setup()
    alpha = np.array([0.2, 0.3, 0.5])
    mu = oracle.rfd_barycenter(pts, mus, area, alpha, 4, spec.eps, 0.0, spec.m, spec.seed)
    np.testing.assert_allclose(mu, np.exp(np.log(mus) @ alpha), rtol=1e-13)


def test_single_input_identity_kernel_is_returned():
    spec, pts, mus, area = _setup()
    mu = oracle.rfd_barycenter(pts, mus[:, :1], area, [1.0], 3, spec.eps, 0.0, spec.m, spec.seed)
    np.testing.assert_allclose(mu, mus[:, 0], rtol=1e-13)


def test_lowrank_action_equals_dense_exponential():
    spec, pts, mus, area = _setup(n_sub=400)
    lam = spec.lam * spec.m / pts.shape[0]
    omega = oracle.sample_frequencies(spec.m, spec.eps, spec.seed)
    r = oracle.weights(omega, spec.eps)
    A, B = oracle.factors(pts, omega, r)
    W = A @ B.T
    W = 0.5 * (W + W.T)
    e, V = np.linalg.eigh(W)
    K = (V * np.exp(lam * e)) @ V.T
    dense = oracle.wasserstein_barycenter(lambda X: K @ X, mus, area, [1 / 3] * 3, 6)
    low = oracle.rfd_barycenter(pts, mus, area, [1 / 3] * 3, 6, spec.eps, lam, spec.m, spec.seed)
    assert oracle.rel_frobenius(low, dense) <= 1e-9


def test_permuting_inputs_with_weights_is_invariant():
    spec, pts, mus, area = _setup()
    lam = spec.lam * spec.m / pts.shape[0]
    alpha = np.array([0.2, 0.3, 0.5])
    a = oracle.rfd_barycenter(pts, mus, area, alpha, 5, spec.eps, lam, spec.m, spec.seed)
    perm = [2, 0, 1]
    b = oracle.rfd_barycenter(pts, mus[:, perm], area, alpha[perm], 5, spec.eps, lam, spec.m, spec.seed)
    np.testing.assert_allclose(a, b, rtol=1e-12)
