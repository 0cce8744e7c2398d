"""Threshold-function variants of step a1 (only tau, hence r = tau/p, changes):

  ball:     f = 1[||z||_2 <= eps] in R^3 (the Bessel-function case of Sec. 2.4);
  cube_l1:  f = ||z||_1 1[||z||_inf <= eps] (the distance-weighted adjacency of the
            paper's brute-force baseline, on the cube of the unweighted reading).

Pins: the oracle's tau against a direct quadrature of the Fourier integral (a
different route to the same number: a radial 1-D integral for the ball, the
3-D integral over the cube for cube_l1); tau(0) = the integral of f; the
estimator's expectation reproduces f where the two kernels differ; the library's
host sampler draws the same weights; and the low-rank oracle equals
exp(lambda W_hat) F formed densely (P1) with the variant's weights."""
import numpy as np
import pytest
import scipy.integrate

import oracle

EPS = 0.1


def _tau_quadrature(w_norm, eps):
    # int_{|z| <= eps} cos(2 pi w.z) dz: integrating over directions leaves
    # 4 pi int_0^eps r^2 sin(2 pi |w| r) / (2 pi |w| r) dr
    q = 2.0 * np.pi * w_norm
    f = lambda rr: 4.0 * np.pi * rr * rr * np.sinc(q * rr / np.pi)
    val, _ = scipy.integrate.quad(f, 0.0, eps, epsabs=0.0, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("w", [0.0, 0.3, 1.0, 2.7, 5.0, 13.0, 40.0, 120.0])
def test_tau_ball_matches_quadrature(w):
    for direction in (np.array([1.0, 0.0, 0.0]), np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0),
                      np.array([0.6, -0.8, 0.0])):
        t = oracle.tau((w * direction)[None, :], EPS, "ball")[0]
        ref = _tau_quadrature(w, EPS)
        assert abs(t - ref) <= 1e-12 * max(abs(ref), 1e-6 * 4.0 / 3.0 * np.pi * EPS ** 3)


def test_tau_ball_at_zero_is_the_volume():
    assert oracle.tau(np.zeros((1, 3)), EPS, "ball")[0] == pytest.approx(4.0 / 3.0 * np.pi * EPS ** 3, rel=1e-15)


def test_estimator_separates_ball_from_cube():
    """z = (0.8 eps, 0.8 eps, 0) lies in the cube (||z||_inf = 0.8 eps) but not in
    the ball (||z||_2 = 1.13 eps): the mean of W_hat(z) over seeds is near 1 for
    the cube and near 0 for the ball (wide band: sigma = 1/eps, R = 3/eps)."""
    z = np.array([0.8 * EPS, 0.8 * EPS, 0.0])
    m, sigma, R = 4096, 1.0 / EPS, 3.0 / EPS
    means = {}
    for kernel in ("cube", "ball"):
        vals = []
        for s in range(16):
            om = oracle.sample_frequencies(m, EPS, 100 + s, sigma, R)
            r = oracle.weights(om, EPS, sigma, R, kernel)
            vals.append((2.0 / m) * np.sum(r * np.cos(2.0 * np.pi * om @ z)))
        means[kernel] = float(np.mean(vals))
    assert means["cube"] > 0.7 and means["ball"] < 0.3, means


@pytest.mark.parametrize("kernel", ["ball", "cube_l1", "l1_ball"])
def test_host_sampler_draws_the_oracle_weights(kernel):
    rfd = pytest.importorskip("paper_2302_00942_gb300")
    for seed in (0, 5):
        om, r = rfd.rfd_sample_weights(256, EPS, seed, kernel=kernel)
        om_ref = oracle.sample_frequencies(256, EPS, seed)
        np.testing.assert_array_equal(om, om_ref)
        ref = oracle.weights(om_ref, EPS, kernel=kernel)
        np.testing.assert_allclose(r, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        om_c, _ = rfd.rfd_sample_weights(256, EPS, seed, kernel="cube")
        np.testing.assert_array_equal(om_c, om)  # the draw does not depend on the kernel


@pytest.mark.parametrize("kernel", ["ball", "cube_l1", "l1_ball"])
def test_lowrank_oracle_equals_dense_exponential(kernel):
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.0, 0.5, size=(300, 3))
    F = rng.standard_normal((300, 2))
    out, parts = oracle.rfd_gfi(pts, F, EPS, 0.05, 64, 11, return_parts=True, kernel=kernel)
    dense = oracle.dense_lowrank_gfi(parts["A"], parts["B"], F, 0.05)
    assert oracle.rel_frobenius(out, dense) <= 1e-10


@pytest.mark.parametrize("w", [[0.0, 0.0, 0.0], [2.0, -3.0, 1.0], [7.0, 0.5, -11.0], [0.01, 40.0, -0.2]])
def test_tau_cube_l1_matches_quadrature(w):
    w = np.array(w)
    f = lambda z2, z1, z0: (abs(z0) + abs(z1) + abs(z2)) * np.cos(2.0 * np.pi * (w[0] * z0 + w[1] * z1 + w[2] * z2))
    ref, _ = scipy.integrate.tplquad(f, -EPS, EPS, -EPS, EPS, -EPS, EPS, epsabs=1e-14, epsrel=1e-10)
    t = oracle.tau(w[None, :], EPS, "cube_l1")[0]
    assert abs(t - ref) <= 1e-9 * max(abs(ref), 1e-3 * 12.0 * EPS ** 4)


def test_tau_cube_l1_at_zero_is_the_integral():
    # int over the cube of |z_1| + |z_2| + |z_3| = 3 eps^2 (2 eps)^2
    assert oracle.tau(np.zeros((1, 3)), EPS, "cube_l1")[0] == pytest.approx(12.0 * EPS ** 4, rel=1e-14)


def test_estimator_reproduces_the_weighted_cube():
    """E[W_hat(z)] ~ ||z||_1 inside the cube, ~0 outside it and at z = 0 (wide band)."""
    m, sigma, R = 4096, 1.0 / EPS, 3.0 / EPS
    def mean_w(z):
        vals = []
        for s in range(16):
            om = oracle.sample_frequencies(m, EPS, 100 + s, sigma, R)
            r = oracle.weights(om, EPS, sigma, R, "cube_l1")
            vals.append((2.0 / m) * np.sum(r * np.cos(2.0 * np.pi * om @ np.asarray(z))))
        return float(np.mean(vals))
    assert abs(mean_w([0.5 * EPS, 0.5 * EPS, 0.0]) - EPS) < 0.4 * EPS
    assert abs(mean_w([1.5 * EPS, 0.0, 0.0])) < 0.4 * EPS
    assert abs(mean_w([0.0, 0.0, 0.0])) < 0.4 * EPS


# ---- the L1 ball (octahedron) -------------------------------------------------

def test_tau_l1_ball_at_zero_is_the_volume():
    assert oracle.tau(np.zeros((1, 3)), EPS, "l1_ball")[0] == pytest.approx(4.0 / 3.0 * EPS ** 3, rel=1e-13)


@pytest.mark.parametrize("w", [3.0, -17.0, 0.4])
def test_tau_l1_ball_on_an_axis(w):
    """w = (w, 0, 0): the cross-section of the octahedron at z_1 is a square of
    area 2 (eps - |z_1|)^2, so tau = int cos(2 pi w z) 2 (eps - |z|)^2 dz."""
    f = lambda z: np.cos(2.0 * np.pi * w * z) * 2.0 * (EPS - abs(z)) ** 2
    ref, _ = scipy.integrate.quad(f, -EPS, EPS, epsabs=0.0, epsrel=1e-13, limit=200, points=[0.0])
    t = oracle.tau(np.array([[w, 0.0, 0.0]]), EPS, "l1_ball")[0]
    assert abs(t - ref) <= 1e-11 * 4.0 / 3.0 * EPS ** 3


@pytest.mark.parametrize("w", [[2.0, -3.0, 1.0], [7.0, 0.5, -11.0], [4.0, 4.0, 4.0], [-6.0, 6.0, 0.0]])
def test_tau_l1_ball_matches_quadrature(w):
    w = np.array(w)
    f = lambda z2, z1, z0: np.cos(2.0 * np.pi * (w[0] * z0 + w[1] * z1 + w[2] * z2))
    r1 = lambda z0: EPS - abs(z0)
    r2 = lambda z0, z1: EPS - abs(z0) - abs(z1)
    ref, _ = scipy.integrate.tplquad(f, -EPS, EPS, lambda z0: -r1(z0), r1, lambda z0, z1: -r2(z0, z1), r2,
                                     epsabs=1e-14, epsrel=1e-10)
    t = oracle.tau(w[None, :], EPS, "l1_ball")[0]
    assert abs(t - ref) <= 1e-8 * 4.0 / 3.0 * EPS ** 3


def test_estimator_separates_l1_ball_from_l2_ball():
    """z = (0.6 eps, 0.6 eps, 0) lies in the L2 ball (||z||_2 = 0.85 eps) but not in
    the L1 ball (||z||_1 = 1.2 eps); z = (0.3 eps, 0.3 eps, 0) lies in both."""
    m, sigma, R = 4096, 1.0 / EPS, 3.0 / EPS
    def mean_w(z, kernel):
        vals = []
        for s in range(16):
            om = oracle.sample_frequencies(m, EPS, 100 + s, sigma, R)
            r = oracle.weights(om, EPS, sigma, R, kernel)
            vals.append((2.0 / m) * np.sum(r * np.cos(2.0 * np.pi * om @ np.asarray(z))))
        return float(np.mean(vals))
    out = [0.6 * EPS, 0.6 * EPS, 0.0]
    assert mean_w(out, "l1_ball") < 0.3 and mean_w(out, "ball") > 0.7
    assert mean_w([0.3 * EPS, 0.3 * EPS, 0.0], "l1_ball") > 0.7


def test_host_l1_ball_weights_in_a_wide_band():
    """The host evaluates the octahedron's divided differences by scaling and
    squaring exp of the bidiagonal node matrix (a power series would cancel at
    nodes of modulus ~6 pi, the frequency radius 3/eps): within 1e-13 of the
    largest weight."""
    rfd = pytest.importorskip("paper_2302_00942_gb300")
    sigma, R = 1.0 / EPS, 3.0 / EPS
    om, r = rfd.rfd_sample_weights(512, EPS, 9, sigma, R, kernel="l1_ball")
    ref = oracle.weights(oracle.sample_frequencies(512, EPS, 9, sigma, R), EPS, sigma, R, "l1_ball")
    np.testing.assert_allclose(r, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
