"""Pins of the CPU FP64 oracle against things other than itself.

Each check_* function states one fact fixed by the paper or by mathematics and
raises AssertionError when the oracle disagrees:

  brute force   exp(lambda A B^T) F by dense eigendecomposition (Sec. 2.4's
                identity not used)                                   -> steps a3..a6
  closed forms  phi1 of scalars, diagonal, nilpotent and rotation matrices
                E[W_hat(z)] = prod_d (Si(2piR(eps+z_d)) + Si(2piR(eps-z_d)))/pi (App. A.4)
                inverse Fourier transform of tau = the smoothed cube kernel
                trace(B^T A) = (2N/m) sum_j r_j  (cos^2 + sin^2 = 1)
  invariants    lambda = 0 gives F bit for bit; semigroup exp(l/2 W)^2 = exp(l W);
                symmetry of exp(lambda W_hat); small-lambda limit F + lambda W_hat F
  statistics    Var(W_hat) ~ 1/m (Lemma lemma:rfd, App. A.4); error to the exact
                kernel shrinks as m grows (App. E ablations)
  published     SplitMix64 reference outputs (tests/golden/)

The mutation tests at the bottom plant plausible mistakes in the oracle (on
the CPU) and check that at least one pin fails for each.
"""
import math
import os

import numpy as np
import pytest
import scipy.special
import scipy.stats

import oracle
import oracle.rfd as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cloud(n, seed=0, radius=1.0):
    return synth.unit_sphere(n, synth.rng_for(seed, 1, n), radius)


# ---------------------------------------------------------------------------
# check functions (also used by the mutation tests)
# ---------------------------------------------------------------------------
def check_brute_force(n=300, m=64, eps=0.1, lam=0.02, seed=1, c=3):
    pts = _cloud(n, seed)
    F = synth.gaussian_field(n, c, seed)
    out, parts = O.rfd_gfi(pts, F, eps, lam, m, seed, return_parts=True)
    # dense reference from W_hat formed straight from its definition (App. A.4):
    # W_hat(i,j) = (1/h) sum_k r_k cos(2 pi w_k^T (x_i - x_j))
    om, r = parts["omega"], parts["r"]
    X = pts.astype(np.float64)
    h = om.shape[0]
    W = np.zeros((n, n))
    for k in range(h):
        t = X @ om[k]
        W += r[k] * np.cos(2 * np.pi * (t[:, None] - t[None, :]))
    W /= h
    e, V = np.linalg.eigh(0.5 * (W + W.T))
    ref = V @ (np.exp(lam * e)[:, None] * (V.T @ F.astype(np.float64)))
    err = oracle.rel_frobenius(out, ref)
    assert err < 1e-10, f"brute force: rel err {err:.3e}"
    return err


def check_lowrank_equals_dense_lowrank(n=16, m=64, eps=0.2, lam=-0.3, seed=4):
    """N < m: B^T A is singular; phi1 still gives exp(lambda A B^T) F."""
    pts = _cloud(n, seed)
    F = synth.gaussian_field(n, 2, seed)
    out, parts = O.rfd_gfi(pts, F, eps, lam, m, seed, return_parts=True)
    assert np.linalg.matrix_rank(parts["M"]) <= n
    ref = O.dense_lowrank_gfi(parts["A"], parts["B"], F, lam)
    err = oracle.rel_frobenius(out, ref)
    assert err < 1e-10, f"singular case: {err:.3e}"


def check_trace_identity(n=500, m=128, eps=0.07, seed=2):
    pts = _cloud(n, seed)
    om = O.sample_frequencies(m, eps, seed)
    r = O.weights(om, eps)
    A, B = O.factors(pts, om, r)
    tr = np.trace(B.T @ A)
    expect = 2.0 * n / m * r.sum()
    assert abs(tr - expect) <= 1e-9 * abs(expect) + 1e-9, (tr, expect)


def check_expectation(eps=0.1, m=256, seeds=120):
    """Sample mean of W_hat(z) over independent frequency draws = f~_R(z)."""
    R = O.default_radius(eps)
    zs = np.array([[0.0, 0.0, 0.0], [0.03, -0.05, 0.02], [0.09, 0.0, -0.095], [0.12, 0.01, 0.0],
                   [0.2, -0.15, 0.1]])
    pts = np.concatenate([np.zeros((1, 3)), zs])
    vals = []
    for s in range(seeds):
        om = O.sample_frequencies(m, eps, 1000 + s)
        r = O.weights(om, eps)
        A, B = O.factors(pts, om, r)
        vals.append(A[1:] @ B[0])          # W_hat(z_i, 0)
    vals = np.array(vals)                  # seeds x len(zs)
    mean = vals.mean(0)
    se = vals.std(0, ddof=1) / math.sqrt(seeds)
    ref = O.smoothed_kernel(zs, eps, R)
    z = np.abs(mean - ref) / np.maximum(se, 1e-12)
    assert np.all(z < 5.0), f"E[W_hat] off by {z} standard errors (mean {mean}, closed form {ref})"


def check_tau_fourier(eps=0.05, R=20.0):
    """int_{-R}^{R} tau_1(w) cos(2 pi w z) dw equals the Si closed form, using the
    oracle's tau on (w, 0, 0) divided by its two other (constant) factors."""
    w = np.linspace(-R, R, 400001)
    t1 = O.tau(np.stack([w, np.zeros_like(w), np.zeros_like(w)], 1), eps) / (2 * eps) ** 2
    for z in (0.0, 0.02, 0.049, 0.051, 0.09):
        num = scipy.integrate.simpson(t1 * np.cos(2 * np.pi * w * z), x=w)
        si = (scipy.special.sici(2 * np.pi * R * (eps + z))[0] + scipy.special.sici(2 * np.pi * R * (eps - z))[0]) / np.pi
        assert abs(num - si) < 2e-6, (z, num, si)
    # as R grows the transform pair recovers the cube indicator: int tau_1 = f(0) = 1
    assert abs(scipy.special.sici(2 * np.pi * 1e6 * eps)[0] * 2 / np.pi - 1) < 1e-5


def check_density(eps=0.05):
    sigma, R = O.default_sigma(eps), O.default_radius(eps)
    w = np.linspace(-R, R, 200001)
    p = O.density(np.stack([w, np.zeros_like(w), np.zeros_like(w)], 1), sigma, R)
    p1_0 = 1.0 / (sigma * math.sqrt(2 * math.pi) * math.erf(R / (sigma * math.sqrt(2))))
    integral = scipy.integrate.simpson(p, x=w)
    assert abs(integral - p1_0 ** 2) < 1e-8 * p1_0 ** 2, (integral, p1_0 ** 2)
    # zero outside the truncation cube
    assert O.density(np.array([[R * 1.01, 0, 0]]), sigma, R)[0] == 0.0


def check_frequency_distribution(eps=0.05, m=4000, seed=3):
    om = O.sample_frequencies(m, eps, seed)
    sigma, R = O.default_sigma(eps), O.default_radius(eps)
    dist = scipy.stats.truncnorm(-R / sigma, R / sigma, scale=sigma)
    for d in range(3):
        p = scipy.stats.kstest(om[:, d], dist.cdf).pvalue
        assert p > 1e-3, (d, p)
    assert np.all(np.abs(om) <= R)


def check_phi1_closed_forms():
    xs = [1e-300, 1e-12, 1e-5, 0.3, -0.7, 2.0, -15.0, 30.0]
    for x in xs:
        got = O.phi1(np.array([[x]]))[0, 0]
        ref = math.expm1(x) / x
        assert abs(got - ref) <= 1e-14 * abs(ref), (x, got, ref)
    d = np.array([-3.0, -0.1, 0.0, 1e-9, 0.5, 4.0])
    ref = np.array([math.expm1(v) / v if v else 1.0 for v in d])
    # scaling and squaring loses ~ s * u * ||X|| (s squarings): a few 1e-13 at ||X|| = 4
    np.testing.assert_allclose(np.diag(O.phi1(np.diag(d))), ref, rtol=2e-12)
    assert np.abs(O.phi1(np.diag(d)) - np.diag(np.diag(O.phi1(np.diag(d))))).max() == 0.0
    rng = np.random.default_rng(0)
    N = np.triu(rng.standard_normal((6, 6)), 1)      # nilpotent: phi1 is a finite sum
    ref = np.zeros((6, 6))
    P = np.eye(6)
    for k in range(6):
        ref += P / math.factorial(k + 1)
        P = P @ N
    np.testing.assert_allclose(O.phi1(N), ref, rtol=1e-13, atol=1e-15)
    for th in (0.1, 1.3, 3.0, 7.5):                   # rotation generator: closed form
        X = np.array([[0.0, -th], [th, 0.0]])
        ref = np.array([[math.sin(th), -(1 - math.cos(th))], [1 - math.cos(th), math.sin(th)]]) / th
        np.testing.assert_allclose(O.phi1(X), ref, rtol=1e-13, atol=1e-15)


def check_lambda_zero():
    pts = _cloud(200, 9)
    F = synth.gaussian_field(200, 4, 9)
    out = O.rfd_gfi(pts, F, 0.1, 0.0, 32, 9)
    np.testing.assert_array_equal(out, F.astype(np.float64))


def check_semigroup_and_symmetry(n=400, m=64, eps=0.1, lam=0.01, seed=5):
    pts = _cloud(n, seed)
    F = synth.gaussian_field(n, 3, seed)
    om = O.sample_frequencies(m, eps, seed)
    r = O.weights(om, eps)
    once = O.rfd_gfi_from_plan(pts, F, lam, om, r)
    twice = O.rfd_gfi_from_plan(pts, O.rfd_gfi_from_plan(pts, F, lam / 2, om, r), lam / 2, om, r)
    assert oracle.rel_frobenius(twice, once) < 1e-11
    F1, F2 = F[:, :1], synth.gaussian_field(n, 1, seed + 1)
    a = float((F1.astype(np.float64) * O.rfd_gfi_from_plan(pts, F2, lam, om, r)).sum())
    b = float((O.rfd_gfi_from_plan(pts, F1, lam, om, r) * F2.astype(np.float64)).sum())
    assert abs(a - b) <= 1e-11 * (abs(a) + abs(b) + 1)


def check_small_lambda(n=300, m=64, eps=0.1, seed=6):
    pts = _cloud(n, seed)
    F = synth.gaussian_field(n, 2, seed).astype(np.float64)
    om = O.sample_frequencies(m, eps, seed)
    r = O.weights(om, eps)
    X = pts.astype(np.float64)
    t = X @ om.T                                          # n x h
    # W_hat F straight from the definition: (1/h) sum_k r_k cos(2 pi (t_ik - t_jk)) F_j
    C, S = np.cos(2 * np.pi * t), np.sin(2 * np.pi * t)
    WF = (C * r) @ (C.T @ F) / len(r) + (S * r) @ (S.T @ F) / len(r)
    errs = []
    for lam in (1e-2, 1e-3, 1e-4):
        out = O.rfd_gfi_from_plan(pts, F, lam, om, r)
        errs.append(oracle.rel_frobenius((out - F) / lam, WF))
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5, errs  # O(lambda)


def check_error_shrinks_with_m(n=128, eps=0.15, seeds=8):
    pts = _cloud(n, 7)
    R = O.default_radius(eps)
    Wt = O.smoothed_adjacency(pts, eps, R)
    errs = {}
    for m in (64, 1024):
        e = []
        for s in range(seeds):
            om = O.sample_frequencies(m, eps, 50 + s)
            r = O.weights(om, eps)
            A, B = O.factors(pts, om, r)
            e.append(np.linalg.norm(A @ B.T - Wt))
        errs[m] = float(np.mean(e))
    ratio = errs[64] / errs[1024]
    assert ratio > 2.5, f"error ratio m=64 -> 1024: {ratio:.2f} (expected ~4 for 1/sqrt(m))"


# ---------------------------------------------------------------------------
# the pins
# ---------------------------------------------------------------------------
def test_brute_force():
    check_brute_force()
    check_brute_force(n=512, m=128, eps=0.15, lam=-0.01, seed=8, c=1)


def test_singular_lowrank():
    check_lowrank_equals_dense_lowrank()


def test_trace_identity():
    check_trace_identity()


def test_expectation_matches_sine_integral_closed_form():
    check_expectation()


def test_tau_is_fourier_transform_of_cube():
    check_tau_fourier()


def test_density_normalised():
    check_density()


def test_frequency_distribution():
    check_frequency_distribution()


def test_phi1_closed_forms():
    check_phi1_closed_forms()


def test_lambda_zero_bitwise():
    check_lambda_zero()


def test_semigroup_and_symmetry():
    check_semigroup_and_symmetry()


def test_small_lambda_limit():
    check_small_lambda()


def test_error_shrinks_with_m():
    check_error_shrinks_with_m()


def test_exact_kernel_error_shrinks_with_m():
    """Against the exact indicator adjacency (N=256, literal lambda=0.1): the
    RFD result approaches exp(lambda W)F as m grows, down to the R-truncation
    floor (reported, asserted only as a decrease)."""
    spec = synth.config_single("tiny")
    pts, F = synth.make_cloud(spec)
    exact = O.dense_exact_gfi(pts, F, spec.eps, spec.lam)
    errs = []
    for m in (64, 512, 4096):
        e = [oracle.rel_frobenius(O.rfd_gfi(pts, F, spec.eps, spec.lam, m, s), exact) for s in range(4)]
        errs.append(float(np.mean(e)))
    print("error to exact exp(lambda W)F vs m=64,512,4096:", errs)
    assert errs[2] < errs[0]


def test_splitmix64_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        vals = [int(x) for x in f.read().split("\n", 3)[3].split()]
    g = O.SplitMix64(1234567)
    assert [g.next_u64() for _ in vals] == vals


def test_uniforms_in_open_interval():
    g = O.SplitMix64(0)
    u = np.array([g.next_uniform() for _ in range(20000)])
    assert u.min() > 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_golden_frequencies():
    """Frequencies for one seed, written by tests/golden/make_golden.py from the
    oracle: the oracle must stay bit-stable across machines (x86 here, Arm on
    the GPU machine) because the library's sampler is compared with it bit for bit."""
    path = os.path.join(GOLDEN, "omega_m64_eps0.1_seed0.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    ref = np.array([[float.fromhex(x) for x in row] for row in rows])
    np.testing.assert_array_equal(O.sample_frequencies(64, 0.1, 0), ref)


# ---------------------------------------------------------------------------
# planted mistakes: each must make at least one pin fail
# ---------------------------------------------------------------------------
def _fails(fn, *a, **k):
    try:
        fn(*a, **k)
    except AssertionError:
        return True
    return False


def test_mutation_scale_without_factor_two(monkeypatch):
    def bad(r, m):
        s = np.sqrt(np.abs(r) / m)
        return np.concatenate([s * np.sign(r)] * 2), np.concatenate([s] * 2)
    monkeypatch.setattr(O, "column_scales", bad)
    assert _fails(check_trace_identity) and _fails(check_expectation, seeds=40)


def test_mutation_sin_half_replaced(monkeypatch):
    def bad(points, omega):
        ang = 2.0 * np.pi * (np.asarray(points, np.float64) @ omega.T)
        return np.concatenate([np.cos(ang), np.cos(ang)], 1)
    monkeypatch.setattr(O, "features", bad)
    assert _fails(check_expectation, seeds=40) or _fails(check_trace_identity)


def test_mutation_paper_literal_tau_constants(monkeypatch):
    def bad(omega, eps):
        w = np.asarray(omega, np.float64)
        safe = np.where(w == 0, 1.0, w)
        return np.prod(np.where(w == 0, 2 * eps, np.sin(2 * eps * w) / safe), axis=-1)
    monkeypatch.setattr(O, "tau", bad)
    assert _fails(check_tau_fourier)


def test_mutation_transposed_gram(monkeypatch):
    orig = O.rfd_gfi

    def bad(points, F, eps, lam, m, seed, sigma=0.0, radius=0.0, *, return_parts=False):
        om = O.sample_frequencies(m, eps, seed, sigma, radius)
        r = O.weights(om, eps, sigma, radius)
        A, B = O.factors(points, om, r)
        M = A.T @ B                                        # wrong: A^T B instead of B^T A
        G = lam * O.phi1(lam * M)
        out = np.asarray(F, np.float64) + A @ (G @ (B.T @ np.asarray(F, np.float64)))
        return (out, dict(omega=om, r=r, A=A, B=B, M=M, G=G)) if return_parts else out
    monkeypatch.setattr(O, "rfd_gfi", bad)
    assert _fails(check_brute_force)
    monkeypatch.setattr(O, "rfd_gfi", orig)


def test_mutation_missing_outer_lambda(monkeypatch):
    orig_phi1 = O.phi1
    monkeypatch.setattr(O, "phi1", lambda X: orig_phi1(X) / 0.02 * 0.02 ** 0 if False else orig_phi1(X) * 50.0)
    assert _fails(check_brute_force)


def test_mutation_sign_of_weights_dropped(monkeypatch):
    orig = O.weights
    monkeypatch.setattr(O, "weights", lambda *a, **k: np.abs(orig(*a, **k)))
    assert _fails(check_expectation, seeds=40)
