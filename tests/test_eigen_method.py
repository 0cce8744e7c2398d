"""The eigenvalue method of the GPU kernel, checked in FP64 on the CPU against
the oracle's route (LAPACK eig of B^T A): with Sigma = diag(sgn r) and
P = M Sigma = Omega_b Phi^T Phi Omega_b (symmetric positive semidefinite),

  * M Sigma is symmetric and P's Cholesky factor L gives eig(L^T Sigma L) = eig(M);
  * the round-robin ordering pairs every (p, q) exactly once per sweep of m - 1
    rounds, with disjoint pairs within a round;
  * cyclic Jacobi with those rounds (two-sided, 2 x 2 blocks) diagonalises
    L^T Sigma L to eigvalsh's values (the FP32-plain path);
  * Householder reduction to tridiagonal form and bisection on Sturm counts (the
    BF16-form path) reach eigvalsh's values, the zeros of a singular M included.
"""
import numpy as np

import oracle
import synth


def round_pairs(m, r):
    pairs = [(r, m - 1)] + [((r + q) % (m - 1), (r - q + m - 1) % (m - 1)) for q in range(1, m // 2)]
    return [(min(a, b), max(a, b)) for a, b in pairs]


def jacobi(H, sweeps=20, tol=1e-14):
    H = H.copy()
    m = len(H)
    fro = np.sum(H * H)
    for _ in range(sweeps):
        off = np.sum(H * H) - np.sum(np.diag(H) ** 2)
        if off <= tol * tol * fro:
            break
        for r in range(m - 1):
            J = np.eye(m)
            for p, q in round_pairs(m, r):
                if H[p, q] == 0.0:
                    continue
                tau = (H[q, q] - H[p, p]) / (2.0 * H[p, q])
                if abs(tau) > 1e150:
                    t = 0.5 / tau
                else:
                    t = np.sign(tau) / (abs(tau) + np.sqrt(1.0 + tau * tau)) if tau != 0 else 1.0
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                J[p, p] = J[q, q] = c
                J[p, q], J[q, p] = s, -s
            H = J.T @ H @ J
    return np.sort(np.diag(H))


def test_round_robin_covers_every_pair_once():
    for m in (2, 4, 10, 64):
        seen = []
        for r in range(m - 1):
            pr = round_pairs(m, r)
            flat = [x for p in pr for x in p]
            assert len(set(flat)) == len(flat) == m  # disjoint, all indices
            seen += pr
        assert sorted(seen) == sorted((a, b) for a in range(m) for b in range(a + 1, m))


def test_cholesky_form_and_jacobi_give_the_spectrum_of_M():
    spec = synth.CloudSpec("sphere", 2048, 64, 1, 0.1, -0.1, 5, sub=2048)
    pts, _ = synth.make_cloud(spec)
    omega = oracle.sample_frequencies(64, 0.1, 5)
    r = oracle.weights(omega, 0.1)
    A, B = oracle.factors(np.asarray(pts, np.float64), omega, r)
    M = B.T @ A
    oa, _ = oracle.column_scales(r, 64)
    sig = np.where(oa < 0, -1.0, 1.0)
    P = M * sig[None, :]
    np.testing.assert_allclose(P, P.T, rtol=0, atol=1e-12 * np.abs(P).max())
    L = np.linalg.cholesky(0.5 * (P + P.T))
    H = L.T @ (sig[:, None] * L)
    ref = np.sort(np.linalg.eigvals(M).real)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(H)), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    np.testing.assert_allclose(jacobi(H), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


# ---- the BF16-form path: Householder tridiagonal form, then Sturm bisection ----

def householder_tridiagonal(H):
    """(d, e2): diagonal and squared off-diagonal of the tridiagonal form, by the
    kernel's steps: v = x - alpha e1 with alpha = -sign(x0) ||x||, beta = 1 / (||x||^2
    - alpha x0), p = beta H' v, w = p - (beta v.p / 2) v, H' -= v w^T + w v^T."""
    H = H.copy()
    m = len(H)
    d = np.zeros(m)
    e2 = np.zeros(max(m - 1, 0))
    for k in range(m - 2):
        x = H[k + 1:, k].copy()
        ss = x @ x
        x0 = x[0]
        alpha = x0
        if ss - x0 * x0 > 1e-30 * ss:
            alpha = -np.sqrt(ss) if x0 > 0 else np.sqrt(ss)
            beta = 1.0 / (ss - alpha * x0)
            v = x.copy()
            v[0] -= alpha
            Hs = H[k + 1:, k + 1:]
            p = beta * (Hs @ v)
            w = p - 0.5 * beta * (v @ p) * v
            H[k + 1:, k + 1:] = Hs - np.outer(v, w) - np.outer(w, v)
        d[k] = H[k, k]
        e2[k] = alpha * alpha
    if m >= 2:
        d[m - 2] = H[m - 2, m - 2]
        e2[m - 2] = H[m - 1, m - 2] ** 2
    d[m - 1] = H[m - 1, m - 1]
    return d, e2


def sturm_bisection(d, e2, tol_rel=1e-15):
    """All eigenvalues of the tridiagonal matrix (d, sqrt(e2)), ascending, each by
    bisection on the count of negative pivots of T - x I (the kernel's Sturm count)."""
    m = len(d)
    e = np.sqrt(e2)
    r = np.array([(e[i - 1] if i > 0 else 0.0) + (e[i] if i + 1 < m else 0.0) for i in range(m)])
    lo, hi = np.min(d - r), np.max(d + r)
    w = max(abs(lo), abs(hi))
    lo, hi = lo - 1e-6 * w - 1e-300, hi + 1e-6 * w + 1e-300
    pivmin = 1e-300 * max(1.0, w)
    out = []
    for i in range(m):
        a, b = lo, hi
        for _ in range(200):
            if b - a <= tol_rel * w:
                break
            x = 0.5 * (a + b)
            cnt, q = 0, 1.0
            for j in range(m):
                q = (d[j] - x) - (e2[j - 1] / q if j > 0 else 0.0)
                if abs(q) < pivmin:
                    q = -pivmin
                cnt += q < 0
            if cnt > i:
                b = x
            else:
                a = x
        out.append(0.5 * (a + b))
    return np.array(out)


def test_tridiagonal_and_bisection_reach_eigvalsh():
    rng = np.random.default_rng(5)
    for m in (1, 2, 3, 7, 32, 64):
        A = rng.standard_normal((m, m))
        H = A + A.T
        d, e2 = householder_tridiagonal(H)
        got = sturm_bisection(d, e2)
        ref = np.linalg.eigvalsh(H)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got - ref).max() <= 1e-11 * scale, (m, np.abs(got - ref).max())


def test_tridiagonal_path_on_rank_deficient_kernel():
    """The kernel's input for a cloud with N < m: M = B^T A is singular, P = M Sigma
    positive semidefinite; with any square root L of P (P = L L^T), the reduction
    and the counts give eig(M), the zeros included."""
    spec = synth.CloudSpec("sphere", 40, 64, 1, 0.1, -0.1, 5, sub=40)
    pts, _ = synth.make_cloud(spec)
    omega = oracle.sample_frequencies(64, 0.1, 5)
    r = oracle.weights(omega, 0.1)
    A, B = oracle.factors(np.asarray(pts, np.float64), omega, r)
    M = B.T @ A
    oa, _ = oracle.column_scales(r, 64)
    sig = np.where(oa < 0, -1.0, 1.0)
    P = 0.5 * (M * sig[None, :] + (M * sig[None, :]).T)
    w, V = np.linalg.eigh(P)
    L = V * np.sqrt(np.clip(w, 0.0, None))
    H = L.T @ (sig[:, None] * L)
    d, e2 = householder_tridiagonal(H)
    got = np.sort(sturm_bisection(d, e2))
    ref = np.sort(np.linalg.eigvals(M).real)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
