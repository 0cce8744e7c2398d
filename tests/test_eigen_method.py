"""The eigenvalue method of the GPU kernel, checked in FP64 on the CPU against
the oracle's route (LAPACK eig of B^T A): with Sigma = diag(sgn r) and
P = M Sigma = Omega_b Phi^T Phi Omega_b (symmetric positive semidefinite),

  * M Sigma is symmetric and P's Cholesky factor L gives eig(L^T Sigma L) = eig(M);
  * the round-robin ordering pairs every (p, q) exactly once per sweep of m - 1
    rounds, with disjoint pairs within a round;
  * cyclic Jacobi with those rounds (two-sided, 2 x 2 blocks) diagonalises
    L^T Sigma L to eigvalsh's values.
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
