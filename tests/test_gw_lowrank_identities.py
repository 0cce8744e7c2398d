"""The re-association the GPU's low-rank GW path relies on, checked in FP64 on
the CPU: with C = I + Psi K Psi^T (Psi the features, K = diag(s sgn r) G diag(s))
and U = Psi K,

  * C^{(.)2} p = p (1 + 2 U_i . Psi_i) + U_i^T S U_i,  S = Psi^T D_p Psi;
  * C T D^T = T + U_C P' + Q U_D^T,  P = Psi_C^T T, Q = T Psi_D, R = P Psi_D,
    P' = P + R U_D^T;
  * <C X D^T, Y> = <X, Y> + sum_j P'_X[:, j] . (K_C^T P_Y[:, j]) + sum_i Q_X[i] . (Q_Y[i] K_D);

each against the dense matrices of the oracle's kernel action."""
import numpy as np

import oracle
import synth


def _factors(pts, eps, lam, m, seed):
    omega = oracle.sample_frequencies(m, eps, seed)
    r = oracle.weights(omega, eps)
    Psi = oracle.features(np.asarray(pts, np.float64), omega)
    oa, ob = oracle.column_scales(r, m)
    A, B = Psi * oa[None, :], Psi * ob[None, :]
    G = lam * oracle.phi1(lam * (B.T @ A))
    K = oa[:, None] * G * ob[None, :]
    C = np.eye(len(pts)) + Psi @ K @ Psi.T
    # the oracle's own action agrees with this dense C
    act = oracle.rfd_kernel_action(pts, eps, lam, m, seed)
    X = np.random.default_rng(0).standard_normal((len(pts), 3))
    assert oracle.rel_frobenius(act(X), C @ X) <= 1e-12
    return Psi, K, C


def test_lowrank_gw_identities():
    X1, X2, T, p, q, Gt, Mf = synth.gw_problem(70, 50, seed=4)
    m, eps = 16, 0.3
    Pc, Kc, C = _factors(X1, eps, -0.2 * m / 70, m, 11)
    Pd, Kd, D = _factors(X2, eps, -0.2 * m / 50, m, 12)
    Uc, Ud = Pc @ Kc, Pd @ Kd
    # Hadamard square (Eq. sq)
    S = Pc.T @ (p[:, None] * Pc)
    v = p * (1.0 + 2.0 * np.sum(Uc * Pc, axis=1)) + np.einsum("if,fg,ig->i", Uc, S, Uc)
    np.testing.assert_allclose(v, (C * C) @ p, rtol=1e-12, atol=1e-15)
    # sandwich C T D^T
    P = Pc.T @ T
    Q = T @ Pd
    R = P @ Pd
    Pp = P + R @ Ud.T
    W = T + Uc @ Pp + Q @ Ud.T
    np.testing.assert_allclose(W, C @ T @ D.T, rtol=1e-12, atol=1e-15)
    # inner products of the line search
    G = np.outer(p, q)
    dG = Gt - G

    def proj(Xm):
        Pm = Pc.T @ Xm
        Qm = Xm @ Pd
        return Pm, Qm, Pm + (Pm @ Pd) @ Ud.T

    for Xm, Ym in ((dG, dG), (dG, G), (G, dG)):
        PX, QX, PpX = proj(Xm)
        PY, QY, _ = proj(Ym)
        lhs = np.sum(Xm * Ym) + np.sum(PpX * (Kc.T @ PY)) + np.sum(QX * (QY @ Kd))
        assert abs(lhs - np.sum((C @ Xm @ D.T) * Ym)) <= 1e-12 * np.abs(C @ Xm @ D.T).sum() * np.abs(Ym).max()
