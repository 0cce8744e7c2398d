"""The oracle's Gromov-Wasserstein tensor product and line search with
implicit structure matrices (App. C.2): pins against direct definitions.

  * Eq. sq: C^{(.)2} p from two actions of C equals the Hadamard square of the
    dense C times p.
  * Algorithm tensor_prod equals the defining four-index sum
    L_ij = sum_kl (C_ik - D_jl)^2 T_kl (brute force on small clouds).
  * Algorithm line_search's a and b are the coefficients of the quadratic
    cost(G + tau dG) in tau (checked by evaluating the cost at three taus), and
    tau minimises it on [0, 1].
"""
import numpy as np

import oracle

rng = np.random.default_rng(5)


def _dense_kernels(n1=30, n2=24):
    X = rng.uniform(0.0, 0.4, size=(n1, 3))
    Y = rng.uniform(0.0, 0.4, size=(n2, 3))
    ac = oracle.rfd_kernel_action(X, 0.1, 0.02, 64, 1)
    ad = oracle.rfd_kernel_action(Y, 0.1, 0.02, 64, 2)
    C = ac(np.eye(n1))
    D = ad(np.eye(n2))
    D = 0.5 * (D + D.T)  # exp(lambda W_hat) is symmetric; remove rounding asymmetry for the brute force
    return ac, ad, C, D


def test_hadamard_square_from_two_actions():
    ac, _, C, _ = _dense_kernels()
    p = rng.uniform(0.1, 1.0, C.shape[0])
    np.testing.assert_allclose(oracle.hadamard_square_action(ac, p), (C * C) @ p, rtol=1e-12)


def test_tensor_product_equals_the_four_index_sum():
    ac, _, C, D = _dense_kernels()
    ad = lambda X: D @ X
    n1, n2 = C.shape[0], D.shape[0]
    T = rng.uniform(0.0, 1.0, (n1, n2))
    T /= T.sum()
    p, q = T.sum(1), T.sum(0)
    L = oracle.gw_tensor_product(ac, ad, T, p, q)
    ref = np.einsum("ikjl,kl->ij", (C[:, :, None, None] - D[None, None, :, :]) ** 2, T)
    np.testing.assert_allclose(L, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_line_search_coefficients_and_step():
    ac, _, C, D = _dense_kernels()
    ad = lambda X: D @ X
    n1, n2 = C.shape[0], D.shape[0]
    p, q = np.full(n1, 1.0 / n1), np.full(n2, 1.0 / n2)
    G = np.outer(p, q)
    Gt = rng.uniform(0.0, 1.0, (n1, n2))
    Gt /= Gt.sum()
    dG = Gt - G
    M = rng.uniform(0.0, 1.0, (n1, n2))
    alpha = 0.6
    tau, a, b = oracle.gw_line_search(ac, ad, alpha, G, dG, M, p, q)
    c_cd = ((C * C) @ p)[:, None] + ((D * D) @ q)[None, :]

    def cost(Gx):  # FGW objective: (1 - alpha) <M, G> + alpha <c_CD - 2 C G D, G>
        return (1 - alpha) * np.sum(M * Gx) + alpha * np.sum((c_cd - 2.0 * C @ Gx @ D) * Gx)

    f = [cost(G + t * dG) for t in (0.0, 0.5, 1.0)]
    a_fit = 2.0 * (f[2] - 2.0 * f[1] + f[0])   # f(t) = a t^2 + b t + c
    b_fit = f[2] - f[0] - a_fit
    assert abs(a - a_fit) <= 1e-9 * max(1.0, abs(a_fit))
    assert abs(b - b_fit) <= 1e-9 * max(1.0, abs(b_fit))
    ts = np.linspace(0.0, 1.0, 1001)
    best = ts[np.argmin([a * t * t + b * t for t in ts])]
    assert abs(tau - best) <= 1e-3 + 1e-12
