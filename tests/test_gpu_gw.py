"""GPU Gromov-Wasserstein building blocks on two resident plans (App. C.2:
Eq. sq, Algorithms tensor_prod and line_search) against the oracle's, through
the C ABI; and the wide-matrix kernel action (column chunks of max_channels).

Inputs: two random 3-D point distributions with a random coupling (the App.
C.2 setting); the experiments' parameters (m = 16, eps = 0.3, lambda = -0.2 in
units of the estimator's mean eigenvalue N/m) and a narrower kernel."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TOL = {rfd.RFD_FP32_PLAIN: 1e-4, rfd.RFD_BF16_TC: 5e-3}
PARAMS = [(16, 0.3, -0.2), (64, 0.1, 0.05)]  # (m, eps, lambda in units of m / N)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def _setup(prec, m, eps, lam, n1=600, n2=500, maxc=64):
    X, Y, T, p, q, Gt, M = synth.gw_problem(n1, n2, seed=3)
    lam1, lam2 = lam * m / n1, lam * m / n2
    st = torch.cuda.current_stream(DEV)
    pc = rfd.Plan(n1, m, eps, lam1, 11, max_channels=maxc, precision=prec, stream=st)
    pd = rfd.Plan(n2, m, eps, lam2, 12, max_channels=maxc, precision=prec, stream=st)
    pc.features(_cuda(X))
    pd.features(_cuda(Y))
    ac = oracle.rfd_kernel_action(X, eps, lam1, m, 11)
    ad = oracle.rfd_kernel_action(Y, eps, lam2, m, 12)
    return pc, pd, ac, ad, (T, p, q, Gt, M)


@pytest.mark.parametrize("prec", [rfd.RFD_FP32_PLAIN, rfd.RFD_BF16_TC])
@pytest.mark.parametrize("m,eps,lam", PARAMS)
def test_fm_apply_wide_matrix(prec, m, eps, lam):
    pc, pd, ac, _, _ = _setup(prec, m, eps, lam)
    try:
        Xm = np.random.default_rng(0).standard_normal((pc.n, 300))  # 300 columns > max_channels = 64
        got = pc.fm_apply(_cuda(Xm))
        pc.sync()
        assert oracle.rel_frobenius(got.cpu().numpy(), ac(Xm)) <= TOL[prec]
    finally:
        pc.close()
        pd.close()


@pytest.mark.parametrize("prec", [rfd.RFD_FP32_PLAIN, rfd.RFD_BF16_TC])
@pytest.mark.parametrize("m,eps,lam", PARAMS)
def test_tensor_product_and_line_search_match_oracle(prec, m, eps, lam):
    pc, pd, ac, ad, (T, p, q, Gt, Mf) = _setup(prec, m, eps, lam)
    try:
        L = rfd.gw_tensor_product(pc, pd, _cuda(T), _cuda(p), _cuda(q))
        pc.sync()
        Lref = oracle.gw_tensor_product(ac, ad, T, p, q)
        err = oracle.rel_frobenius(L.cpu().numpy(), Lref)
        print(f"tensor product prec={prec} m={m}: rel err {err:.3e}")
        assert err <= TOL[prec]
        G = np.outer(p, q)
        dG = Gt - G
        alpha = 0.6
        tau, a, b = rfd.gw_line_search(pc, pd, alpha, _cuda(G), _cuda(dG), _cuda(Mf), _cuda(p), _cuda(q))
        tr, ar, br = oracle.gw_line_search(ac, ad, alpha, G, dG, Mf, p, q)
        print(f"line search prec={prec} m={m}: tau {tau} vs {tr}, a {a} vs {ar}, b {b} vs {br}")
        # Cauchy-Schwarz bounds: operands with relative error <= TOL move each
        # inner product by at most ~TOL times the product of the norms
        nrm = np.linalg.norm
        a1 = ad(np.ascontiguousarray(ac(dG).T)).T
        b1 = ad(np.ascontiguousarray(ac(G).T)).T
        c_cd = Lref + 2.0 * ad(np.ascontiguousarray(ac(T).T)).T  # v1 1^T + 1 v2^T
        scale_a = 2 * alpha * nrm(a1) * nrm(dG)
        scale_b = (nrm((1 - alpha) * Mf + alpha * c_cd) * nrm(dG) +
                   2 * alpha * (nrm(a1) * nrm(G) + nrm(b1) * nrm(dG)))
        assert abs(a - ar) <= 10 * TOL[prec] * scale_a
        assert abs(b - br) <= 10 * TOL[prec] * scale_b
        # tau follows the rule of Algorithm line_search from the device's (a, b)
        rule = min(1.0, max(0.0, -b / (2 * a))) if a > 0 else (1.0 if a + b < 0 else 0.0)
        assert tau == rule
        if abs(ar + br) > 10 * TOL[prec] * (scale_a + scale_b):
            assert abs(tau - tr) <= 0.05
    finally:
        pc.close()
        pd.close()


@pytest.mark.parametrize("n1,n2", [(300, 203), (77, 1000)])
def test_tensor_product_ragged_sizes(n1, n2):
    """Column counts that are not a multiple of 4 take the scalar assembly;
    row counts below one tile, and tiles cut by the row groups."""
    pc, pd, ac, ad, (T, p, q, _, _) = _setup(rfd.RFD_FP32_PLAIN, 16, 0.3, -0.2, n1=n1, n2=n2)
    try:
        L = rfd.gw_tensor_product(pc, pd, _cuda(T), _cuda(p), _cuda(q))
        pc.sync()
        assert oracle.rel_frobenius(L.cpu().numpy(), oracle.gw_tensor_product(ac, ad, T, p, q)) <= 1e-4
    finally:
        pc.close()
        pd.close()


def test_gw_argument_checks():
    pc, pd, _, _, (T, p, q, _, _) = _setup(rfd.RFD_FP32_PLAIN, 16, 0.3, -0.2, n1=100, n2=80)
    other = torch.cuda.Stream(DEV)
    pe = rfd.Plan(80, 16, 0.3, -0.01, 13, max_channels=64, precision=rfd.RFD_FP32_PLAIN, stream=other)
    try:
        with pytest.raises(RuntimeError):  # features not yet computed on pe, and another stream
            rfd.gw_tensor_product(pc, pe, _cuda(T), _cuda(p), _cuda(q))
        with pytest.raises(RuntimeError):
            rfd.gw_line_search(pc, pd, float("nan"), _cuda(T), _cuda(T), _cuda(T), _cuda(p), _cuda(q))
        with pytest.raises(RuntimeError):
            pc.fm_apply(torch.empty((100, 0), dtype=torch.float32, device=DEV))
    finally:
        pc.close()
        pd.close()
        pe.close()
