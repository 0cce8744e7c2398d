"""GPU Gromov-Wasserstein building blocks on two resident plans (App. C.2:
Eq. sq, Algorithms tensor_prod and line_search) against the oracle's, through
the C ABI; and the wide-matrix kernel action (column chunks of max_channels)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
EPS, M_FEAT = 0.1, 64


def _cloud(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    return (u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)


def _plans(prec, n1=600, n2=500, maxc=64):
    X, Y = _cloud(n1, 1), _cloud(n2, 2)
    lam1, lam2 = 0.05 * M_FEAT / n1, 0.05 * M_FEAT / n2
    st = torch.cuda.current_stream(DEV)
    pc = rfd.Plan(n1, M_FEAT, EPS, lam1, 11, max_channels=maxc, precision=prec, stream=st)
    pd = rfd.Plan(n2, M_FEAT, EPS, lam2, 12, max_channels=maxc, precision=prec, stream=st)
    pc.features(torch.from_numpy(X).to(DEV))
    pd.features(torch.from_numpy(Y).to(DEV))
    ac = oracle.rfd_kernel_action(X, EPS, lam1, M_FEAT, 11)
    ad = oracle.rfd_kernel_action(Y, EPS, lam2, M_FEAT, 12)
    return pc, pd, ac, ad


TOL = {rfd.RFD_FP32_PLAIN: 1e-4, rfd.RFD_BF16_TC: 5e-3}


@pytest.mark.parametrize("prec", [rfd.RFD_FP32_PLAIN, rfd.RFD_BF16_TC])
def test_fm_apply_wide_matrix(prec):
    pc, pd, ac, _ = _plans(prec)
    try:
        rng = np.random.default_rng(0)
        Xm = rng.standard_normal((pc.n, 300)).astype(np.float32)  # 300 columns > max_channels = 64
        got = pc.fm_apply(torch.from_numpy(Xm).to(DEV))
        pc.sync()
        assert oracle.rel_frobenius(got.cpu().numpy(), ac(Xm.astype(np.float64))) <= TOL[prec]
    finally:
        pc.close()
        pd.close()


@pytest.mark.parametrize("prec", [rfd.RFD_FP32_PLAIN, rfd.RFD_BF16_TC])
def test_tensor_product_and_line_search_match_oracle(prec):
    pc, pd, ac, ad = _plans(prec)
    try:
        rng = np.random.default_rng(1)
        n1, n2 = pc.n, pd.n
        T = rng.uniform(0.0, 1.0, (n1, n2))
        T /= T.sum()
        p, q = T.sum(1), T.sum(0)
        cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)
        L = rfd.gw_tensor_product(pc, pd, cuda(T), cuda(p), cuda(q))
        pc.sync()
        Lref = oracle.gw_tensor_product(ac, ad, T, p, q)
        err = oracle.rel_frobenius(L.cpu().numpy(), Lref)
        print(f"tensor product prec={prec}: rel err {err:.3e}")
        assert err <= TOL[prec]
        G = np.outer(p, q)
        Gt = rng.uniform(0.0, 1.0, (n1, n2))
        Gt /= Gt.sum()
        dG = Gt - G
        Mf = rng.uniform(0.0, 1.0, (n1, n2))
        alpha = 0.6
        tau, a, b = rfd.gw_line_search(pc, pd, alpha, cuda(G), cuda(dG), cuda(Mf), cuda(p), cuda(q))
        tr, ar, br = oracle.gw_line_search(ac, ad, alpha, G, dG, Mf, p, q)
        print(f"line search prec={prec}: tau {tau} vs {tr}, a {a} vs {ar}, b {b} vs {br}")
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
