"""GPU entropic Wasserstein barycenter (rfd_barycenter: repeated GFI on a resident
plan, App. C Algorithm wass_barycenter) against the oracle's, through the C ABI.

The scaling iteration needs a positive kernel action.  The random-feature
kernel exp(lambda W_hat) is positive only while lambda |W_hat - W| stays small
(many features, a short diffusion time): m = 1024 features on the 2048-point
sphere with lambda = 1e-3 and smooth inputs keep every kernel output positive
over the 8 passes compared here (the oracle checks this too)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


M_FEAT, LAM = 1024, 1e-3


def _case():
    spec = synth.config_single("small", None)
    pts, _ = synth.make_cloud(spec)
    n = spec.n
    p64 = np.asarray(pts, dtype=np.float64)

    def bump(c, s=0.5):
        d = np.linalg.norm(p64 - p64[c], axis=1)
        b = 1.0 + 0.5 * np.exp(-(d / s) ** 2)
        return b / b.sum()

    mus = np.stack([bump(0), bump(n // 4), bump(3 * n // 4)], axis=1).astype(np.float32)
    area = np.full(n, 1.0 / n, dtype=np.float32)
    return spec, pts, mus, area


def _gpu(spec, pts, mus, area, lam, prec, alpha, iters):
    plan = rfd.Plan(spec.n, M_FEAT, spec.eps, lam, spec.seed, max_channels=3, precision=prec)
    try:
        P = torch.from_numpy(pts).to(DEV)
        plan.features(P)
        out = plan.barycenter(torch.from_numpy(mus).to(DEV), torch.from_numpy(area).to(DEV), alpha, iters)
        plan.sync()
        return out.cpu().numpy().astype(np.float64)
    finally:
        plan.close()


@pytest.mark.parametrize("prec,tol", [(rfd.RFD_FP32_PLAIN, 1e-4), (rfd.RFD_BF16_TC, 1e-3)])
def test_barycenter_matches_oracle(prec, tol):
    spec, pts, mus, area = _case()
    alpha = [0.2, 0.3, 0.5]
    got = _gpu(spec, pts, mus, area, LAM, prec, alpha, 8)
    ref = oracle.rfd_barycenter(pts, mus.astype(np.float64), area.astype(np.float64), alpha, 8, spec.eps, LAM,
                                M_FEAT, spec.seed)
    err = oracle.rel_frobenius(got, ref)
    print(f"barycenter prec={prec}: rel err {err:.3e}")
    assert err <= tol


def test_barycenter_lambda_zero_is_the_geometric_mean():
    spec, pts, mus, area = _case()
    alpha = np.array([0.2, 0.3, 0.5])
    got = _gpu(spec, pts, mus, area, 0.0, rfd.RFD_FP32_PLAIN, alpha, 3)
    ref = np.exp(np.log(mus.astype(np.float64)) @ alpha)
    assert oracle.rel_frobenius(got, ref) <= 1e-5


def test_barycenter_argument_checks():
    spec, pts, mus, area = _case()
    plan = rfd.Plan(spec.n, spec.m, spec.eps, LAM, spec.seed, max_channels=2, precision=rfd.RFD_BF16_TC)
    try:
        M = torch.from_numpy(mus).to(DEV)
        A = torch.from_numpy(area).to(DEV)
        with pytest.raises(rfd.RfdError):  # before the features
            plan.barycenter(M[:, :2].contiguous(), A, [0.5, 0.5], 2)
        plan.features(torch.from_numpy(pts).to(DEV))
        with pytest.raises(rfd.RfdError):  # k > max_channels
            plan.barycenter(M, A, [1 / 3] * 3, 2)
        with pytest.raises(rfd.RfdError):  # negative weight
            plan.barycenter(M[:, :2].contiguous(), A, [1.5, -0.5], 2)
        out = plan.barycenter(M[:, :2].contiguous(), A, [0.5, 0.5], 0)  # no pass: mu = 1
        plan.sync()
        assert torch.all(out == 1.0)
    finally:
        plan.close()
