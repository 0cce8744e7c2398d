"""Kernel eigenvalues on the GPU (Sec. 3.3 / App. E: the k smallest or largest
eigenvalues of exp(lambda W_hat) from the low-rank factors) against the
oracle's, through the C ABI: single plans in both precisions, the rank-
deficient case N < m, ragged N, lambda = 0, batches of uneven N and m, and
the argument checks.

Tolerance: FP32 plain form 2e-5 relative per eigenvalue; BF16 form
2e-3 max(1, |lambda| ||M||_2) relative (an eigenvalue perturbation of M moves
exp(lambda mu) by |lambda| |d mu| relative, and the BF16 Gram moves M by
~1e-3 of its size)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _tol(prec, pts, eps, lam, m, seed):
    if prec == rfd.RFD_FP32_PLAIN:
        return 2e-5
    omega = oracle.sample_frequencies(m, eps, seed)
    A, B = oracle.factors(np.asarray(pts, np.float64), omega, oracle.weights(omega, eps))
    return 2e-3 * max(1.0, abs(lam) * np.linalg.norm(B.T @ A, 2))


def _check(got, ref, tol):
    got = np.asarray(got, np.float64)
    rel = np.max(np.abs(got - ref) / np.abs(ref))
    assert rel <= tol, (rel, tol)
    return rel


def _run_plan(pts, m, eps, lam, seed, prec, k, largest):
    st = torch.cuda.current_stream(DEV)
    pl = rfd.Plan(len(pts), m, eps, lam, seed, max_channels=4, precision=prec, stream=st)
    try:
        pl.features(torch.from_numpy(np.ascontiguousarray(pts, np.float32)).to(DEV))
        out = pl.eigenvalues(k, largest=largest)
        pl.sync()
        return out.cpu().numpy()
    finally:
        pl.close()


@pytest.mark.parametrize("prec", [rfd.RFD_FP32_PLAIN, rfd.RFD_BF16_TC])
@pytest.mark.parametrize("n,m,k,largest", [(2048, 64, 32, False), (2048, 64, 16, True), (1000, 128, 48, False),
                                           (40, 64, 40, False), (64, 64, 64, True), (300, 2, 5, True)])
def test_plan_eigenvalues_match_oracle(prec, n, m, k, largest):
    spec = synth.CloudSpec("sphere", n, m, 1, 0.1, -0.1, 5, sub=n)
    pts, _ = synth.make_cloud(spec)
    lam = -0.1 * m / n
    got = _run_plan(pts, m, 0.1, lam, 5, prec, k, largest)
    ref = oracle.rfd_kernel_eigenvalues(pts, 0.1, lam, m, 5, k=k, largest=largest)
    rel = _check(got, ref, _tol(prec, pts, 0.1, lam, m, 5))
    print(f"prec={prec} n={n} m={m} k={k} largest={largest}: max rel err {rel:.2e}")
    step = np.diff(got)
    assert np.all(step <= 0) if largest else np.all(step >= 0)


def test_lambda_zero_gives_ones():
    pts, _ = synth.make_cloud(synth.CloudSpec("torus", 500, 32, 1, 0.1, 0.0, 2))
    got = _run_plan(pts, 32, 0.1, 0.0, 2, rfd.RFD_BF16_TC, 20, False)
    np.testing.assert_array_equal(got, np.ones(20, np.float32))


def test_batch_eigenvalues_match_oracle_and_single_plans():
    specs = synth.batched_specs(count=12, seed=9, n_lo=300, n_hi=20000, ms=(32, 64, 128), c=1)
    clouds = [synth.make_cloud(s)[0] for s in specs]
    lams = [-0.1 * s.m / s.n for s in specs]
    st = torch.cuda.current_stream(DEV)
    plans = [rfd.Plan(s.n, s.m, s.eps, lam, s.seed, max_channels=4, precision=rfd.RFD_BF16_TC, stream=st)
             for s, lam in zip(specs, lams)]
    batch = rfd.Batch(plans, stream=st, timing=True)
    items = [{"points": torch.from_numpy(p).to(DEV)} for p in clouds]
    k = 16
    try:
        got = batch.eigenvalues(items, k).cpu().numpy()
        batch.sync()
        assert batch.stats()["step_ms"]["eigen"] > 0
        for i, (s, pts, lam) in enumerate(zip(specs, clouds, lams)):
            ref = oracle.rfd_kernel_eigenvalues(pts, s.eps, lam, s.m, s.seed, k=k)
            rel = _check(got[i], ref, _tol(rfd.RFD_BF16_TC, pts, s.eps, lam, s.m, s.seed))
            print(f"cloud {i}: N={s.n} m={s.m}: max rel err {rel:.2e}")
        # G is not computed by the eigenvalue pass
        with pytest.raises(RuntimeError):
            plans[0].integrate(torch.zeros((specs[0].n, 1), dtype=torch.float32, device=DEV))
        # the same clouds alone
        for i in (0, len(specs) - 1):
            plans[i].features(items[i]["points"])
            alone = plans[i].eigenvalues(k).cpu().numpy()
            # the tensor-core Gram's FP32 accumulation chains differ between the
            # batch and the lone plan (split-K lanes), so the two agree to the
            # BF16 form's tolerance, not bitwise
            rel = _check(alone, got[i].astype(np.float64), _tol(rfd.RFD_BF16_TC, clouds[i], specs[i].eps, lams[i],
                                                               specs[i].m, specs[i].seed))
            print(f"cloud {i} alone vs batch: max rel diff {rel:.2e}")
    finally:
        batch.close()
        for p in plans:
            p.close()


def test_eigenvalue_argument_checks():
    st = torch.cuda.current_stream(DEV)
    pts = torch.from_numpy(synth.make_cloud(synth.CloudSpec("sphere", 100, 16, 1, 0.1, 0.0, 1))[0]).to(DEV)
    pl = rfd.Plan(100, 16, 0.1, -0.01, 1, precision=rfd.RFD_BF16_TC, stream=st)
    big = rfd.Plan(100, 256, 0.1, -0.01, 1, precision=rfd.RFD_BF16_TC, stream=st)
    try:
        with pytest.raises(RuntimeError):  # features not yet computed
            pl.eigenvalues(4)
        pl.features(pts)
        big.features(pts)
        for bad in (0, 101):
            with pytest.raises(RuntimeError):
                pl.eigenvalues(bad)
        with pytest.raises(RuntimeError):  # m > 128
            big.eigenvalues(4)
        pl.sync()
    finally:
        pl.close()
        big.close()
