"""Step a6, out = F + Phi Z, on the tensor cores (the BF16 form's apply for up to
64 channels, forced here; by default the batch takes it above 16 channels, or
above 8 when m >= 512) against the FP32 SIMT apply of the same plan and against
the CPU FP64 oracle.

The tensor-core form recomputes Phi in FP32 exactly as the SIMT kernel does,
splits Phi and Z into BF16 hi and lo parts and sums Phi_hi Z_hi + Phi_hi Z_lo +
Phi_lo Z_hi in FP32: each term keeps a relative error of about 3 x 2^-16 (the
two 16-bit splits and the dropped Phi_lo Z_lo), so its increment differs from
the SIMT kernel's by about 2^-16 of the terms' magnitude -- far inside the BF16
form's own bound, whose error comes from the BF16 Phi of B^T F.  Asserted here:
  - against the oracle: the BF16 form's three bounds (parity_checks);
  - against the SIMT apply (two identical plans: same features, Gram, G and Z):
    ||out_tc - out_simt||_F <= 2e-4 ||out_simt - F||_F, and every element within
    2e-3 of the largest increment element;
  - in place (out == F) bit for bit equal to out of place, and columns beyond c
    of a wider leading dimension never written.
Shapes span ragged point counts (a partial last 256-point tile), m with a
partial last chunk of 32 frequencies (m = 66, 130), channel counts that are not
multiples of 16 or of 4, and leading dimensions above c.
"""
import numpy as np
import pytest

import oracle
import parity_checks as pc
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
BF16 = rfd.RFD_BF16_TC


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _gfi(pts, F, eps, lam, m, seed, ld, tc, *, inplace=False):
    n, c = F.shape
    Fp = np.zeros((n, ld), np.float32)
    Fp[:, :c] = F
    P, Ft = _cuda(pts), _cuda(Fp)
    out = Ft if inplace else torch.full((n, ld), float("nan"), device=DEV)
    plan = rfd.Plan(n, m, eps, lam, seed, max_channels=c, precision=BF16, stream=torch.cuda.current_stream(DEV))
    try:
        assert rfd.lib.rfd_debug_plan_set_apply_tc(plan.handle, 2 if tc else 0) == 0, rfd.rfd_last_error()
        rfd.rfd_gfi(plan.handle, P, Ft, c, ld, out, ld)
        plan.sync()
        launches = plan.stats()["kernel_launches"]
    finally:
        plan.close()
    res = out.cpu().numpy()
    if ld > c and not inplace:
        assert np.isnan(res[:, c:]).all(), "columns beyond c were written"
    return res[:, :c], launches


CASES = [(3001, 130, 5, 8), (5000, 256, 12, 12), (1000, 64, 16, 19), (2600, 512, 33, 40), (700, 256, 64, 64),
         (513, 66, 64, 67), (257, 128, 7, 7)]


@pytest.mark.parametrize("n,m,c,ld", CASES)
def test_tensor_core_apply_matches_simt_and_oracle(n, m, c, ld):
    rng = synth.rng_for(23, c, n)
    pts = synth.unit_sphere(n, rng)
    F = synth.gaussian_field(n, c, 23, n)
    eps, seed = 0.1, 5
    lam = 0.1 * m / max(n, m)
    ref = oracle.rfd_gfi(pts, F, eps, lam, m, seed)
    out_tc, _ = _gfi(pts, F, eps, lam, m, seed, ld, True)
    out_simt, _ = _gfi(pts, F, eps, lam, m, seed, ld, False)
    e = pc.assert_matches(out_tc, ref, F, BF16, label=f"tensor-core apply N={n} m={m} c={c} ld={ld}")
    inc = out_simt.astype(np.float64) - F
    d = out_tc.astype(np.float64) - out_simt
    rel = np.linalg.norm(d) / np.linalg.norm(inc)
    worst = np.abs(d).max() / np.abs(inc).max()
    print(f"N={n} m={m} c={c}: vs oracle {e}, vs SIMT apply: frobenius {rel:.3e}, worst element {worst:.3e}")
    assert rel <= 2e-4, rel
    assert worst <= 2e-3, worst
    inpl, _ = _gfi(pts, F, eps, lam, m, seed, c, True, inplace=True)
    outp, _ = _gfi(pts, F, eps, lam, m, seed, c, True)
    np.testing.assert_array_equal(inpl, outp)


def test_tensor_core_apply_on_compact_plan_and_batch():
    """A compact plan's warm integration (Phi^T F from the points) with 24 channels,
    and a batch whose clouds take 1, 9 and 64 channels in one tensor-core launch
    (the default choice: the largest c is above 16)."""
    specs = synth.batched_specs(count=3, seed=31, n_lo=900, n_hi=9000, ms=(64, 128, 256), c=8)
    for s, c in zip(specs, (1, 9, 64)):
        s.c = c
    stream = torch.cuda.current_stream(DEV)
    clouds = [synth.make_cloud(s) for s in specs]
    lams = [s.lam * s.m / s.n for s in specs]
    plans = [rfd.Plan(s.n, s.m, s.eps, lam, s.seed, max_channels=64, precision=BF16, stream=stream)
             for s, lam in zip(specs, lams)]
    try:
        batch = rfd.Batch(plans, stream=stream)
        outs = batch.gfi([{"points": _cuda(p), "F": _cuda(F)} for p, F in clouds])
        batch.sync()
        for k, (s, (pts, F)) in enumerate(zip(specs, clouds)):
            ref = oracle.rfd_gfi(pts, F, s.eps, lams[k], s.m, s.seed)
            pc.assert_matches(outs[k].cpu().numpy(), ref, F, BF16, label=f"batched cloud {k} c={s.c}")
        batch.close()
        # compact: the same plan, integration from the points, 24 channels
        p0 = plans[2]
        p0.compact()
        F24 = synth.gaussian_field(specs[2].n, 24, 77, 2)
        got = p0.integrate(_cuda(F24))
        p0.sync()
        ref = oracle.rfd_gfi(clouds[2][0], F24, specs[2].eps, lams[2], specs[2].m, specs[2].seed)
        pc.assert_matches(got.cpu().numpy(), ref, F24, BF16, label="compact plan, 24 channels")
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("n,m,c,ld", [(3001, 130, 9, 9), (5000, 514, 17, 20), (2047, 256, 40, 40),
                                      (777, 1024, 64, 67)])
def test_tensor_core_field_from_points_matches_simt(n, m, c, ld):
    """A compact plan's B^T F from the points on the tensor cores (Phi^T and F split
    into BF16 hi / lo parts, K over the points) against the SIMT kernel of the same
    plan and against the oracle: point counts that are not multiples of 64 (a
    partial last step of a chunk), frequency tiles of 128 that the cloud's h fills
    only in part (m = 130, 514), leading dimensions above c."""
    rng = synth.rng_for(29, c, n)
    pts = synth.unit_sphere(n, rng)
    F = synth.gaussian_field(n, c, 29, n)
    eps, seed = 0.1, 7
    lam = 0.1 * m / max(n, m)
    ref = oracle.rfd_gfi(pts, F, eps, lam, m, seed)
    Fp = np.zeros((n, ld), np.float32)
    Fp[:, :c] = F
    P, Ft = _cuda(pts), _cuda(Fp)
    outs = {}
    for mode in (2, 0):
        plan = rfd.Plan(n, m, eps, lam, seed, max_channels=c, precision=BF16, stream=torch.cuda.current_stream(DEV))
        try:
            plan.features(P)
            plan.compact()
            assert rfd.lib.rfd_debug_plan_set_apply_tc(plan.handle, mode) == 0, rfd.rfd_last_error()
            out = torch.full((n, ld), float("nan"), device=DEV)
            rfd.rfd_integrate(plan.handle, Ft, c, ld, out, ld)
            plan.sync()
        finally:
            plan.close()
        res = out.cpu().numpy()
        if ld > c:
            assert np.isnan(res[:, c:]).all(), "columns beyond c were written"
        outs[mode] = res[:, :c]
    e = pc.assert_matches(outs[2], ref, F, BF16, label=f"tensor-core B^T F N={n} m={m} c={c} ld={ld}")
    inc = outs[0].astype(np.float64) - F
    d = outs[2].astype(np.float64) - outs[0]
    rel = np.linalg.norm(d) / np.linalg.norm(inc)
    worst = np.abs(d).max() / np.abs(inc).max()
    print(f"N={n} m={m} c={c}: vs oracle {e}, vs SIMT: frobenius {rel:.3e}, worst element {worst:.3e}")
    assert rel <= 2e-4, rel
    assert worst <= 2e-3, worst
