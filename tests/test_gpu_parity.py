"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Every whole-path check asserts, on the same seeded inputs (parity_checks):
  the whole output   FP32 plain <= 1e-5, BF16 tensor core <= 1e-3 (relative Frobenius);
  the increment      out - F against ref - F: FP32 <= 1e-4, BF16 <= 2e-2;
  every row          max_i ||out_i - ref_i|| <= the increment bound x max_i ||ref_i - F_i||.
Step a4 alone (FP64 on both sides): <= 1e-12.
"""
import numpy as np
import pytest

import oracle
import parity_checks as pc
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

TOL = {rfd.RFD_FP32_PLAIN: 1e-5, rfd.RFD_BF16_TC: 1e-3}
PRECS = [rfd.RFD_FP32_PLAIN, rfd.RFD_BF16_TC]
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def gpu_gfi(pts, F, eps, lam, m, seed, precision, *, api="gfi", max_channels=None, ld=None, inplace=False,
            kernel="cube"):
    n, c = F.shape
    ld = ld or c
    Fp = np.zeros((n, ld), np.float32)
    Fp[:, :c] = F
    P, Ft = _cuda(pts), _cuda(Fp)
    out = Ft if inplace else torch.full((n, ld), float("nan"), device=DEV)
    plan = rfd.Plan(n, m, eps, lam, seed, max_channels=max_channels or c, precision=precision,
                    stream=torch.cuda.current_stream(DEV), kernel=kernel)
    try:
        if api == "gfi":
            rfd.rfd_gfi(plan.handle, P, Ft, c, ld, out, ld)
        else:
            plan.features(P)
            rfd.rfd_integrate(plan.handle, Ft, c, ld, out, ld)
        plan.sync()
        stats = plan.stats()
        om, r, G = plan.export()
    finally:
        plan.close()
    res = out.cpu().numpy()
    if ld > c and not inplace:
        assert np.isnan(res[:, c:]).all(), "columns beyond c were written"
    return res[:, :c], stats, (om, r, G)


def small_case(name="small", c=None):
    spec = synth.config_single(name, c)
    pts, F = synth.make_cloud(spec)
    lam = spec.lam * spec.m / spec.n
    return spec, pts, F, lam


@pytest.mark.parametrize("prec", PRECS)
def test_small_config_matches_oracle(prec):
    spec, pts, F, lam = small_case()
    ref, parts = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, return_parts=True)
    out, stats, (om, r, G) = gpu_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, prec)
    print(f"stats {stats}")
    pc.assert_matches(out, ref, F, prec, label="small")
    np.testing.assert_array_equal(om, parts["omega"])
    np.testing.assert_allclose(r, parts["r"], rtol=1e-13)
    # G from the device-side M against the oracle's G: limited by the reductions' precision
    gerr = oracle.rel_frobenius(G, parts["G"])
    assert gerr <= (1e-5 if prec == rfd.RFD_FP32_PLAIN else 2e-2), gerr


@pytest.mark.parametrize("m,norm,lam", [(1, 0.5, 1.0), (7, 0.01, 1.0), (64, 0.2, -1.0), (64, 0.9, 1.0),
                                        (96, 2.0, 0.5), (200, 5.0, 1.0), (130, 40.0, -1.0), (64, 300.0, 1.0)])
def test_phi1_matches_oracle(m, norm, lam):
    rng = np.random.default_rng(m * 1000 + int(norm * 10))
    M = rng.standard_normal((m, m))
    M *= norm / (np.abs(lam) * np.abs(M).sum(0).max())
    G = torch.zeros((m, m), dtype=torch.float64, device=DEV)
    stats = rfd.rfd_phi1(m, lam, _cuda(M), G)
    ref = lam * oracle.phi1(lam * M)
    err = oracle.rel_frobenius(G.cpu().numpy(), ref)
    print(m, norm, stats, err)
    assert abs(stats["norm1"] - norm) <= 1e-9 * norm
    assert err <= 1e-12 * max(1.0, norm)


def test_phi1_singular_and_zero():
    m = 48
    rng = np.random.default_rng(5)
    Bm = rng.standard_normal((m, 10))
    M = Bm @ Bm.T * 0.05                      # rank 10
    G = torch.zeros((m, m), dtype=torch.float64, device=DEV)
    rfd.rfd_phi1(m, 0.7, _cuda(M), G)
    assert oracle.rel_frobenius(G.cpu().numpy(), 0.7 * oracle.phi1(0.7 * M)) <= 1e-12
    rfd.rfd_phi1(m, 0.0, _cuda(M), G)
    assert not G.cpu().numpy().any()
    rfd.rfd_phi1(m, 2.0, _cuda(np.zeros((m, m))), G)
    np.testing.assert_array_equal(G.cpu().numpy(), 2.0 * np.eye(m))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,m,c,ld", [(1000, 66, 5, 7), (40, 64, 3, 3), (1, 8, 2, 2), (3001, 130, 1, 1),
                                      (700, 2, 4, 4), (5000, 256, 64, 64)])
def test_ragged_and_degenerate_shapes(prec, n, m, c, ld):
    rng = synth.rng_for(11, 1, n)
    pts = synth.unit_sphere(n, rng)
    F = synth.gaussian_field(n, c, 11, n)
    eps, seed = 0.1, 3
    lam = 0.1 * m / max(n, m)
    ref = oracle.rfd_gfi(pts, F, eps, lam, m, seed)
    out, stats, _ = gpu_gfi(pts, F, eps, lam, m, seed, prec, ld=ld)
    print(stats)
    pc.assert_matches(out, ref, F, prec, label=f"N={n} m={m} c={c} ld={ld}")


@pytest.mark.parametrize("prec", PRECS)
def test_lambda_zero_is_identity_bitwise(prec):
    spec, pts, F, _ = small_case()
    out, _, _ = gpu_gfi(pts, F, spec.eps, 0.0, spec.m, spec.seed, prec)
    np.testing.assert_array_equal(out, F)


@pytest.mark.parametrize("prec", PRECS)
def test_negative_lambda(prec):
    # W_hat is indefinite (r_j of both signs), so lambda < 0 amplifies through its
    # negative eigenvalues exactly as lambda > 0 does through the positive ones.
    spec, pts, F, lam = small_case()
    ref = oracle.rfd_gfi(pts, F, spec.eps, -lam, spec.m, spec.seed)
    out, _, _ = gpu_gfi(pts, F, spec.eps, -lam, spec.m, spec.seed, prec)
    pc.assert_matches(out, ref, F, prec, label="negative lambda")


@pytest.mark.parametrize("prec", PRECS)
def test_warm_path_equals_cold_and_inplace(prec):
    spec, pts, F, lam = small_case()
    cold, _, _ = gpu_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, prec)
    warm, _, _ = gpu_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, prec, api="split", max_channels=8)
    inpl, _, _ = gpu_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, prec, inplace=True)
    ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
    pc.assert_matches(warm, ref, F, prec, label="warm")
    pc.assert_matches(cold, ref, F, prec, label="cold")
    np.testing.assert_array_equal(inpl, cold)


def test_warm_integrate_of_few_channels_has_no_bf16_rounding():
    """A full BF16 plan integrates a field of few channels (c <= 4) with B^T F
    from the points in FP32, the compact plans' path, so its increment error
    drops well below the cold pass's, whose B^T F rides on the BF16 Psi; with
    more channels it passes over Psi, within the BF16 bounds."""
    spec, pts, F, lam = small_case("torus")
    plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=16, precision=rfd.RFD_BF16_TC,
                    stream=torch.cuda.current_stream(DEV))
    try:
        F3 = np.ascontiguousarray(F[:, :3])
        cold = plan.gfi(_cuda(pts), _cuda(F3))
        warm = plan.integrate(_cuda(F3))
        wide = plan.integrate(_cuda(F))
        plan.sync()
        ref3 = oracle.rfd_gfi(pts, F3, spec.eps, lam, spec.m, spec.seed)
        ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
        e_cold = pc.assert_matches(cold.cpu().numpy(), ref3, F3, rfd.RFD_BF16_TC, label="cold, c=3")
        e_warm = pc.assert_matches(warm.cpu().numpy(), ref3, F3, rfd.RFD_BF16_TC, label="warm, c=3")
        pc.assert_matches(wide.cpu().numpy(), ref, F, rfd.RFD_BF16_TC, label=f"warm, c={F.shape[1]}")
        assert e_warm["inc"] < 0.2 * e_cold["inc"], (e_warm, e_cold)
    finally:
        plan.close()


@pytest.mark.parametrize("prec", PRECS)
def test_resident_plan_reuse_new_fields(prec):
    """One plan, resident Phi and G, several fields of different widths (Sec. 2.4 inference)."""
    spec, pts, F, lam = small_case()
    plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=32, precision=prec,
                    stream=torch.cuda.current_stream(DEV))
    try:
        plan.features(_cuda(pts))
        for k, c in enumerate((1, 32, 7)):
            Fk = synth.gaussian_field(spec.n, c, 99, k)
            out = plan.integrate(_cuda(Fk))
            plan.sync()
            ref = oracle.rfd_gfi(pts, Fk, spec.eps, lam, spec.m, spec.seed)
            pc.assert_matches(out.cpu().numpy(), ref, Fk, prec, label=f"resident c={c}")
    finally:
        plan.close()


@pytest.mark.parametrize("prec", PRECS)
def test_torus_config(prec):
    spec, pts, F, lam = small_case("torus")
    ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
    out, stats, _ = gpu_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, prec)
    print(f"torus N={spec.n} m={spec.m} c={spec.c} stats={stats}")
    pc.assert_matches(out, ref, F, prec, label="torus")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,factor", [("small", 2.5), ("torus", 6.0)])
def test_large_relative_increment(prec, name, factor):
    """A longer diffusion time, where the integrated part is a large share of the
    output (relative increment 0.36 on the small workload, 0.44 on the torus):
    the whole-output bounds of both forms still hold, so they do not rest on a
    small increment."""
    spec, pts, F, lam = small_case(name)
    lam *= factor
    ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
    out, _, _ = gpu_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, prec)
    e = pc.assert_matches(out, ref, F, prec, label=f"{name} x{factor}")
    assert e["relative_increment"] >= 0.3


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["small", "torus"])
@pytest.mark.parametrize("kernel", ["ball", "cube_l1", "l1_ball"])
def test_kernel_variants_match_oracle(prec, name, kernel):
    """Threshold-function variants (the L2 ball, the Bessel case of Sec. 2.4; the L1 ball; the
    distance-weighted cube): only step a1's weights change; the whole path
    against the oracle with the same kernel."""
    spec, pts, F, lam = small_case(name)
    ref, parts = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, return_parts=True, kernel=kernel)
    out, stats, (om, r, G) = gpu_gfi(pts, F, spec.eps, lam, spec.m, spec.seed, prec, kernel=kernel)
    pc.assert_matches(out, ref, F, prec, label=f"{kernel} {name}")
    np.testing.assert_array_equal(om, parts["omega"])
    np.testing.assert_allclose(r, parts["r"], rtol=0, atol=1e-13 * np.abs(parts["r"]).max())


def test_plan_graph_replay_is_bitwise_identical():
    """A BF16 plan with RFD_FLAG_GRAPH replays each call's launches from CUDA graphs:
    the output equals the plain plan's bit for bit, call after call (gfi and integrate)."""
    spec, pts, F, lam = small_case("torus")
    P, Ft = _cuda(pts), _cuda(F)
    outs = {}
    for graph in (False, True):
        plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=F.shape[1],
                        precision=rfd.RFD_BF16_TC, stream=torch.cuda.current_stream(DEV), graph=graph)
        try:
            res = []
            for _ in range(3):
                o = torch.empty_like(Ft)
                plan.gfi(P, Ft, o)
                res.append(o)
            o2 = torch.empty_like(Ft)
            plan.integrate(Ft * 0.5, o2)
            res.append(o2)
            plan.sync()
            outs[graph] = [r.cpu().numpy() for r in res]
        finally:
            plan.close()
    for a, b in zip(outs[False], outs[True]):
        np.testing.assert_array_equal(a, b)
    ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
    pc.assert_matches(outs[True][2], ref, F, rfd.RFD_BF16_TC, label="graph replay")


def test_invalid_arguments_and_alloc_failure():
    spec, pts, F, lam = small_case()
    plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=3, precision=rfd.RFD_BF16_TC)
    try:
        Ft = _cuda(F)
        out = torch.empty_like(Ft)
        with pytest.raises(rfd.RfdError) as e:
            rfd.rfd_integrate(plan.handle, Ft, 3, 3, out, 3)   # before rfd_features
        assert e.value.status == rfd.RFD_EINVAL
        F4 = _cuda(np.zeros((spec.n, 4), np.float32))
        with pytest.raises(rfd.RfdError) as e:
            rfd.rfd_gfi(plan.handle, _cuda(pts), F4, 4, 4, F4, 4)  # c > max_channels
        assert e.value.status == rfd.RFD_EINVAL
        # the plan stays usable after failed calls
        out = plan.gfi(_cuda(pts), Ft)
        plan.sync()
        pc.assert_matches(out.cpu().numpy(), oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed), F,
                          rfd.RFD_BF16_TC, label="after failed calls")
    finally:
        plan.close()
    for k in (0, 1, 2):  # the plan chunk, its batch tables, their pinned staging
        rfd.rfd_debug_fail_alloc_after(k)
        with pytest.raises(rfd.RfdError) as e:
            rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=3)
        assert e.value.status == rfd.RFD_ENOMEM
    rfd.rfd_debug_fail_alloc_after(-1)
    free0 = torch.cuda.mem_get_info()[0]
    p = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=3)
    p.close()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)


@pytest.mark.parametrize("m,norm,lam", [(64, 0.5, 1.0), (256, 0.97, 1.0), (256, 3.0, -1.0), (1024, 0.5, 1.0),
                                        (130, 40.0, 1.0), (96, 1e-6, 1.0)])
def test_batched_phi1_matches_oracle(m, norm, lam):
    """Step a4 as rfd_features runs it for BF16 plans (the batched, emulated path:
    Taylor degree 16 in Paterson-Stockmeyer form, scaling and squaring above
    ||X||_1 = 0.977), on a given M, against the oracle's expm-based phi1: FP64
    accuracy, ~s u ||X|| after s squarings."""
    rng = np.random.default_rng(m * 7 + int(norm * 100))
    M = rng.standard_normal((m, m))
    M *= norm / (abs(lam) * np.abs(M).sum(0).max())
    plan = rfd.Plan(64, m, 0.1, lam, 1, precision=rfd.RFD_BF16_TC, stream=torch.cuda.current_stream(DEV))
    try:
        _check(rfd.lib.rfd_debug_plan_phi1(plan.handle, _cuda(M).data_ptr()), "rfd_debug_plan_phi1")
        st = plan.stats()
        _, _, G = plan.export()
    finally:
        plan.close()
    ref = lam * oracle.phi1(lam * M)
    err = oracle.rel_frobenius(G, ref)
    print(m, norm, st["squarings"], st["phi1_gemms"], err)
    assert abs(st["norm1"] - norm) <= 1e-9 * norm
    assert st["pade_degree"] == 16 and st["phi1_gemms"] == 6 + 2 * st["squarings"]
    assert err <= 1e-13 * max(1.0, norm)


def _check(status, where):
    if status != 0:
        raise RuntimeError(f"{where}: {rfd.rfd_last_error()}")


@pytest.mark.parametrize("phase_blocks", [64, 300, 1])
def test_multi_phase_point_axis_matches_oracle(phase_blocks):
    """The tensor-core reductions walk the point axis in phases (one launch each,
    later phases adding into the split-K lanes' FP32 partials, Sec. 2.4's
    reduction over N).  The large workload takes several phases; here a short
    phase makes the torus cloud (1563 blocks of 64 points) take 25, 6 and 1563
    of them, and the result must match the oracle and the one-phase result."""
    spec, pts, F, lam = small_case("torus")
    ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
    P, Ft = _cuda(pts), _cuda(F)
    outs = []
    for ph in (phase_blocks, 1 << 20):
        plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=F.shape[1],
                        precision=rfd.RFD_BF16_TC, stream=torch.cuda.current_stream(DEV))
        try:
            _check(rfd.lib.rfd_debug_plan_set_phase(plan.handle, ph), "rfd_debug_plan_set_phase")
            o = plan.gfi(P, Ft)
            plan.sync()
            assert plan.stats()["tune_phase_blocks"] == ph
            outs.append(o.cpu().numpy())
        finally:
            plan.close()
    pc.assert_matches(outs[0], ref, F, rfd.RFD_BF16_TC, label=f"{phase_blocks}-block phases")
    # against the single-phase run: the same products, summed in another order (FP32)
    pc.assert_matches(outs[0], outs[1], F, rfd.RFD_BF16_TC, label="phases vs one phase", tol_out=1e-5,
                      tol_inc=2e-3, tol_row=2e-3)


@pytest.mark.parametrize("phase_blocks", [64, 512])
def test_features_beside_gram_matches_oracle(phase_blocks):
    """The schedule that runs the features phase by phase on a side stream beside
    the Gram (the Gram of phase p waits for the features of phase p only) gives
    the oracle's result, and bit for bit the serial schedule's: the same kernels
    on the same data, only their overlap differs.  A single phase, or a phase
    length that is not a multiple of 8 blocks, refuses the schedule."""
    spec, pts, F, lam = small_case("torus")
    ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
    P, Ft = _cuda(pts), _cuda(F)
    outs = []
    for overlap in (1, 0):
        plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=F.shape[1],
                        precision=rfd.RFD_BF16_TC, stream=torch.cuda.current_stream(DEV))
        try:
            _check(rfd.lib.rfd_debug_plan_set_phase(plan.handle, phase_blocks), "rfd_debug_plan_set_phase")
            _check(rfd.lib.rfd_debug_plan_set_overlap(plan.handle, overlap), "rfd_debug_plan_set_overlap")
            o = plan.gfi(P, Ft)
            o2 = plan.gfi(P, Ft)  # a second call through the same schedule
            plan.sync()
            assert plan.stats()["tune_overlap"] == overlap
            assert torch.equal(o, o2)
            outs.append(o.cpu().numpy())
            if overlap:
                assert rfd.lib.rfd_debug_plan_set_phase(plan.handle, 300) == 0
                assert rfd.lib.rfd_debug_plan_set_overlap(plan.handle, 1) != 0   # 300 % 8 != 0
                assert rfd.lib.rfd_debug_plan_set_phase(plan.handle, 1 << 20) == 0
                assert rfd.lib.rfd_debug_plan_set_overlap(plan.handle, 1) != 0   # one phase
                assert plan.stats()["tune_overlap"] == 0
        finally:
            plan.close()
    pc.assert_matches(outs[0], ref, F, rfd.RFD_BF16_TC, label=f"features beside the Gram, {phase_blocks}-block phases")
    assert np.array_equal(outs[0], outs[1])
