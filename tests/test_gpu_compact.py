"""Compact resident plans (rfd_plan_compact): after the cold pass a BF16 plan
keeps its points, frequencies, M and G, and integrates new fields by
recomputing the features from the points (Sec. 2.4 inference: "linear in N,
quadratic in m").  Checked against the FP64 oracle with the parity bounds;
B^T F no longer carries the BF16 rounding of the feature matrix, so the
increment error also drops below the full plan's."""
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


@pytest.mark.parametrize("name", ["small", "torus"])
@pytest.mark.parametrize("cs", [(1, 3), (32, 40)])
def test_compact_plan_integrates_new_fields(name, cs):
    spec = synth.config_single(name)
    pts, F = synth.make_cloud(spec)
    lam = spec.lam * spec.m / spec.n
    cmax = max(max(cs), F.shape[1])
    plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=cmax, precision=BF16,
                    stream=torch.cuda.current_stream(DEV))
    try:
        P = torch.from_numpy(pts).to(DEV)
        full_out = plan.gfi(P, torch.from_numpy(F).to(DEV))
        plan.sync()
        full_bytes = plan.device_bytes()
        plan.compact()
        plan.compact()   # a second call does nothing
        small_bytes = plan.device_bytes()
        print(f"{name}: {full_bytes / 2**20:.1f} MiB -> {small_bytes / 2**20:.2f} MiB")
        assert small_bytes * 4 < full_bytes
        errs = []
        for k, c in enumerate(cs):
            Fk = synth.gaussian_field(spec.n, c, 50 + k, 1)
            out = plan.integrate(torch.from_numpy(Fk).to(DEV))
            plan.sync()
            ref = oracle.rfd_gfi(pts, Fk, spec.eps, lam, spec.m, spec.seed)
            errs.append(pc.assert_matches(out.cpu().numpy(), ref, Fk, BF16, label=f"compact {name} c={c}"))
        # the full plan's increment error (BF16 Phi in B^T F) against the compact plan's (FP32 features)
        ref0 = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
        full = pc.errors(full_out.cpu().numpy(), ref0, F)
        out0 = plan.integrate(torch.from_numpy(F).to(DEV))
        plan.sync()
        comp = pc.assert_matches(out0.cpu().numpy(), ref0, F, BF16, label=f"compact {name}, the cold field")
        assert comp["inc"] < full["inc"], (comp, full)
        # no feature matrix: the cold path is refused, the plan stays usable
        with pytest.raises(rfd.RfdError) as e:
            plan.features(P)
        assert e.value.status == rfd.RFD_EINVAL
        with pytest.raises(rfd.RfdError) as e:
            plan.gfi(P, torch.from_numpy(F).to(DEV))
        assert e.value.status == rfd.RFD_EINVAL
        again = plan.integrate(torch.from_numpy(F).to(DEV))
        plan.sync()
        np.testing.assert_array_equal(again.cpu().numpy(), out0.cpu().numpy())
    finally:
        plan.close()


def test_compact_refused_before_features_and_for_fp32():
    spec = synth.config_single("small")
    p = rfd.Plan(spec.n, spec.m, spec.eps, 0.01, 0, precision=BF16)
    with pytest.raises(rfd.RfdError) as e:
        p.compact()
    assert e.value.status == rfd.RFD_EINVAL
    p.close()
    q = rfd.Plan(spec.n, spec.m, spec.eps, 0.01, 0, precision=rfd.RFD_FP32_PLAIN)
    pts, F = synth.make_cloud(spec)
    q.gfi(torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV))
    q.sync()
    with pytest.raises(rfd.RfdError) as e:
        q.compact()
    assert e.value.status == rfd.RFD_EINVAL
    q.close()


def test_compact_plan_in_a_batch_and_eigenvalues():
    """Compact plans integrate together in one batch; a batch may not mix compact
    and full plans; the kernel eigenvalues still come from the resident M."""
    specs = synth.batched_specs(count=4, seed=17, n_lo=800, n_hi=6000, ms=(64, 128), c=4)
    stream = torch.cuda.current_stream(DEV)
    clouds = [synth.make_cloud(s) for s in specs]
    plans = [rfd.Plan(s.n, s.m, s.eps, s.lam * s.m / s.n, s.seed, max_channels=4, precision=BF16, stream=stream)
             for s in specs]
    try:
        for p, (pts, F) in zip(plans, clouds):
            p.gfi(torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV))
        for p in plans:
            p.sync()
        ev_full = plans[0].eigenvalues(8).cpu().numpy()
        for p in plans[:3]:
            p.compact()
        with pytest.raises(rfd.RfdError) as e:
            rfd.Batch(plans, stream=stream)
        assert e.value.status == rfd.RFD_EINVAL
        plans[3].compact()
        np.testing.assert_array_equal(plans[0].eigenvalues(8).cpu().numpy(), ev_full)
        batch = rfd.Batch(plans, stream=stream)
        fields = [synth.gaussian_field(s.n, 3, 70, k) for k, s in enumerate(specs)]
        outs = batch.integrate([{"F": torch.from_numpy(F).to(DEV)} for F in fields])
        batch.sync()
        for k, s in enumerate(specs):
            ref = oracle.rfd_gfi(clouds[k][0], fields[k], s.eps, s.lam * s.m / s.n, s.m, s.seed)
            pc.assert_matches(outs[k].cpu().numpy(), ref, fields[k], BF16, label=f"compact batch cloud {k}")
        batch.close()
    finally:
        for p in plans:
            p.close()


def test_compact_graph_replay_tracks_channel_count():
    """A compact plan with CUDA-graph replay: calls whose channel counts share the
    per-block channel group (9 and 13 channels: one group of 16) but not the grid
    of the sum over the chunks (one warp per 4 channels) each get a graph of
    their own, and each matches the oracle."""
    spec = synth.config_single("small")
    pts, F = synth.make_cloud(spec)
    lam = spec.lam * spec.m / spec.n
    plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=16, precision=BF16,
                    stream=torch.cuda.current_stream(DEV), graph=True)
    try:
        plan.gfi(torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV))
        plan.sync()
        plan.compact()
        for k, c in enumerate((9, 13, 9, 16)):
            Fk = synth.gaussian_field(spec.n, c, 80 + k, 1)
            out = plan.integrate(torch.from_numpy(Fk).to(DEV))
            plan.sync()
            ref = oracle.rfd_gfi(pts, Fk, spec.eps, lam, spec.m, spec.seed)
            pc.assert_matches(out.cpu().numpy(), ref, Fk, BF16, label=f"compact, graphs, c={c}")
    finally:
        plan.close()
