"""Parity at the large workload, in the launch configuration the benchmark times.

N = 1,000,000 points on 8 ellipsoid surfaces, eps = 0.02, m = 1024, lambda =
0.02 (applied as 0.02 m / N), F with 3 and with 64 channels, against the FP64
oracle at full N (every output element).  The BF16 plan is built as bench.py
builds its timed plan (RFD_FLAG_AUTOTUNE and RFD_FLAG_GRAPH), so the tuned
split-K lanes, phase length, Gram form and schedule and the CUDA-graph replay
are the ones compared; the FP32 plain form runs its own plan.  Two more BF16
plans fix the point axis at four phases of 4096 blocks (15,625 blocks of 64
points), once with the features run before the Gram and once beside it, so
that the multi-phase accumulation is compared at full size whatever the
tuner picks.  Feature phases reach ~|w| |x| ~ 10^2 cycles here, the largest
of any workload.  The oracle holds ~24 GB of host memory for a minute."""
import numpy as np
import pytest

import oracle
import parity_checks as pc
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.fixture(scope="module")
def large_case():
    spec3 = synth.config_single("large", 3)
    spec64 = synth.config_single("large", 64)
    pts, F3 = synth.make_cloud(spec3)
    pts64, F64 = synth.make_cloud(spec64)
    assert np.array_equal(pts, pts64)
    lam = spec3.lam * spec3.m / spec3.n
    # one oracle pass for both fields: the columns of F are integrated independently
    ref = oracle.rfd_gfi(pts, np.concatenate([F3, F64], axis=1), spec3.eps, lam, spec3.m, spec3.seed)
    return spec3, pts, lam, {3: (F3, ref[:, :3]), 64: (F64, ref[:, 3:])}


@pytest.mark.parametrize("prec,c,fixed", [(rfd.RFD_BF16_TC, 3, None), (rfd.RFD_BF16_TC, 64, None),
                                          (rfd.RFD_FP32_PLAIN, 3, None), (rfd.RFD_BF16_TC, 3, "serial"),
                                          (rfd.RFD_BF16_TC, 3, "beside")])
def test_large_workload_matches_oracle(large_case, prec, c, fixed):
    spec, pts, lam, fields = large_case
    F, ref = fields[c]
    bf16 = prec == rfd.RFD_BF16_TC
    tuned = bf16 and fixed is None
    P, Fd = torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV)
    plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=c, precision=prec,
                    stream=torch.cuda.current_stream(DEV), autotune=tuned, graph=tuned)
    try:
        if fixed:  # four phases of 4096 blocks, features before or beside the Gram
            assert rfd.lib.rfd_debug_plan_set_phase(plan.handle, 4096) == 0, rfd.rfd_last_error()
            assert rfd.lib.rfd_debug_plan_set_overlap(plan.handle, int(fixed == "beside")) == 0, rfd.rfd_last_error()
        out = torch.empty_like(Fd)
        for _ in range(3):        # the first call tunes, the second captures the graphs, the third replays
            plan.gfi(P, Fd, out)
        plan.sync()
        st = plan.stats()
        got = out.cpu().numpy()
    finally:
        plan.close()
    if tuned:
        assert st["tuned"] == 1, st
    if fixed:
        assert st["tune_phase_blocks"] == 4096 and st["tune_overlap"] == int(fixed == "beside"), st
    print(f"large c={c} prec={prec} {fixed or 'tuned'}: norm1 {st['norm1']:.3f}, squarings {st['squarings']}, "
          f"phase {st['tune_phase_blocks']}, lanes {st['tune_lanes_pct']}%, overlap {st['tune_overlap']}")
    pc.assert_matches(got, ref, F, prec, label=f"large N=1e6 m=1024 c={c} {fixed or 'tuned'}")
