"""Failure detection on the device without a fault: a bounded device-side
wait that runs out is reported as RFD_ETIMEDOUT, and the plan stays usable.

Every mbarrier wait in the tensor-core kernels gives up after a %globaltimer
limit, records a code in the plan's device error word, frees its TMEM and
returns; rfd_sync maps the word to RFD_ETIMEDOUT.  Here that unwind path runs
on its own (rfd_debug_plan_wait_timeout): one CTA waits 1 ms on an mbarrier
that nothing ever arrives on.  Nothing faults, traps or hangs, and no copy is
in flight."""
import time

import numpy as np
import pytest

import oracle
import parity_checks as pc
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.mark.parametrize("prec", [rfd.RFD_FP32_PLAIN, rfd.RFD_BF16_TC])
def test_device_wait_runs_out_and_plan_stays_usable(prec):
    spec = synth.config_single("small")
    pts, F = synth.make_cloud(spec)
    lam = spec.lam * spec.m / spec.n
    ref = oracle.rfd_gfi(pts, F, spec.eps, lam, spec.m, spec.seed)
    P, Fd = torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV)
    plan = rfd.Plan(spec.n, spec.m, spec.eps, lam, spec.seed, max_channels=spec.c, precision=prec,
                    stream=torch.cuda.current_stream(DEV))
    try:
        out = plan.gfi(P, Fd)
        plan.sync()                                   # a clean pass first: no error recorded
        t0 = time.monotonic()
        assert rfd.lib.rfd_debug_plan_wait_timeout(plan.handle, 1000) == rfd.RFD_OK
        with pytest.raises(rfd.RfdError) as e:
            plan.sync()
        waited = time.monotonic() - t0
        assert e.value.status == rfd.RFD_ETIMEDOUT, str(e.value)
        assert "code 21" in str(e.value)              # the probe's own code
        assert waited < 5.0, waited                   # the wait ended at its limit, not at a watchdog
        plan.sync()                                   # the word was cleared: the next sync is clean
        # the same plan integrates again and matches the oracle
        out = plan.gfi(P, Fd, out)
        plan.sync()
        pc.assert_matches(out.cpu().numpy(), ref, F, prec, label="after a timed-out wait")
        # so does a second timeout after normal work, then normal work again
        assert rfd.lib.rfd_debug_plan_wait_timeout(plan.handle, 200) == rfd.RFD_OK
        with pytest.raises(rfd.RfdError) as e:
            plan.sync()
        assert e.value.status == rfd.RFD_ETIMEDOUT
        out2 = plan.gfi(P, Fd)
        plan.sync()
        np.testing.assert_array_equal(out2.cpu().numpy(), out.cpu().numpy())
    finally:
        plan.close()


def test_wait_probe_rejects_bad_limits():
    plan = rfd.Plan(64, 8, 0.1, 0.01, 0, precision=rfd.RFD_BF16_TC)
    try:
        for bad in (0, -5, 1000001):
            assert rfd.lib.rfd_debug_plan_wait_timeout(plan.handle, bad) == rfd.RFD_EINVAL
        plan.sync()
    finally:
        plan.close()
