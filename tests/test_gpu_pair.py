"""The 2-SM form of the tensor-core reductions (Sec. 2.4, M = B^T A and
Y = B^T F over N): BF16 plans with m >= 512 run their Gram on CTA pairs
(tcgen05.mma.cta_group::2, each SM of a pair loading half of B).  Checked
against the FP64 oracle (whole output, increment, rows) and against the
one-SM kernel on the same inputs, at ragged m (528, 640: row blocks of 512
with empty or partial second halves), several point-axis phases, and 64
field channels (the widest field the pair form takes)."""
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


def _run(pts, F, eps, lam, m, seed, pairs, phase=None):
    rfd.rfd_debug_gram_pairs(1 if pairs else 0)
    try:
        plan = rfd.Plan(len(pts), m, eps, lam, seed, max_channels=F.shape[1], precision=BF16,
                        stream=torch.cuda.current_stream(DEV))
    finally:
        rfd.rfd_debug_gram_pairs(1)
    try:
        if phase:
            assert rfd.lib.rfd_debug_plan_set_phase(plan.handle, phase) == 0, rfd.rfd_last_error()
        out = plan.gfi(torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV))
        warm = plan.integrate(torch.from_numpy(F).to(DEV))   # the warm path stays on the one-SM field tiles
        plan.sync()
        return out.cpu().numpy(), warm.cpu().numpy(), plan.stats()
    finally:
        plan.close()


@pytest.mark.parametrize("m,c,n,phase", [(512, 3, 20000, None), (528, 3, 20000, None), (640, 5, 15000, None),
                                         (1024, 3, 30000, None), (1024, 64, 12000, None), (1024, 3, 30000, 64),
                                         (768, 8, 9000, 16)])
def test_pair_gram_matches_oracle_and_one_sm_form(m, c, n, phase):
    rng = synth.rng_for(21, 1, n + m)
    pts = synth.unit_sphere(n, rng)
    F = synth.gaussian_field(n, c, 21, m)
    eps, seed = 0.1, 5
    lam = 0.1 * m / n
    ref = oracle.rfd_gfi(pts, F, eps, lam, m, seed)
    out2, warm2, st = _run(pts, F, eps, lam, m, seed, True, phase)
    out1, warm1, st1 = _run(pts, F, eps, lam, m, seed, False, phase)
    assert st["tune_pair_gram"] == 1 and st1["tune_pair_gram"] == 0   # each run took the form it names
    pc.assert_matches(out2, ref, F, BF16, label=f"pairs m={m} c={c} N={n} phase={phase}")
    pc.assert_matches(warm2, ref, F, BF16, label="pairs, then the warm path")
    pc.assert_matches(out1, ref, F, BF16, label="one-SM form")
    # the same BF16 products, summed in another order: far inside the BF16 bounds
    pc.assert_matches(out2, out1, F, BF16, label="pairs vs one-SM", tol_out=1e-5, tol_inc=2e-3, tol_row=2e-3)


def test_pair_form_not_used_below_512():
    """m < 512 (or not a multiple of 16) stays on the one-SM kernel: the toggle changes nothing."""
    n, m, c = 5000, 256, 3
    pts = synth.unit_sphere(n, synth.rng_for(3, 1, 0))
    F = synth.gaussian_field(n, c, 3, 0)
    a, _, _ = _run(pts, F, 0.1, 0.1 * m / n, m, 1, True)
    b, _, _ = _run(pts, F, 0.1, 0.1 * m / n, m, 1, False)
    np.testing.assert_array_equal(a, b)
