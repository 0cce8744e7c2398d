"""Batched integration (many clouds of uneven N and m in shared launches)
against the CPU FP64 oracle and against each cloud integrated alone."""
import numpy as np
import pytest

import oracle
import parity_checks as pc
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
BF16 = 1  # RFD_BF16_TC: every comparison asserts the output, increment and per-row bounds of parity_checks


def _specs(count=9, seed=4):
    specs = synth.batched_specs(count=count, seed=seed, n_lo=500, n_hi=12000, ms=(64, 128, 256), c=8)
    # uneven channel counts too
    for k, s in enumerate(specs):
        s.c = (1, 3, 8)[k % 3]
    return specs


def _lam(s):
    return s.lam * s.m / s.n   # diffusion time in units of the estimator's mean eigenvalue


def _plans(specs, stream):
    return [rfd.Plan(s.n, s.m, s.eps, _lam(s), s.seed, max_channels=8, precision=rfd.RFD_BF16_TC, stream=stream)
            for s in specs]


def test_batch_gfi_matches_oracle_and_single_cloud_runs():
    specs = _specs()
    clouds = [synth.make_cloud(s) for s in specs]
    stream = torch.cuda.current_stream(DEV)
    plans = _plans(specs, stream)
    batch = rfd.Batch(plans, stream=stream, timing=True)
    items = [{"points": torch.from_numpy(p).to(DEV), "F": torch.from_numpy(F).to(DEV)} for p, F in clouds]
    outs = batch.gfi(items)
    batch.sync()
    st = batch.stats()
    assert st["timed_calls"] == 1 and st["kernel_launches"] > 0
    for k, (s, (pts, F)) in enumerate(zip(specs, clouds)):
        ref = oracle.rfd_gfi(pts, F, s.eps, _lam(s), s.m, s.seed)
        got = outs[k].cpu().numpy()
        pc.assert_matches(got, ref, F, BF16, label=f"cloud {k}: N={s.n} m={s.m} c={s.c}")
        # the same cloud alone (its own plan, a batch of one)
        alone = plans[k].gfi(items[k]["points"], items[k]["F"])
        plans[k].sync()
        pc.assert_matches(got, alone.cpu().numpy(), F, BF16, label=f"cloud {k} batched vs alone")
    batch.close()
    for p in plans:
        p.close()


def test_batch_warm_integrate_reuses_resident_G():
    specs = _specs(count=5, seed=7)
    clouds = [synth.make_cloud(s) for s in specs]
    stream = torch.cuda.current_stream(DEV)
    plans = _plans(specs, stream)
    batch = rfd.Batch(plans, stream=stream)
    batch.features([{"points": torch.from_numpy(p).to(DEV)} for p, _ in clouds])
    for rep in range(2):
        fields = [synth.gaussian_field(s.n, s.c, 1000 + rep, k) for k, s in enumerate(specs)]
        outs = batch.integrate([{"F": torch.from_numpy(F).to(DEV)} for F in fields])
        batch.sync()
        for k, s in enumerate(specs):
            ref = oracle.rfd_gfi(clouds[k][0], fields[k], s.eps, _lam(s), s.m, s.seed)
            pc.assert_matches(outs[k].cpu().numpy(), ref, fields[k], BF16, label=f"warm cloud {k}")
    batch.close()
    for p in plans:
        p.close()


def test_batch_rejects_fp32_and_repeated_plans():
    s = _specs(count=2)
    p16 = rfd.Plan(s[0].n, s[0].m, s[0].eps, _lam(s[0]), 0, precision=rfd.RFD_BF16_TC)
    p32 = rfd.Plan(s[1].n, s[1].m, s[1].eps, _lam(s[1]), 0, precision=rfd.RFD_FP32_PLAIN)
    with pytest.raises(rfd.RfdError) as e:
        rfd.Batch([p16, p32])
    assert e.value.status == rfd.RFD_EINVAL
    with pytest.raises(rfd.RfdError) as e:
        rfd.Batch([p16, p16])
    assert e.value.status == rfd.RFD_EINVAL
    p16.close()
    p32.close()


def test_batch_graph_replay_matches_direct_launches():
    specs = _specs(count=6, seed=12)
    clouds = [synth.make_cloud(s) for s in specs]
    stream = torch.cuda.current_stream(DEV)
    plans = _plans(specs, stream)
    direct = rfd.Batch(plans, stream=stream)
    items = [{"points": torch.from_numpy(p).to(DEV), "F": torch.from_numpy(F).to(DEV)} for p, F in clouds]
    ref = [o.cpu().numpy() for o in direct.gfi(items)]
    direct.sync()
    direct.close()
    graph = rfd.Batch(plans, stream=stream, graph=True)
    for rep in range(3):   # first call captures, the others replay
        outs = graph.gfi(items)
        graph.sync()
        for k in range(len(specs)):
            np.testing.assert_array_equal(outs[k].cpu().numpy(), ref[k])   # same launches, same bits
    # warm integrate under a graph as well
    fields = [synth.gaussian_field(s.n, s.c, 500, k) for k, s in enumerate(specs)]
    outs = graph.integrate([{"F": torch.from_numpy(F).to(DEV)} for F in fields])
    graph.sync()
    for k, s in enumerate(specs):
        want = oracle.rfd_gfi(clouds[k][0], fields[k], s.eps, _lam(s), s.m, s.seed)
        pc.assert_matches(outs[k].cpu().numpy(), want, fields[k], BF16, label=f"graph warm cloud {k}")
    assert graph.stats()["kernel_launches"] > 0
    graph.close()
    for p in plans:
        p.close()


def test_nonfinite_G_is_reported_at_sync():
    s = _specs(count=1, seed=2)[0]
    pts, F = synth.make_cloud(s)
    p = rfd.Plan(s.n, s.m, s.eps, 1e30, s.seed, max_channels=8, precision=rfd.RFD_BF16_TC)
    P, Fd = torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV)
    p.gfi(P, Fd)   # enqueues; ||lambda M||_1 needs more than 60 squarings: flagged on the device
    with pytest.raises(rfd.RfdError) as e:
        p.sync()
    assert e.value.status == rfd.RFD_ENUMERIC
    assert p.stats()["nonfinite"] == 1
    with pytest.raises(rfd.RfdError) as e:   # G is not resident after a failed features pass
        p.integrate(Fd)
    assert e.value.status == rfd.RFD_EINVAL
    p.sync()   # the flags were cleared by the first sync
    p.close()


def test_autotuned_batch_and_plan():
    specs = _specs(count=5, seed=21)
    clouds = [synth.make_cloud(s) for s in specs]
    stream = torch.cuda.current_stream(DEV)
    plans = _plans(specs, stream)
    batch = rfd.Batch(plans, stream=stream, autotune=True)
    items = [{"points": torch.from_numpy(p).to(DEV), "F": torch.from_numpy(F).to(DEV)} for p, F in clouds]
    for rep in range(2):   # the first call tunes, the second runs the chosen tables
        outs = batch.gfi(items)
        batch.sync()
        for k, s in enumerate(specs):
            ref = oracle.rfd_gfi(clouds[k][0], clouds[k][1], s.eps, _lam(s), s.m, s.seed)
            pc.assert_matches(outs[k].cpu().numpy(), ref, clouds[k][1], BF16, label=f"tuned batch cloud {k}")
    st = batch.stats()
    assert st["tuned"] == 1 and st["tune_waves"] in (2, 4, 8) and st["tune_phase_blocks"] in (1024, 2048, 4096, 8192, 16384)
    batch.close()
    # a lone autotuned plan, then a second plan of the same bucket (taken from the cache)
    s = specs[0]
    for _ in range(2):
        p = rfd.Plan(s.n, s.m, s.eps, _lam(s), s.seed, max_channels=8, precision=rfd.RFD_BF16_TC, autotune=True)
        P, Fd = items[0]["points"], items[0]["F"]
        for rep in range(2):
            out = p.gfi(P, Fd)
            p.sync()
            ref = oracle.rfd_gfi(clouds[0][0], clouds[0][1], s.eps, _lam(s), s.m, s.seed)
            pc.assert_matches(out.cpu().numpy(), ref, clouds[0][1], BF16, label="tuned plan")
        st = p.stats()
        assert st["tuned"] == 1 and st["tune_lanes_pct"] in (50, 100, 200)
        p.close()
    for p in plans:
        p.close()
