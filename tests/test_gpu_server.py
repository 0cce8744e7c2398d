"""The GFI request loop (rfd_server_create / rfd_submit / rfd_poll): results in
a mixed stream of requests equal the same requests run alone (within the BF16
tolerance) and the FP64 oracle; resident clouds are reused; admission, poll
timeouts and eviction behave as the header states.  Every failure is made on
the host (a paused scheduler, a full queue, a budget too small)."""
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
BF16 = 1  # RFD_BF16_TC: every comparison asserts the output, increment and per-row bounds of parity_checks
WAIT_US = 60_000_000


def _lam(s):
    return s.lam * s.m / s.n   # diffusion time in units of the estimator's mean eigenvalue


def _specs(count, seed, n_hi=20000):
    specs = synth.batched_specs(count=count, seed=seed, n_lo=500, n_hi=n_hi, ms=(64, 128, 256), c=8)
    for k, s in enumerate(specs):
        s.c = (1, 3, 8, 5)[k % 4]
    return specs


def _upload(specs):
    clouds = [synth.make_cloud(s) for s in specs]
    return clouds, [(torch.from_numpy(p).to(DEV), torch.from_numpy(F).to(DEV)) for p, F in clouds]


def _submit(srv, s, P, F, out, **kw):
    return srv.submit(F, out, points=P, m=s.m, eps=s.eps, lam=_lam(s), seed=s.seed, **kw)


def _wait(srv, t):
    st, res = srv.poll(t, WAIT_US)
    assert st == rfd.RFD_OK, rfd.rfd_last_error()
    return res


def test_server_mix_equals_alone_and_oracle():
    specs = _specs(12, seed=11)
    clouds, dev = _upload(specs)
    srv = rfd.Server(4 << 30, executors=2, max_batch=8)
    try:
        alone = []
        for s, (P, F) in zip(specs, dev):
            out = torch.empty_like(F)
            res = _wait(srv, _submit(srv, s, P, F, out))
            assert res["status"] == rfd.RFD_OK and res["batch_size"] == 1
            alone.append(out.cpu().numpy())
        # the same requests in one burst: batched together, on two streams
        outs = [torch.empty_like(F) for _, F in dev]
        tickets = [_submit(srv, s, P, F, o) for s, (P, F), o in zip(specs, dev, outs)]
        sizes = []
        for t in tickets:
            res = _wait(srv, t)
            assert res["status"] == rfd.RFD_OK
            sizes.append(res["batch_size"])
        assert max(sizes) > 1, "the burst was not batched"
        for k, s in enumerate(specs):
            mixed = outs[k].cpu().numpy()
            pc.assert_matches(mixed, alone[k], clouds[k][1], BF16, label=f"request {k} mixed vs alone")
            if k < 4:
                ref = oracle.rfd_gfi(clouds[k][0], clouds[k][1], s.eps, _lam(s), s.m, s.seed)
                pc.assert_matches(mixed, ref, clouds[k][1], BF16, label=f"request {k}: N={s.n} m={s.m} c={s.c}")
        st = srv.stats()
        assert st["completed"] == 24 and st["batches"] >= 13 and st["kernel_launches"] > 0
    finally:
        srv.close()


def test_server_resident_cloud_reused_with_new_field():
    s = _specs(1, seed=3)[0]
    (pts, F), = [synth.make_cloud(s)]
    P, Fd = torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV)
    srv = rfd.Server(2 << 30)
    try:
        out = torch.empty_like(Fd)
        res = _wait(srv, _submit(srv, s, P, Fd, out, keep=True, max_channels=16))
        assert res["status"] == rfd.RFD_OK and res["cloud"] > 0 and res["reused"] == 0
        cid = res["cloud"]
        F2 = synth.gaussian_field(s.n, 16, 77)
        F2d = torch.from_numpy(F2).to(DEV)
        out2 = torch.empty_like(F2d)
        res2 = _wait(srv, srv.submit(F2d, out2, cloud=cid))
        assert res2["status"] == rfd.RFD_OK and res2["reused"] == 1 and res2["cloud"] == cid
        ref = oracle.rfd_gfi(pts, F2, s.eps, _lam(s), s.m, s.seed)
        pc.assert_matches(out2.cpu().numpy(), ref, F2, BF16, label="reused cloud")
        # more channels than the cloud was kept for: the request fails, the cloud stays usable
        F3 = torch.zeros((s.n, 17), device=DEV)
        t0 = time.monotonic()
        res3 = _wait(srv, srv.submit(F3, torch.empty_like(F3), cloud=cid))
        assert res3["status"] == rfd.RFD_EINVAL
        assert time.monotonic() - t0 < 5.0   # a request refused at admission wakes its poller at once
        res4 = _wait(srv, srv.submit(F2d, out2, cloud=cid))
        assert res4["status"] == rfd.RFD_OK
        assert srv.stats()["reused"] == 2
    finally:
        srv.close()


def test_server_admission_and_poll_timeouts():
    s = _specs(1, seed=5)[0]
    (pts, F), = [synth.make_cloud(s)]
    P, Fd = torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV)
    srv = rfd.Server(256 << 20, max_queue=3, executors=2)
    try:
        outs = [torch.empty_like(Fd) for _ in range(4)]
        srv.pause(True)
        tickets = [_submit(srv, s, P, Fd, outs[k]) for k in range(3)]
        st, t = srv.try_submit(Fd, outs[3], points=P, m=s.m, eps=s.eps, lam=_lam(s), seed=s.seed)
        assert st == rfd.RFD_EBUSY and t is None   # queue full
        assert srv.poll(tickets[0], 0)[0] == rfd.RFD_ENOTREADY
        assert srv.poll(tickets[0], 2000)[0] == rfd.RFD_ETIMEDOUT   # nothing runs while paused
        srv.pause(False)
        for t in tickets:
            assert _wait(srv, t)["status"] == rfd.RFD_OK
        assert srv.poll(tickets[0], 0)[0] == rfd.RFD_EINVAL   # retired
        # a request that alone needs more than the budget is refused at once
        big = torch.zeros((2_000_000, 3), device=DEV)
        st, t = srv.try_submit(big, big, points=big, m=1024, eps=0.02, lam=1e-5, seed=0)
        assert st == rfd.RFD_EBUSY
        # invalid arguments are refused at submit
        st, _ = srv.try_submit(Fd, outs[0], points=P, m=63, eps=s.eps, lam=_lam(s), seed=s.seed)
        assert st == rfd.RFD_EINVAL
        st, _ = srv.try_submit(Fd, outs[0], cloud=12345)   # unknown cloud, no points
        assert st == rfd.RFD_EINVAL
        assert srv.stats()["rejected"] == 2
    finally:
        srv.close()


def test_server_chained_reuse_waits_for_its_root():
    """A request may name the cloud of a keep = 1 request that has not finished
    (a cloud's id is the ticket of the request that keeps it): it waits behind
    it, runs on the compact resident cloud, and matches the oracle."""
    s = _specs(1, seed=13)[0]
    (pts, F), = [synth.make_cloud(s)]
    P, Fd = torch.from_numpy(pts).to(DEV), torch.from_numpy(F).to(DEV)
    fields = [synth.gaussian_field(s.n, 8, 300 + k) for k in range(3)]
    srv = rfd.Server(2 << 30, executors=3)
    try:
        srv.pause(True)   # everything is queued before any of it runs
        root_out = torch.empty_like(Fd)
        root = _submit(srv, s, P, Fd, root_out, keep=True, max_channels=8)
        outs, tickets = [], []
        for Fk in fields:
            Fk_d = torch.from_numpy(Fk).to(DEV)
            o = torch.empty_like(Fk_d)
            tickets.append(srv.submit(Fk_d, o, cloud=root))   # no points: the root's cloud
            outs.append(o)
        srv.pause(False)
        res = _wait(srv, root)
        assert res["status"] == rfd.RFD_OK and res["cloud"] == root
        for t, o, Fk in zip(tickets, outs, fields):
            r = _wait(srv, t)
            assert r["status"] == rfd.RFD_OK and r["reused"] == 1 and r["cloud"] == root
            ref = oracle.rfd_gfi(pts, Fk, s.eps, _lam(s), s.m, s.seed)
            pc.assert_matches(o.cpu().numpy(), ref, Fk, BF16, label="chained reuse")
        # a request that names a finished request which kept nothing is refused at once
        t2 = _submit(srv, s, P, Fd, torch.empty_like(Fd))
        _wait(srv, t2)
        st, _ = srv.try_submit(Fd, torch.empty_like(Fd), cloud=t2)
        assert st == rfd.RFD_EINVAL
    finally:
        srv.close()


def test_server_evicts_idle_clouds_and_rebuilds_from_points():
    # resident clouds are compact (points, M, G: 2 m^2 doubles dominate at m = 1024), so 20
    # clouds of m = 1024 overflow a 512 MB plan pool that also has to hold one full plan
    specs = synth.batched_specs(count=20, seed=9, n_lo=1500, n_hi=2000, ms=(1024,), c=3)
    clouds, dev = _upload(specs)
    srv = rfd.Server((64 + 512) << 20, executors=2)
    try:
        ids = []
        for s, (P, F) in zip(specs, dev):
            res = _wait(srv, _submit(srv, s, P, F, torch.empty_like(F), keep=True))
            assert res["status"] == rfd.RFD_OK
            ids.append(res["cloud"])
        st = srv.stats()
        assert st["evicted"] > 0 and st["resident"] < len(specs)
        assert st["mem_peak"] <= st["mem_budget"]
        # the first cloud was evicted: reusing it without points fails, with points rebuilds it
        F0 = dev[0][1]
        st, _ = srv.try_submit(F0, torch.empty_like(F0), cloud=ids[0])
        assert st == rfd.RFD_EINVAL
        out = torch.empty_like(F0)
        res = _wait(srv, _submit(srv, specs[0], dev[0][0], F0, out, cloud=ids[0]))
        assert res["status"] == rfd.RFD_OK and res["reused"] == 0
        ref = oracle.rfd_gfi(clouds[0][0], clouds[0][1], specs[0].eps, _lam(specs[0]), specs[0].m, specs[0].seed)
        pc.assert_matches(out.cpu().numpy(), ref, clouds[0][1], BF16, label="rebuilt cloud")
    finally:
        srv.close()
