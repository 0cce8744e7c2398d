"""The benchmark's multi-rank plumbing on the CPU: two gloo ranks, the barrier
and the max over ranks that bracket the timed region, and the whole-job value
(replicas: every rank integrates its own cloud, units add up)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    D = bench.Dist("gloo")
    assert (D.ws, D.rank) == (ws, rank)
    D.barrier()
    ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    q.put((rank, D.max(ms), bench.dist_env()))
    D.barrier()
    D.close()


def test_two_gloo_ranks_take_the_max_over_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(r for r, _, _ in out) == [0, 1]
    assert all(m == 15.0 for _, m, _ in out)
    assert {env for _, _, env in out} == {(2, 0, 0), (2, 1, 1)}


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    D = bench.Dist("gloo")
    assert D.dist is None and D.max(3.5) == 3.5
    D.barrier()
    D.close()


def test_whole_job_value_adds_the_ranks_units():
    sys.path.insert(0, ROOT)
    import bench
    # two replicas of 1e6 points x 3 channels in 7 ms (the max over ranks)
    assert bench.whole_job_value(2, 1_000_000 * 3, 7.0) == pytest.approx(2 * 3e6 / 7e-3)
