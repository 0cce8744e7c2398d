#!/usr/bin/env python
"""Benchmark of the RFD graph-field integration hot path on GB300.

One step = one pass of the whole path (Sec. 2.4): features (a2), the
reductions B^T A and B^T F over N (a3), G = lambda phi1(lambda M) in FP64 (a4),
Z = diag(s sgn r) G Y (a5) and out = F + Phi Z (a6), through rfd_gfi on inputs
already resident in HBM.  Default workload: N = 1,000,000 points on 8 random
ellipsoid surfaces, eps = 0.02, m = 1024, c = 3 (BF16 tensor-core form).

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU FP64 oracle
(the reference arm of this project) on a bounded sample of the same workload.

Multi-GPU: the clouds are independent problems, so N ranks each integrate
their own cloud (weak scaling, no collective on the data path); the timed
region is bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 (profiling recipe's table); a DFMA probe measured ~1.0
MUFU_PER_SM_CLK = 16            # sin or cos results per SM per clock (SFU)
GRAM_DRAM_BYTES_PER_BLOCK = 548.81e6 / 4096  # Gram kernel DRAM bytes per 64-point block, m = 1024 (ncu)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["large", "torus", "small"], default="large")
    ap.add_argument("--channels", type=int, default=None, help="field channels (default: the workload's)")
    ap.add_argument("--precision", choices=["bf16", "fp32"], default="bf16")
    ap.add_argument("--fp32-steps", type=int, default=2, help="timed steps of the FP32 plain form (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--c64-steps", type=int, default=20, help="timed steps of the c = 64 line (0: skip)")
    ap.add_argument("--cpu-sample", type=int, default=65536, help="points in the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the FP64 oracle at full N (the headline result's error; ~30 s, ~24 GB host memory)")
    ap.add_argument("--n", type=int, default=None, help="override the workload's point count (profiling runs)")
    ap.add_argument("--batched-clouds", type=int, default=512, help="clouds of the batched workload (0: skip)")
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="length of the serving trace (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-executors", type=int, default=6, help="batches in flight at once (one stream each)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the reductions' default launch parameters (a fixed launch sequence for profiling)")
    ap.add_argument("--gw-n", type=int, default=8192, help="points per cloud of the GW workload (0: skip)")
    ap.add_argument("--gw-steps", type=int, default=5)
    ap.add_argument("--eigen-clouds", type=int, default=1024, help="clouds of the kernel-eigenvalue workload (0: skip)")
    ap.add_argument("--sections", default="main,batched,serving,gw,eigen",
                    help="comma list of main, batched, serving (profiling runs select one; the JSON line then "
                         "carries only what ran)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (torchrun: one rank per GPU)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    def __init__(self, backend):
        import torch
        import torch.distributed as dist
        self.ws, self.rank, self.local = dist_env()
        self.dist = dist if self.ws > 1 else None
        if self.dist:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend)
        self.torch = torch

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if not self.dist:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64,
                              device="cuda" if self.dist.get_backend() == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


def whole_job_value(ws: int, units_per_rank: float, ms_max: float) -> float:
    """Replicas: every rank processes its own units; the job's rate is their sum
    over the slowest rank's time."""
    return ws * units_per_rank / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"rfd_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per step: tensor flops of the Gram and Phi^T F, HBM bytes of points, F and out
# ---------------------------------------------------------------------------
def work_model(n, m, c):
    gram_flops = n * m * (m + 1) + 2 * n * m * c          # symmetric Phi^T Phi + Phi^T F
    apply_flops = 2 * n * m * c
    hbm_bytes = 12 * n * (1 + c)                           # points, F read twice, out
    sincos = n * m                                         # feature values (cos + sin)
    return dict(gram_flops=gram_flops, apply_flops=apply_flops, hbm_bytes=hbm_bytes, sincos=sincos)


def phi1_flops(m, q, s):
    """FP64 flops of the block-triangular Pade evaluation: its m x m x m GEMMs
    (2 m^3 each: the even powers, X Sp, Higham's two grouped products for q = 13,
    two per squaring but the last), the LU (2/3 m^3) and the two triangular
    solves with m (s = 0) or 2m right-hand sides (2 m^2 per right-hand side)."""
    if not q:
        return 0.0
    gemms = (3 if q == 13 else (q - 1) // 2) + (2 if q == 13 else 0) + 1 + (2 * s - 1 if s > 0 else 0)
    nrhs = 2 * m if s > 0 else m
    return gemms * 2.0 * m ** 3 + (2.0 / 3.0) * m ** 3 + 2.0 * m * m * nrhs


# ---------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def accuracy_vs_oracle(pts, F, eps, lam, m, seed, outs):
    """Every output element of the GPU results against the FP64 oracle at full
    N (outside the timed region): the whole output, the increment out - F, and
    the worst row, as the parity tests measure them."""
    import oracle
    t0 = time.perf_counter()
    ref = oracle.rfd_gfi(pts, F, eps, lam, m, seed)
    F64 = np.asarray(F, dtype=np.float64)
    inc = ref - F64
    inc_norm = float(np.linalg.norm(inc))
    row_inc = float(np.sqrt((inc * inc).sum(axis=1)).max())
    res = {"oracle": "FP64 CPU oracle at full N, every element", "oracle_s": round(time.perf_counter() - t0, 1),
           "relative_increment": inc_norm / float(np.linalg.norm(F64))}
    for name, out in outs.items():
        if out is None:
            continue
        d = np.asarray(out, dtype=np.float64) - ref
        res[name] = {"rel_err_out": float(np.linalg.norm(d) / np.linalg.norm(ref)),
                     "rel_err_increment": float(np.linalg.norm(d) / inc_norm),
                     "max_row_err_over_max_row_increment": float(np.sqrt((d * d).sum(axis=1)).max() / row_inc)}
    return res


def time_oracle(pts, F, eps, lam, m, seed, steps=1):
    import oracle
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.rfd_gfi(pts, F, eps, lam, m, seed)
    return (time.perf_counter() - t0) / steps


def time_oracle_stages(pts, F, eps, lam, m, seed):
    """The oracle's steps timed one by one (ms), as the GPU's step breakdown is."""
    import oracle
    F64 = np.asarray(F, dtype=np.float64)
    t = {}
    t0 = time.perf_counter()
    omega = oracle.sample_frequencies(m, eps, seed)
    r = oracle.weights(omega, eps)
    t["a1 frequencies and weights"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    A, B = oracle.factors(pts, omega, r)
    t["a2 features"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    M = B.T @ A
    Y = B.T @ F64
    t["a3 reductions"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    G = lam * oracle.phi1(lam * M)
    t["a4 phi1"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    _ = F64 + A @ (G @ Y)
    t["a5-a6 apply"] = time.perf_counter() - t0
    return {k: round(v * 1e3, 3) for k, v in t.items()}


def time_oracle_single_thread(name="small", sample=None, reps=5):
    """The oracle on a workload (by default the small one: N = 2048, m = 64, c = 3),
    or on its first `sample` points, with one BLAS / OpenMP thread, in a child
    process (the thread count is fixed at import)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, time, oracle, synth\n"
            f"s = synth.config_single({name!r})\n"
            "pts, F = synth.make_cloud(s)\n"
            f"k = {sample or 0} or s.n\n"
            "pts, F = pts[:k], F[:k]\n"
            "lam = s.lam * s.m / s.n\n"
            "oracle.rfd_gfi(pts, F, s.eps, lam, s.m, s.seed)\n"
            "t0 = time.perf_counter()\n"
            f"for _ in range({reps}): oracle.rfd_gfi(pts, F, s.eps, lam, s.m, s.seed)\n"
            f"t = (time.perf_counter() - t0) / {reps}\n"
            "print(json.dumps({'ms': t * 1e3, 'value': k * F.shape[1] / t, 'n': s.n, 'm': s.m, 'c': F.shape[1],"
            " 'eps': s.eps}))\n")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, cwd=os.path.dirname(os.path.abspath(__file__)),
                             capture_output=True, text=True, timeout=300)
        d = json.loads(out.stdout.strip().splitlines()[-1])
        what = f"{name}: N={d['n']}, eps={d['eps']}, m={d['m']}, c={d['c']}"
        if sample:
            what += f"; the first {sample} points (lambda kept at the full cloud's lambda m/N)"
        return {"workload": what, "cores": 1, "ms_per_step": d["ms"], "value": d["value"], "unit": "points*ch/s"}
    except Exception as e:  # a missing measurement is reported, not fatal
        return {"unavailable": str(e)[:200]}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def arm_config(args, spec, n, m, c, lam, ws):
    """The `config` object of the JSON line, the same for both arms."""
    fbytes = 2 if args.precision == "bf16" else 4
    return {"workload": f"{args.workload}: N={n} points ({spec.kind}), eps={spec.eps}, m={m}, c={c}, "
                        f"lambda={spec.lam} x m/N = {lam:.4g}, seed={spec.seed}",
            "l2": "inputs > L2: the step rewrites and rereads the feature matrix "
                  f"({(m + 16) * n * fbytes / 1e9:.2f} GB)",
            "parallelism": f"replicas x{ws}"}


def reference_arm(args, spec, pts, F, lam):
    ns = min(args.cpu_sample, spec.n)
    c = F.shape[1]
    for _ in range(args.warmup if args.warmup < 2 else 1):
        time_oracle(pts[:ns], F[:ns], spec.eps, lam, spec.m, spec.seed)
    t = time_oracle(pts[:ns], F[:ns], spec.eps, lam, spec.m, spec.seed, steps=args.steps)
    val = ns * c / t
    unit = "points*ch/s"
    cb = {"value": val, "unit": unit, "cores": cpu_cores(), "kind": "oracle",
          "sample": f"first {ns} of {spec.n} points, m={spec.m}, c={c}, FP64 NumPy/SciPy, whole path per step"}
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args, spec, spec.n, spec.m, c, lam, args.gpus),
            "cpu_baseline": cb, "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


METRIC = "RFD GFI points*ch/s at N=1M, m=1024 (BF16 tensor-core form; FP32 plain form alongside)"


# ---------------------------------------------------------------------------
# batched workload: 512 clouds of uneven N and m in shared launches (CUDA graphs)
# ---------------------------------------------------------------------------
def bench_batched(args, dev, stream, D):
    import torch
    import paper_2302_00942_gb300 as rfd
    specs = synth.batched_specs(count=args.batched_clouds, seed=0)
    plans, items = [], []
    for s in specs:
        pts, F = synth.make_cloud(s)
        plans.append(rfd.Plan(s.n, s.m, s.eps, s.lam * s.m / s.n, s.seed, max_channels=s.c,
                              precision=rfd.RFD_BF16_TC, stream=stream))
        items.append({"points": torch.from_numpy(pts).to(dev), "F": torch.from_numpy(F).to(dev)})
    for it in items:
        it["out"] = torch.empty_like(it["F"])
    units = sum(s.n * s.c for s in specs)
    res = {"workload": f"{len(specs)} clouds, N log-uniform [1e3, 2e5] (sum {sum(s.n for s in specs)}), "
                       "sphere/torus, m in {64,128,256}, c=8, eps=0.05, lambda U[0.01,0.2] x m/N"}
    # the timed path: graph replay (the first warm-up call autotunes the reductions)
    gb = rfd.Batch(plans, stream=stream, graph=True, autotune=True)
    for _ in range(max(3, args.warmup)):
        gb.gfi(items)
    gb.sync()
    gb.stats_reset()
    D.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batched_steps):
        gb.gfi(items)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    gb.sync()
    ms = D.max(e0.elapsed_time(e1) / args.batched_steps)
    gst = gb.stats()
    gb.close()
    # per-step breakdown from direct launches with CUDA-event timing (same tuning, from the cache)
    tb = rfd.Batch(plans, stream=stream, timing=True, autotune=True)
    for _ in range(2):
        tb.gfi(items)
    tb.sync()
    tb.stats_reset()
    tb.gfi(items)
    tb.sync()
    st = tb.stats()
    tb.close()
    res["step_ms"] = {k: round(v, 4) for k, v in st["step_ms"].items()}
    for p in plans:
        p.close()
    res["autotune"] = {"waves": gst["tune_waves"], "phase_blocks": gst["tune_phase_blocks"], "tuned": gst["tuned"]}
    res.update({"value": D.ws * units / (ms * 1e-3), "unit": "points*ch/s", "ms_per_step": ms,
                "gpu_launches_per_step": gst["kernel_launches"] / args.batched_steps, "cuda_graphs": True,
                "steps": args.batched_steps})
    return res


# ---------------------------------------------------------------------------
# serving: Poisson arrivals of GFI requests through rfd_submit / rfd_poll
# ---------------------------------------------------------------------------
def bench_gw(args, dev, stream, D):
    """One (F)GW conditional-gradient iteration's FM-heavy steps (App. C.2) between
    two random 3-D distributions of gw_n points, at the experiments' m = 16,
    eps = 0.3, lambda = -0.2 (x m/N): the tensor product L(C, D, T) and the line
    search, on two resident BF16 plans (graph replay, 256-column chunks)."""
    import torch
    import paper_2302_00942_gb300 as rfd
    n, m, eps, lam = args.gw_n, 16, 0.3, -0.2
    X, Y, T, p, q, Gt, M = synth.gw_problem(n, n, seed=0)
    lam_a = lam * m / n
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)  # noqa: E731
    pc = rfd.Plan(n, m, eps, lam_a, 21, max_channels=256, precision=rfd.RFD_BF16_TC, stream=stream, graph=True)
    pd = rfd.Plan(n, m, eps, lam_a, 22, max_channels=256, precision=rfd.RFD_BF16_TC, stream=stream, graph=True)
    pc.features(cu(X))
    pd.features(cu(Y))
    Td, pv, qv = cu(T), cu(p), cu(q)
    G = np.outer(p, q)
    Gd, dGd, Md = cu(G), cu(Gt - G), cu(M)
    L = rfd.gw_tensor_product(pc, pd, Td, pv, qv)  # warm-up (captures the graphs)
    rfd.gw_line_search(pc, pd, 0.5, Gd, dGd, Md, pv, qv)
    torch.cuda.synchronize(dev)
    D.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = max(1, args.gw_steps)
    e0.record(stream)
    for _ in range(k):
        rfd.gw_tensor_product(pc, pd, Td, pv, qv, out=L)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    tp_ms = D.max(e0.elapsed_time(e1) / k)
    e0.record(stream)
    for _ in range(k):
        ls = rfd.gw_line_search(pc, pd, 0.5, Gd, dGd, Md, pv, qv)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ls_ms = D.max(e0.elapsed_time(e1) / k)
    io = 8.0 * n * n  # T in, L out (FP32)
    peaks, _ = load_peaks()
    res = {"workload": f"two uniform random 3-D clouds of {n} points, m={m}, eps={eps}, lambda={lam} x m/N, "
                       "dense coupling T (n x n, FP32)",
           "tensor_product_ms": tp_ms, "line_search_ms": ls_ms, "line_search": {"tau": ls[0], "a": ls[1], "b": ls[2]},
           "tensor_product_io": {"bytes": io, "achieved_gbs": io / (tp_ms * 1e-3) / 1e9,
                                 "frac_of_measured_hbm": io / (tp_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}}
    if D.rank == 0 and D.ws == 1 and not args.no_cpu:
        import oracle
        ac = oracle.rfd_kernel_action(X, eps, lam_a, m, 21)
        ad = oracle.rfd_kernel_action(Y, eps, lam_a, m, 22)
        t0 = time.perf_counter()
        Lref = oracle.gw_tensor_product(ac, ad, T, p, q)
        t_or = time.perf_counter() - t0
        res["cpu_baseline"] = {"tensor_product_ms": t_or * 1e3, "cores": cpu_cores(), "kind": "oracle",
                               "sample": "one FP64 tensor product at the same size",
                               "rel_err_vs_oracle": oracle.rel_frobenius(L.cpu().numpy(), Lref)}
    pc.close()
    pd.close()
    return res


def bench_eigen(args, dev, stream, D):
    """Kernel eigenvalues for shape classification (Sec. 3.3): the 32 smallest
    eigenvalues of exp(lambda W_hat) for every cloud of a batch of 2048-point
    shapes (eps = 0.1, lambda = -0.1 x m/N, m = 64), from points: steps a2-a3
    batched (graph replay), then one CTA per cloud on the m x m problem."""
    import torch
    import paper_2302_00942_gb300 as rfd
    specs = synth.eigen_specs(count=args.eigen_clouds, seed=0)
    clouds = [synth.make_cloud(s)[0] for s in specs]
    lams = [s.lam * s.m / s.n for s in specs]
    k = 32

    def mk_plans():
        return [rfd.Plan(s.n, s.m, s.eps, lam, s.seed, max_channels=1, precision=rfd.RFD_BF16_TC, stream=stream)
                for s, lam in zip(specs, lams)]
    plans = mk_plans()
    items = [{"points": torch.from_numpy(p).to(dev)} for p in clouds]
    gb = rfd.Batch(plans, stream=stream, graph=True)
    out = gb.eigenvalues(items, k)
    gb.eigenvalues(items, k, out=out)
    torch.cuda.synchronize(dev)
    D.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 5
    e0.record(stream)
    for _ in range(steps):
        gb.eigenvalues(items, k, out=out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = D.max(e0.elapsed_time(e1) / steps)
    gb.close()
    tb = rfd.Batch(plans, stream=stream, timing=True)
    tb.eigenvalues(items, k)
    tb.stats_reset()
    for _ in range(3):
        tb.eigenvalues(items, k, out=out)
    tb.sync()
    st = tb.stats()
    tb.close()
    got = out.cpu().numpy()
    for p in plans:
        p.close()
    n_cl = len(specs)
    res = {"workload": f"{n_cl} shapes (sphere / torus / ellipsoid union, 2048 points each), m=64, eps=0.1, "
                       f"lambda=-0.1 x m/N, k={k} smallest eigenvalues of exp(lambda W_hat)",
           "value": D.ws * n_cl / (ms * 1e-3), "unit": "clouds/s", "ms_per_batch": ms,
           "step_ms": {kk: round(v, 4) for kk, v in st["step_ms"].items() if v}}
    if D.rank == 0 and D.ws == 1 and not args.no_cpu:
        import oracle
        sample = min(16, n_cl)
        t0 = time.perf_counter()
        refs = [oracle.rfd_kernel_eigenvalues(clouds[i], specs[i].eps, lams[i], specs[i].m, specs[i].seed, k=k)
                for i in range(sample)]
        t = time.perf_counter() - t0
        err = max(float(np.max(np.abs(got[i] - refs[i]) / refs[i])) for i in range(sample))
        res["cpu_baseline"] = {"value": sample / t, "unit": "clouds/s", "cores": cpu_cores(), "kind": "oracle",
                               "sample": f"first {sample} clouds, FP64", "max_rel_err_vs_oracle": err}
    return res


def bench_serving(args, dev):
    import torch
    import paper_2302_00942_gb300 as rfd
    trace = synth.serving_trace(rate=args.serve_rate, duration=args.serve_seconds, seed=0)
    # point sources: 16 templates of 5e5 points (8 spheres, 8 tori of random scale); a request
    # of N points uses the first N points of one template (a prefix of an i.i.d. sample is one too)
    n_max = 500_000
    templates = []
    for k in range(16):
        kind = "sphere" if k % 2 == 0 else "torus"
        spec = synth.CloudSpec(kind, n_max, 64, 1, 0.05, 0.1, 4242 + k, scale=0.5 + 1.5 * k / 15, sub=k)
        templates.append(torch.from_numpy(synth.make_cloud(spec)[0]).to(dev))
    F_pool = torch.randn(n_max * 32 + 4096, device=dev)
    srv = rfd.Server(int(args.serve_budget_gb * (1 << 30)), max_batch=256, executors=args.serve_executors)
    ticket_of = {}  # trace index of a root request -> its ticket (= the id of the cloud it keeps)

    def submit(i, spec, j):
        n, c = spec.n, spec.c
        off = (i * 7919) % 4096
        F = F_pool[off:off + n * c].view(n, c)
        out = torch.empty((n, c), device=dev)
        pts = templates[(i if j < 0 else j) % 16][:n]
        kw = dict(points=pts, m=spec.m, eps=spec.eps, lam=spec.lam * spec.m / n, seed=spec.seed)
        if j >= 0 and j in ticket_of:
            # the root's cloud, resident or still being made (the request waits behind its root);
            # the points are passed as well, so an evicted cloud is rebuilt
            kw["cloud"] = ticket_of[j]
        else:
            kw.update(keep=True, max_channels=32)
        st, t = srv.try_submit(F, out, **kw)
        return st, t, out

    # warm-up: a short burst, not timed
    warm = []
    for i, (_, spec, j) in enumerate(trace[:64]):
        st, t, out = submit(i, spec, -1)
        if t:
            warm.append((t, out))
    for t, _ in warm:
        srv.poll(t, 120_000_000)
    pending = {}
    results = []
    rejected = 0
    t0 = time.perf_counter()

    def retire(timeout_us=0):
        # every pending request that has finished: its latency to this poll's return
        for t in list(pending):
            st, r = srv.poll(t, timeout_us)
            if st != rfd.RFD_OK:
                continue
            now = time.perf_counter()
            n, c, _, t_sub = pending.pop(t)
            r["n"], r["c"] = n, c
            r["client_ms"] = (now - t_sub) * 1e3
            results.append(r)

    for i, (ta, spec, j) in enumerate(trace):
        while True:
            retire()
            now = time.perf_counter() - t0
            if now >= ta:
                break
            time.sleep(min(ta - now, 1e-4))
        t_sub = time.perf_counter()
        st, t, out = submit(i, spec, j)
        if t is None:
            rejected += 1
            continue
        if j < 0:
            ticket_of[i] = t
        pending[t] = (spec.n, spec.c, out, t_sub)
    while pending:
        retire(1000)
    wall = time.perf_counter() - t0
    sst = srv.stats()
    srv.close()
    ok = [r for r in results if r["status"] == rfd.RFD_OK]
    lat = np.array([r["latency_ms"] for r in ok]) if ok else np.zeros(1)
    clat = np.array([r["client_ms"] for r in ok]) if ok else np.zeros(1)
    units = sum(r["n"] * r["c"] for r in ok)
    return {"workload": f"Poisson {args.serve_rate:.0f} req/s for {args.serve_seconds:.0f} s: N log-uniform "
                        "[500, 5e5], m in {64..512}, c in 1..32, lambda U[0.01,0.2] x m/N, eps=0.05, 30% reuse "
                        "(a reuse names its root's ticket: resident compact cloud, or waits for the root)",
            "executors": args.serve_executors,
            "requests": len(trace), "completed_ok": len(ok), "failed": len(results) - len(ok), "rejected": rejected,
            "p50_ms": float(np.percentile(clat, 50)), "p99_ms": float(np.percentile(clat, 99)),
            "latency": "rfd_submit to the rfd_poll that returns the result (the client polls every pending "
                       "ticket about every 0.1 ms)",
            "server_p50_ms": float(np.percentile(lat, 50)), "server_p99_ms": float(np.percentile(lat, 99)),
            "mean_batch": float(np.mean([r["batch_size"] for r in ok])) if ok else 0.0,
            "reused": sum(r["reused"] for r in ok), "evicted": sst["evicted"], "batches": sst["batches"],
            "throughput": units / wall, "unit": "points*ch/s", "req_per_s": len(ok) / wall,
            "mem_peak_gb": sst["mem_peak"] / 2 ** 30, "gpu_launches": sst["kernel_launches"]}


def main():
    args = parse()
    ws, rank, local = dist_env()
    spec = synth.config_single(args.workload, args.channels)
    if args.n:
        import dataclasses
        spec = dataclasses.replace(spec, n=args.n)
    if args.impl == "reference":
        if rank != 0:
            return 0
        pts, F = synth.make_cloud(spec)
        lam = spec.lam * spec.m / spec.n
        print(json.dumps(reference_arm(args, spec, pts, F, lam)))
        return 0

    import torch
    import paper_2302_00942_gb300 as rfd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    D = Dist("nccl")
    sections = set(args.sections.split(","))
    if "main" not in sections:   # a profiling run of one section
        stream = torch.cuda.current_stream(dev)
        res = {"metric": METRIC, "sections": sorted(sections)}
        if "batched" in sections and args.batched_clouds > 0:
            res["batched"] = bench_batched(args, dev, stream, D)
        if "serving" in sections and args.serve_seconds > 0:
            res["serving"] = bench_serving(args, dev)
        if "gw" in sections and args.gw_n > 0:
            res["gw"] = bench_gw(args, dev, stream, D)
        if "eigen" in sections and args.eigen_clouds > 0:
            res["eigen"] = bench_eigen(args, dev, stream, D)
        if rank == 0:
            print(json.dumps(res))
        D.close()
        return 0
    # each rank integrates its own cloud (independent problems)
    if ws > 1:
        import dataclasses
        spec = dataclasses.replace(spec, sub=rank)
    pts, F = synth.make_cloud(spec)
    n, c, m = spec.n, F.shape[1], spec.m
    lam = spec.lam * m / n   # diffusion time in units of the estimator's mean eigenvalue N/m
    stream = torch.cuda.current_stream(dev)
    P = torch.from_numpy(pts).to(dev)
    Ft = torch.from_numpy(F).to(dev)
    out = torch.empty_like(Ft)
    prec = rfd.RFD_BF16_TC if args.precision == "bf16" else rfd.RFD_FP32_PLAIN
    tune = prec == rfd.RFD_BF16_TC and not args.no_autotune
    # the timed plan replays each call from CUDA graphs (BF16 form); a second plan with per-step
    # CUDA events gives the step breakdown (events between kernels would sit in the timed path)
    gplan = rfd.Plan(n, m, spec.eps, lam, spec.seed, max_channels=c, precision=prec, stream=stream, autotune=tune,
                     graph=(prec == rfd.RFD_BF16_TC))
    plan = rfd.Plan(n, m, spec.eps, lam, spec.seed, max_channels=c, precision=prec, stream=stream, timing=True,
                    autotune=tune)

    for _ in range(args.warmup):
        gplan.gfi(P, Ft, out)
    gplan.sync()
    gplan.stats_reset()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    D.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        gplan.gfi(P, Ft, out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    D.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = D.max(ms)
    gst = gplan.stats()
    out_bf = out.clone()
    # step breakdown (per-step events), outside the timed region
    for _ in range(max(1, min(args.warmup, 3))):
        plan.gfi(P, Ft, out)
    plan.sync()
    plan.stats_reset()
    for _ in range(args.steps):
        plan.gfi(P, Ft, out)
    plan.sync()
    st = plan.stats()
    st["kernel_launches"] = gst["kernel_launches"]

    # warm: a new field on the resident features and G (rfd_integrate: steps a3(Y) to a6)
    F2 = torch.from_numpy(synth.gaussian_field(n, c, spec.seed + 1)).to(dev)
    out2 = torch.empty_like(F2)
    for _ in range(2):
        plan.integrate(F2, out2)
    plan.sync()
    plan.stats_reset()
    D.barrier()
    torch.cuda.synchronize(dev)
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    for _ in range(args.steps):
        plan.integrate(F2, out2)
    w1.record(stream)
    torch.cuda.synchronize(dev)
    wst = plan.stats()
    for _ in range(2):
        gplan.integrate(F2, out2)
    gplan.sync()
    torch.cuda.synchronize(dev)
    w0.record(stream)
    for _ in range(args.steps):
        gplan.integrate(F2, out2)
    w1.record(stream)
    torch.cuda.synchronize(dev)
    warm_ms = D.max(w0.elapsed_time(w1) / args.steps)

    # Wasserstein barycenter (App. C): repeated GFI on the resident plan, k = 3 bumps, 10 passes
    p64 = np.asarray(pts, dtype=np.float64)
    bumps = []
    for cidx in (0, n // 3, (2 * n) // 3):
        dd = np.linalg.norm(p64 - p64[cidx], axis=1)
        bb = 1.0 + 0.5 * np.exp(-(dd / 0.5) ** 2)
        bumps.append(bb / bb.sum())
    bary_k = min(3, c)
    Mu = torch.from_numpy(np.stack(bumps[:bary_k], axis=1).astype(np.float32)).to(dev)
    Ar = torch.full((n,), 1.0 / n, dtype=torch.float32, device=dev)
    bary_out = gplan.barycenter(Mu, Ar, [1.0 / bary_k] * bary_k, 2)
    gplan.sync()
    torch.cuda.synchronize(dev)
    y0, y1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bary_passes = 10
    y0.record(stream)
    gplan.barycenter(Mu, Ar, [1.0 / bary_k] * bary_k, bary_passes, out=bary_out)
    y1.record(stream)
    torch.cuda.synchronize(dev)
    bary_ms = D.max(y0.elapsed_time(y1) / bary_passes)

    # end to end: host buffers, H2D of every step's inputs and D2H of its result inside the
    # timed region, pipelined over the steps with double buffers: step k's inputs go up on an
    # upload stream while step k-1 computes, and its result comes back on a download stream
    # while step k+1 computes (the copy engines run beside the kernels)
    Ph = torch.from_numpy(pts).pin_memory()
    Fh = torch.from_numpy(F).pin_memory()
    Oh = [torch.empty_like(Fh).pin_memory() for _ in range(2)]
    Pd = [torch.empty_like(P) for _ in range(2)]
    Fd = [torch.empty_like(Ft) for _ in range(2)]
    Od = [torch.empty_like(Ft) for _ in range(2)]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    D.barrier()
    torch.cuda.synchronize(dev)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(up)
    for k in range(args.e2e_steps):
        b = k % 2
        if k >= 2:
            up.wait_event(ev_done[b])        # step k-2 has read Pd[b], Fd[b]
        with torch.cuda.stream(up):
            Pd[b].copy_(Ph, non_blocking=True)
            Fd[b].copy_(Fh, non_blocking=True)
        ev_in[b].record(up)
        stream.wait_event(ev_in[b])
        if k >= 2:
            stream.wait_event(ev_out[b])     # step k-2's result has left Od[b]
        rfd.rfd_gfi(gplan.handle, Pd[b], Fd[b], c, c, Od[b], c)
        ev_done[b].record(stream)
        down.wait_event(ev_done[b])
        with torch.cuda.stream(down):
            Oh[b].copy_(Od[b], non_blocking=True)
        ev_out[b].record(down)
    up.wait_stream(down)
    a1.record(up)
    torch.cuda.synchronize(dev)
    D.barrier()
    e2e_ms = D.max(a0.elapsed_time(a1) / args.e2e_steps)
    # the pipelined steps return what the device-timed step returned
    e2e_same = bool(torch.equal(Oh[(args.e2e_steps - 1) % 2], out_bf.cpu()))

    # compact warm path: the same plan with Phi released (rfd_plan_compact); a new field is
    # integrated from the points alone (Phi^T F from the points in FP32, then a5, a6), the cost
    # of generating the features on the fly instead of keeping them resident
    out2_full = out2.clone()
    full_bytes = gplan.device_bytes()
    gplan.compact()
    compact_bytes = gplan.device_bytes()
    out3 = torch.empty_like(F2)
    for _ in range(2):
        gplan.integrate(F2, out3)
    gplan.sync()
    torch.cuda.synchronize(dev)
    w0.record(stream)
    for _ in range(args.steps):
        gplan.integrate(F2, out3)
    w1.record(stream)
    torch.cuda.synchronize(dev)
    compact_ms = D.max(w0.elapsed_time(w1) / args.steps)
    # the step breakdown of the compact path, on the event-timed plan compacted the same way
    plan.compact()
    for _ in range(2):
        plan.integrate(F2, out3)
    plan.sync()
    plan.stats_reset()
    for _ in range(args.steps):
        plan.integrate(F2, out3)
    plan.sync()
    cst = plan.stats()
    inc_full = (out2_full.double() - F2.double())
    compact_dev = float((out3.double() - out2_full.double()).norm() / inc_full.norm())
    compact = {"value": whole_job_value(ws, n * c, compact_ms), "unit": "points*ch/s", "ms_per_step": compact_ms,
               "what": "rfd_integrate on the compact plan: B^T F from the points (FP32 SIMT), a5, a6",
               "step_ms": {k: round(v, 4) for k, v in cst["step_ms"].items() if v},
               "device_bytes": int(compact_bytes), "full_plan_device_bytes": int(full_bytes),
               "increment_rel_diff_vs_resident": compact_dev}
    plan.close()
    gplan.close()

    # the same cloud with 64 channels (the large workload's second field width): its own
    # autotuned, graph-replayed plan, timed the same way
    c64 = None
    if prec == rfd.RFD_BF16_TC and c != 64 and args.c64_steps > 0:
        F64 = torch.from_numpy(synth.gaussian_field(n, 64, spec.seed + 2)).to(dev)
        o64 = torch.empty_like(F64)
        p64 = rfd.Plan(n, m, spec.eps, lam, spec.seed, max_channels=64, precision=prec, stream=stream,
                       autotune=tune, graph=True)
        for _ in range(max(args.warmup, 3)):
            p64.gfi(P, F64, o64)
        p64.sync()
        torch.cuda.synchronize(dev)
        D.barrier()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(args.c64_steps):
            p64.gfi(P, F64, o64)
        q1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = D.max(q0.elapsed_time(q1) / args.c64_steps)
        wm64, (pk, _) = work_model(n, m, 64), load_peaks()
        t64 = max(wm64["hbm_bytes"] / (pk["hbm_gbs"] * 1e9),
                  (wm64["gram_flops"] + wm64["apply_flops"]) / (pk["bf16_tflops"] * 1e12))
        s64 = p64.stats()
        c64 = {"value": whole_job_value(ws, n * 64, ms64), "unit": "points*ch/s", "ms_per_step": ms64,
               "what": "rfd_gfi with c = 64 on the same cloud (own plan, CUDA graphs, autotuned)",
               "path_roofline": {"t_roofline_ms": t64 * 1e3, "frac_of_step": t64 * 1e3 / ms64},
               "autotune": {"lanes_pct": s64["tune_lanes_pct"], "phase_blocks": s64["tune_phase_blocks"],
                            "gram_form": "CTA pairs (2-SM MMA)" if s64["tune_pair_gram"] else "one SM per tile"}}
        p64.close()
        # its step breakdown (direct launches, CUDA-event timing; same tuning, from the cache), and
        # the apply (step a6) in both forms: tensor cores (BF16 hi/lo splits) and FP32 SIMT
        t64p = rfd.Plan(n, m, spec.eps, lam, spec.seed, max_channels=64, precision=prec, stream=stream,
                        autotune=tune, timing=True)
        apply_ms = {}
        for form, flag in (("tensor_core", 2), ("simt_fp32", 0)):
            assert rfd.lib.rfd_debug_plan_set_apply_tc(t64p.handle, flag) == 0, rfd.rfd_last_error()
            for _ in range(2):
                t64p.gfi(P, F64, o64)
            t64p.sync()
            t64p.stats_reset()
            t64p.gfi(P, F64, o64)
            t64p.sync()
            sm64 = t64p.stats()["step_ms"]
            if flag:
                c64["step_ms"] = {k: round(v, 4) for k, v in sm64.items() if v}
            apply_ms[form] = round(sm64["apply"], 4)
        c64["apply_ms"] = apply_ms
        t64p.close()
        del F64, o64

    # FP32 plain form on the same inputs (the form the BF16 path must beat), and the BF16 form's
    # deviation from it (the FP32 form matches the FP64 oracle to <= 1e-5 in the parity tests)
    fp32 = None
    out_fp32 = None
    if args.fp32_steps > 0 and prec == rfd.RFD_BF16_TC:
        p32 = rfd.Plan(n, m, spec.eps, lam, spec.seed, max_channels=c, precision=rfd.RFD_FP32_PLAIN, stream=stream,
                       timing=True)
        o32 = torch.empty_like(Ft)
        p32.gfi(P, Ft, o32)
        p32.sync()
        p32.stats_reset()
        torch.cuda.synchronize(dev)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.fp32_steps):
            p32.gfi(P, Ft, o32)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        ms32 = D.max(b0.elapsed_time(b1) / args.fp32_steps)
        st32 = p32.stats()
        p32.close()
        out_fp32 = o32.cpu().numpy()
        diff = float(torch.linalg.norm((out_bf - o32).double()) / torch.linalg.norm(o32.double()))
        inc = float(torch.linalg.norm((o32 - Ft).double()) / torch.linalg.norm(Ft.double()))
        fp32 = {"value": ws * n * c / (ms32 * 1e-3), "ms_per_step": ms32,
                "step_ms": {k: round(v, 4) for k, v in st32["step_ms"].items()},
                "bf16_rel_err_vs_fp32": diff, "relative_increment": inc}

    peaks, peak_src = load_peaks()
    wm = work_model(n, m, c)
    steps = st["step_ms"]
    dom = max(steps, key=steps.get)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mufu_peak = sms * MUFU_PER_SM_CLK * (clk["sm_mhz"] or 1900.0) * 1e6
    # phi1 (emulated FP64): phi1_gemms m x m x m FP64 products (the Taylor form: X^2, X^3, X^4, three
    # Horner products, two per squaring), each at most 16 BF16 residue products (one per modulus)
    ngemm = st.get("phi1_gemms", 0) if st.get("phi1_emulated") else 0
    pf = ngemm * 2.0 * m ** 3 if ngemm else phi1_flops(m, st["pade_degree"], st["squarings"])
    phi1_tc_flops = ngemm * 16 * 2.0 * m ** 3
    # the apply's sin/cos count: the SIMT kernel recomputes Phi per channel group; the tensor-core
    # form (BF16 form, 5..64 channels) once per point and frequency
    tc_apply = prec == rfd.RFD_BF16_TC and (16 < c <= 64 or (8 < c <= 64 and m >= 512))
    groups = 1 if tc_apply else -(-c // (4 if c <= 4 else 8 if c <= 8 else 16 if c <= 16 else 32))
    step_roof = {
        "gram": {"bound": "tensor", "achieved": wm["gram_flops"] / (steps["gram"] * 1e-3) / 1e12,
                 "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                 "work": "N m(m+1) + 2 N m c flops per launch (symmetric Gram + Phi^T F)"},
        "phi1": ({"bound": "tensor", "achieved": phi1_tc_flops / (steps["phi1"] * 1e-3) / 1e12,
                  "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                  "work": f"{ngemm} emulated FP64 products x at most 16 BF16 residue products x 2 m^3 "
                          "(an upper bound: the first two Horner products use fewer moduli; residue splits "
                          "and reconstruction included in the time)",
                  "fp64_equivalent_tflops": pf / (steps["phi1"] * 1e-3) / 1e12}
                 if ngemm else
                 {"bound": "fp64", "achieved": pf / (steps["phi1"] * 1e-3) / 1e12, "peak": FP64_NOMINAL_TFLOPS,
                  "unit": "TFLOP/s", "work": "native FP64 Pade products, LU and solves"}),
        "features": {"bound": "alu", "achieved": wm["sincos"] / (steps["features"] * 1e-3) / 1e9,
                     "peak": mufu_peak / 1e9, "unit": "Gsincos/s", "work": "N m sin/cos values (MUFU)"},
        "apply": {"bound": "alu", "achieved": wm["sincos"] * groups / (steps["apply"] * 1e-3) / 1e9,
                  "peak": mufu_peak / 1e9, "unit": "Gsincos/s",
                  "work": ("N m sin/cos values (Phi recomputed once in FP32, its BF16 hi/lo parts times Z's "
                           "on the tensor cores); reads points, F; writes out") if tc_apply else
                          f"N m sin/cos values recomputed per channel group ({groups}); reads points, F; writes out"},
    }
    for v in step_roof.values():
        v["frac"] = v["achieved"] / v["peak"]
    # the dominant single kernel: the Gram kernel is one launch per step (the phi1 step is ~50 launches)
    roof = {k: v for k, v in step_roof["gram"].items() if k != "work"}
    roof["kernel"] = "gram_tc_kernel (step a3)"
    # DRAM bytes of the Gram kernel per 64-point block of the feature matrix, from one ncu capture at
    # N = 262,144, m = 1024 (dram__bytes_read.sum + dram__bytes_write.sum = 548.81 MB over 4096 blocks,
    # field rows padded to 16); the kernel reads the matrix once, so the bytes scale with the blocks a
    # launch covers.  Null for other shapes.
    roof["traffic"] = None
    cpad = -(-min(2 * c, 256) // 16) * 16 if prec == rfd.RFD_BF16_TC and 2 * c <= 256 else None
    if prec == rfd.RFD_BF16_TC and m == 1024 and cpad == 16:
        nblocks = -(-n // 128) * 2  # points padded to 128, blocks of 64
        phase = st["tune_phase_blocks"] or 4096
        launches = -(-nblocks // phase)
        roof["traffic"] = GRAM_DRAM_BYTES_PER_BLOCK * nblocks / launches
    roof["peak_source"] = (f"{peak_src} (burst bf16: the kernel runs at full SM clock inside a ~2 ms step; "
                           f"the sustained figure is for seconds-long loops under the power cap)")
    roof["scope"] = "the dominant kernel alone; the whole step's fraction is path_roofline.frac_of_step"
    # the same time against the paper-literal work of a general B^T A (2 N m^2) and B^T F
    roof["frac_paper_literal"] = (2.0 * n * m * m + 2.0 * n * m * c) / (steps["gram"] * 1e-3) / 1e12 / peaks["bf16_tflops"]
    roof["dominant_step"] = dom
    # whole-path roofline: slower of HBM bytes at peak bandwidth and tensor flops at peak
    t_roof = max(wm["hbm_bytes"] / (peaks["hbm_gbs"] * 1e9),
                 (wm["gram_flops"] + wm["apply_flops"]) / (peaks["bf16_tflops"] * 1e12))

    res = {
        "metric": METRIC, "value": whole_job_value(ws, n * c, ms_max), "unit": "points*ch/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": arm_config(args, spec, n, m, c, lam, ws),
        "roofline": roof,
        "path_roofline": {"t_roofline_ms": t_roof * 1e3, "frac_of_step": t_roof * 1e3 / ms_max,
                          "bound": "tensor" if wm["gram_flops"] / peaks["bf16_tflops"] / 1e12 >
                          wm["hbm_bytes"] / peaks["hbm_gbs"] / 1e9 else "hbm",
                          "peak": "measured burst bf16 and copy bandwidth",
                          "target_frac": 0.60, "target_met": t_roof * 1e3 / ms_max >= 0.60,
                          # against the paper-literal tensor work (a general B^T A: 2 N m^2, plus 4 N m c)
                          "frac_of_step_paper_literal": max(wm["hbm_bytes"] / (peaks["hbm_gbs"] * 1e9),
                                                            (2.0 * n * m * m + 4.0 * n * m * c) /
                                                            (peaks["bf16_tflops"] * 1e12)) * 1e3 / ms_max},
        "step_ms": {k: round(v, 4) for k, v in steps.items()},
        "step_roofline": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                          for k, v in step_roof.items()},
        "phi1": {"pade_degree": st["pade_degree"], "squarings": st["squarings"], "norm1": st["norm1"]},
        "clocks": clk,
        "e2e": {"value": ws * n * c / (e2e_ms * 1e-3), "unit": "points*ch/s", "ms_per_step": e2e_ms,
                "pipelined": "double-buffered: upload of step k+1 and download of step k-1 beside step k's kernels",
                "steps": args.e2e_steps, "result_equals_device_timed_step": e2e_same,
                "h2d_bytes_per_step": int(Ph.numel() * 4 + Fh.numel() * 4), "d2h_bytes_per_step": int(Oh[0].numel() * 4)},
        "gpu_launches": int(st["kernel_launches"]),
        "barycenter": {"what": f"entropic Wasserstein barycenter of {bary_k} bump distributions on the same cloud "
                               "(App. C): 2 GFI of k columns + 2 element-wise kernels per pass, resident plan",
                       "passes": bary_passes, "ms_per_pass": bary_ms},
        "autotune": {"lanes_pct": st["tune_lanes_pct"], "phase_blocks": st["tune_phase_blocks"], "tuned": st["tuned"],
                     "gram_form": "CTA pairs (2-SM MMA)" if st.get("tune_pair_gram") else "one SM per tile",
                     "features_beside_gram": bool(st.get("tune_overlap")),
                     "form_ms": {"one_sm": round(st["tune_form_ms"][0], 4), "cta_pairs": round(st["tune_form_ms"][1], 4)}},
        "warm": {"value": whole_job_value(ws, n * c, warm_ms), "unit": "points*ch/s", "ms_per_step": warm_ms,
                 "what": "rfd_integrate: a new field on the resident plan (steps a3(Y) to a6; with c <= 4 B^T F comes from the points in FP32, with more channels from a pass over the resident BF16 Psi)",
                 "step_ms": {k: round(v, 4) for k, v in wst["step_ms"].items() if v}},
        "warm_compact": compact,
        "fp32_plain": fp32,
        "headline_c64": c64,
    }
    if "batched" in sections and args.batched_clouds > 0 and prec == rfd.RFD_BF16_TC:
        res["batched"] = bench_batched(args, dev, stream, D)
    if "serving" in sections and args.serve_seconds > 0 and prec == rfd.RFD_BF16_TC:
        res["serving"] = bench_serving(args, dev)
        res["p99_ms"] = res["serving"]["p99_ms"]
    if "gw" in sections and args.gw_n > 0 and prec == rfd.RFD_BF16_TC:
        res["gw"] = bench_gw(args, dev, stream, D)
    if "eigen" in sections and args.eigen_clouds > 0 and prec == rfd.RFD_BF16_TC:
        res["eigen"] = bench_eigen(args, dev, stream, D)
    if rank == 0 and ws == 1 and not args.no_oracle_check:
        acc = accuracy_vs_oracle(pts, F, spec.eps, lam, m, spec.seed,
                                 {"bf16" if prec == rfd.RFD_BF16_TC else "fp32": out_bf.cpu().numpy(),
                                  "fp32": out_fp32})
        res["accuracy_vs_oracle"] = acc
        main_form = acc.get("bf16" if prec == rfd.RFD_BF16_TC else "fp32", {})
        res["rel_err_vs_oracle"] = main_form.get("rel_err_out")
        res["increment_rel_err_vs_oracle"] = main_form.get("rel_err_increment")
    if rank == 0 and ws == 1 and not args.no_cpu:
        ns = min(args.cpu_sample, n)
        t = time_oracle(pts[:ns], F[:ns], spec.eps, lam, m, spec.seed)
        res["cpu_baseline"] = {"value": ns * c / t, "unit": "points*ch/s", "cores": cpu_cores(), "kind": "oracle",
                               "sample": f"first {ns} of {n} points, same m, c, eps, lambda; whole path, FP64",
                               "stages_ms": time_oracle_stages(pts[:ns], F[:ns], spec.eps, lam, m, spec.seed),
                               "single_thread": time_oracle_single_thread(),
                               "single_thread_torus": time_oracle_single_thread("torus", None, 1)}
    if rank == 0:
        print(json.dumps(res))
    D.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
