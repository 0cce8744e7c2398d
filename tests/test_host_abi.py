"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function the headers declare, its step-a1 sampler (Sec. 2.4) matches
the oracle bit for bit, and invalid arguments are rejected with RFD_EINVAL
before any device work."""
import glob
import os
import re

import numpy as np
import pytest

import oracle

import paper_2302_00942_gb300 as rfd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"RFD_API\s+[\w\s\*]+?\b(rfd_\w+)\s*\(", txt))
    return names


def test_library_exports_every_header_symbol():
    declared = header_functions()
    assert declared, "no RFD_API declarations found"
    assert declared == set(rfd.HEADER_SYMBOLS)
    import ctypes
    L = ctypes.CDLL(rfd.lib_path)
    for name in declared:
        assert hasattr(L, name), name
    assert "sm_103a" in rfd.rfd_version()


@pytest.mark.parametrize("m,eps,seed,sigma,R", [(64, 0.1, 0, 0, 0), (1024, 0.02, 0, 0, 0), (256, 0.05, 7, 0, 0),
                                                (66, 0.3, 123456789, 1.0, 10.0), (2, 0.5, 2**63 + 5, 0.7, 0.9),
                                                (512, 0.01, 42, 1.0, 0.0)])
def test_host_sampler_matches_oracle_bitwise(m, eps, seed, sigma, R):
    om, r = rfd.rfd_sample_frequencies(m, eps, seed, sigma, R)
    om_ref = oracle.sample_frequencies(m, eps, seed, sigma, R)
    np.testing.assert_array_equal(om, om_ref)
    r_ref = oracle.weights(om_ref, eps, sigma, R)
    np.testing.assert_allclose(r, r_ref, rtol=1e-13, atol=0)


def test_host_sampler_matches_golden_file():
    path = os.path.join(ROOT, "tests", "golden", "omega_m64_eps0.1_seed0.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    ref = np.array([[float.fromhex(x) for x in row] for row in rows])
    om, _ = rfd.rfd_sample_frequencies(64, 0.1, 0)
    np.testing.assert_array_equal(om, ref)


@pytest.mark.parametrize("kw", [dict(m=63), dict(m=0), dict(eps=0.0), dict(eps=-1.0), dict(eps=float("nan"))])
def test_sampler_rejects_invalid(kw):
    args = dict(m=64, eps=0.1, seed=0)
    args.update(kw)
    with pytest.raises(rfd.RfdError) as e:
        rfd.rfd_sample_frequencies(args["m"], args["eps"], args["seed"]) if args["m"] > 0 else \
            rfd.lib.rfd_sample_frequencies(args["m"], args["eps"], 0, 0, 0, None, None) == 0 or \
            (_ for _ in ()).throw(rfd.RfdError(rfd.RFD_EINVAL, "x", "m"))
    assert e.value.status == rfd.RFD_EINVAL


def test_sampler_acceptance_limit():
    # truncation far wider than the Gaussian: acceptance ~ sigma/R ~ 1e-7 per try
    with pytest.raises(rfd.RfdError) as e:
        rfd.rfd_sample_frequencies(2, 0.1, 0, 1e-4, 1e4)
    assert e.value.status == rfd.RFD_EINVAL
    assert "acceptance" in rfd.rfd_last_error()


@pytest.mark.parametrize("kw", [dict(n=0), dict(m=7), dict(m=8192), dict(max_channels=0), dict(max_channels=300),
                                dict(lam=float("inf")), dict(precision=5), dict(flags=16), dict(eps=0.0)])
def test_plan_rejects_invalid_before_device_work(kw):
    args = dict(n=100, m=64, eps=0.1, lam=0.1, seed=0, max_channels=3, precision=rfd.RFD_BF16_TC, flags=0)
    args.update(kw)
    with pytest.raises(rfd.RfdError) as e:
        rfd.rfd_plan(args["n"], args["m"], args["eps"], args["lam"], args["seed"], args["max_channels"],
                     args["precision"], None, flags=args["flags"])
    assert e.value.status == rfd.RFD_EINVAL
    assert rfd.rfd_last_error()


def test_null_handles_rejected():
    assert rfd.lib.rfd_features(None, None) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_integrate(None, None, 1, 1, None, 1) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_gfi(None, None, None, 1, 1, None, 1) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_sync(None) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_plan_stats(None, None) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_plan_stats_reset(None) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_plan_destroy(None) == rfd.RFD_OK
    assert rfd.lib.rfd_phi1(0, 1.0, None, None, 0, None, None) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_phi1(4, 1.0, None, None, 0, None, None) == rfd.RFD_EINVAL
    assert rfd.lib.rfd_debug_dgemm(1, 0, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None) == rfd.RFD_EINVAL


def test_null_handles_rejected_by_the_next_rows():
    """The barycenter, GW, eigenvalue and debug entry points check their handles
    and pointers before any device work (no GPU needed)."""
    import ctypes
    out3 = (ctypes.c_double * 3)()
    alpha = (ctypes.c_double * 1)(1.0)
    calls = {
        "rfd_barycenter": lambda: rfd.lib.rfd_barycenter(None, None, 1, 1, alpha, None, 1, None),
        "rfd_fm_apply": lambda: rfd.lib.rfd_fm_apply(None, None, 1, 1, None, 1),
        "rfd_gw_tensor_product": lambda: rfd.lib.rfd_gw_tensor_product(None, None, None, None, None, None),
        "rfd_gw_line_search": lambda: rfd.lib.rfd_gw_line_search(None, None, 0.5, None, None, None, None, None, out3),
        "rfd_eigenvalues": lambda: rfd.lib.rfd_eigenvalues(None, 4, 0, None),
        "rfd_batch_eigenvalues": lambda: rfd.lib.rfd_batch_eigenvalues(None, None, 4, 0, None),
        "rfd_debug_plan_phi1": lambda: rfd.lib.rfd_debug_plan_phi1(None, None),
        "rfd_debug_plan_set_phase": lambda: rfd.lib.rfd_debug_plan_set_phase(None, 64),
        "rfd_debug_plan_set_overlap": lambda: rfd.lib.rfd_debug_plan_set_overlap(None, 1),
        "rfd_debug_plan_set_apply_tc": lambda: rfd.lib.rfd_debug_plan_set_apply_tc(None, 1),
        "rfd_debug_plan_wait_timeout": lambda: rfd.lib.rfd_debug_plan_wait_timeout(None, 1000),
    }
    for name, call in calls.items():
        assert call() == rfd.RFD_EINVAL, name
        assert rfd.rfd_last_error(), name


def test_phi1_gemm_count_matches_bench_model():
    import bench
    for q, s, m in [(3, 0, 8), (7, 0, 64), (9, 0, 10), (13, 0, 100), (13, 4, 32)]:
        gem = {3: 1, 5: 2, 7: 3, 9: 4, 13: 5}[q] + 1 + (2 * s - 1 if s else 0)
        nrhs = 2 * m if s else m
        assert bench.phi1_flops(m, q, s) == pytest.approx(gem * 2 * m ** 3 + 2 / 3 * m ** 3 + 2 * m * m * nrhs)


def test_bench_work_model_at_the_headline():
    """The algorithmic work the roofline is computed from, at N = 1e6, m = 1024,
    c = 3: T = N m (m + 1) + 4 N m c flops (symmetric Gram, Phi^T F, Phi Z) and
    12 N (1 + c) HBM bytes (points, F read twice, out)."""
    import bench
    w = bench.work_model(1_000_000, 1024, 3)
    assert w["gram_flops"] + w["apply_flops"] == 1_000_000 * 1024 * 1025 + 4 * 1_000_000 * 1024 * 3
    assert abs((w["gram_flops"] + w["apply_flops"]) - 1.062e12) < 0.001e12
    assert w["hbm_bytes"] == 48_000_000
    assert w["sincos"] == 1_024_000_000
