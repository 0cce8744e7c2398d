"""GB300-native RFDiffusion (RFD) graph-field integrator (arXiv 2302.00942, Sec. 2.4).

Thin Python binding of the C ABI in include/rfd.h: argument marshalling only.
Every step of the integrator runs in the CUDA kernels of librfd_gb300.so; this
module never computes any of it.  Importing it loads the library and raises
if it is missing (build it with ``python -m paper_2302_00942_gb300.build``):
there is no CPU fallback.

Device buffers are passed as torch CUDA tensors (PyTorch is used for device
memory and streams only) or as raw integer device pointers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "RFD_OK", "RFD_EINVAL", "RFD_ENOMEM", "RFD_ECUDA", "RFD_ENOTREADY", "RFD_ETIMEDOUT", "RFD_ENUMERIC",
    "RFD_EBUSY", "RFD_ENOTSUP", "RFD_FP32_PLAIN", "RFD_BF16_TC", "RfdError", "rfd_params", "rfd_stats",
    "lib", "lib_path", "gw_tensor_product", "gw_line_search", "rfd_sample_frequencies", "rfd_sample_weights", "RFD_KERNEL_CUBE", "RFD_KERNEL_BALL", "rfd_plan", "rfd_plan_destroy", "rfd_features",
    "rfd_integrate", "rfd_gfi", "rfd_phi1", "rfd_sync", "rfd_plan_export", "rfd_plan_stats", "rfd_plan_stats_reset", "rfd_last_error",
    "rfd_version", "RFD_FLAG_TIMING", "STEP_NAMES", "rfd_debug_fail_alloc_after", "rfd_debug_dgemm", "Plan", "Batch", "rfd_batch_item", "HEADER_SYMBOLS",
    "RFD_FLAG_NATIVE_FP64", "RFD_FLAG_GRAPH", "RFD_FLAG_AUTOTUNE", "Server", "rfd_request", "rfd_result", "rfd_server_config",
    "rfd_server_stats",
]

RFD_OK, RFD_EINVAL, RFD_ENOMEM, RFD_ECUDA, RFD_ENOTREADY, RFD_ETIMEDOUT, RFD_ENUMERIC, RFD_EBUSY, RFD_ENOTSUP = range(9)
RFD_FP32_PLAIN, RFD_BF16_TC = 0, 1
_STATUS = {0: "RFD_OK", 1: "RFD_EINVAL", 2: "RFD_ENOMEM", 3: "RFD_ECUDA", 4: "RFD_ENOTREADY",
           5: "RFD_ETIMEDOUT", 6: "RFD_ENUMERIC", 7: "RFD_EBUSY", 8: "RFD_ENOTSUP"}

lib_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "librfd_gb300.so")


class rfd_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int32), ("max_channels", ctypes.c_int32),
                ("eps", ctypes.c_double), ("lambda_", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32), ("freq_sigma", ctypes.c_double),
                ("freq_radius", ctypes.c_double), ("kernel", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


RFD_KERNEL_CUBE, RFD_KERNEL_BALL, RFD_KERNEL_CUBE_L1, RFD_KERNEL_L1_BALL = 0, 1, 2, 3  # rfd_kernel: the eps-NN threshold function
KERNELS = {"cube": RFD_KERNEL_CUBE, "ball": RFD_KERNEL_BALL, "cube_l1": RFD_KERNEL_CUBE_L1,
           "l1_ball": RFD_KERNEL_L1_BALL}


RFD_FLAG_TIMING = 1
RFD_FLAG_NATIVE_FP64 = 2
RFD_FLAG_GRAPH = 4
RFD_FLAG_AUTOTUNE = 8
STEP_NAMES = ("features", "field", "gram", "reduce", "phi1", "small", "apply", "eigen")


class rfd_stats(ctypes.Structure):
    _fields_ = [("norm1", ctypes.c_double), ("pade_degree", ctypes.c_int32), ("squarings", ctypes.c_int32),
                ("nonfinite", ctypes.c_int32), ("splits", ctypes.c_int32), ("phi1_emulated", ctypes.c_int32),
                ("phi1_gemms", ctypes.c_int32), ("step_ms", ctypes.c_double * len(STEP_NAMES)), ("timed_calls", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("tune_lanes_pct", ctypes.c_int32), ("tune_waves", ctypes.c_int32),
                ("tune_phase_blocks", ctypes.c_int32), ("tuned", ctypes.c_int32), ("tune_pair_gram", ctypes.c_int32),
                ("tune_overlap", ctypes.c_int32), ("tune_form_ms", ctypes.c_double * 2)]


class rfd_batch_item(ctypes.Structure):
    _fields_ = [("d_points", ctypes.c_void_p), ("d_F", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("c", ctypes.c_int32), ("reserved_", ctypes.c_int32), ("ldF", ctypes.c_int64),
                ("ldOut", ctypes.c_int64)]


class rfd_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_queue", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("executors", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class rfd_request(ctypes.Structure):
    _fields_ = [("d_points", ctypes.c_void_p), ("d_F", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("ldF", ctypes.c_int64), ("ldOut", ctypes.c_int64), ("m", ctypes.c_int32),
                ("c", ctypes.c_int32), ("eps", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("cloud", ctypes.c_uint64), ("keep", ctypes.c_int32),
                ("max_channels", ctypes.c_int32)]


class rfd_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reused", ctypes.c_int32), ("cloud", ctypes.c_uint64),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("batch_size", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]


class rfd_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "rejected", "batches", "reused", "evicted",
                                               "resident", "mem_used", "mem_peak", "mem_budget", "kernel_launches")]


def _stats_dict(s: "rfd_stats") -> dict:
    d = {k: getattr(s, k) for k, _ in rfd_stats._fields_ if k not in ("step_ms", "tune_form_ms")}
    d["step_ms"] = dict(zip(STEP_NAMES, list(s.step_ms)))
    d["tune_form_ms"] = list(s.tune_form_ms)
    return d


class RfdError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(lib_path):
        raise ImportError(f"{lib_path} is missing: build it with `python -m paper_2302_00942_gb300.build` "
                          "(this package has no CPU fallback)")
    L = ctypes.CDLL(lib_path)
    P, D, I32, I64, U64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "rfd_sample_frequencies": (I32, [I32, D, U64, D, D, DP, DP]),
        "rfd_sample_weights": (I32, [I32, D, U64, D, D, I32, DP, DP]),
        "rfd_barycenter": (I32, [P, P, I32, I64, DP, P, I32, P]),
        "rfd_fm_apply": (I32, [P, P, I64, I64, P, I64]),
        "rfd_gw_tensor_product": (I32, [P, P, P, P, P, P]),
        "rfd_gw_line_search": (I32, [P, P, D, P, P, P, P, P, DP]),
        "rfd_eigenvalues": (I32, [P, I32, I32, P]),
        "rfd_plan": (I32, [ctypes.POINTER(rfd_params), P, ctypes.POINTER(P)]),
        "rfd_plan_destroy": (I32, [P]),
        "rfd_features": (I32, [P, P]),
        "rfd_integrate": (I32, [P, P, I32, I64, P, I64]),
        "rfd_gfi": (I32, [P, P, P, I32, I64, P, I64]),
        "rfd_sync": (I32, [P]),
        "rfd_phi1": (I32, [I32, D, P, P, I32, P, ctypes.POINTER(rfd_stats)]),
        "rfd_phi1_noalloc": (I32, [I32, D, P, P, I32, P, ctypes.POINTER(rfd_stats)]),
        "rfd_plan_export": (I32, [P, DP, DP, DP]),
        "rfd_plan_stats": (I32, [P, ctypes.POINTER(rfd_stats)]),
        "rfd_plan_stats_reset": (I32, [P]),
        "rfd_plan_compact": (I32, [P]),
        "rfd_plan_device_bytes": (I32, [P, ctypes.POINTER(I64)]),
        "rfd_last_error": (ctypes.c_char_p, []),
        "rfd_version": (ctypes.c_char_p, []),
        "rfd_debug_fail_alloc_after": (None, [I32]),
        "rfd_debug_dgemm": (I32, [I32, I32, I32, I32, D, P, I32, P, I32, D, P, I32, P]),
        "rfd_debug_plan_phi1": (I32, [P, P]),
        "rfd_debug_plan_set_phase": (I32, [P, I32]),
        "rfd_debug_plan_set_overlap": (I32, [P, I32]),
        "rfd_debug_plan_set_apply_tc": (I32, [P, I32]),
        "rfd_debug_gram_pairs": (None, [I32]),
        "rfd_debug_plan_wait_timeout": (I32, [P, I32]),
        "rfd_batch_create": (I32, [ctypes.POINTER(P), I32, I32, P, ctypes.POINTER(P)]),
        "rfd_batch_destroy": (I32, [P]),
        "rfd_batch_features": (I32, [P, ctypes.POINTER(rfd_batch_item)]),
        "rfd_batch_integrate": (I32, [P, ctypes.POINTER(rfd_batch_item)]),
        "rfd_batch_gfi": (I32, [P, ctypes.POINTER(rfd_batch_item)]),
        "rfd_batch_eigenvalues": (I32, [P, ctypes.POINTER(rfd_batch_item), I32, I32, P]),
        "rfd_batch_sync": (I32, [P]),
        "rfd_batch_stats": (I32, [P, ctypes.POINTER(rfd_stats)]),
        "rfd_batch_stats_reset": (I32, [P]),
        "rfd_server_create": (I32, [ctypes.c_size_t, ctypes.POINTER(rfd_server_config), ctypes.POINTER(P)]),
        "rfd_server_destroy": (I32, [P]),
        "rfd_submit": (I32, [P, ctypes.POINTER(rfd_request), ctypes.POINTER(U64)]),
        "rfd_poll": (I32, [P, U64, I32, ctypes.POINTER(rfd_result)]),
        "rfd_server_stats_get": (I32, [P, ctypes.POINTER(rfd_server_stats)]),
        "rfd_debug_server_pause": (None, [P, I32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype, fn.argtypes = res, args
    return L


lib = _load()

# Every function include/rfd.h and include/rfd_testing.h declare (checked against the headers by a test).
HEADER_SYMBOLS = ("rfd_sample_frequencies", "rfd_sample_weights", "rfd_barycenter", "rfd_fm_apply",
                  "rfd_gw_tensor_product", "rfd_gw_line_search", "rfd_eigenvalues", "rfd_batch_eigenvalues", "rfd_plan", "rfd_plan_destroy", "rfd_features", "rfd_integrate",
                  "rfd_gfi", "rfd_phi1", "rfd_phi1_noalloc", "rfd_sync", "rfd_plan_export", "rfd_plan_stats", "rfd_plan_stats_reset", "rfd_plan_compact",
                  "rfd_plan_device_bytes", "rfd_last_error",
                  "rfd_version", "rfd_debug_fail_alloc_after", "rfd_debug_dgemm", "rfd_debug_plan_phi1", "rfd_debug_plan_set_phase", "rfd_debug_plan_set_overlap",
                  "rfd_debug_plan_set_apply_tc",
                  "rfd_debug_plan_wait_timeout", "rfd_debug_gram_pairs", "rfd_batch_create",
                  "rfd_batch_destroy", "rfd_batch_features", "rfd_batch_integrate", "rfd_batch_gfi",
                  "rfd_batch_sync", "rfd_batch_stats", "rfd_batch_stats_reset", "rfd_server_create",
                  "rfd_server_destroy", "rfd_submit", "rfd_poll", "rfd_server_stats_get", "rfd_debug_server_pause")


def rfd_last_error() -> str:
    return lib.rfd_last_error().decode()


def rfd_version() -> str:
    return lib.rfd_version().decode()


def _check(st: int, where: str) -> None:
    if st != RFD_OK:
        raise RfdError(st, where, rfd_last_error())


def _dptr(x) -> int:
    """Device pointer of a CUDA tensor (or an int pointer)."""
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return x.data_ptr()


def rfd_sample_frequencies(m: int, eps: float, seed: int, freq_sigma: float = 0.0, freq_radius: float = 0.0):
    """Step a1 on the host: (omega (m/2, 3) float64, r (m/2,) float64)."""
    om = np.zeros((m // 2, 3), dtype=np.float64)
    r = np.zeros(m // 2, dtype=np.float64)
    _check(lib.rfd_sample_frequencies(m, eps, seed, freq_sigma, freq_radius,
                                      om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "rfd_sample_frequencies")
    return om, r


def rfd_sample_weights(m: int, eps: float, seed: int, freq_sigma: float = 0.0, freq_radius: float = 0.0,
                       kernel: str = "cube"):
    """Step a1 for the threshold function `kernel` ("cube" or "ball"): (omega, r)."""
    om = np.zeros((m // 2, 3), dtype=np.float64)
    r = np.zeros(m // 2, dtype=np.float64)
    _check(lib.rfd_sample_weights(m, eps, seed, freq_sigma, freq_radius, KERNELS[kernel],
                                  om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "rfd_sample_weights")
    return om, r


def rfd_plan(n, m, eps, lam, seed=0, max_channels=3, precision=RFD_BF16_TC, stream=None, freq_sigma=0.0,
             freq_radius=0.0, flags=0, kernel="cube") -> int:
    p = rfd_params(n=n, m=m, max_channels=max_channels, eps=eps, lambda_=lam, seed=seed, precision=precision,
                   flags=flags, freq_sigma=freq_sigma, freq_radius=freq_radius, kernel=KERNELS[kernel])
    h = ctypes.c_void_p()
    _check(lib.rfd_plan(ctypes.byref(p), stream, ctypes.byref(h)), "rfd_plan")
    return h.value


def rfd_plan_destroy(plan: int) -> None:
    _check(lib.rfd_plan_destroy(plan), "rfd_plan_destroy")


def rfd_features(plan: int, points) -> None:
    _check(lib.rfd_features(plan, _dptr(points)), "rfd_features")


def rfd_integrate(plan: int, F, c: int, ldF: int, out, ldOut: int) -> None:
    _check(lib.rfd_integrate(plan, _dptr(F), c, ldF, _dptr(out), ldOut), "rfd_integrate")


def rfd_gfi(plan: int, points, F, c: int, ldF: int, out, ldOut: int) -> None:
    _check(lib.rfd_gfi(plan, _dptr(points), _dptr(F), c, ldF, _dptr(out), ldOut), "rfd_gfi")


def rfd_sync(plan: int) -> None:
    _check(lib.rfd_sync(plan), "rfd_sync")


def rfd_phi1(m: int, lam: float, M, G, stream=None, native_fp64: bool = False) -> dict:
    """G = lam * phi1(lam * M) for float64 CUDA tensors M, G (m x m)."""
    s = rfd_stats()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    flags = RFD_FLAG_NATIVE_FP64 if native_fp64 else 0
    _check(lib.rfd_phi1(m, lam, _dptr(M), _dptr(G), flags, st, ctypes.byref(s)), "rfd_phi1")
    return _stats_dict(s)


def rfd_phi1_noalloc(m: int, lam: float, M, G, stream=None, native_fp64: bool = False) -> dict:
    """rfd_phi1 for callers that cannot allocate device memory (m <= 128; the
    workspace is a fixed device array shared by all calls -- serialise them)."""
    s = rfd_stats()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    flags = RFD_FLAG_NATIVE_FP64 if native_fp64 else 0
    _check(lib.rfd_phi1_noalloc(m, lam, _dptr(M), _dptr(G), flags, st, ctypes.byref(s)), "rfd_phi1_noalloc")
    return _stats_dict(s)


def rfd_plan_export(plan: int, m: int, with_G: bool = True):
    om = np.zeros((m // 2, 3)), np.zeros(m // 2)
    G = np.zeros((m, m)) if with_G else None
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.rfd_plan_export(plan, om[0].ctypes.data_as(dp), om[1].ctypes.data_as(dp),
                               G.ctypes.data_as(dp) if G is not None else None), "rfd_plan_export")
    return om[0], om[1], G


def rfd_plan_stats(plan: int) -> dict:
    s = rfd_stats()
    _check(lib.rfd_plan_stats(plan, ctypes.byref(s)), "rfd_plan_stats")
    return _stats_dict(s)


def rfd_plan_stats_reset(plan: int) -> None:
    _check(lib.rfd_plan_stats_reset(plan), "rfd_plan_stats_reset")


def rfd_debug_fail_alloc_after(k: int) -> None:
    lib.rfd_debug_fail_alloc_after(k)


def rfd_debug_gram_pairs(enable: bool) -> None:
    """Plans created from now on may (True, the default) or may not run their Gram on CTA pairs."""
    lib.rfd_debug_gram_pairs(1 if enable else 0)


def rfd_debug_dgemm(method: int, A, B, C, alpha=1.0, beta=0.0, stream=None) -> None:
    """C = alpha A B + beta C on float64 CUDA tensors (method 0 native FP64, 1 emulated)."""
    M, K = A.shape
    N = B.shape[1]
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(lib.rfd_debug_dgemm(method, M, N, K, alpha, _dptr(A), A.stride(0), _dptr(B), B.stride(0), beta,
                               _dptr(C), C.stride(0), st), "rfd_debug_dgemm")


class Plan:
    """Owning wrapper of an rfd_plan_t (one point cloud's integrator).

    All tensors are torch CUDA float32, contiguous: points (N, 3), F and out (N, c).
    """

    def __init__(self, n, m, eps, lam, seed=0, max_channels=3, precision=RFD_BF16_TC, stream=None,
                 freq_sigma=0.0, freq_radius=0.0, timing=False, native_fp64=False, autotune=False, kernel="cube",
                 graph=False):
        self.n, self.m, self.max_channels = int(n), int(m), int(max_channels)
        self.handle = None
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self.handle = rfd_plan(n, m, eps, lam, seed, max_channels, precision, s, freq_sigma, freq_radius,
                               (RFD_FLAG_TIMING if timing else 0) | (RFD_FLAG_NATIVE_FP64 if native_fp64 else 0) |
                               (RFD_FLAG_AUTOTUNE if autotune else 0) | (RFD_FLAG_GRAPH if graph else 0), kernel)

    @staticmethod
    def _chk(t, shape_last=None):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
            raise TypeError("expected a float32 CUDA tensor")
        if t.dim() != 2 or t.stride(1) != 1:
            raise ValueError("expected a 2-D row-major tensor")
        return t

    def features(self, points):
        self._chk(points)
        rfd_features(self.handle, points)

    def integrate(self, F, out=None):
        import torch
        self._chk(F)
        out = torch.empty_like(F) if out is None else self._chk(out)
        rfd_integrate(self.handle, F, F.shape[1], F.stride(0), out, out.stride(0))
        return out

    def barycenter(self, mu, area, alpha, iters, out=None):
        """Entropic Wasserstein barycenter of the columns of mu (N x k) on the
        resident plan (rfd_barycenter): returns the N-vector barycenter."""
        import torch
        self._chk(mu)
        if not (isinstance(area, torch.Tensor) and area.is_cuda and area.dtype == torch.float32 and area.dim() == 1
                and area.is_contiguous()):
            raise TypeError("area must be a contiguous float32 CUDA vector")
        k = mu.shape[1]
        al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(k))
        out = torch.empty(mu.shape[0], dtype=torch.float32, device=mu.device) if out is None else out
        _check(lib.rfd_barycenter(self.handle, mu.data_ptr(), k, mu.stride(0),
                                  al.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), area.data_ptr(), int(iters),
                                  out.data_ptr()), "rfd_barycenter")
        return out

    def fm_apply(self, X, out=None):
        """Y = exp(lambda W_hat) X for an N x k float32 CUDA matrix (any k; rfd_fm_apply)."""
        import torch
        self._chk(X)
        out = torch.empty_like(X) if out is None else self._chk(out)
        _check(lib.rfd_fm_apply(self.handle, X.data_ptr(), X.shape[1], X.stride(0), out.data_ptr(), out.stride(0)),
               "rfd_fm_apply")
        return out

    def eigenvalues(self, k, largest=False, out=None):
        """The k smallest (ascending) or largest (descending) eigenvalues of
        exp(lambda W_hat) from the resident M (rfd_eigenvalues): float32 CUDA (k,)."""
        import torch
        out = torch.empty(int(k), dtype=torch.float32, device="cuda") if out is None else out
        _check(lib.rfd_eigenvalues(self.handle, int(k), 1 if largest else 0, out.data_ptr()), "rfd_eigenvalues")
        return out

    def gfi(self, points, F, out=None):
        import torch
        self._chk(points)
        self._chk(F)
        out = torch.empty_like(F) if out is None else self._chk(out)
        rfd_gfi(self.handle, points, F, F.shape[1], F.stride(0), out, out.stride(0))
        return out

    def sync(self):
        rfd_sync(self.handle)

    def export(self, with_G=True):
        return rfd_plan_export(self.handle, self.m, with_G)

    def stats(self):
        return rfd_plan_stats(self.handle)

    def stats_reset(self):
        rfd_plan_stats_reset(self.handle)

    def compact(self):
        """Release Phi, the partials and the phi1 workspace (rfd_plan_compact)."""
        _check(lib.rfd_plan_compact(self.handle), "rfd_plan_compact")

    def device_bytes(self) -> int:
        v = ctypes.c_int64(0)
        _check(lib.rfd_plan_device_bytes(self.handle, ctypes.byref(v)), "rfd_plan_device_bytes")
        return v.value

    def close(self):
        if self.handle:
            rfd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many BF16 plans integrated by shared launches (include/rfd.h, batches).

    items: a list with one dict per plan: {"points": (N, 3) tensor, "F": (N, c)
    tensor, "out": (N, c) tensor or None}; all float32 CUDA, row-major.
    """

    def __init__(self, plans, stream=None, timing=False, graph=False, autotune=False):
        self.plans = list(plans)
        self.handle = None
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = ctypes.c_void_p()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        flags = (RFD_FLAG_TIMING if timing else 0) | (RFD_FLAG_GRAPH if graph else 0) | (RFD_FLAG_AUTOTUNE if autotune else 0)
        _check(lib.rfd_batch_create(arr, len(self.plans), flags, s, ctypes.byref(h)), "rfd_batch_create")
        self.handle = h.value

    def _items(self, items, need_f):
        arr = (rfd_batch_item * len(self.plans))()
        outs = []
        for k, it in enumerate(items):
            P = it.get("points")
            F = it.get("F")
            arr[k].d_points = _dptr(P) if P is not None else None
            if need_f:
                import torch
                out = it.get("out")
                if out is None:
                    out = torch.empty_like(F)
                arr[k].d_F, arr[k].d_out = _dptr(F), _dptr(out)
                arr[k].c, arr[k].ldF, arr[k].ldOut = F.shape[1], F.stride(0), out.stride(0)
                outs.append(out)
            else:
                arr[k].c, arr[k].ldF, arr[k].ldOut = 1, 1, 1
        return arr, outs

    def gfi(self, items):
        arr, outs = self._items(items, True)
        _check(lib.rfd_batch_gfi(self.handle, arr), "rfd_batch_gfi")
        return outs

    def features(self, items):
        arr, _ = self._items(items, False)
        _check(lib.rfd_batch_features(self.handle, arr), "rfd_batch_features")

    def integrate(self, items):
        arr, outs = self._items(items, True)
        _check(lib.rfd_batch_integrate(self.handle, arr), "rfd_batch_integrate")
        return outs

    def eigenvalues(self, items, k, largest=False, out=None):
        """Steps a2-a3 from items[i]["points"], then every cloud's k smallest /
        largest kernel eigenvalues (rfd_batch_eigenvalues): float32 CUDA (count, k)."""
        import torch
        arr, _ = self._items(items, False)
        if out is None:
            out = torch.empty((len(self.plans), int(k)), dtype=torch.float32, device=items[0]["points"].device)
        _check(lib.rfd_batch_eigenvalues(self.handle, arr, int(k), 1 if largest else 0, out.data_ptr()),
               "rfd_batch_eigenvalues")
        return out

    def sync(self):
        _check(lib.rfd_batch_sync(self.handle), "rfd_batch_sync")

    def stats(self):
        st = rfd_stats()
        _check(lib.rfd_batch_stats(self.handle, ctypes.byref(st)), "rfd_batch_stats")
        return _stats_dict(st)

    def stats_reset(self):
        _check(lib.rfd_batch_stats_reset(self.handle), "rfd_batch_stats_reset")

    def close(self):
        if self.handle:
            _check(lib.rfd_batch_destroy(self.handle), "rfd_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning wrapper of an rfd_server_t (the GFI request loop, include/rfd.h).

    submit() takes float32 CUDA tensors (points (N, 3), F and out (N, c)) that
    must stay alive until poll() reports the ticket; it returns the ticket.
    poll() returns (status, result dict or None).
    """

    def __init__(self, mem_budget, max_queue=0, max_batch=0, executors=0):
        self.handle = None
        cfg = rfd_server_config(mem_budget=int(mem_budget), max_queue=max_queue, max_batch=max_batch,
                                executors=executors)
        h = ctypes.c_void_p()
        _check(lib.rfd_server_create(int(mem_budget), ctypes.byref(cfg), ctypes.byref(h)), "rfd_server_create")
        self.handle = h.value

    def submit(self, F, out, points=None, m=0, eps=0.0, lam=0.0, seed=0, cloud=0, keep=False, max_channels=0,
               n=None):
        r = rfd_request(d_points=_dptr(points) if points is not None else None, d_F=_dptr(F), d_out=_dptr(out),
                        n=int(F.shape[0] if n is None else n), ldF=F.stride(0), ldOut=out.stride(0), m=m,
                        c=F.shape[1], eps=eps, lambda_=lam, seed=seed, cloud=cloud, keep=1 if keep else 0,
                        max_channels=max_channels)
        t = ctypes.c_uint64()
        _check(lib.rfd_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "rfd_submit")
        return t.value

    def try_submit(self, *args, **kw):
        """submit(), but returns (status, ticket or None) instead of raising."""
        try:
            return RFD_OK, self.submit(*args, **kw)
        except RfdError as e:
            return e.status, None

    def poll(self, ticket, timeout_us=0):
        res = rfd_result()
        st = lib.rfd_poll(self.handle, ticket, int(timeout_us), ctypes.byref(res))
        if st != RFD_OK:
            return st, None
        return st, {k: getattr(res, k) for k, _ in rfd_result._fields_ if k != "reserved_"}

    def stats(self):
        s = rfd_server_stats()
        _check(lib.rfd_server_stats_get(self.handle, ctypes.byref(s)), "rfd_server_stats_get")
        return {k: getattr(s, k) for k, _ in rfd_server_stats._fields_}

    def pause(self, paused=True):
        lib.rfd_debug_server_pause(self.handle, 1 if paused else 0)

    def close(self):
        if self.handle:
            _check(lib.rfd_server_destroy(self.handle), "rfd_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gw_tensor_product(plan_C, plan_D, T, p, q, out=None):
    """Algorithm tensor_prod (App. C.2) on two resident plans: L = (C^2 p) 1^T + 1 (D^2 q)^T - 2 C T D^T."""
    import torch
    out = torch.empty_like(T) if out is None else out
    for t in (T, p, q, out):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError("expected contiguous float32 CUDA tensors")
    _check(lib.rfd_gw_tensor_product(plan_C.handle, plan_D.handle, T.data_ptr(), p.data_ptr(), q.data_ptr(),
                                     out.data_ptr()), "rfd_gw_tensor_product")
    return out


def gw_line_search(plan_C, plan_D, alpha, G, dG, M, p, q):
    """Algorithm line_search (App. C.2) on two resident plans: (tau, a, b)."""
    import torch
    for t in (G, dG, M, p, q):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError("expected contiguous float32 CUDA tensors")
    res = np.zeros(3, dtype=np.float64)
    _check(lib.rfd_gw_line_search(plan_C.handle, plan_D.handle, float(alpha), G.data_ptr(), dG.data_ptr(),
                                  M.data_ptr(), p.data_ptr(), q.data_ptr(),
                                  res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "rfd_gw_line_search")
    return float(res[0]), float(res[1]), float(res[2])
