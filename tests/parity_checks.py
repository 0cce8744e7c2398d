"""Element-wise comparison of a GPU result with the FP64 oracle's (test helper).

The output of the method is out = F + increment, increment = A (G (B^T F))
(Sec. 2.4).  F passes through unchanged, so a whole-output bound alone says
little when the increment is small (at the large workload it is 0.3 % of
||F||).  Every GPU parity check therefore asserts three things on the same
seeded inputs:

  1. the whole output:  ||out - ref||_F / ||ref||_F               <= TOL_OUT
  2. the increment:     ||(out - F) - (ref - F)||_F / ||ref - F||_F <= TOL_INC
  3. every row:         max_i ||out_i - ref_i||_2 <= TOL_ROW * max_i ||ref_i - F_i||_2

Bounds per form (derivation: the design notes, "Precision of the BF16 form"):

  FP32 plain form.  Phi in FP32 (phase error ~|w^T x| 2^-24 cycles), compensated
  FP32 reductions, FP64 G, FP32 apply: the increment carries relative error of
  order sqrt(m) 2^-24 ~ 1e-6 .. 1e-5 from the apply's sum over m columns;
  TOL_INC = 1e-4, TOL_OUT = 1e-5 (the stated tolerance of the form).
  BF16 tensor-core form.  Phi is rounded to BF16 (relative 2^-9 per entry)
  inside B^T F, and F is zero-mean, so that rounding does not average away:
  Y = B^T F, and with it the increment, carries relative error ~2^-9 ~ 2e-3;
  TOL_INC = 2e-2 (ten times that), TOL_OUT = 1e-3 (the stated tolerance of
  the form; met while the relative increment stays below ~0.5).
TOL_ROW equals TOL_INC: a row's error is a projection of the same coefficient
error, so a tail (the last partial 64-point block, the last tile of a ragged
m) that went wrong shows up here even when the norms hide it.
"""
from __future__ import annotations

import numpy as np

FP32_PLAIN, BF16_TC = 0, 1
TOL_OUT = {FP32_PLAIN: 1e-5, BF16_TC: 1e-3}
TOL_INC = {FP32_PLAIN: 1e-4, BF16_TC: 2e-2}
TOL_ROW = TOL_INC


def errors(out, ref, F) -> dict:
    """Whole-output, increment and per-row errors of out against ref (both N x c)."""
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    d = out - ref
    inc = ref - F
    inc_norm = float(np.linalg.norm(inc))
    row_err = np.sqrt((d * d).sum(axis=1))
    row_inc = np.sqrt((inc * inc).sum(axis=1))
    return {
        "out": float(np.linalg.norm(d) / np.linalg.norm(ref)),
        "inc": float(np.linalg.norm(d) / inc_norm) if inc_norm > 0 else float(np.linalg.norm(d)),
        "row": float(row_err.max() / row_inc.max()) if row_inc.max() > 0 else float(row_err.max()),
        "worst_row": int(row_err.argmax()) if row_err.size else -1,
        "relative_increment": inc_norm / float(np.linalg.norm(F)) if np.linalg.norm(F) > 0 else 0.0,
    }


def assert_matches(out, ref, F, prec, *, label="", tol_out=None, tol_inc=None, tol_row=None) -> dict:
    """Assert the three bounds for precision `prec` (0: FP32 plain, 1: BF16 tensor core)."""
    e = errors(out, ref, F)
    to = TOL_OUT[prec] if tol_out is None else tol_out
    ti = TOL_INC[prec] if tol_inc is None else tol_inc
    tr = TOL_ROW[prec] if tol_row is None else tol_row
    print(f"{label} prec={prec}: out {e['out']:.3e} (<= {to:g}), increment {e['inc']:.3e} (<= {ti:g}), "
          f"row {e['row']:.3e} (<= {tr:g}; worst row {e['worst_row']}), relative increment "
          f"{e['relative_increment']:.3e}")
    assert np.isfinite(np.asarray(out, dtype=np.float64)).all(), f"{label}: non-finite output"
    assert e["out"] <= to, (label, "out", e)
    assert e["inc"] <= ti, (label, "increment", e)
    assert e["row"] <= tr, (label, "row", e)
    return e
