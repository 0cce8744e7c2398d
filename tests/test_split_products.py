"""The arithmetic of the tensor-core apply and of the tensor-core B^T F (CPU).

Both kernels split each FP32 operand value v into BF16 parts hi = bf16(v) and
lo = bf16(v - hi) (round to nearest even) and form a product x z as
x_hi z_hi + x_hi z_lo + x_lo z_hi, dropping x_lo z_lo.  With u = 2^-8 the unit
roundoff of BF16 (8 significant bits): |v - hi| <= u |v| and |v - hi - lo| <=
u |v - hi| <= u^2 |v|, so each of the two representation errors and the
dropped term is at most u^2 |x z|, and a product keeps a relative error of at
most 3 u^2 = 3 x 2^-16 (plus the FP32 accumulation, not modelled here).  The
GPU tests compare those kernels with the FP32 SIMT kernels at 2e-4 of the
increment, which is this bound with the margin of the FP32 sums over m terms.

Here the bound is checked on BF16 rounding written out bit by bit, and
planted mistakes (a dropped cross term, truncation instead of rounding for
hi) are shown to break it.
"""
import numpy as np

U2 = 2.0 ** -16


def bf16_rn(x):
    """FP32 -> nearest BF16 (ties to even), returned as FP32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def bf16_trunc(x):
    b = np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    return b.view(np.float32)


def split(v, hi_round=bf16_rn):
    v = np.asarray(v, np.float32)
    hi = hi_round(v)
    lo = bf16_rn((v - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def three_products(x, z, *, drop=None, hi_round=bf16_rn):
    xh, xl = split(x, hi_round)
    zh, zl = split(z, hi_round)
    terms = {"hh": xh * zh, "hl": xh * zl, "lh": xl * zh}
    if drop:
        terms.pop(drop)
    return sum(terms.values())


def _operands(n, seed):
    rng = np.random.default_rng(seed)
    # Phi values in [-1, 1] (cos / sin), Z or F values of several magnitudes
    x = np.cos(rng.uniform(0, 2 * np.pi, n)).astype(np.float32)
    z = (rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))).astype(np.float32)
    return x, z


def test_bf16_rounding_is_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even significand (1)
    assert bf16_rn(np.float32(1 + 2 ** -8)) == 1.0
    assert bf16_rn(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    assert bf16_rn(np.float32(1 + 2 ** -8 + 2 ** -20)) == np.float32(1 + 2 ** -7)
    v = np.float32(np.pi)
    assert abs(float(bf16_rn(v)) - float(v)) <= 2 ** -8 * abs(float(v))


def test_split_represents_to_two_bf16_unit_roundoffs():
    x, _ = _operands(200000, 1)
    hi, lo = split(x)
    err = np.abs(hi + lo - x.astype(np.float64))
    assert (err <= U2 * np.abs(x)).all()
    assert (np.abs(lo) <= 2 ** -8 * np.abs(x)).all()


def test_three_products_within_three_u_squared():
    x, z = _operands(200000, 2)
    exact = x.astype(np.float64) * z.astype(np.float64)
    p = three_products(x, z)
    rel = np.abs(p - exact) / np.abs(exact)
    assert rel.max() <= 3 * U2, rel.max()
    # a dot product over m = 1024 terms: relative to the sum of magnitudes
    xs, zs = x[: 1024 * 150].reshape(150, 1024), z[: 1024 * 150].reshape(150, 1024)
    d_exact = (xs.astype(np.float64) * zs).sum(axis=1)
    d = three_products(xs, zs).sum(axis=1)
    mag = (np.abs(xs.astype(np.float64) * zs)).sum(axis=1)
    assert (np.abs(d - d_exact) <= 3 * U2 * mag).all()


def test_planted_mistakes_break_the_bound():
    x, z = _operands(200000, 3)
    exact = x.astype(np.float64) * z.astype(np.float64)
    for drop in ("hl", "lh"):  # a dropped cross term: the error of one BF16 rounding, ~2^-9
        rel = np.abs(three_products(x, z, drop=drop) - exact) / np.abs(exact)
        assert rel.max() > 3 * U2 * 10, (drop, rel.max())
    # hi by truncation: lo can reach 2^-7 |v| and its own rounding then exceeds the bound
    rel = np.abs(three_products(x, z, hi_round=bf16_trunc) - exact) / np.abs(exact)
    assert rel.max() > 3 * U2, rel.max()
