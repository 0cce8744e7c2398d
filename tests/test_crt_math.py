"""Host-side pins of the integer arithmetic of the modular FP64 emulation
(paper_2302_00942_gb300/csrc/crt_math.h, shared with the step-a4 kernels):
the header is compiled as plain C++ and checked against Python integers and
exact rationals -- residues, the Chinese-remainder reconstruction, the choice
of integer width for a contraction length, the integer extraction of FP64
entries and the correctly rounded conversion back to FP64."""
import ctypes
import pathlib
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HEADER = pathlib.Path(__file__).resolve().parents[1] / "paper_2302_00942_gb300" / "csrc" / "crt_math.h"
MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 211, 199, 197, 193, 191]

SHIM = r"""
#include "crt_math.h"
using namespace rfd::crt;
static Constants g;
static bool ok = make_constants(&g);
template <int j> void res_all(const Limbs& L, long long X, float* r) {
  r[j] = residue<j>(L, X);
  if constexpr (j + 1 < kNumMod) res_all<j + 1>(L, X, r);
}
extern "C" {
int c_ok() { return ok; }
unsigned c_modulus(int j) { return modulus(j); }
int c_kbits(int K) { return kbits(K); }
void c_residues(long long X, float* r) { Limbs L = limbs_of(X); res_all<0>(L, X, r); }
void c_recon(const unsigned* r, unsigned long long* lo, unsigned long long* hi) {
  uint32_t rr[kNumMod];
  for (int j = 0; j < kNumMod; ++j) rr[j] = r[j];
  reconstruct(rr, g, lo, hi);
}
int c_to_double(unsigned long long lo, unsigned long long hi, int E, int flip, double* out) {
  return to_double(lo, hi, E, flip != 0, out);
}
long long c_scaled_int(unsigned long long b, int emax, int sh0) { return scaled_int(b, emax, sh0); }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("crt")
    (d / "shim.cpp").write_text(SHIM)
    so = d / "libcrt.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", str(HEADER.parent), str(d / "shim.cpp"),
                    "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    L.c_to_double.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_double)]
    L.c_scaled_int.restype = ctypes.c_longlong
    L.c_scaled_int.argtypes = [ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int]
    L.c_residues.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_float)]
    L.c_modulus.restype = ctypes.c_uint
    assert L.c_ok()
    return L


def _P():
    P = 1
    for p in MODULI:
        P *= p
    return P


def test_moduli_pairwise_coprime_and_range(lib):
    from math import gcd
    assert [lib.c_modulus(j) for j in range(16)] == MODULI
    for i, a in enumerate(MODULI):
        assert a <= 256
        for b in MODULI[i + 1:]:
            assert gcd(a, b) == 1
    assert 2 ** 125 < _P() < 2 ** 126


def test_kbits_keeps_products_inside_half_the_modulus(lib):
    P = _P()
    for K in (1, 2, 64, 1000, 1024, 1025, 2048, 4096):
        k = lib.c_kbits(K)
        assert k <= 57 and K * 2 ** (2 * k) <= P // 2 and K * 2 ** (2 * k + 2) > P // 2 or k == 57
    assert lib.c_kbits(1024) == 57 and lib.c_kbits(4096) == 56


def test_residues_symmetric_and_exact(lib):
    rng = random.Random(7)
    r = (ctypes.c_float * 16)()
    for it in range(20000):
        X = rng.randrange(-(1 << 57) + 1, 1 << 57) if it % 2 else rng.randrange(-(1 << rng.randrange(1, 57)),
                                                                                1 << rng.randrange(1, 57))
        lib.c_residues(X, r)
        for j, p in enumerate(MODULI):
            v = r[j]
            assert v == int(v) and abs(v) <= 128 and (int(v) - X) % p == 0, (X, p, v)


def test_reconstruction_recovers_every_integer_in_range(lib):
    rng = random.Random(11)
    lo, hi = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    bound = 1 << 124
    cases = [0, 1, -1, bound - 1, -(bound - 1), 1 << 123, -(1 << 123)]
    cases += [rng.randrange(-bound, bound) for _ in range(20000)]
    cases += [rng.randrange(-(1 << rng.randrange(1, 124)), 1 << rng.randrange(1, 124)) for _ in range(20000)]
    for C in cases:
        res = (ctypes.c_uint * 16)(*[C % p for p in MODULI])
        lib.c_recon(res, ctypes.byref(lo), ctypes.byref(hi))
        v = (hi.value << 64) | lo.value
        if v >= 1 << 127:
            v -= 1 << 128
        assert v == C


def test_to_double_rounds_to_nearest_even(lib):
    rng = random.Random(13)
    out = ctypes.c_double()
    for it in range(40000):
        if it % 5 == 0:  # exact ties and near ties
            b = rng.randrange(54, 126)
            C = ((rng.randrange(1 << 52, 1 << 53) << 1) | 1) << (b - 54)
            C += rng.choice([0, 0, 1, -1])
        else:
            C = rng.randrange(-(1 << rng.randrange(1, 127)), 1 << rng.randrange(1, 127))
        if rng.random() < 0.5:
            C = -C
        E, flip = rng.randrange(-1200, 900), rng.randrange(2)
        u = C & ((1 << 128) - 1)
        ok = lib.c_to_double(u & ((1 << 64) - 1), u >> 64, E, flip, ctypes.byref(out))
        exact = Fraction(C) * Fraction(2) ** E * (-1 if flip else 1)
        try:
            ref = float(exact)
        except OverflowError:
            ref = float("inf")
        if C == 0:
            assert ok and out.value == 0.0
        elif ok:
            assert out.value == ref, (C, E, flip)
        else:  # only results outside the normal range take the plain route
            assert ref == 0.0 or abs(ref) < 2.0 ** -1022 or abs(ref) == float("inf") or abs(ref) >= 2.0 ** 1023


def test_scaled_int_truncates_toward_zero(lib):
    rng = random.Random(17)
    for _ in range(20000):
        x = rng.uniform(-1, 1) * 2.0 ** rng.randrange(-60, 60)
        b = struct.unpack("<Q", struct.pack("<d", x))[0]
        E = (b >> 52) & 0x7FF
        emax, sh0 = E + rng.randrange(0, 70), rng.choice([3, 4])
        X = lib.c_scaled_int(b, emax, sh0)
        assert X == int(Fraction(x) / Fraction(2) ** (emax - 1075 - sh0))
        assert abs(X) < 1 << (53 + sh0)
