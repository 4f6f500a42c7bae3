"""The double-float arithmetic that implements the library's FP64 precision
(paper_1309_2256_gb300/csrc/dl_df.cuh), compiled for the host with g++ and checked
against exact rational arithmetic: sums, products and long dot products stay within
a few units of 2^-48 of the exact result of the represented inputs."""
import ctypes
import os
import random
import shutil
import subprocess
import tempfile
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_1309_2256_gb300", "csrc", "dl_df.cuh")

SRC = r"""
#include "%s"
extern "C" {
void df_split(double v, float* o) { dfloat a(v); o[0] = a.hi; o[1] = a.lo; }
void df_add2(const float* a, const float* b, float* o) { dfloat r = dfloat(a[0], a[1]) + dfloat(b[0], b[1]); o[0] = r.hi; o[1] = r.lo; }
void df_mul2(const float* a, const float* b, float* o) { dfloat r = dfloat(a[0], a[1]) * dfloat(b[0], b[1]); o[0] = r.hi; o[1] = r.lo; }
void df_dot(int n, const float* a, const float* b, float* o) {
  dfloat acc(0);
  for (int i = 0; i < n; ++i) acc += dfloat(a[2 * i], a[2 * i + 1]) * dfloat(b[2 * i], b[2 * i + 1]);
  o[0] = acc.hi; o[1] = acc.lo;
}
// the stencil's lazy sums: products accumulated unnormalised, normalised once
void df_dot_lazy(int n, const float* a, const float* b, float* o) {
  dfloat acc = df_mul_lazy(dfloat(a[0], a[1]), dfloat(b[0], b[1]));
  for (int i = 1; i < n; ++i) df_acc_mul(acc, dfloat(a[2 * i], a[2 * i + 1]), dfloat(b[2 * i], b[2 * i + 1]));
  acc = df_normalize(acc);
  o[0] = acc.hi; o[1] = acc.lo;
}
void df_sum_lazy(int n, const float* a, float* o) {
  dfloat acc = df_add_lazy(dfloat(a[0], a[1]), dfloat(a[2], a[3]));
  for (int i = 2; i < n; ++i) df_acc(acc, dfloat(a[2 * i], a[2 * i + 1]));
  acc = df_normalize(acc);
  o[0] = acc.hi; o[1] = acc.lo;
}
}
"""


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "df.cpp")
    so = os.path.join(d, "libdf.so")
    with open(src, "w") as f:
        f.write(SRC % os.path.abspath(HEADER))
    # -ffp-contract=off: the header's FMA is explicit; no other contraction on the host
    subprocess.check_call([cxx, "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, src])
    h = ctypes.CDLL(so)
    return h


def _f2(vals):
    return (ctypes.c_float * len(vals))(*vals)


def _split(h, v):
    o = _f2([0.0, 0.0])
    h.df_split(ctypes.c_double(v), o)
    return [o[0], o[1]]


def _exact(p):
    return Fraction(p[0]) + Fraction(p[1])


def test_split_keeps_48_bits(lib):
    rng = random.Random(1)
    for _ in range(2000):
        v = rng.uniform(-1, 1) * 10 ** rng.randint(-3, 3)
        p = _split(lib, v)
        assert abs(_exact(p) - Fraction(v)) <= abs(Fraction(v)) * Fraction(1, 2 ** 47)
        assert abs(p[1]) <= abs(p[0]) * 2.0 ** -23


def test_sum_and_product_error_bounds(lib):
    rng = random.Random(2)
    worst_add = worst_mul = Fraction(0)
    for _ in range(3000):
        a = _split(lib, rng.uniform(-1, 1) * 10 ** rng.randint(-2, 2))
        b = _split(lib, rng.uniform(-1, 1) * 10 ** rng.randint(-2, 2))
        o = _f2([0.0, 0.0])
        lib.df_add2(_f2(a), _f2(b), o)
        ex = _exact(a) + _exact(b)
        worst_add = max(worst_add, abs(_exact(o) - ex) / (abs(_exact(a)) + abs(_exact(b))))
        lib.df_mul2(_f2(a), _f2(b), o)
        ex = _exact(a) * _exact(b)
        worst_mul = max(worst_mul, abs(_exact(o) - ex) / abs(ex))
    assert worst_add <= Fraction(1, 2 ** 46)
    assert worst_mul <= Fraction(1, 2 ** 45)


def test_cancellation_is_exact(lib):
    """x + (-(x + d)) for a tiny d: the two-sum recovers d exactly from the representations."""
    rng = random.Random(3)
    for _ in range(500):
        x = rng.uniform(0.5, 1.0)
        a = _split(lib, x)
        b = _split(lib, -(x + x * 1e-9))
        o = _f2([0.0, 0.0])
        lib.df_add2(_f2(a), _f2(b), o)
        assert _exact(o) == _exact(a) + _exact(b)


def test_dot_product_of_200_terms(lib):
    rng = random.Random(4)
    for _ in range(50):
        n = 200
        a = [c for _ in range(n) for c in _split(lib, rng.uniform(-1, 1))]
        b = [c for _ in range(n) for c in _split(lib, rng.uniform(-1, 1))]
        o = _f2([0.0, 0.0])
        lib.df_dot(n, _f2(a), _f2(b), o)
        ex = sum(_exact(a[2 * i:2 * i + 2]) * _exact(b[2 * i:2 * i + 2]) for i in range(n))
        mag = sum(abs(_exact(a[2 * i:2 * i + 2]) * _exact(b[2 * i:2 * i + 2])) for i in range(n))
        assert abs(_exact(o) - ex) <= mag * Fraction(1, 2 ** 46)


@pytest.mark.parametrize("n", [3, 6, 8, 48])
def test_lazy_dot_products(lib, n):
    """The stencil's SU(3) sums (6 products per output) accumulated without intermediate
    normalisation, normalised (|lo| <= ulp(hi)/2) at the end.  The unnormalised low part
    grows with the terms added, each FP32 addition into it erring by 2^-24 of it, so the
    error bound is linear in the length: (n + 2) 2^-48 of the sum of the magnitudes
    (6 terms: 2^-45)."""
    rng = random.Random(5 + n)
    for _ in range(1000):
        a = [c for _ in range(n) for c in _split(lib, rng.uniform(-1, 1) * 10 ** rng.randint(-2, 2))]
        b = [c for _ in range(n) for c in _split(lib, rng.uniform(-1, 1))]
        o = _f2([0.0, 0.0])
        lib.df_dot_lazy(n, _f2(a), _f2(b), o)
        ex = sum(_exact(a[2 * i:2 * i + 2]) * _exact(b[2 * i:2 * i + 2]) for i in range(n))
        mag = sum(abs(_exact(a[2 * i:2 * i + 2]) * _exact(b[2 * i:2 * i + 2])) for i in range(n))
        assert abs(_exact(o) - ex) <= mag * Fraction(n + 2, 2 ** 48)
        assert abs(o[1]) <= abs(o[0]) * 2.0 ** -23


def test_lazy_sum_with_cancellation(lib):
    """The hop sum of the stencil (eight terms of either sign that may nearly cancel):
    absolute error within 2^-47 of the summed magnitudes, also when the result is far
    smaller than the terms."""
    rng = random.Random(6)
    for k in range(300):
        x = [rng.uniform(-1, 1) for _ in range(7)]
        x.append(-sum(x) + (rng.uniform(-1, 1) * 1e-9 if k % 2 else 0.0))  # near or exact cancellation
        a = [c for v in x for c in _split(lib, v)]
        o = _f2([0.0, 0.0])
        lib.df_sum_lazy(len(x), _f2(a), o)
        ex = sum(_exact(a[2 * i:2 * i + 2]) for i in range(len(x)))
        mag = sum(abs(_exact(a[2 * i:2 * i + 2])) for i in range(len(x)))
        assert abs(_exact(o) - ex) <= mag * Fraction(1, 2 ** 47)
