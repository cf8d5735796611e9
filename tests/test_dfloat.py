"""The double-float arithmetic of the mixed-precision solvers' FP64-accuracy operator
(paper_1612_06424_gb300/csrc/dfloat.h), compiled for the host with g++ (no FP contraction) and
checked against exact rational arithmetic:
  TwoSum and TwoProduct are error-free: s + e = a + b and p + e = a * b exactly;
  a double rounds to a double-float within 2^-48 of its magnitude;
  sums and products of double-floats are within 2^-45 of the exact result of their inputs
  (a few units of the 2^-48 double-float rounding; a wrong sign or a dropped error term breaks
  this by orders of magnitude).
"""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1612_06424_gb300", "csrc", "dfloat.h")

HARNESS = r"""
#include "dfloat.h"
using lq::dfloat;
extern "C" {
void t_two_sum(float a, float b, float* s, float* e) { lq::two_sum(a, b, *s, *e); }
void t_two_prod(float a, float b, float* p, float* e) { lq::two_prod(a, b, *p, *e); }
void t_from(double x, float* hi, float* lo) { dfloat d(x); *hi = d.hi; *lo = d.lo; }
void t_add(float ah, float al, float bh, float bl, float* h, float* l) { dfloat r = dfloat(ah, al) + dfloat(bh, bl); *h = r.hi; *l = r.lo; }
void t_mul(float ah, float al, float bh, float bl, float* h, float* l) { dfloat r = dfloat(ah, al) * dfloat(bh, bl); *h = r.hi; *l = r.lo; }
void t_fma(float ah, float al, float bh, float bl, float ch, float cl, float* h, float* l) {
  dfloat r = fma(dfloat(ah, al), dfloat(bh, bl), dfloat(ch, cl)); *h = r.hi; *l = r.lo; }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("dfloat")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    so = d / "libdf.so"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I", os.path.dirname(HEADER), "-o",
                    str(so), str(src)], check=True)
    L = ctypes.CDLL(str(so))
    f, fp, dd = ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.c_double
    L.t_two_sum.argtypes = [f, f, fp, fp]
    L.t_two_prod.argtypes = [f, f, fp, fp]
    L.t_from.argtypes = [dd, fp, fp]
    L.t_add.argtypes = [f, f, f, f, fp, fp]
    L.t_mul.argtypes = [f, f, f, f, fp, fp]
    L.t_fma.argtypes = [f, f, f, f, f, f, fp, fp]
    return L


def _out():
    return ctypes.c_float(), ctypes.c_float()


def _fr(x):
    return Fraction(float(x))


def _rand_floats(rng, n):
    # signs, mantissas and exponents spread over +-2^20
    return (rng.choice([-1.0, 1.0], n) * rng.random(n) * np.exp2(rng.integers(-20, 21, n))).astype(np.float32)


def _df(L, x):
    h, l = _out()
    L.t_from(float(x), ctypes.byref(h), ctypes.byref(l))
    return h.value, l.value


def test_error_free_transformations(lib):
    rng = np.random.default_rng(1)
    a, b = _rand_floats(rng, 2000), _rand_floats(rng, 2000)
    for x, y in zip(a, b):
        s, e = _out()
        lib.t_two_sum(float(x), float(y), ctypes.byref(s), ctypes.byref(e))
        assert _fr(np.float32(s.value)) + _fr(np.float32(e.value)) == _fr(x) + _fr(y)
        assert np.float32(s.value) == np.float32(x) + np.float32(y)
        p, e = _out()
        lib.t_two_prod(float(x), float(y), ctypes.byref(p), ctypes.byref(e))
        assert _fr(np.float32(p.value)) + _fr(np.float32(e.value)) == _fr(x) * _fr(y)


def test_rounding_and_arithmetic_accuracy(lib):
    rng = np.random.default_rng(2)
    xs = rng.standard_normal(3000) * np.exp2(rng.integers(-30, 31, 3000))
    bound_round = Fraction(1, 2 ** 48)
    bound_op = Fraction(1, 2 ** 45)
    for i in range(0, len(xs) - 2, 3):
        x, y, z = xs[i], xs[i + 1], xs[i + 2]
        dx, dy, dz = _df(lib, x), _df(lib, y), _df(lib, z)
        for v, d in ((x, dx), (y, dy)):
            assert abs(_fr(d[0]) + _fr(d[1]) - _fr(v)) <= bound_round * abs(_fr(v))
        X, Y, Z = (_fr(d[0]) + _fr(d[1]) for d in (dx, dy, dz))
        h, l = _out()
        lib.t_add(dx[0], dx[1], dy[0], dy[1], ctypes.byref(h), ctypes.byref(l))
        exact = X + Y
        assert abs(_fr(h.value) + _fr(l.value) - exact) <= bound_op * max(abs(X), abs(Y)), (x, y)
        lib.t_mul(dx[0], dx[1], dy[0], dy[1], ctypes.byref(h), ctypes.byref(l))
        exact = X * Y
        assert abs(_fr(h.value) + _fr(l.value) - exact) <= bound_op * abs(exact), (x, y)
        lib.t_fma(dx[0], dx[1], dy[0], dy[1], dz[0], dz[1], ctypes.byref(h), ctypes.byref(l))
        exact = X * Y + Z
        assert abs(_fr(h.value) + _fr(l.value) - exact) <= 2 * bound_op * (abs(X * Y) + abs(Z)), (x, y, z)
