"""The exact fixed-point sums of the FP64 CG kernels' dot products (csrc/pcg_fixed.cuh), checked
on the host: the arithmetic is the device's own, compiled for the host.  The fixed-point sum
of a set of doubles equals the exact rational sum of the values truncated at the window's
bottom, rounded once to nearest (ties to even), whatever the order; values beyond the window
or not finite are reported, never summed silently."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
from fractions import Fraction

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_10698_gb300", "csrc")


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    from paper_2211_10698_gb300 import build

    so = str(tmp_path_factory.mktemp("fx") / "libfxh.so")
    src = os.path.join(ROOT, "tests", "native", "fixed_sum_host.cu")
    subprocess.check_call([build._nvcc(), "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-shared", "-I",
                           os.path.join(ROOT, "include"), "-I", CSRC, "-o", so, src])
    L = ctypes.CDLL(so)
    L.fxh_window.restype = ctypes.c_int
    L.fxh_window.argtypes = [ctypes.c_double] * 3
    L.fxh_digits.restype = ctypes.c_int
    L.fxh_digits.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.fxh_sum.restype = ctypes.c_double
    L.fxh_sum.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_long, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    return L


def _sum(L, v, lo):
    a = np.ascontiguousarray(v, dtype=np.float64)
    bad = ctypes.c_int()
    s = L.fxh_sum(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(a), lo, ctypes.byref(bad))
    return s, bad.value


def _exact(v, lo):
    """float(sum of trunc(v_i 2^-lo)) 2^lo: Fraction -> float rounds to nearest, ties to even."""
    u = Fraction(2) ** lo
    return float(sum(int(Fraction(float(x)) / u) for x in v) * u)


def test_sums_are_exact_and_order_free(fx):
    rng = np.random.default_rng(2211)
    for trial in range(200):
        n = int(rng.integers(1, 2000))
        scale = 10.0 ** rng.uniform(-250, 250)
        kind = trial % 4
        if kind == 0:
            v = rng.standard_normal(n) * scale
        elif kind == 1:
            v = np.abs(rng.standard_normal(n)) * scale
        elif kind == 2:  # values spread over 30 decades
            v = rng.standard_normal(n) * scale * 10.0 ** rng.uniform(-30, 0, n)
        else:  # near-cancelling halves
            w = rng.standard_normal(n) * scale
            v = np.concatenate([w, -w * (1 + 1e-9 * rng.standard_normal(n))])
        lo = fx.fxh_window(float(np.abs(v).sum()), 0.0, 0.0)
        s, bad = _sum(fx, v, lo)
        assert bad == 0
        assert s == _exact(v, lo), trial
        assert _sum(fx, rng.permutation(v), lo)[0] == s  # bit for bit in any order
        true = float(sum(Fraction(float(x)) for x in v))
        assert abs(s - true) <= 2.0 ** -60 * float(np.abs(v).sum()) + abs(true) * 2.0 ** -53


def test_window_limits(fx):
    lo = fx.fxh_window(1.0, 0.5, -3.0)  # the largest power of two is 2
    d = (ctypes.c_int * 5)()
    assert fx.fxh_digits(2.0 ** 20, lo, d) == 1        # up to 2^20 times the largest previous sum fits
    assert fx.fxh_digits(2.0 ** 22, lo, d) == 0        # beyond it: reported
    assert fx.fxh_digits(float("nan"), lo, d) == 0 and fx.fxh_digits(float("inf"), lo, d) == 0
    assert fx.fxh_digits(-3.0, lo, d) == 1 and all(x <= 0 for x in d)  # sign on every digit
    s, bad = _sum(fx, [2.0 ** 22, 1.0], lo)
    assert bad == 1
    # subnormals and zeros around an all-zero reference
    lo0 = fx.fxh_window(0.0, 0.0, 0.0)
    v = [5e-324, 1e-310, -2e-320, 0.0]
    assert _sum(fx, v, lo0) == (float(sum(Fraction(x) for x in v)), 0)


def test_rounding_is_to_nearest_even(fx):
    big = 2.0 ** 53
    lo = fx.fxh_window(big, 0.0, 0.0)
    assert _sum(fx, [big, 1.0], lo)[0] == big                 # tie, even below
    assert _sum(fx, [big + 2.0, 1.0], lo)[0] == big + 4.0     # tie, even above
    assert _sum(fx, [big, 1.0, 2.0 ** -20], lo)[0] == big + 2.0  # above the tie
