"""CPU tests of the line subproblem's numerical helpers, from a host build of
the device header (tests/host/line_helpers.cpp):

* the FP64 reciprocal square root by one third-order step from an FP32
  estimate meets its error bound (an estimate with relative error up to 2^-21
  ends within a few units in the last place of 1/sqrt(a));
* the FP64 -> FP32 truncation and the FP32 -> FP64 widening in integer
  operations (IEEE 754 binary64 and binary32) agree with numpy's
  conversions: rounding toward zero, and exact widening;
* the exact FP64 line solve by a predicted active set (eq. line_kernel: a
  strictly convex 4-variable QP with box, two line-limit rows and the angle
  rows) returns the same KKT point as the dual active-set method of Goldfarb
  and Idnani on random subproblems, and never accepts a subproblem with no
  feasible point.
"""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("host") / "line_helpers.so")
    subprocess.check_call(["g++", "-O2", "-shared", "-fPIC", "-o", out, os.path.join(HERE, "host", "line_helpers.cpp")])
    L = C.CDLL(out)
    L.host_rsqrt_newton.restype = C.c_double
    L.host_rsqrt_newton.argtypes = [C.c_double, C.c_double]
    return L


def test_rsqrt_newton_error_bound(lib):
    rng = np.random.default_rng(5)
    a = np.exp(rng.uniform(math.log(1e-8), math.log(1e12), 4000))
    worst = 0.0
    for v in a:
        ref = 1.0 / math.sqrt(v)
        for e0 in (0.0, 2.0 ** -21, -(2.0 ** -21), rng.uniform(-1, 1) * 2.0 ** -21):
            y = lib.host_rsqrt_newton(float(v), ref * (1.0 + e0))
            worst = max(worst, abs(y - ref) / ref)
    assert worst <= 4 * 2.0 ** -53, worst


def test_integer_float_conversions(lib):
    FP = C.POINTER(C.c_float)
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.standard_normal(3000) * np.exp(rng.uniform(-80, 80, 3000)),  # across the FP32 range
        rng.standard_normal(200),
        [0.0, -0.0, 1.0, -1.0, 1e30, -1e30, 3.4028234663852886e38, 1e-40, -1e-40, 1e39, -1e39, np.inf, -np.inf,
         np.nan, 2.0 ** -126, 2.0 ** -127],
    ])
    out = np.zeros(len(x), dtype=np.float32)
    lib.host_f32_trunc(len(x), np.ascontiguousarray(x).ctypes.data_as(DP), out.ctypes.data_as(FP))
    # numpy rounds to nearest; step toward zero where that overshot |x|
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    over = np.isfinite(x) & (np.abs(want.astype(np.float64)) > np.abs(x))
    want[over] = np.nextafter(want[over], np.float32(0))
    tiny = np.isfinite(x) & (np.abs(x) < 2.0 ** -126)  # below the FP32 normal range: a signed zero
    want[tiny] = np.copysign(np.float32(0), x[tiny]).astype(np.float32)
    big = np.isfinite(x) & (np.abs(x) >= 2.0 ** 128)  # above it: an infinity
    want[big] = np.copysign(np.float32(np.inf), x[big]).astype(np.float32)
    nan = np.isnan(x)
    assert np.isnan(out[nan]).all()
    np.testing.assert_array_equal(out[~nan], want[~nan])
    assert (np.signbit(out[~nan]) == np.signbit(x[~nan])).all()
    # widening: exact for normal numbers, zeros and infinities; FP32 subnormals give a signed zero
    f = np.concatenate([out[np.isfinite(out)], np.array([1e-40, -1e-40, np.inf, -np.inf, np.nan], dtype=np.float32)])
    f = np.ascontiguousarray(f, dtype=np.float32)
    w = np.zeros(len(f))
    lib.host_f64_widen(len(f), f.ctypes.data_as(FP), w.ctypes.data_as(DP))
    ref = f.astype(np.float64)
    sub = np.isfinite(ref) & (np.abs(ref) < 2.0 ** -126)
    ref[sub] = np.copysign(0.0, ref[sub])
    fn = np.isnan(f)
    assert np.isnan(w[fn]).all()
    np.testing.assert_array_equal(w[~fn], ref[~fn])
    assert (np.signbit(w[~fn]) == np.signbit(ref[~fn])).all()


def _random_problems(rng, n):
    """Line subproblems shaped like the sweep's: Q = A'A + rho (F'F + I) with
    rho 2e4, boxes from voltage bands and a trust region (some degenerate),
    two normalised line-limit rows and the angle rows."""
    P = np.zeros((n, 41))
    iu = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
    rho = 2e4
    for k in range(n):
        A = rng.standard_normal((4, 4)) * 10.0
        F = rng.standard_normal((4, 4)) * rng.uniform(0.1, 3.0)
        Q = A.T @ A + rho * (F.T @ F + np.eye(4))
        for j, (a, b) in enumerate(iu):
            P[k, j] = Q[a, b]
        xstar = rng.standard_normal(4) * 0.05
        P[k, 10:14] = -Q @ xstar + rng.standard_normal(4) * rho * 0.01
        lo = -rng.uniform(0.0, 0.06, 4)
        hi = rng.uniform(0.0, 0.06, 4)
        if rng.random() < 0.2:  # a reference-bus angle: fixed at zero
            lo[1] = hi[1] = 0.0
        P[k, 14:18], P[k, 18:22] = lo, hi
        for e in range(2):
            r = rng.standard_normal(4)
            P[k, 22 + 4 * e:26 + 4 * e] = r / np.linalg.norm(r)
            P[k, 30 + e] = rng.uniform(-0.01, 0.05)
            P[k, 32 + e] = 1.0 if rng.random() < 0.9 else 0.0
        P[k, 34], P[k, 35], P[k, 36] = -rng.uniform(0.0, 0.05), rng.uniform(0.0, 0.05), 1.0
        P[k, 37:41] = np.clip(rng.standard_normal(4) * 0.02, lo, hi)
    return P


def test_predicted_line_solve_matches_the_dual_method(lib):
    rng = np.random.default_rng(11)
    n = 3000
    P = np.ascontiguousarray(_random_problems(rng, n))
    ok = np.zeros(n, dtype=np.int32)
    st = np.zeros(n, dtype=np.int32)
    xp, up, xe, ue = (np.zeros((n, 4)) for _ in range(4))
    lib.host_line_solves(n, P.ctypes.data_as(DP), ok.ctypes.data_as(IP), xp.ctypes.data_as(DP), up.ctypes.data_as(DP),
                         st.ctypes.data_as(IP), xe.ctypes.data_as(DP), ue.ctypes.data_as(DP))
    feas = st >= 0
    assert feas.sum() > n // 2 and (~feas).sum() > 0  # both kinds occur
    assert not (ok.astype(bool) & ~feas).any()  # no point accepted where none is feasible
    both = ok.astype(bool) & feas
    assert both.sum() >= 0.9 * feas.sum(), (int(both.sum()), int(feas.sum()))
    sx = np.maximum(1e-3, np.abs(xe).max(1))
    su = np.maximum(1.0, np.abs(ue).max(1))
    assert (np.abs(xp - xe).max(1) / sx)[both].max() <= 1e-10
    assert (np.abs(up - ue).max(1) / su)[both].max() <= 1e-8
