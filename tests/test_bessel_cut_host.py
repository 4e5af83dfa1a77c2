"""CPU checks of the projection kernels' Bessel cutoff (abcmb_bessel.cuh
built for the host): the last l each (k, tau) node keeps is the Debye rule it
states (the smallest l whose decay exponent nu (alpha - tanh alpha),
nu = l + 1/2, cosh alpha = nu / x, reaches 16 + 2 ln(1/x) for x < 1), the
spherical Bessel functions it drops are below ~e^-16 of their largest value
(scipy's spherical_jn), and the benchmark's count of evaluated (node, l)
points follows the same rule."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
LMAX = 2500


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("bessel_cut") / "libbessel_cut.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "bessel_cut_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bessel_cut.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
    return L


def cut(H, x, lmax=LMAX):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(x.size, dtype=np.int32)
    H.h_bessel_cut(x.ctypes.data_as(P), x.size, lmax, out.ctypes.data_as(P))
    return out


def debye_rule(x, lmax):
    """The rule in float64: nu* solves nu (alpha - tanh alpha) = T(x) by
    bisection on nu > x + 1/2, l = ceil(nu* - 1/2) clipped to [2, lmax];
    l = lmax for x > lmax + 200.  -> (l, nu*)."""
    def expo(nu, xi):
        al = np.arccosh(max(nu / xi, 1.0))
        return nu * (al - np.tanh(al))
    out, roots = [], []
    for xi in x:
        T = 16.0 + 2.0 * max(0.0, -np.log(xi))
        lo, hi = xi + 0.5, xi + 0.5 + 1e5
        for _ in range(200):
            m = 0.5 * (lo + hi)
            lo, hi = (m, hi) if expo(m, xi) < T else (lo, m)
        out.append(lmax if xi > lmax + 200 else min(max(np.ceil(hi - 0.5), 2), lmax))
        roots.append(hi)
    return np.array(out), np.array(roots)


def assert_rule(got, x, lmax):
    """got equals the float64 rule, except by one l where nu* - 1/2 lies
    within 1e-6 nu* of an integer (the kernel finds nu* in float32)."""
    ref, nu = debye_rule(x, lmax)
    d = np.abs(got - ref)
    edge = np.abs(nu - 0.5 - np.round(nu - 0.5)) <= 1e-6 * nu
    assert d.max() <= 1 and np.all(edge[d > 0]), (x[d > 0], got[d > 0], ref[d > 0])


def nodes_x():
    # float32 inputs, as the kernel receives them
    return np.exp(np.linspace(np.log(1e-3), np.log(LMAX + 400.0), 3001)).astype(np.float32).astype(np.float64)


def test_cutoff_is_the_debye_rule(H):
    x = nodes_x()
    assert_rule(cut(H, x), x, LMAX)
    # a small lmax clips
    xs = x[x < 300]
    assert_rule(cut(H, xs, 40), xs, 40)


@pytest.mark.parametrize("x", [0.01, 0.3, 2.0, 10.0, 100.0, 1000.0, 2400.0])
def test_dropped_bessel_functions_are_below_e_minus_16_of_the_largest(H, x):
    from scipy.special import spherical_jn
    lc = int(cut(H, np.array([x]))[0])
    j = np.abs(spherical_jn(np.arange(lc + 60), x))
    # the T2 and E kernels carry j_l / x^2, hence the x < 1 threshold shift
    w = 1.0 / min(x, 1.0) ** 2
    # (the Debye exponent leaves out the prefactor: measured at most 2.1e-8)
    assert w * j[lc + 1:].max() <= 5e-8 * j[:lc + 1].max(), (x, lc)
    # and it keeps no l it need not: one l earlier the function is still
    # above 2e-8 of the largest (measured 3.5e-8 to 1e-4)
    assert w * j[lc - 1] >= 2e-8 * j[:lc + 1].max(), (x, lc)


def test_the_benchmark_counts_the_points_the_kernel_evaluates(H):
    sys.path.insert(0, ROOT)
    import bench
    x = nodes_x()
    # the projection kernels stop nodes with x < 1 (power-series j_l) at l = 30
    series = x < 1.0
    kern = cut(H, x)
    kern = np.where(series, np.minimum(kern, 30), kern)
    ours = bench.bessel_cut(x, LMAX)
    np.testing.assert_array_equal(ours[series], kern[series])
    assert_rule(ours[~series], x[~series], LMAX)
    assert_rule(kern[~series], x[~series], LMAX)
