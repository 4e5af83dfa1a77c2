"""CPU checks of the adjoint building blocks (abcmb_adjoint_ops.cuh, built for
the host): every transpose satisfies <v, X y> = <X^T v, y>, the IMEX solve
inverts I - h T and its transpose inverts the transpose, and every reverse-mode
gradient (background quantities, node data, initial time and R_nu) matches
central finite differences of the forward expression."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
D = ctypes.c_double


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("adj") / "libadjops.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "adjoint_ops_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_apply.argtypes = [ctypes.c_int, ctypes.c_int, D, P, D, P, P]
    L.h_bgrad.argtypes = [ctypes.c_int, ctypes.c_int, D, P, P, P, P]
    L.h_sources.argtypes = [ctypes.c_int, D, P, P, P, P, P]
    L.h_sources_rev.argtypes = [ctypes.c_int, D, P, P, P, P, P, P, P, P]
    L.h_initial.argtypes = [ctypes.c_int, D, D, D, P]
    L.h_initial_d.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, P]
    L.h_initial_d.restype = D
    return L


def p(a):
    return a.ctypes.data_as(P)


def bg_point(rng):
    # ih, iht, fc, fb, fg, fnu, nu, rnu, cs2, hc (positive, O(1) spreads)
    return rng.uniform(0.2, 2.0, size=10)


def apply(H, which, L, k, b, y, h=0.0):
    out = np.zeros_like(y)
    H.h_apply(which, L, k, p(b), h, p(np.ascontiguousarray(y)), p(out))
    return out


@pytest.mark.parametrize("L", [4, 12, 30])
def test_transposes(H, L):
    rng = np.random.default_rng(L)
    N = H.h_nstate(L)
    for _ in range(5):
        k, b = rng.uniform(0.01, 2.0), bg_point(rng)
        y, v = rng.normal(size=N), rng.normal(size=N)
        for fwd, tr in ((0, 1), (2, 3)):
            lhs = v @ apply(H, fwd, L, k, b, y)
            rhs = apply(H, tr, L, k, b, v) @ y
            assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(v) * np.linalg.norm(y))


@pytest.mark.parametrize("L", [5, 30])
def test_imex_solve_and_its_transpose(H, L):
    rng = np.random.default_rng(100 + L)
    N = H.h_nstate(L)
    for h in (1e-3, 0.3, 50.0):
        k, b, w = rng.uniform(0.01, 2.0), bg_point(rng), rng.normal(size=N)
        y = apply(H, 4, L, k, b, w, h)
        r = y - h * apply(H, 2, L, k, b, y) - w  # (I - h T) y = w
        assert np.max(np.abs(r)) <= 1e-12 * (1 + np.max(np.abs(w)))
        v = rng.normal(size=N)
        assert abs(v @ y - apply(H, 5, L, k, b, v, h) @ w) <= 1e-11 * np.linalg.norm(v) * np.linalg.norm(w)


@pytest.mark.parametrize("which", [0, 1])
def test_background_gradients(H, which):
    rng = np.random.default_rng(7 + which)
    L = 8
    N = H.h_nstate(L)
    k, b = 0.3, bg_point(rng)
    y, v = rng.normal(size=N), rng.normal(size=N)
    g = np.zeros(10)
    H.h_bgrad(which, L, k, p(b), p(v), p(y), p(g))
    op = 0 if which == 0 else 2
    for q in range(10):
        e = 1e-6 * max(1.0, abs(b[q]))
        bp, bm = b.copy(), b.copy()
        bp[q] += e
        bm[q] -= e
        fd = (v @ apply(H, op, L, k, bp, y) - v @ apply(H, op, L, k, bm, y)) / (2 * e)
        assert abs(g[q] - fd) <= 1e-7 * (1 + abs(fd)), q


def test_sources_reverse_mode(H):
    rng = np.random.default_rng(3)
    L = 10
    N = H.h_nstate(L)
    k, b = 0.07, bg_point(rng)
    nd = np.array([0.8, -0.3, 1.7, 0.4, 0.6])  # Hc, dHc, g, dg, e^-kappa
    sw = np.array([1.0, 1.0, 1.0])
    y, Sb = rng.normal(size=N), rng.normal(size=3)

    def S(yv, bv, nv):
        out = np.zeros(3)
        H.h_sources(L, k, p(bv), p(nv), p(sw), p(np.ascontiguousarray(yv)), p(out))
        return out

    yb, bb, nb = np.zeros(N), np.zeros(10), np.zeros(5)
    H.h_sources_rev(L, k, p(b), p(nd), p(sw), p(y), p(Sb), p(yb), p(bb), p(nb))
    for i in range(N):  # linear in y: the transposed Jacobian exactly
        e = np.zeros(N)
        e[i] = 1.0
        assert abs(yb[i] - Sb @ (S(y + e, b, nd) - S(y, b, nd))) <= 1e-10 * (1 + abs(yb[i])), i
    for arr, grad, name in ((b, bb, "b"), (nd, nb, "node")):
        for q in range(arr.size):
            e = 1e-4 * max(1.0, abs(arr[q]))  # sources are ~1/k^2: a larger step keeps rounding down
            ap, am = arr.copy(), arr.copy()
            ap[q] += e
            am[q] -= e
            args_p = (y, ap, nd) if name == "b" else (y, b, ap)
            args_m = (y, am, nd) if name == "b" else (y, b, am)
            fd = Sb @ (S(*args_p) - S(*args_m)) / (2 * e)
            assert abs(grad[q] - fd) <= 1e-6 * (1 + abs(fd)), (name, q)


def test_initial_state_derivatives(H):
    rng = np.random.default_rng(5)
    L = 6
    N = H.h_nstate(L)
    k, tau, Rn = 0.2, 0.37, 0.41
    yb = rng.normal(size=N)

    def y0(t, r):
        out = np.zeros(N)
        H.h_initial(L, k, t, r, p(out))
        return out

    fd_t = yb @ (y0(tau + 1e-6, Rn) - y0(tau - 1e-6, Rn)) / 2e-6
    fd_r = yb @ (y0(tau, Rn + 1e-6) - y0(tau, Rn - 1e-6)) / 2e-6
    assert abs(H.h_initial_d(0, L, k, tau, Rn, p(yb)) - fd_t) <= 1e-7 * (1 + abs(fd_t))
    assert abs(H.h_initial_d(1, L, k, tau, Rn, p(yb)) - fd_r) <= 1e-7 * (1 + abs(fd_r))
