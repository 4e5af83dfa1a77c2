"""CPU checks of one mode's discrete adjoint (abcmb_adjoint.cuh built for the
host): a step's transpose is exact, and the gradient of <Sbar, S> with respect
to the background record (ODE table, node data) matches central finite
differences of the taped forward."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2602_15104_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
D = ctypes.c_double
I = ctypes.c_int


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("adjmode") / "libadjmode.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "adjoint_mode_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_fwd.argtypes = [P, D, I, D, P, P]
    L.h_grad.argtypes = [P, D, I, D, P, P]
    L.h_step.argtypes = [P, D, I, D, D, I, I, P, P]
    L.h_step_adj.argtypes = [P, D, I, D, D, I, I, P, P, P]
    return L


@pytest.fixture(scope="module")
def rec(H):
    n_tau = 120
    p = W.BATCH64.params()[0]
    r = np.zeros(H.h_bg_len(n_tau))
    H.h_build_bg(p.ctypes.data_as(P), n_tau, r.ctypes.data_as(P))
    return r


def ptr(a):
    return a.ctypes.data_as(P)


@pytest.mark.parametrize("x,H_,J,gbs", [(-9.0, 0.01, 2, 0), (-6.95, 0.004, 5, 0), (-3.0, 0.05, 4, 1),
                                        (-3.0, 0.05, 6, 1)])
def test_step_transpose_and_table_gradient(H, rec, x, H_, J, gbs):
    L, k = 8, 0.02
    N = 4 + 3 * (L + 1)
    rng = np.random.default_rng(J + 10 * gbs)
    y, v = rng.normal(size=N), rng.normal(size=N)
    out = np.zeros(N)
    H.h_step(ptr(rec), k, L, x, H_, J, gbs, ptr(y), ptr(out))
    yb, rb = v.copy(), np.zeros_like(rec)
    H.h_step_adj(ptr(rec), k, L, x, H_, J, gbs, ptr(y), ptr(yb), ptr(rb))
    assert abs(v @ out - yb @ y) <= 1e-12 * abs(v @ out)
    a, b = 64 + 8 * 18433, 64 + 28 * 18433
    for e in a + np.argsort(-np.abs(rb[a:b]))[:3]:
        h = 1e-6 * abs(rec[e])
        rp, rm = rec.copy(), rec.copy()
        rp[e] += h
        rm[e] -= h
        op, om = np.zeros(N), np.zeros(N)
        H.h_step(ptr(rp), k, L, x, H_, J, gbs, ptr(y), ptr(op))
        H.h_step(ptr(rm), k, L, x, H_, J, gbs, ptr(y), ptr(om))
        fd = v @ (op - om) / (2 * h)
        assert abs(rb[e] - fd) <= 1e-4 * abs(fd), e


@pytest.mark.parametrize("k,node", [(0.02, 30), (0.02, 80), (0.003, 60)])
def test_mode_gradient_against_finite_differences(H, rec, k, node):
    # An adaptive forward flips an accept/reject decision or a column count
    # (err within ~1e-7 of 1) for perturbations as small as 1e-7 of a table
    # entry, which changes the discrete map by the integration error; the
    # differences are therefore taken with steps of ~1e-8 relative and only
    # where the three runs took the same steps with the same column counts.
    # The forward's rounding moves <Sbar, S> by ~3e-12 of itself, so a
    # difference is used only where the perturbation moves it by 1e-8 of
    # itself or more, and the entries tried are those it is most sensitive to
    # in relative terms (|rbar_e rec_e|).
    n_tau, L, rtol = 120, 8, 1e-9
    rng = np.random.default_rng(node)
    Sb = np.zeros((n_tau, 3))
    Sb[node] = rng.normal(size=3)

    def phi(r):
        S, sig = np.zeros((n_tau, 3)), np.zeros(3, dtype=np.int32)
        assert H.h_fwd(ptr(r), k, L, rtol, ptr(S), ptr(sig)) == 0
        return (Sb * S).sum(), tuple(sig)

    _, acc0 = phi(rec)
    rb = np.zeros_like(rec)
    assert H.h_grad(ptr(rec), k, L, rtol, ptr(Sb), ptr(rb)) == 0
    regions = [(64 + 8 * 18433, 64 + 28 * 18433), (64 + 28 * 18433, 64 + 28 * 18433 + 8 * n_tau)]  # ODE table, nodes
    checked = 0
    for a, b in regions:
        for e in a + np.argsort(-np.abs(rb[a:b] * rec[a:b]))[:6]:
            for hr in (3e-8, 1e-8, 3e-9, 1e-9):
                h = hr * abs(rec[e])
                rp, rm = rec.copy(), rec.copy()
                rp[e] += h
                rm[e] -= h
                (fp, ap), (fm, am) = phi(rp), phi(rm)
                if ap == am == acc0 and abs(fp - fm) > 1e-8 * max(abs(fp), abs(fm)):
                    fd = (fp - fm) / (2 * h)
                    assert abs(rb[e] - fd) <= 2e-3 * abs(fd), (e, rb[e], fd)
                    checked += 1
                    break
    assert checked >= 4


@pytest.mark.parametrize("k,node", [(0.02, 80), (0.003, 100)])
def test_node_position_gradient(H, rec, k, node):
    # a node's ln a moves the sources there with the ODE flow and the
    # background's slope; later nodes are unaffected up to the integration error
    # (rtol 2e-9: at 1e-9 the unperturbed k = 0.02 run sits on an accept/reject
    # boundary that every node perturbation flips, leaving no step to compare)
    n_tau, L, rtol = 120, 8, 2e-9
    rng = np.random.default_rng(7 + node)
    Sb = rng.normal(size=(n_tau, 3))

    def phi(r):
        S, sig = np.zeros((n_tau, 3)), np.zeros(3, dtype=np.int32)
        assert H.h_fwd(ptr(r), k, L, rtol, ptr(S), ptr(sig)) == 0
        return (Sb * S).sum(), tuple(sig)

    _, acc0 = phi(rec)
    rb = np.zeros_like(rec)
    assert H.h_grad(ptr(rec), k, L, rtol, ptr(Sb), ptr(rb)) == 0
    e = 64 + 28 * 18433 + 8 * node  # the node's ln a
    for hr in (3e-8, 1e-8, 3e-9, 1e-9):
        h = hr * abs(rec[e])
        rp, rm = rec.copy(), rec.copy()
        rp[e] += h
        rm[e] -= h
        (fp, ap), (fm, am) = phi(rp), phi(rm)
        if ap == am == acc0:
            fd = (fp - fm) / (2 * h)
            assert abs(rb[e] - fd) <= 2e-3 * abs(fd), (rb[e], fd)
            return
    pytest.fail("no step size kept the accepted steps fixed")
