"""CPU check of the adjoint's warp layout (abcmb_adjoint.cuh and
abcmb_adjoint_ops.cuh, one warp per mode as taped_kernel and adjoint_kernel
run them): built for the host with the 32 lanes as threads
(tests/host/warp_emu.h), one mode's taped forward and reverse sweep equal the
one-lane host build (tests/test_adjoint_mode.py holds that against finite
differences), and repeated runs agree bit for bit.  Lanes that run ahead of a
lane still reading a shared vector break the second and the first: this is
how the barriers closing op_E_bgrad and op_T_bgrad were found missing.
"""
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


def _build(tmp_path_factory, name, src, extra=()):
    so = str(tmp_path_factory.mktemp(name) / f"lib{name}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", *extra, "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", src), "-o", so])
    return ctypes.CDLL(so)


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    one = _build(tmp_path_factory, "adjone", "adjoint_mode_harness.cpp")
    one.h_bg_len.restype = ctypes.c_long
    one.h_fwd.argtypes = [P, D, I, D, P, P]
    one.h_grad.argtypes = [P, D, I, D, P, P]
    warp = _build(tmp_path_factory, "adjwarp", "adjoint_warp_harness.cpp", ("-pthread",))
    warp.h_fwd_warp.argtypes = [P, D, I, D, P, P]
    warp.h_grad_warp.argtypes = [P, D, I, D, P, P]
    return one, warp


def ptr(a):
    return a.ctypes.data_as(P)


def test_warp_adjoint_equals_the_one_lane_adjoint(libs):
    one, warp = libs
    n_tau, k, L, rtol = 120, 0.05, 8, 1e-6  # implicit and explicit (Gragg) regimes both
    p = W.BATCH64.params()[0]
    rec = np.zeros(one.h_bg_len(n_tau))
    one.h_build_bg(ptr(p), n_tau, ptr(rec))
    S1, Sw = np.zeros((n_tau, 3)), np.zeros((n_tau, 3))
    sig1, sigw = np.zeros(3, np.int32), np.zeros(3, np.int32)
    assert one.h_fwd(ptr(rec), k, L, rtol, ptr(S1), ptr(sig1)) == 0
    assert warp.h_fwd_warp(ptr(rec), k, L, rtol, ptr(Sw), ptr(sigw)) == 0
    np.testing.assert_array_equal(sigw, sig1)  # the same discrete map
    assert np.abs(Sw - S1).max() <= 1e-13 * np.abs(S1).max()
    Sb = np.random.default_rng(3).normal(size=(n_tau, 3)) / np.abs(S1).max(axis=0)
    g1 = np.zeros_like(rec)
    assert one.h_grad(ptr(rec), k, L, rtol, ptr(Sb), ptr(g1)) == 0
    gw = [np.zeros_like(rec), np.zeros_like(rec)]
    for g in gw:
        assert warp.h_grad_warp(ptr(rec), k, L, rtol, ptr(Sb), ptr(g)) == 0
    np.testing.assert_array_equal(gw[1], gw[0])
    # measured 8e-18 of the largest entry
    assert np.abs(gw[0] - g1).max() <= 1e-12 * np.abs(g1).max()
