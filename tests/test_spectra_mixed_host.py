"""CPU parity of the mixed-precision projection and k-quadrature kernels
(abcmb_spectra_mixed.cuh: the FP32 form behind abcmb_project_mixed and
abcmb_cl_mixed), built for the host with every CTA's threads run as host
threads (tests/host/warp_emu.h) and every FP32 operation rounded once, against
the oracle's FP64 exact-Bessel projection (App. B.4 transfer functions) and
k-quadrature (App. B.4 eq. c_ell_def): the double-float recurrence, the FP32
products and Kahan sums.  The same kernels run on a GB300 in
tests/test_gpu_mixed.py, at the same sizes and bars.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2602_15104_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("mixed") / "libmixed.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-pthread", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "spectra_mixed_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_build_bg.argtypes = [P, ctypes.c_int, P]
    L.h_project_mixed.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, P]
    L.h_cl_mixed.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int, P]
    return L


def records(H, params, n_tau):
    params = np.atleast_2d(params)
    r = np.zeros((len(params), H.h_bg_len(n_tau)))
    for b, p in enumerate(params):
        H.h_build_bg(np.ascontiguousarray(p).ctypes.data_as(P), n_tau, r[b].ctypes.data_as(P))
    return r


def test_mixed_projection_against_oracle_at_full_size(H):
    # 6000 nodes, l <= 2500, k from 1e-5 to 0.5: within 2e-5 of each row's
    # peak, the GPU test's bar (measured 1.9e-6)
    params = W.BATCH64.params()[[0, 63]]
    k = np.array([1e-5, 3e-4, 0.004, 0.05, 0.18, 0.5])
    n_tau, lmax = 6000, 2500
    S = np.stack([W.synthetic_sources(k.size, n_tau, 100 + b) for b in range(2)])
    bg = records(H, params, n_tau)
    D = np.zeros((2, k.size, lmax - 1, 2), dtype=np.float32)
    H.h_project_mixed(2, bg.ctypes.data_as(P), S.ctypes.data_as(P), k.ctypes.data_as(P), k.size, lmax, 1.0,
                      D.ctypes.data_as(P))
    for b in range(2):
        lna, tau, w = O.nodes(params[b], n_tau)
        ref = O.project(tau, w, O.scalars(params[b])["tau0"], k, S[b], lmax)
        for i in range(k.size):
            for c in range(2):
                scale = np.abs(ref[i, :, c]).max()
                assert np.max(np.abs(D[b, i, :, c] - ref[i, :, c])) < 2e-5 * scale, (b, k[i], c)


def test_mixed_quadrature_against_oracle(H):
    # FP32 transfer functions: products rounded in FP32, Kahan-summed over
    # 400 k; within 1e-6 of each spectrum's largest value (measured 7e-8)
    rng = np.random.default_rng(12)
    params = W.BATCH64.params()[:2]
    k = W.log_k_nodes(400, 1e-5, 0.5)
    lmax = 300
    bg = records(H, params, 64)
    D = rng.normal(size=(2, k.size, lmax - 1, 2)).astype(np.float32)
    C = np.zeros((2, 3, lmax - 1))
    H.h_cl_mixed(2, bg.ctypes.data_as(P), D.ctypes.data_as(P), k.ctypes.data_as(P), k.size, lmax,
                 C.ctypes.data_as(P))
    for b in range(2):
        ref = O.cl(k, D[b].astype(np.float64), lmax, O.scalars(params[b])["A_s"], params[b][3])
        assert np.all(np.abs(C[b] - ref) <= 1e-6 * np.abs(ref).max(axis=1, keepdims=True)), b
