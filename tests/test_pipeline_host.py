"""The whole hot path on the CPU: the calls Pipeline.run makes on the GPU
(the background builder on one warp per cosmology, perturb_quad_kernel,
project_kernel, cl_kernel, and for the mixed form project_mixed_kernel and
cl_mixed_kernel), with their grids and arguments, built for the host
with every CTA's threads run as host threads (tests/host/warp_emu.h), against
the oracle's C_l (App. B.4 eq. c_ell_def) on the single-cosmology TT workload's
grids (l <= 500, hierarchies 12, 2000 tau nodes) at every fourth of its 100 k
up to 0.1 /Mpc (k chi* ~ 1400 there, past every l kept).  The GPU runs the same
kernels on the full workload in tests/test_gpu_parity.py.
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
D = ctypes.c_double
I = ctypes.c_int


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("pipeline") / "libpipe.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "pipeline_harness.cpp"), "-o", so])
    H = ctypes.CDLL(so)
    H.h_bg_len.restype = ctypes.c_long
    H.h_pipeline.argtypes = [I, P, P, I, I, I, I, D, D, P, P, P, P, P]
    return H


def test_hot_path_kernels_on_the_host_against_the_oracle(H):
    wl = W.SMALL_TT
    k = wl.k()[::4]
    params, k = np.ascontiguousarray(wl.params()), np.ascontiguousarray(k[k <= 0.1])
    n_tau, lmax, L = wl.n_tau, wl.l_max_cl, wl.l_max_hier
    bg = np.zeros((1, H.h_bg_len(n_tau)))
    S = np.zeros((1, k.size, n_tau, 3))
    Dl = np.zeros((1, k.size, lmax - 1, 2))
    C = np.zeros((1, 3, lmax - 1))
    st = np.full((1, k.size), -1, np.int32)
    ptr = lambda a: a.ctypes.data_as(P)
    # the library's defaults: rtol 1e-6, error floor 1e-4
    H.h_pipeline(1, ptr(params), ptr(k), k.size, L, n_tau, lmax, 1e-6, 1e-4, ptr(bg), ptr(S), ptr(Dl), ptr(C),
                 ptr(st))
    assert bg[0, 0] == 0 and np.all(st == 0)
    ref = O.run(params[0], k, n_tau, lmax, O.opts(lmax=L), want=("Cl",))["Cl"]
    tt = np.abs(C[0, 0] - ref[0]) / np.abs(ref[0])
    ee = np.abs(C[0, 2] - ref[2]) / np.abs(ref[2])
    te = np.abs(C[0, 1] - ref[1]) / np.sqrt(np.abs(ref[0] * ref[2]))
    # the FP64 bar, 1e-5 (measured 8.7e-7 TT, 6.3e-7 TE, 2.0e-7 EE)
    assert tt.max() < 1e-5 and te.max() < 1e-5 and ee.max() < 1e-5, (tt.max(), te.max(), ee.max())
    # the mixed-precision end (FP32 projection and quadrature) on the same sources: the 1e-4 bar
    H.h_mixed_tail.argtypes = [I, P, P, P, I, I, I, P, P]
    D32, C32 = np.zeros((1, k.size, lmax - 1, 2), np.float32), np.zeros((1, 3, lmax - 1))
    H.h_mixed_tail(1, ptr(bg), ptr(S), ptr(k), k.size, n_tau, lmax, ptr(D32), ptr(C32))
    tt = np.abs(C32[0, 0] - ref[0]) / np.abs(ref[0])
    ee = np.abs(C32[0, 2] - ref[2]) / np.abs(ref[2])
    te = np.abs(C32[0, 1] - ref[1]) / np.sqrt(np.abs(ref[0] * ref[2]))
    assert tt.max() < 1e-4 and te.max() < 1e-4 and ee.max() < 1e-4, (tt.max(), te.max(), ee.max())


def test_the_smoke_run_on_the_host(H):
    """The configuration __graft_entry__.smoke() runs on the GPU -- two seeded
    cosmologies, eight k on [1e-3, 0.05], hierarchies 8, 256 tau nodes,
    l <= 64, rtol 1e-9 -- through the same kernels on the host, held to the
    same check: C_l within 1e-5 of the oracle (measured 7.7e-8)."""
    B, n_tau, lmax, L = 2, 256, 64, 8
    params = np.ascontiguousarray(W.draw_cosmologies(B, 20260101))
    k = np.ascontiguousarray(W.log_k_nodes(8, 1e-3, 0.05))
    bg = np.zeros((B, H.h_bg_len(n_tau)))
    S = np.zeros((B, k.size, n_tau, 3))
    Dl = np.zeros((B, k.size, lmax - 1, 2))
    C = np.zeros((B, 3, lmax - 1))
    st = np.full((B, k.size), -1, np.int32)
    ptr = lambda a: a.ctypes.data_as(P)
    H.h_pipeline(B, ptr(params), ptr(k), k.size, L, n_tau, lmax, 1e-9, 1e-4, ptr(bg), ptr(S), ptr(Dl), ptr(C),
                 ptr(st))
    assert np.all(bg[:, 0] == 0) and np.all(st == 0)
    for b in range(B):
        ref = O.run(params[b], k, n_tau, lmax, O.opts(lmax=L), want=("Cl",))["Cl"]
        tt = np.abs(C[b, 0] - ref[0]) / np.abs(ref[0])
        ee = np.abs(C[b, 2] - ref[2]) / np.abs(ref[2])
        te = np.abs(C[b, 1] - ref[1]) / np.sqrt(ref[0] * ref[2])
        assert max(tt.max(), te.max(), ee.max()) < 1e-5, (b, tt.max(), te.max(), ee.max())
