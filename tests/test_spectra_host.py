"""CPU parity of the line-of-sight projection and k-quadrature kernels
(abcmb_spectra.cuh: project_kernel and cl_kernel, the calls abcmb_project,
abcmb_project_interp and abcmb_cl launch), built for the host with every CTA's
threads run as host threads (tests/host/warp_emu.h), against the oracle's
exact-Bessel projection (App. B.4 transfer functions, App. B.6 trapezoid in
tau) and its k-quadrature (App. B.4 eq. c_ell_def): the collapsed kernels
(A0 + l A1 + l^2 A2) j_l + B j_{l-1}, the upward recurrence and its Debye
cutoff, the power series below x = 1, the warp butterfly and the CTA's
atomic accumulation, the E factor, the ln k interpolation of the transfer
grid.  The same kernels run on a GB300 in tests/test_gpu_parity.py and
tests/test_gpu_transfer.py, at the same sizes and bars.
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
    so = str(tmp_path_factory.mktemp("spectra") / "libspectra.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "spectra_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_build_bg.argtypes = [P, ctypes.c_int, P]
    L.h_project.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, P]
    L.h_project_interp.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, P]
    L.h_cl.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int, P]
    return L


def records(H, params, n_tau):
    params = np.atleast_2d(params)
    r = np.zeros((len(params), H.h_bg_len(n_tau)))
    for b, p in enumerate(params):
        H.h_build_bg(np.ascontiguousarray(p).ctypes.data_as(P), n_tau, r[b].ctypes.data_as(P))
    return r


def assert_transfer_close(D, ref, bar):
    """|Delta - ref| below bar times each (k, T/E) row's largest |ref|."""
    for i in range(ref.shape[0]):
        for c in range(2):
            scale = np.abs(ref[i, :, c]).max()
            assert np.max(np.abs(D[i, :, c] - ref[i, :, c])) < bar * scale, (i, c)


def test_projection_against_oracle_at_full_size(H):
    # the 64-cosmology workload's grids: 6000 nodes, l <= 2500, k from
    # 1e-5 to 0.5 (series nodes, recurrence, cutoff); 1e-6 of each row's
    # peak, the GPU test's bar (measured 1.1e-7)
    params = W.BATCH64.params()[[0, 63]]
    k = np.array([1e-5, 3e-4, 0.004, 0.05, 0.18, 0.5])
    n_tau, lmax = 6000, 2500
    S = np.stack([W.synthetic_sources(k.size, n_tau, 100 + b) for b in range(2)])
    bg = records(H, params, n_tau)
    D = np.zeros((2, k.size, lmax - 1, 2))
    H.h_project(2, bg.ctypes.data_as(P), S.ctypes.data_as(P), k.ctypes.data_as(P), k.size, lmax, 1.0,
                D.ctypes.data_as(P))
    for b in range(2):
        lna, tau, w = O.nodes(params[b], n_tau)
        ref = O.project(tau, w, O.scalars(params[b])["tau0"], k, S[b], lmax)
        assert_transfer_close(D[b], ref, 1e-6)


def test_polarization_switch_scales_the_temperature_only(H):
    # scale_pol multiplies S_T2 in Delta_T alone (the E kernel reads S_P as is)
    params = W.BATCH64.params()[[5]]
    k = np.array([0.01, 0.1])
    n_tau, lmax = 600, 400
    S = W.synthetic_sources(k.size, n_tau, 7)[None]
    bg = records(H, params, n_tau)
    D1, D0 = np.zeros((2, 1, k.size, lmax - 1, 2))
    for D, s in ((D1, 1.0), (D0, 0.0)):
        H.h_project(1, bg.ctypes.data_as(P), S.ctypes.data_as(P), k.ctypes.data_as(P), k.size, lmax, s,
                    D.ctypes.data_as(P))
    # (the CTA's atomic additions may come in another order: rounding only)
    np.testing.assert_allclose(D0[..., 1], D1[..., 1], rtol=0, atol=1e-14 * np.abs(D1[..., 1]).max())
    lna, tau, w = O.nodes(params[0], n_tau)
    ref = O.project(tau, w, O.scalars(params[0])["tau0"], k, S[0], lmax, scale_pol=0.0)
    assert_transfer_close(D0[0], ref, 1e-6)
    assert np.abs(D0[0, :, :, 0] - D1[0, :, :, 0]).max() > 1e-3 * np.abs(D1[0, :, :, 0]).max()


def test_interpolating_projection_against_oracle(H):
    # smooth synthetic sources on 60 ODE nodes projected at 37 other k, some
    # outside the nodes (the end cubics extend); 1e-6 as on the GPU
    params = W.BATCH64.params()[[4, 50]]
    n_tau, lmax = 3000, 1200
    k = np.exp(np.linspace(np.log(2e-4), np.log(0.1), 60))
    kt = np.exp(np.linspace(np.log(1.5e-4), np.log(0.11), 37))
    S = np.stack([W.synthetic_sources_smooth(k, n_tau, 300 + b) for b in range(2)])
    bg = records(H, params, n_tau)
    D = np.zeros((2, kt.size, lmax - 1, 2))
    H.h_project_interp(2, bg.ctypes.data_as(P), S.ctypes.data_as(P), k.ctypes.data_as(P), k.size,
                       kt.ctypes.data_as(P), kt.size, lmax, 1.0, D.ctypes.data_as(P))
    for b in range(2):
        lna, tau, w = O.nodes(params[b], n_tau)
        ref = O.project(tau, w, O.scalars(params[b])["tau0"], kt, O.interp_sources(S[b], k, kt), lmax)
        assert_transfer_close(D[b], ref, 1e-6)


def test_k_quadrature_against_oracle(H):
    # random transfer functions: the trapezoid in ln k with the primordial
    # spectrum, compensated sums; to rounding (rtol 1e-12)
    rng = np.random.default_rng(11)
    params = W.BATCH64.params()[:3]
    k = W.log_k_nodes(37, 1e-4, 0.3)
    lmax = 300
    bg = records(H, params, 64)
    D = rng.normal(size=(3, k.size, lmax - 1, 2))
    C = np.zeros((3, 3, lmax - 1))
    H.h_cl(3, bg.ctypes.data_as(P), D.ctypes.data_as(P), k.ctypes.data_as(P), k.size, lmax, C.ctypes.data_as(P))
    for b in range(3):
        ref = O.cl(k, D[b], lmax, O.scalars(params[b])["A_s"], params[b][3])
        np.testing.assert_allclose(C[b], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
