"""CPU parity of the lensing kernels (abcmb_lens_kernels.cuh: lens_kernel,
lens_finish and cl_psi_kernel, behind abcmb_lens and abcmb_cl_psi), built for
the host with every CTA's threads run as host threads (tests/host/warp_emu.h),
against the oracle (App. B.5): the lensed spectra from the correlation-function
method, summed over the Gauss-Legendre nodes by warp shuffles and atomic
additions, and the Limber lensing potential.  The same kernels run on a GB300
in tests/test_gpu_lensing.py and tests/test_gpu_limber.py."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import lensing as LZ
from paper_2602_15104_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
I = ctypes.c_int
BG_LEN = lambda n_tau: 64 + 28 * (18 * 1024 + 1) + 8 * n_tau + 40 * 18 * 1024  # ABCMB_BG_LEN
NODES = 64 + 28 * (18 * 1024 + 1)  # ABCMB_BG_NODES
S = dict(H0=1, OMB=2, OMC=3, AS=10, NS=11, TAU0=15, NTAU=18)  # ABCMB_S_*


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("lensk") / "liblensk.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "lens_kernels_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_lens.argtypes = [I, P, I, P, I, I, P]
    L.h_cl_psi.argtypes = [I, P, ctypes.c_long, P, P, I, I, P]
    return L


def ptr(a):
    return a.ctypes.data_as(P)


def test_lensed_spectra_against_oracle(H):
    from test_lensing_host import spectra
    L, lout = 400, 300
    sp = [spectra(L, 7 + b) for b in range(2)]
    Cl = np.ascontiguousarray(np.stack([np.stack([s[0][2:], s[2][2:], s[1][2:]]) for s in sp]))
    Cpsi = np.ascontiguousarray(np.stack([s[3][2:] for s in sp]))
    out = np.zeros((2, 4, lout - 1))
    H.h_lens(2, ptr(Cl), L, ptr(Cpsi), lout, L + 100, ptr(out))
    for b, (ctt, cee, cte, cpsi) in enumerate(sp):
        TT, EE, TE, BB = LZ.lensed_cls(ctt, cee, cte, cpsi, lout, n_mu=L + 100)
        for c, ref, scale in [(0, TT, ctt), (2, EE, cee), (1, TE, np.sqrt(ctt * cee)), (3, BB, cee)]:
            assert np.abs(out[b, c] - ref[2:]).max() < 1e-10 * np.abs(scale).max(), (b, c)


def test_limber_potential_against_oracle(H):
    # the oracle's nodes, background and delta_m in a record: the kernel's
    # Limber sum against the oracle's C_l^psi, same quadrature, rounding only
    p = W.SMALL_TT.params()[0]
    n_tau, lmax = 300, 150
    k = np.exp(np.linspace(np.log(1e-4), np.log(0.15), 24))
    o = O.opts(lmax=8)
    ref = LZ.cl_psi(p, k, n_tau, lmax, o)
    lna, tau, w = O.nodes(p, n_tau)
    bg = O.background(p, lna)
    sc = O.scalars(p)
    rec = np.zeros((1, BG_LEN(n_tau)))
    rec[0, S["H0"]], rec[0, S["OMB"]], rec[0, S["OMC"]] = sc["H0"], sc["Om_b"], sc["Om_c"]
    rec[0, S["AS"]], rec[0, S["NS"]], rec[0, S["TAU0"]], rec[0, S["NTAU"]] = sc["A_s"], sc["n_s"], sc["tau0"], n_tau
    nodes = rec[0, NODES:NODES + 8 * n_tau].reshape(n_tau, 8)
    nodes[:, 0], nodes[:, 1], nodes[:, 2], nodes[:, 3], nodes[:, 6] = lna, tau, w, bg["g"], bg["Hc"]
    dm = np.ascontiguousarray(O.delta_m_nodes(p, k, n_tau, o))
    out = np.zeros((1, lmax - 1))
    H.h_cl_psi(1, ptr(rec), rec.shape[1], ptr(dm), ptr(k), k.size, lmax, ptr(out))
    np.testing.assert_allclose(out[0], ref[2:], rtol=1e-10)
