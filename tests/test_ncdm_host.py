"""CPU parity of the massive-neutrino path (App. B.3 "Massive neutrinos",
App. C.6) against the oracle: the library's background builder and its
one-warp-per-mode forward, built for the host (one lane), on a cosmology with
one massive neutrino -- background scalars, tau nodes and the CMB sources."""
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
    so = str(tmp_path_factory.mktemp("ncdm") / "libncdm.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "ncdm_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_build_bg_m.argtypes = [P, I, D, P]
    L.h_fwd_m.argtypes = [P, D, I, I, D, P]
    return L


S_INDEX = dict(OML=6, RNU=7, TAU0=15, NTAU=18)


def record(H, p, n_tau, m):
    r = np.zeros(H.h_bg_len(n_tau))
    H.h_build_bg_m(np.ascontiguousarray(p).ctypes.data_as(P), n_tau, m, r.ctypes.data_as(P))
    assert r[0] == 0
    return r


@pytest.mark.parametrize("m", [0.06, 0.5])
def test_background_with_a_massive_neutrino(H, m):
    p = W.BATCH64.params()[7]
    n_tau = 400
    r = record(H, p, n_tau, m)
    s = O.scalars(p, m_ncdm=m)
    assert abs(r[S_INDEX["OML"]] - s["Om_L"]) < 1e-12
    assert abs(r[S_INDEX["RNU"]] / s["R_nu"] - 1) < 1e-12
    assert abs(r[S_INDEX["TAU0"]] / s["tau0"] - 1) < 1e-9
    lna, tau, w = O.nodes(p, n_tau, m_ncdm=m)
    nodes = r[64 + 28 * 18433: 64 + 28 * 18433 + 8 * n_tau].reshape(n_tau, 8)
    np.testing.assert_allclose(nodes[:, 0], lna, rtol=0, atol=1e-9)
    # the neutrino's relativistic-to-matter transition enters the conformal-time
    # integrand; the two quadratures agree to a few 1e-9
    np.testing.assert_allclose(nodes[:, 1], tau, rtol=1e-8)


@pytest.mark.parametrize("k", [3e-4, 0.01, 0.08])
def test_sources_with_a_massive_neutrino(H, k):
    p = W.BATCH64.params()[7]
    m, n_tau, L, Lm = 0.1, 300, 8, 6
    r = record(H, p, n_tau, m)
    S = np.zeros((n_tau, 3))
    assert H.h_fwd_m(r.ctypes.data_as(P), k, L, Lm, 1e-9, S.ctypes.data_as(P)) == 0
    ref = O.run(p, np.array([k]), n_tau, 40, O.opts(lmax=L, m_ncdm=m, lmax_ncdm=Lm), want=("S",))["S"][0]
    err = np.abs(S - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert np.all(err < 1e-6), err
    # and the neutrino mass is visible: the massless run differs well beyond that
    ref0 = O.run(p, np.array([k]), n_tau, 40, O.opts(lmax=L), want=("S",))["S"][0]
    assert (np.abs(ref0 - ref).max(axis=0) / np.abs(ref).max(axis=0)).max() > 1e-4
