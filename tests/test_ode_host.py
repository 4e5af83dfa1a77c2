"""CPU parity of the thread-per-mode perturbation solver (abcmb_ode.cuh, the
path abcmb_perturb takes for hierarchies above 63), built for the host,
against the oracle's CMB sources: the initial state, the IMEX extrapolation
integrator, node landing and the source functions of that path."""
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
    so = str(tmp_path_factory.mktemp("ode") / "libode.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "ode_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_build_bg.argtypes = [P, ctypes.c_int, P]
    L.h_integrate.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_double, P, P]
    L.h_integrate_batch.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P]
    return L


# the oracle's dense Radau solve is O(N^3) per step: a deep hierarchy only on a
# slow mode (30 s), the fast mode with a short one
@pytest.mark.parametrize("k,L", [(3e-4, 64), (0.02, 12), (0.1, 12)])
def test_sources_against_oracle(H, k, L):
    p = W.BATCH64.params()[11]
    n_tau = 200
    r = np.zeros(H.h_bg_len(n_tau))
    H.h_build_bg(np.ascontiguousarray(p).ctypes.data_as(P), n_tau, r.ctypes.data_as(P))
    S = np.zeros((n_tau, 3))
    steps = np.zeros(2, dtype=np.int32)
    assert H.h_integrate(r.ctypes.data_as(P), k, L, 1e-9, S.ctypes.data_as(P), steps.ctypes.data_as(P)) == 0
    ref = O.run(p, np.array([k]), n_tau, 40, O.opts(lmax=L), want=("S",))["S"][0]
    err = np.abs(S - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert np.all(err < 1e-6), (err, steps)


def test_interleaved_workspace_of_concurrent_modes(H):
    # perturb_kernel's layout: the modes' working vectors interleaved in one
    # workspace (stride M), the modes integrated at once; each equals the mode
    # integrated alone with its vectors contiguous, bit for bit
    p = W.BATCH64.params()[11]
    n_tau, L = 120, 70
    r = np.zeros(H.h_bg_len(n_tau))
    H.h_build_bg(p.ctypes.data_as(P), n_tau, r.ctypes.data_as(P))
    k = np.array([3e-4, 1e-3, 2e-3, 4e-3, 6e-3])
    S = np.zeros((k.size, n_tau, 3))
    st = np.full(k.size, -1, np.int32)
    H.h_integrate_batch(r.ctypes.data_as(P), k.ctypes.data_as(P), k.size, L, 1e-6, S.ctypes.data_as(P),
                        st.ctypes.data_as(P))
    assert np.all(st == 0)
    for i, kk in enumerate(k):
        S1, steps = np.zeros((n_tau, 3)), np.zeros(2, dtype=np.int32)
        assert H.h_integrate(r.ctypes.data_as(P), kk, L, 1e-6, S1.ctypes.data_as(P), steps.ctypes.data_as(P)) == 0
        np.testing.assert_array_equal(S[i], S1)
