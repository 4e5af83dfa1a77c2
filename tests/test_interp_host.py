"""CPU checks of the library's interpolation in ln k (abcmb_interp.cuh built
for the host), used on the GPU by the projection onto the transfer k grid and
by the Limber lensing potential: against the oracle's source interpolation and
against its exactness for quadratics in ln k."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("interp") / "libinterp.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "interp_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_interp.argtypes = [P, ctypes.c_int, P, P, ctypes.c_int, P]
    return L


def interp(H, kn, f, kt):
    kn, f, kt = (np.ascontiguousarray(a, dtype=np.float64) for a in (kn, f, kt))
    out = np.zeros(kt.size)
    H.h_interp(kn.ctypes.data_as(P), kn.size, f.ctypes.data_as(P), kt.ctypes.data_as(P), kt.size,
               out.ctypes.data_as(P))
    return out


@pytest.mark.parametrize("n", [4, 5, 37])
def test_matches_the_oracle_interpolation(H, n):
    rng = np.random.default_rng(n)
    kn = np.sort(np.exp(rng.uniform(np.log(1e-5), np.log(0.5), n)))  # uneven spacing
    f = rng.normal(size=n)
    kt = np.exp(rng.uniform(np.log(kn[0]), np.log(kn[-1]), 300))
    kt = np.concatenate([kt, kn])  # the nodes themselves
    ref = O.interp_sources(np.broadcast_to(f[:, None, None], (n, 1, 3)).copy(), kn, kt)[:, 0, 0]
    np.testing.assert_allclose(interp(H, kn, f, kt), ref, rtol=1e-12, atol=1e-12 * np.abs(f).max())


def test_exact_for_quadratics_in_lnk_inside_and_beyond_the_nodes(H):
    kn = np.exp(np.sort(np.random.default_rng(1).uniform(-8.0, 0.0, 12)))
    q = lambda k: 0.3 - 1.7 * np.log(k) + 0.45 * np.log(k) ** 2
    kt = np.exp(np.linspace(-9.0, 1.0, 401))  # the end cubics extend outside
    # exact up to rounding, which the divided differences of close random nodes and
    # the extrapolated cubics amplify to ~1e-9 of the largest value
    np.testing.assert_allclose(interp(H, kn, q(kn), kt), q(kt), rtol=0, atol=1e-8 * np.abs(q(kt)).max())
