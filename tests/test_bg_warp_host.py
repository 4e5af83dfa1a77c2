"""CPU check of the background builder's warp split (abcmb_bg.cuh): the
record background_kernel writes with the 32 lanes of a warp (its Gauss-Legendre
sums, chunked cumulative sums and scans split over the lanes, through the warp
emulation of tests/host/warp_emu.h) equals the one-lane host build, which
tests/test_host_parity.py and tests/test_ncdm_host.py hold against the oracle,
to rounding: the lanes add the same terms in another order.  The ODE table's
cubic section is compared through the cubics it defines (its highest
coefficients are differences of nearly equal values, so the coefficients
themselves carry the rounding amplified)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2602_15104_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
NLNA = 18 * 1024 + 1  # ABCMB_BG_NLNA
TABLE, ODETAB = 64, 64 + 8 * NLNA  # ABCMB_BG_TABLE, ABCMB_BG_ODETAB
NODES = ODETAB + 20 * NLNA  # ABCMB_BG_NODES


def _build(tmp_path_factory, name, src, extra=()):
    so = str(tmp_path_factory.mktemp(name) / f"lib{name}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", *extra, "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", src), "-o", so])
    return ctypes.CDLL(so)


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    warp = _build(tmp_path_factory, "bgwarp", "bg_warp_harness.cpp", ("-pthread",))
    warp.h_bg_len.restype = ctypes.c_long
    warp.h_build_bg_warp.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P]
    lane = _build(tmp_path_factory, "bglane", "ncdm_harness.cpp")
    lane.h_build_bg_r.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P]
    return warp, lane


@pytest.mark.parametrize("b,recipe,m_ncdm", [(0, 0, 0.0), (63, 1, 0.0), (17, 0, 0.06)])
def test_warp_record_equals_the_one_lane_record(libs, b, recipe, m_ncdm):
    warp, lane = libs
    p = np.ascontiguousarray(W.BATCH64.params()[b])
    n_tau = 2000
    r1 = np.zeros(warp.h_bg_len(n_tau))
    r32 = np.full_like(r1, np.nan)
    lane.h_build_bg_r(p.ctypes.data_as(P), n_tau, m_ncdm, recipe, r1.ctypes.data_as(P))
    warp.h_build_bg_warp(p.ctypes.data_as(P), n_tau, m_ncdm, recipe, r32.ctypes.data_as(P))
    assert r1[0] == 0 and r32[0] == 0  # status
    again = np.full_like(r1, np.nan)  # a second build repeats the first bit for bit
    warp.h_build_bg_warp(p.ctypes.data_as(P), n_tau, m_ncdm, recipe, again.ctypes.data_as(P))
    np.testing.assert_array_equal(again, r32)
    np.testing.assert_allclose(r32[:TABLE], r1[:TABLE], rtol=1e-14, atol=0)
    poly = NODES + 8 * n_tau
    for name, a, e, ncol in [("table", TABLE, ODETAB, 8), ("ode table", ODETAB, NODES, 20), ("nodes", NODES, poly, 8)]:
        X1, X32 = r1[a:e].reshape(-1, ncol), r32[a:e].reshape(-1, ncol)
        err = (np.abs(X32 - X1) / np.maximum(np.abs(X1).max(axis=0), 1e-300)).max()
        assert err < 1e-12, (name, err)
    # the cubics c0 + c1 u + c2 u^2 + c3 u^3 on u in [0, 1] move by at most
    # sum |dc_i|, against each quantity's largest value (measured <= 2.4e-15)
    C1 = r1[poly:poly + 40 * (NLNA - 1)].reshape(NLNA - 1, 10, 4)
    C32 = r32[poly:poly + 40 * (NLNA - 1)].reshape(NLNA - 1, 10, 4)
    shift = np.abs(C32 - C1).sum(axis=2).max(axis=0) / np.abs(C1[:, :, 0]).max(axis=0)
    assert np.all(shift < 1e-13), shift
    assert r32.size == poly + 40 * (NLNA - 1) and not np.isnan(r32).any()
