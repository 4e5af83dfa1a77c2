"""CPU parity of the library's massless-neutrino background and per-mode
forward (abcmb_bg.cuh and the one-warp-per-mode forward of abcmb_adjoint.cuh,
built for the host with one lane) against the oracle: the background record
(scalars, ln a table, tau nodes) and the CMB sources of single modes.  The
GPU tests check the same record and the four-lane kernel's sources on the
device; these run without one."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2602_15104_gb300 import workload as W

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
D = ctypes.c_double
I = ctypes.c_int


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("hostpar") / "libhostpar.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "ncdm_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_build_bg_m.argtypes = [P, I, D, P]
    L.h_build_bg_r.argtypes = [P, I, D, I, P]
    L.h_fwd_m.argtypes = [P, D, I, I, D, P]
    return L


def record(H, p, n_tau, recipe=0):
    r = np.zeros(H.h_bg_len(n_tau))
    H.h_build_bg_r(np.ascontiguousarray(p).ctypes.data_as(P), n_tau, 0.0, recipe, r.ctypes.data_as(P))
    return r


@pytest.mark.parametrize("b,recipe", [(0, 0), (63, 0), (17, 1)])
def test_background_record(H, b, recipe):
    from paper_2602_15104_gb300 import abcmb as A
    p = W.BATCH64.params()[b]
    n_tau = 2000
    scal, tab, nodes = A.bg_view(torch.tensor(record(H, p, n_tau, recipe)), n_tau)
    assert scal["STATUS"] == 0
    s = O.scalars(p)
    for gk, ok in [("H0", "H0"), ("OMB", "Om_b"), ("OMC", "Om_c"), ("OMG", "Om_g"), ("OML", "Om_L"),
                   ("RNU", "R_nu"), ("NH0", "nH0"), ("AS", "A_s"), ("TAU0", "tau0")]:
        assert abs(scal[gk] / s[ok] - 1) < 1e-12, gk
    for gk, ok in [("ZREION", "z_reion"), ("LNA_TC", "lna_tc"), ("LNA_SW", "lna_sw")]:
        assert abs(scal[gk] - s[ok]) < 1e-9 * abs(s[ok]), gk
    lna, tau, w = O.nodes(p, n_tau, node_recipe=recipe)
    np.testing.assert_allclose(nodes[:, 0], lna, rtol=0, atol=1e-9)
    np.testing.assert_allclose(nodes[:, 1], tau, rtol=1e-10)
    np.testing.assert_allclose(nodes[:, 2], w, rtol=1e-8)
    bg = O.background(p, lna)
    for c, name in [(3, "g"), (4, "dg"), (6, "Hc"), (7, "dHc")]:
        assert np.max(np.abs(nodes[:, c] - bg[name])) < 1e-8 * np.max(np.abs(bg[name])), name
    np.testing.assert_allclose(nodes[:, 5], np.exp(-bg["kappa"]), rtol=1e-8, atol=1e-14)
    lt = A.BG_LNA0 + np.arange(A.BG_NLNA) / A.BG_PER_UNIT
    sel = np.arange(500, A.BG_NLNA, 1013)
    ob = O.background(p, lt[sel])
    for c, name in [(0, "nuT"), (2, "tau"), (4, "cs2"), (7, "xe")]:
        np.testing.assert_allclose(tab[sel, c], ob[name], rtol=1e-9, err_msg=name)


@pytest.mark.parametrize("k,recipe", [(2e-4, 0), (0.01, 0), (0.1, 0), (0.01, 1)])
def test_sources_of_single_modes(H, k, recipe):
    p = W.BATCH64.params()[5]
    n_tau, L = 300, 8
    r = record(H, p, n_tau, recipe)
    S = np.zeros((n_tau, 3))
    assert H.h_fwd_m(r.ctypes.data_as(P), k, L, 0, 1e-9, S.ctypes.data_as(P)) == 0
    ref = O.run(p, np.array([k]), n_tau, 40, O.opts(lmax=L, node_recipe=recipe), want=("S",))["S"][0]
    err = np.abs(S - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert np.all(err < 1e-6), err


@pytest.mark.parametrize("recipe", [0, 1])
@pytest.mark.parametrize("n_tau", [8, 9, 13, 101])
def test_nodes_of_small_and_ragged_counts(H, n_tau, recipe):
    # the segment sizes round down; every count from the minimum of 8 gives
    # strictly increasing nodes before tau_0 that match the oracle's
    p = W.BATCH64.params()[3]
    r = record(H, p, n_tau, recipe)
    assert r[0] == 0  # status
    nodes = r[64 + 28 * 18433: 64 + 28 * 18433 + 8 * n_tau].reshape(n_tau, 8)
    lna, tau, w = O.nodes(p, n_tau, node_recipe=recipe)
    assert np.all(np.diff(nodes[:, 1]) > 0) and nodes[-1, 1] < O.scalars(p)["tau0"]
    np.testing.assert_allclose(nodes[:, 0], lna, rtol=0, atol=1e-9)
    np.testing.assert_allclose(nodes[:, 2], w, rtol=1e-8)


def test_ode_table_cubics_are_the_hermite_interpolants(H):
    # the record's polynomial section (read by the four-lane ODE kernel) holds,
    # per interval and quantity, the cubic Hermite interpolant of the (value,
    # d/dln a) pairs of the ODE table: compare at points inside intervals
    from paper_2602_15104_gb300 import abcmb as A
    n_tau = 400
    r = record(H, W.BATCH64.params()[5], n_tau)
    assert r.size == A.BG_NODES + 8 * n_tau + A.BG_ODEPOLY_DOUBLES
    pairs = r[A.BG_ODETAB:A.BG_NODES].reshape(A.BG_NLNA, 10, 2)
    poly = r[A.BG_NODES + 8 * n_tau:].reshape(A.BG_NLNA - 1, 10, 4)
    rng = np.random.default_rng(2)
    dx = 1.0 / 1024
    for j in np.concatenate([[0, A.BG_NLNA - 2], rng.integers(0, A.BG_NLNA - 1, 200)]):
        for u in (0.0, 0.31, 0.77, 1.0):
            h00, h10 = (1 + 2 * u) * (1 - u) ** 2, u * (1 - u) ** 2
            h01, h11 = u * u * (3 - 2 * u), u * u * (u - 1)
            v0, d0 = pairs[j, :, 0], pairs[j, :, 1]
            v1, d1 = pairs[j + 1, :, 0], pairs[j + 1, :, 1]
            herm = h00 * v0 + h10 * dx * d0 + h01 * v1 + h11 * dx * d1
            c = poly[j]
            cub = c[:, 0] + u * (c[:, 1] + u * (c[:, 2] + u * c[:, 3]))
            scale = np.maximum(np.abs(v0), np.abs(v1))
            assert np.all(np.abs(cub - herm) <= 2e-15 * scale + 1e-300), (j, u)
