"""CPU parity of the library's lensing math (abcmb_lensing.cuh built for the
host) against the oracle's lensed spectra (App. B.5)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import lensing as LZ

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("lens") / "liblens.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "lensing_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_lens.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    L.h_cl_psi.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, ctypes.c_int,
                           ctypes.c_double, ctypes.c_double, ctypes.c_int, P]
    return L


def spectra(L, seed):
    rng = np.random.default_rng(seed)
    l = np.arange(L + 1.0)
    on = l >= 2
    ph = rng.uniform(0, 2 * np.pi, 3)
    ctt = np.where(on, 1e-9 * 6e3 / (l * (l + 1) + 10) * (1.3 + np.cos(l / 40 + ph[0])) * np.exp(-(l / 900) ** 2), 0)
    cee = np.where(on, 1e-9 * 80 / (l * (l + 1) + 10) * (1.3 + np.sin(l / 40 + ph[1])) * (l / 300) ** 1.5
                   * np.exp(-(l / 900) ** 2), 0)
    cte = np.where(on, 0.4 * np.sqrt(ctt * cee) * np.cos(l / 60 + ph[2]), 0)
    lp = np.maximum(l, 1)
    cpsi = np.where(on, 2e-7 * 2 * np.pi / (lp * (lp + 1)) ** 2 * (lp / (lp + 40)), 0)
    return ctt, cee, cte, cpsi


@pytest.mark.parametrize("L,lout", [(300, 250), (1200, 1000)])
def test_lensed_spectra_match_oracle(H, L, lout):
    ctt, cee, cte, cpsi = spectra(L, L)
    n_mu = L + 100
    TT, EE, TE, BB = LZ.lensed_cls(ctt, cee, cte, cpsi, lout, n_mu=n_mu)
    Cl = np.ascontiguousarray(np.stack([ctt[2:], cte[2:], cee[2:]]))
    out = np.zeros((4, lout - 1))
    H.h_lens(Cl.ctypes.data_as(P), np.ascontiguousarray(cpsi[2:]).ctypes.data_as(P), L, lout, n_mu,
             out.ctypes.data_as(P))
    for got, ref, scale in [(out[0], TT[2:], ctt[2:lout + 1]), (out[2], EE[2:], cee[2:lout + 1]),
                            (out[1], TE[2:], np.sqrt(ctt * cee)[2:lout + 1]), (out[3], BB[2:], cee[2:lout + 1])]:
        assert np.all(np.abs(got - ref) <= 1e-10 * np.abs(scale).max() + 1e-9 * np.abs(scale)), \
            np.abs(got - ref).max()
    # lensing changed them (well beyond the tolerance): B modes from E, E smoothed
    assert out[3].max() > 1e-4 * cee.max()
    assert np.abs(out[2] - cee[2:lout + 1]).max() > 1e-4 * cee.max()


def test_limber_lensing_potential_matches_oracle(H):
    # the library's Limber sum on the oracle's nodes, background and delta_m
    # against the oracle's C_l^psi (App. B.5): same quadrature, so rounding only
    import oracle as O
    from paper_2602_15104_gb300 import workload as W
    p = W.SMALL_TT.params()[0]
    n_tau, lmax = 300, 150
    k = np.exp(np.linspace(np.log(1e-4), np.log(0.15), 24))
    o = O.opts(lmax=8)
    ref = LZ.cl_psi(p, k, n_tau, lmax, o)
    lna, tau, w = O.nodes(p, n_tau)
    bg = O.background(p, lna)
    sc = O.scalars(p)
    nodes = np.zeros((n_tau, 8))
    nodes[:, 0], nodes[:, 1], nodes[:, 2], nodes[:, 3], nodes[:, 6] = lna, tau, w, bg["g"], bg["Hc"]
    dm = np.ascontiguousarray(O.delta_m_nodes(p, k, n_tau, o))
    out = np.zeros(lmax - 1)
    H.h_cl_psi(nodes.ctypes.data_as(P), n_tau, sc["tau0"], sc["Om_b"] + sc["Om_c"], sc["H0"], dm.ctypes.data_as(P),
               k.ctypes.data_as(P), k.size, sc["A_s"], sc["n_s"], lmax, out.ctypes.data_as(P))
    assert np.all(np.isfinite(out)) and out.min() > 0
    np.testing.assert_allclose(out, ref[2:], rtol=1e-10)
