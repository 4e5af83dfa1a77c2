"""CPU checks of the four-lane ODE kernel's extrapolation tables
(abcmb_ode_quad.cuh, evaluated on the host by tests/host/extrap_harness.cu):
the weighted sums of a step's column values reproduce the Aitken-Neville
tableau they replace -- the extrapolated value T_jj and the error estimate
T_jj - T_j,j-1 -- for the implicit-Euler sequence n_j = j (expansion in h) and
the Gragg sequence n_j = 2j (expansion in h^2), and extrapolate polynomials in
the expansion variable exactly."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = str(tmp_path_factory.mktemp("ext") / "libext.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-Xcompiler",
                           "-fPIC", "--expt-relaxed-constexpr", "-shared", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "extrap_harness.cu"), "-o", so])
    L = ctypes.CDLL(so)
    lam, mu, inv = np.zeros((2, 8, 8)), np.zeros((2, 8, 8)), np.zeros(15)
    K = L.h_ext_tables(lam.ctypes.data_as(P), mu.ctypes.data_as(P), inv.ctypes.data_as(P))
    assert K == 7
    return lam, mu, inv


def neville(z, g):
    """Aitken-Neville tableau of column values z[0..J-1]: T[j][s] with the
    factor 1 / ((n_j / n_{j-s})^p - 1), p = 1 for n_j = j, p = 2 for n_j = 2j."""
    J = len(z)
    T = [[0.0] * J for _ in range(J)]
    for j in range(J):
        T[j][0] = z[j]
        for s in range(1, j + 1):
            n_j, n_js = (j + 1), (j + 1 - s)
            r = (n_j / n_js) ** (2 if g else 1)
            T[j][s] = T[j][s - 1] + (T[j][s - 1] - T[j - 1][s - 1]) / (r - 1.0)
    return T


@pytest.mark.parametrize("g", [0, 1])
def test_weighted_sums_are_the_neville_tableau(tables, g):
    lam, mu, _ = tables
    rng = np.random.default_rng(3 + g)
    for _ in range(20):
        z = 1.0 + 1e-3 * rng.normal(size=7)  # nearly equal columns, as in a converging step
        T = neville(list(z), g)
        for j in range(1, 8):
            val = sum(lam[g, j, i] * z[i - 1] for i in range(1, j + 1))
            assert abs(val - T[j - 1][j - 1]) <= 2e-12, (g, j)  # weights up to ~400: rounding ~1e-13
            if j >= 2:
                err = sum(mu[g, j, i] * z[i - 1] for i in range(1, j + 1))
                assert abs(err - (T[j - 1][j - 1] - T[j - 1][j - 2])) <= 2e-12, (g, j)


@pytest.mark.parametrize("g", [0, 1])
def test_extrapolation_is_exact_for_polynomials(tables, g):
    # column j from n_j substeps; the error expansion is in x = 1/n (implicit
    # Euler) or 1/n^2 (Gragg): a polynomial of degree < j in x is reproduced
    # at x = 0 exactly, and the weights sum to one
    lam, _, inv = tables
    rng = np.random.default_rng(11 + g)
    x = np.array([(1.0 / (2 * i)) ** 2 if g else 1.0 / i for i in range(1, 8)])
    for j in range(1, 8):
        assert abs(lam[g, j, 1:j + 1].sum() - 1.0) <= 1e-12
        c = rng.normal(size=j)
        z = np.polyval(c[::-1], x[:j])
        assert abs(lam[g, j, 1:j + 1] @ z - c[0]) <= 1e-10 * np.abs(c).max(), (g, j)
    np.testing.assert_allclose(inv[1:], 1.0 / np.arange(1, 15), rtol=0, atol=0)
