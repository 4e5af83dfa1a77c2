"""Pins of the oracle's forward sensitivities (oracle.sensitivity and the
*_sensitivity helpers: the oracle built over double complex, orc_real.h).
They are checked against what fixes them independently: closed forms of the
derived parameters, the exact dependence of C_l on A_s and n_s (App. B.4,
eq. c_ell_def with eq. PK_pivot), and Richardson-extrapolated central
differences of the double oracle for everything else (the root finds of the
thermal history and of the tau nodes included)."""
import numpy as np
import pytest

import oracle as O
from paper_2602_15104_gb300 import workload as W

P = W.BATCH16_GRAD.params()[0]
NAMES = ("omega_b", "omega_cdm", "h", "n_s", "ln10As", "tau_reio")


def richardson(f, j, rel):
    est = []
    for r in (2 * rel, rel):
        h = r * abs(P[j])
        pp, pm = P.copy(), P.copy()
        pp[j] += h
        pm[j] -= h
        est.append((np.asarray(f(pp)) - np.asarray(f(pm))) / (2 * h))
    return (4 * est[1] - est[0]) / 3


def test_derived_parameters_closed_forms():
    ob, oc, h, ns, las, tr = P
    d = {j: O.scalars_sensitivity(P, j) for j in range(6)}
    v = {f: x[0] for f, x in d[0].items()}
    exact = [  # (field, parameter, derivative)
        ("H0", 2, v["H0"] / h), ("Om_b", 0, 1 / h**2), ("Om_b", 2, -2 * v["Om_b"] / h), ("Om_c", 1, 1 / h**2),
        ("Om_c", 2, -2 * v["Om_c"] / h), ("Om_L", 1, -1 / h**2), ("A_s", 4, v["A_s"]), ("n_s", 3, 1.0),
        ("H0", 0, 0.0), ("R_nu", 2, 0.0), ("Om_g", 2, -2 * v["Om_g"] / h),
        ("nH0", 0, v["nH0"] / ob), ("nH0", 2, 0.0)]
    for f, j, ref in exact:
        got = d[j][f][1]
        assert abs(got - ref) <= 1e-13 * max(abs(ref), abs(v[f]) / abs(P[j])), (f, NAMES[j], got, ref)
    s = O.scalars(P)
    for f in O.SCALAR_FIELDS:
        assert d[0][f][0] == pytest.approx(s[f], rel=1e-12, abs=1e-300), f


@pytest.mark.parametrize("j", [0, 1, 2, 5])
def test_root_finds_carry_their_derivatives(j):
    # z_reion, the Saha switch, the HeIII switch, the tight-coupling start and
    # tau_0 are roots or integrals over roots: their sensitivities come from
    # the first-order imaginary correction of each bisection
    fields = ("z_reion", "lna_tc", "lna_sw", "lna_He3", "tau0")
    cs = O.scalars_sensitivity(P, j)
    fd = richardson(lambda p: [O.scalars(p)[f] for f in fields], j, 1e-4)
    for f, ref in zip(fields, fd):
        scale = max(abs(ref), 1e-4 * abs(cs[f][0]) / abs(P[j]))  # floor: derivatives that vanish
        assert abs(cs[f][1] - ref) <= 1e-6 * scale, (f, NAMES[j], cs[f][1], ref)


@pytest.mark.parametrize("recipe", [0, 1])
def test_node_sensitivities(recipe):
    # the nodes uniform in tau are roots of tau(ln a) = target, whose targets
    # move with tau(z = 900 or 300) and tau_0
    n = 200
    (lna, tau, w), (dlna, dtau, dw) = O.nodes_sensitivity(P, 2, n, recipe)
    fd = richardson(lambda p: np.array(O.nodes(p, n, node_recipe=recipe)), 2, 1e-4)
    for got, ref in ((dlna, fd[0]), (dtau, fd[1]), (dw, fd[2])):
        assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref).max()), np.abs(got - ref).max()
    assert np.abs(dlna).max() > 0.0 and np.abs(dtau).max() > 0.0


K = W.log_k_nodes(8, 1e-4, 0.15)
N_TAU, LMAX = 200, 120
OPTS = O.opts(lmax=8)


@pytest.fixture(scope="module")
def plain():
    return O.run(P, K, N_TAU, LMAX, OPTS)


def test_amplitude_and_tilt_sensitivities_are_exact(plain):
    C = plain["Cl"]
    v, d = O.sensitivity(P, 4, K, N_TAU, LMAX, OPTS)["Cl"]
    assert np.all(np.abs(v - C) <= 1e-10 * np.abs(C).max(axis=1, keepdims=True))
    assert np.all(np.abs(d - C) <= 1e-12 * np.abs(C).max(axis=1, keepdims=True))  # C_l is linear in A_s
    # dC_l/dn_s = 4 pi sum_k w_k A_s (k/k_p)^(n_s-1) ln(k/k_p) Delta_X Delta_Y
    D = plain["Delta"]
    x = np.log(K)
    wk = np.empty_like(x)
    wk[1:-1] = 0.5 * (x[2:] - x[:-2])
    wk[0], wk[-1] = 0.5 * (x[1] - x[0]), 0.5 * (x[-1] - x[-2])
    As = np.exp(P[4]) * 1e-10
    f = 4 * np.pi * wk * As * (K / 0.05) ** (P[3] - 1) * np.log(K / 0.05)
    ref = np.stack([np.einsum("k,kl->l", f, D[:, :, a] * D[:, :, b]) for a, b in ((0, 0), (0, 1), (1, 1))])
    _, dns = O.sensitivity(P, 3, K, N_TAU, LMAX, OPTS)["Cl"]
    assert np.all(np.abs(dns - ref) <= 1e-11 * np.abs(ref).max(axis=1, keepdims=True))


@pytest.mark.parametrize("j", [0, 1, 2, 5])
def test_sensitivities_match_richardson_differences(plain, j):
    _, d = O.sensitivity(P, j, K, N_TAU, LMAX, OPTS)["Cl"]
    fd = richardson(lambda p: O.run(p, K, N_TAU, LMAX, OPTS, want=("Cl",))["Cl"], j, 1e-4)
    err = np.abs(d - fd) / np.abs(fd).max(axis=1, keepdims=True)
    assert err.max() <= 2e-6, (NAMES[j], err.max())


@pytest.mark.parametrize("case", ["small", "full"])
def test_stored_forward_sensitivities_agree_with_the_stored_differences(case):
    # tests/golden/grad_forward_<case>.npz (complex step) against
    # grad_oracle_<case>.npz (Richardson-extrapolated central differences),
    # both written by tests/golden/make_grad_reference.py: per multipole they
    # agree to ~1e-7 of each spectrum's largest derivative; the differences
    # carry the jumps of the oracle's step counts, the complex step does not
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    f = np.load(os.path.join(here, f"grad_forward_{case}.npz"))
    d = np.load(os.path.join(here, f"grad_oracle_{case}.npz"))
    np.testing.assert_array_equal(f["params"], d["params"])
    np.testing.assert_array_equal(f["k"], d["k"])
    assert np.all(np.abs(f["Cl"] - d["Cl"]) <= 1e-10 * np.abs(d["Cl"]).max(axis=1, keepdims=True))
    for j in range(6):
        err = np.abs(f["dCl"][j] - d["dCl"][j]) / np.abs(f["dCl"][j]).max(axis=1, keepdims=True)
        assert err.max() <= 1e-6, (NAMES[j], err.max())
