"""Pins of the oracle's lensing (App. B.5): Wigner functions against closed
forms and a library routine; the Limber integral against a closed form; the
lensed spectra of the cited correlation-function method against the exact
first-order lensing of the spectra, computed independently here from the
harmonic convolution (full sky, Wigner-3j couplings obtained by the
three-d-function integral identity), and the unlensed limit."""
import numpy as np
import pytest

from oracle import lensing as LZ


def test_wigner_d_closed_forms():
    from scipy.special import eval_legendre
    mu = np.linspace(-0.999, 0.999, 41)
    np.testing.assert_allclose(LZ.wigner_d(40, mu, 0, 0)[37], eval_legendre(37, mu), atol=1e-13)
    np.testing.assert_allclose(LZ.wigner_d(5, mu, 2, 2)[2], ((1 + mu) / 2) ** 2, atol=1e-15)
    np.testing.assert_allclose(LZ.wigner_d(5, mu, 2, -2)[2], ((1 - mu) / 2) ** 2, atol=1e-15)
    np.testing.assert_allclose(LZ.wigner_d(5, mu, 1, 0)[1], -np.sqrt((1 - mu * mu) / 2), atol=1e-15)
    np.testing.assert_allclose(LZ.wigner_d(5, mu, 2, 0)[2], np.sqrt(3.0 / 8.0) * (1 - mu * mu), atol=1e-15)


def test_wigner_d_against_sympy_and_orthogonality():
    sp = pytest.importorskip("sympy")
    from sympy.physics.quantum.spin import Rotation
    b = sp.Symbol("b")
    mu = np.array([-0.7, -0.1, 0.4, 0.95])
    for m, n in [(3, 1), (3, -3), (4, -4), (-2, 4), (1, -1)]:
        f = sp.lambdify(b, Rotation.d(6, m, n, b).doit())
        ref = np.array([float(f(np.arccos(x))) for x in mu])
        np.testing.assert_allclose(LZ.wigner_d(6, mu, m, n)[6], ref, atol=1e-14)
    # orthogonality: int d^l_mn d^l'_mn dmu = 2 delta_ll' / (2l + 1)
    x, w = np.polynomial.legendre.leggauss(400)
    d = LZ.wigner_d(300, x, 2, -2)
    G = (d * w) @ d.T
    ref = np.diag(np.where(np.arange(301) >= 2, 2.0 / (2 * np.arange(301) + 1), 0.0))
    assert np.abs(G - ref).max() < 1e-12


def test_limber_integral_closed_form():
    # P_psi(k) = c / k^2 makes the integrand c chi (chi* - chi)^2 / ((l+1/2)^2 chi*^2),
    # zero at chi = 0: C_l = 8 pi^2 / (l+1/2)^5 c chi*^2 / 12
    chi_star = 1.0e4
    chi = np.linspace(chi_star, 0.0, 20001)[:-1]  # 0 < chi <= chi*
    w = np.full(chi.size, chi_star / 20000)
    w[0] *= 0.5
    ell = np.array([2.0, 30.0, 700.0])
    c = 3e-9
    out = LZ.limber_cl_psi(ell, chi, w, chi_star, lambda k, i: c / k ** 2)
    ref = 8 * np.pi ** 2 * c * chi_star ** 2 / (12 * (ell + 0.5) ** 5)
    np.testing.assert_allclose(out, ref, rtol=1e-7)


def _spectra(L, Lt=600, Lp=80):
    l = np.arange(L + 1)
    on = (l >= 2) & (l <= Lt)
    ctt = np.where(on, 1e3 / (l * (l + 1) + 10.0) * (1.2 + np.cos(l / 35.0)) * np.exp(-(l / 450.0) ** 2), 0.0)
    cee = np.where(on, 30.0 / (l * (l + 1) + 10.0) * (1.2 + np.sin(l / 35.0)) * np.exp(-(l / 450.0) ** 2)
                   * (l / 100.0) ** 1.5, 0.0)
    cte = np.where(on, 0.3 * np.sqrt(ctt * cee) * np.cos(l / 50.0), 0.0)
    lp = np.maximum(l, 1).astype(float)
    cpsi = np.where((l >= 2) & (l <= Lp), 1.0 / (lp * (lp + 1.0)) ** 2 * (lp / (lp + 40.0)), 0.0)
    return ctt, cee, cte, cpsi


def _exact_first_order(ctt, cee, cte, cpsi, lout, n_mu):
    """First-order lensing of the spectra in harmonic space: C~_l - C_l =
    -(l(l+1) - s^2) R C_l + sum_{l1 l2} C^psi_l1 C_l2 (F^s_{l l1 l2})^2 / (2l+1)
    (parity-split for E/B, F^0 F^2 for TE), F^s = [l1(l1+1) + l2(l2+1) - l(l+1)]/2
    sqrt((2l+1)(2l1+1)(2l2+1)/4pi) (l l1 l2; s 0 -s), R = sum (2l+1) l(l+1) C^psi / 8pi;
    the 3j products come from int d^l d^l1 d^l2 dmu = 2 (3j)(3j)."""
    L = len(ctt) - 1
    l = np.arange(L + 1.0)
    A = l * (l + 1)
    mu, wm = np.polynomial.legendre.leggauss(n_mu)
    d = {mn: LZ.wigner_d(L, mu, *mn) for mn in [(0, 0), (2, 2), (2, -2), (-2, -2), (-2, 2), (0, 2), (0, -2)]}
    R = np.sum(A * (2 * l + 1) * cpsi) / (8 * np.pi)
    f = [((2 * l + 1) * cpsi * A ** n) @ d[(0, 0)] for n in range(3)]

    def conv(X, dl, dx):
        g = [((2 * l + 1) * X * A ** n) @ dx for n in range(3)]
        out = np.zeros(lout + 1)
        for ll in range(lout + 1):
            a = ll * (ll + 1.0)
            integ = f[2] * g[0] + f[0] * g[2] + a * a * f[0] * g[0] + 2 * f[1] * g[1] - 2 * a * f[1] * g[0] \
                - 2 * a * f[0] * g[1]
            out[ll] = np.sum(wm * dl[ll] * integ) / (32 * np.pi)
        return out

    lo = np.arange(lout + 1.0)
    Ao = lo * (lo + 1)
    dTT = -Ao * R * ctt[: lout + 1] + conv(ctt, d[(0, 0)], d[(0, 0)])
    s, p = conv(cee, d[(2, 2)], d[(-2, -2)]), conv(cee, d[(2, -2)], d[(-2, 2)])
    dEE = -(Ao - 4) * R * cee[: lout + 1] + 0.5 * (s + p)
    dBB = 0.5 * (s - p)
    dTE = -(Ao - 2) * R * cte[: lout + 1] + conv(cte, d[(0, 2)], d[(0, -2)])
    return dTT, dEE, dBB, dTE


def test_lensed_spectra_match_first_order_lensing():
    # weak lensing of spectra whose structure sits at l ~ 100-600 by a potential
    # at l <= 80: the correlation-function method's small-angle approximations
    # hold, and it must reproduce the exact first-order change
    L, lout, eps = 680, 500, 1e-6
    ctt, cee, cte, cpsi = _spectra(L)
    TT, EE, TE, BB = LZ.lensed_cls(ctt, cee, cte, eps * cpsi, lout, n_mu=900)
    dTT, dEE, dBB, dTE = _exact_first_order(ctt, cee, cte, cpsi, lout, 800)
    sl = slice(20, lout + 1)
    for got, ref, tol in [((TT - ctt[: lout + 1]) / eps, dTT, 3e-3), ((EE - cee[: lout + 1]) / eps, dEE, 8e-3),
                          (BB / eps, dBB, 2e-3), ((TE - cte[: lout + 1]) / eps, dTE, 1e-2)]:
        assert np.abs(got[sl] - ref[sl]).max() < tol * np.abs(ref[sl]).max()


def test_no_lensing_leaves_the_spectra():
    ctt, cee, cte, cpsi = _spectra(300, Lt=250, Lp=40)
    TT, EE, TE, BB = LZ.lensed_cls(ctt, cee, cte, 0.0 * cpsi, 250, n_mu=400)
    np.testing.assert_allclose(TT[2:], ctt[2:251], rtol=0, atol=1e-12 * ctt.max())
    np.testing.assert_allclose(EE[2:], cee[2:251], rtol=0, atol=1e-12 * cee.max())
    np.testing.assert_allclose(TE[2:], cte[2:251], rtol=0, atol=1e-12 * np.abs(cte).max())
    assert np.abs(BB).max() < 1e-12 * cee.max()


def test_lensing_potential_spectrum_of_a_lcdm_cosmology():
    # the Limber C_l^psi of a Planck-like cosmology peaks near l ~ 40 at
    # [l(l+1)]^2 C_l^psi / 2 pi ~ 1.2e-7 (the familiar LCDM lensing spectrum)
    import oracle as O
    from paper_2602_15104_gb300 import workload as W
    p = W.SMALL_TT.params()[0]
    k = np.exp(np.linspace(np.log(1e-4), np.log(0.3), 40))
    c = LZ.cl_psi(p, k, 400, 200, O.opts(lmax=8))
    l = np.arange(201)
    v = (l * (l + 1.0)) ** 2 * c / (2 * np.pi)
    lpk = int(np.argmax(v))
    assert 20 <= lpk <= 60, lpk
    assert 0.8e-7 < v[lpk] < 1.6e-7, v[lpk]
