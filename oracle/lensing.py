"""ORACLE (test infrastructure only): CMB lensing (App. B.5).

Plain numpy restatement, slow and direct:

  * the lensing potential's angular spectrum in the Limber approximation
      C_l^psi = 8 pi^2 / (l + 1/2)^3 int_0^chi* dchi / chi
                P_psi(k = (l + 1/2) / chi, tau0 - chi) ((chi* - chi) / chi*)^2,
      P_psi(k, a) = 9 Omega_m(a)^2 H^4 / (8 pi^2 k) P(k, a),
    with P(k, a) = (2 pi^2 / k^3) A_s (k/k_pivot)^(n_s - 1) delta_m^2 (eq. PK),
    Omega_m(a) = (rho_c + rho_b) / rho_tot and H the conformal Hubble rate
    (App. B.5).  Readings (the paper is silent): chi* = tau0 - tau* with tau*
    the node where the visibility g peaks; the chi integral is the trapezoid
    rule over the tau nodes between tau* and tau0; P(k, a) at k = (l+1/2)/chi
    comes from delta_m on the given k nodes interpolated in ln k (the cubic
    Hermite rule of interp_sources) and is zero outside them.

  * the lensed spectra by the all-sky correlation-function method the paper
    cites (Challinor & Lewis 2005), integrated over the whole of mu in [-1, 1]
    with Gauss-Legendre nodes (the paper rejects the restricted "fast" range):
    the lensed correlation functions xi~(beta) for T, (+), (-) and the cross
    term are built from the unlensed spectra, sigma^2(beta) = C_gl(0) -
    C_gl(beta) and C_gl,2(beta) (second order in C_gl,2), and transformed back
    with the Wigner functions d^l_00, d^l_22, d^l_2-2 and d^l_20.  Only the
    difference lensed - unlensed is transformed, as the cited method advises.

Wigner small-d functions d^l_mn(beta) of the usual convention (d^l_mn(0) =
delta_mn, d^1_10 = -sin(beta)/sqrt 2) start at l = max(|m|, |n|) from the
explicit sum over s and rise in l by the three-term recurrence.
"""
from __future__ import annotations

from math import factorial, sqrt

import numpy as np


def wigner_d(lmax, mu, m, n):
    """d^l_mn(arccos mu) for l = 0..lmax: array [lmax + 1, len(mu)] (zero below
    l = max(|m|, |n|))."""
    mu = np.asarray(mu, dtype=np.float64)
    out = np.zeros((lmax + 1, mu.size))
    j = max(abs(m), abs(n))
    if j > lmax:
        return out
    c = np.sqrt(np.clip((1.0 + mu) / 2.0, 0.0, None))  # cos(beta/2)
    s = np.sqrt(np.clip((1.0 - mu) / 2.0, 0.0, None))  # sin(beta/2)
    mp, mm = m, n
    tot = np.zeros(mu.size)
    for k in range(0, 2 * j + 1):
        a, b_, c_, d_ = j + mm - k, k, mp - mm + k, j - mp - k
        if min(a, b_, c_, d_) < 0:
            continue
        coef = (-1) ** (mp - mm + k) * sqrt(factorial(j + mp) * factorial(j - mp) * factorial(j + mm)
                                            * factorial(j - mm)) / (factorial(a) * factorial(b_) * factorial(c_)
                                                                    * factorial(d_))
        tot += coef * c ** (2 * j + mm - mp - 2 * k) * s ** (mp - mm + 2 * k)
    out[j] = tot
    for l in range(j, lmax):
        num = (2 * l + 1) * (l * (l + 1) * mu - m * n) * out[l]
        if l > j:
            num -= (l + 1) * sqrt((l * l - m * m) * (l * l - n * n)) * out[l - 1]
        den = l * sqrt(((l + 1) ** 2 - m * m) * ((l + 1) ** 2 - n * n)) if l > 0 else None
        if l == 0:
            # j = 0: d^1_00 = mu
            out[1] = mu * out[0]
        else:
            out[l + 1] = num / den
    return out


def limber_cl_psi(ell, chi, w, chi_star, Ppsi):
    """C_l^psi = 8 pi^2 / (l+1/2)^3 sum_i w_i / chi_i Ppsi((l+1/2)/chi_i, i)
    ((chi* - chi_i)/chi*)^2 over nodes with 0 < chi_i <= chi*; Ppsi(k, i)."""
    ell = np.asarray(ell, dtype=np.float64)
    out = np.zeros(ell.size)
    for i in range(chi.size):
        if not (0.0 < chi[i] <= chi_star):
            continue
        kk = (ell + 0.5) / chi[i]
        out += w[i] / chi[i] * Ppsi(kk, i) * ((chi_star - chi[i]) / chi_star) ** 2
    return 8.0 * np.pi ** 2 / (ell + 0.5) ** 3 * out


def cl_psi(params, k, n_tau, lmax, o, m_ncdm=0.0):
    """C_l^psi for l = 0..lmax of one cosmology from the oracle's delta_m on the k nodes."""
    import oracle as O
    k = np.asarray(k, dtype=np.float64)
    lna, tau, w = O.nodes(params, n_tau, m_ncdm=m_ncdm)
    sc = O.scalars(params, m_ncdm=m_ncdm)
    bg = O.background(params, lna, m_ncdm=m_ncdm)
    istar = int(np.argmax(bg["g"]))
    tau0 = sc["tau0"]
    chi = tau0 - tau
    chi_star = tau0 - tau[istar]
    # trapezoid weights in chi over the nodes istar..n_tau-1 and chi = 0 at tau0
    wchi = np.zeros(n_tau)
    for i in range(istar, n_tau):
        lo = tau[i - 1] if i > istar else tau[i]
        hi = tau[i + 1] if i < n_tau - 1 else tau0
        wchi[i] = 0.5 * (hi - lo)
    dm = O.delta_m_nodes(params, k, n_tau, o)  # [n_k, n_tau]
    from oracle import interp_sources
    logk = np.log(k)
    As, ns = sc["A_s"], sc["n_s"]

    def Ppsi(kk, i):
        inside = (kk >= k[0]) & (kk <= k[-1])
        res = np.zeros(kk.size)
        if not inside.any():
            return res
        d = interp_sources(dm[:, i][:, None, None] * np.ones((1, 1, 3)), k, kk[inside])[:, 0, 0]
        P = 2.0 * np.pi ** 2 / kk[inside] ** 3 * As * (kk[inside] / 0.05) ** (ns - 1.0) * d * d
        om = bg["fc"][i] + bg["fb"][i]
        res[inside] = 9.0 * om * om * bg["Hc"][i] ** 4 / (8.0 * np.pi ** 2 * kk[inside]) * P
        return res

    ell = np.arange(lmax + 1)
    out = limber_cl_psi(ell, chi, wchi, chi_star, Ppsi)
    out[:2] = 0.0
    return out


def _corr(C, d, l):
    """sum_l (2l+1)/(4 pi) C_l d_l(mu)"""
    return ((2 * l + 1) / (4 * np.pi) * C)[:, None] * d


def lensed_cls(cl_tt, cl_ee, cl_te, cl_psi, lmax_out, n_mu=None):
    """Lensed TT, EE, TE, BB for l = 0..lmax_out from unlensed spectra and
    C_l^psi given for l = 0..L (L >= lmax_out; arrays indexed by l)."""
    L = len(cl_tt) - 1
    l = np.arange(L + 1, dtype=np.float64)
    n_mu = n_mu or (L + 200)
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    llp1 = l * (l + 1)
    d00, d11, d1m1 = wigner_d(L, mu, 0, 0), wigner_d(L, mu, 1, 1), wigner_d(L, mu, 1, -1)
    d22, d2m2, d20 = wigner_d(L, mu, 2, 2), wigner_d(L, mu, 2, -2), wigner_d(L, mu, 2, 0)
    d31, d3m1, d3m3 = wigner_d(L, mu, 3, 1), wigner_d(L, mu, 3, -1), wigner_d(L, mu, 3, -3)
    d40, d4m4, dm24 = wigner_d(L, mu, 4, 0), wigner_d(L, mu, 4, -4), wigner_d(L, mu, -2, 4)
    cpsi = np.asarray(cl_psi, dtype=np.float64)[: L + 1]
    Cgl = (_corr(llp1 * cpsi, d11, l)).sum(0)
    Cgl2 = (_corr(llp1 * cpsi, d1m1, l)).sum(0)
    Cgl0 = ((2 * l + 1) / (4 * np.pi) * llp1 * cpsi).sum()  # d^l_11(0) = 1
    sig2 = Cgl0 - Cgl
    S = sig2[None, :]
    lp = llp1[:, None]
    X000 = np.exp(-lp * S / 4)
    Xp000 = -lp / 4 * X000  # d X_000 / d sigma^2
    X220 = 0.25 * np.sqrt(np.clip((l + 2) * (l - 1) * l * (l + 1), 0, None))[:, None] * np.exp(-(lp - 2) * S / 4)
    X022 = np.exp(-(lp - 4) * S / 4)
    Xp022 = -(lp - 4) / 4 * X022
    X121 = -0.5 * np.sqrt(np.clip((l + 2) * (l - 1), 0, None))[:, None] * np.exp(-(lp - 8.0 / 3) * S / 4)
    X132 = -0.5 * np.sqrt(np.clip((l + 3) * (l - 2), 0, None))[:, None] * np.exp(-(lp - 20.0 / 3) * S / 4)
    X242 = 0.25 * np.sqrt(np.clip((l + 4) * (l + 3) * (l - 2) * (l - 3), 0, None))[:, None] * \
        np.exp(-(lp - 10) * S / 4)
    G = Cgl2[None, :]
    pre = ((2 * l + 1) / (4 * np.pi))[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_llp1 = np.where(lp > 0, 1.0 / lp, 0.0)
    # differences lensed - unlensed of the correlation functions
    tt = np.asarray(cl_tt, dtype=np.float64)[:, None]
    xT = (pre * tt * ((X000 ** 2 - 1) * d00 + 8 * inv_llp1 * G * Xp000 ** 2 * d1m1
                      + G * G * (Xp000 ** 2 * d00 + X220 ** 2 * d2m2))).sum(0)
    ee = np.asarray(cl_ee, dtype=np.float64)[:, None]
    xP = (pre * ee * ((X022 ** 2 - 1) * d22 + 2 * G * X132 * X121 * d31
                      + G * G * (Xp022 ** 2 * d22 + X242 * X220 * d40))).sum(0)
    xM = (pre * ee * ((X022 ** 2 - 1) * d2m2 + G * (X121 ** 2 * d1m1 + X132 ** 2 * d3m3)
                      + 0.5 * G * G * (2 * Xp022 ** 2 * d2m2 + X220 ** 2 * d00 + X242 ** 2 * d4m4))).sum(0)
    te = np.asarray(cl_te, dtype=np.float64)[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        sq = np.where(lp > 0, 1.0 / np.sqrt(np.where(lp > 0, lp, 1.0)), 0.0)
    xX = (pre * te * ((X022 * X000 - 1) * d20 + G * 2 * Xp000 * sq * (X121 * d11 + X132 * d3m1)
                      + 0.5 * G * G * ((2 * Xp022 * Xp000 + X220 ** 2) * d20 + X220 * X242 * dm24))).sum(0)
    lo = np.arange(lmax_out + 1)
    dTT = 2 * np.pi * (d00[: lmax_out + 1] * (wmu * xT)[None, :]).sum(1)
    dP = 2 * np.pi * (d22[: lmax_out + 1] * (wmu * xP)[None, :]).sum(1)
    dM = 2 * np.pi * (d2m2[: lmax_out + 1] * (wmu * xM)[None, :]).sum(1)
    dX = 2 * np.pi * (d20[: lmax_out + 1] * (wmu * xX)[None, :]).sum(1)
    TT = np.asarray(cl_tt)[lo] + dTT
    EE = np.asarray(cl_ee)[lo] + 0.5 * (dP + dM)
    BB = 0.5 * (dP - dM)
    TE = np.asarray(cl_te)[lo] + dX
    for a in (TT, EE, BB, TE):
        a[:2] = 0.0
    return TT, EE, TE, BB
