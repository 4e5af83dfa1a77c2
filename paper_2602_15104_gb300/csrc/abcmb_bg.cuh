// Background and thermal history of one cosmology, built by one thread into
// the background record whose layout include/abcmb.h defines.
//
// Follows arXiv 2602.15104: densities (App. C.1-C.5), conformal time
// (Sec. 2.4 "Background"), helium Saha phases (App. B.1.1), hydrogen Saha
// (App. B.1.2, eq. SahaH) then a Peebles three-level atom (the TLA cited in
// App. B.1.2; rates from the literature: Pequignot et al. 1991 case-B fit,
// detailed-balance photo-ionisation at T_CMB, Lambda_2s1s = 8.2245809/s,
// Sobolev escape K = lambda_a^3/(8 pi H)), matter temperature (App. B.1.2:
// quasi-static T_CMB (1 - H/Gamma_C) above z = 700, its ODE below), tanh
// reionization (App. B.2) with z_reion solved from tau_reion (App. A.2),
// kappa and g (App. B.4), baryon sound speed (App. C.3), tight-coupling start
// H tau_c = R_tc (App. A.1) and the tau nodes of the line-of-sight integral
// with trapezoid weights (App. B.6).
//
// Compiled for sm_103a; it also compiles as plain C++ so that the same code
// can be stepped through on a host for debugging.
#pragma once

#include <math.h>

#include "../../include/abcmb.h"

#ifdef __CUDACC__
#define ABCMB_HD __host__ __device__ __forceinline__
#else
#define ABCMB_HD inline
#endif

// storage shared by the threads of a CTA; a host build of the kernels (the
// CPU tests, which run a CTA's threads as host threads) makes it static
#ifndef ABCMB_CTA_SHARED
#define ABCMB_CTA_SHARED __shared__
#endif

namespace abcmb {

// ---- physical constants ----
constexpr double kPi = 3.141592653589793238;
constexpr double kC = 2.99792458e10;           // cm/s
constexpr double kMpc = 3.0856775814913673e24; // cm
constexpr double kSigmaT = 6.6524587321e-25;   // cm^2
constexpr double kHc = 1.239841984e-4;         // h c, eV cm
constexpr double kHbarC = 1.973269804e-5;      // hbar c, eV cm
constexpr double kKB = 8.617333262e-5;         // eV/K
constexpr double kMe = 510998.95;              // eV
constexpr double kMH = 938783073.6;            // eV, hydrogen atom
constexpr double kMHeOverMH = 3.971480;        // 4He atom / H atom
constexpr double kEH = 13.598434005;           // eV
constexpr double kEHe1 = 24.587387;            // eV
constexpr double kEHe2 = 54.417760;            // eV
constexpr double kL2s1s = 8.2245809;           // 1/s
constexpr double kG = 6.67430e-8;              // cgs
constexpr double kEvErg = 1.602176634e-12;

// ---- fixed cosmological inputs (paper defaults, App. A.2) ----
constexpr double kYHe = 0.245;
constexpr double kTcmb0 = 2.34865418e-4; // eV
constexpr double kTnuRatio = 0.71636856;
constexpr double kNnu = 3.0;
constexpr double kTncdmRatio = 0.71611; // massive neutrino temperature today / T_gamma (App. A.1)
constexpr double kZreHe = 3.5, kDzReHe = 0.5, kDzRe = 0.5, kBetaRe = 1.5;
constexpr double kRtc = 1.5e-3, kRlarge = 7e-2, kKpivot = 0.05;
constexpr double kLna700 = -6.55250788703459; // ln(1/701)
// RK4 steps of the TLA in ln a: fine through the stiff transient after the
// Saha switch, one table cell afterwards
constexpr double kTlaFine = 0.125 / ABCMB_BG_PER_UNIT;
constexpr double kTlaFineSpan = 0.05;

constexpr int kNlna = ABCMB_BG_NLNA;
constexpr double kLna0 = ABCMB_BG_LNA0;
constexpr double kDlna = 1.0 / ABCMB_BG_PER_UNIT;
// table columns
enum { C_NUT = 0, C_DNUT, C_TAU, C_DTAU, C_CS2, C_DCS2, C_KAPPA, C_XE };
// tau-node columns
enum { N_LNA = 0, N_TAU, N_W, N_G, N_DG, N_EXPMK, N_HC, N_DHC };

// 4-point Gauss-Legendre rule on [-1, 1]
ABCMB_HD double gl4_x(int i)
{
    return i == 0 ? -0.8611363115940526 : i == 1 ? -0.3399810435848563
         : i == 2 ? 0.3399810435848563 : 0.8611363115940526;
}
ABCMB_HD double gl4_w(int i) { return (i == 0 || i == 3) ? 0.3478548451374538 : 0.6521451548625461; }

// Scalars of one cosmology (record header).
struct Cosmo {
    double H0, Om_b, Om_c, Om_g, Om_nu, Om_L, Om_r, Om_m;
    double R_nu, f_He, nH0, A_s, n_s;
    double z_reion, lna_tc, lna_sw, tau0, lna_He3;
    double rho_g0; // photon energy density today, eV/cm^3
    // one massive neutrino (0 when absent); Om_r includes its relativistic limit
    double ncdm_pref, ncdm_x1, Om_ncdm_rel;
};

// Massive neutrino (App. B.3 "Massive neutrinos"): energy density and pressure
// in units of today's critical density, by the paper's 5-point rule for the
// background, rho = PREF a^-4 sum_i K_i (1 + e^-q_i) eps_i / q_i^2 and
// p = PREF a^-4 sum_i K_i (1 + e^-q_i) / (3 eps_i), eps_i = sqrt(q_i^2 + x^2),
// x = a m / T_ncdm (Fermi-Dirac in the comoving momentum q).
ABCMB_HD void ncdm_rho_p(const Cosmo &c, double a, double *rho, double *p)
{
    *rho = *p = 0.0;
    if (c.ncdm_pref == 0.0) return;
    const double q5[5] = {0.583165, 2.0, 4.0, 7.26582, 13.0};
    const double k5[5] = {0.0081201, 0.689407, 2.8063, 2.05156, 0.12681};
    const double x = a * c.ncdm_x1, a4 = a * a * a * a;
    double sr = 0.0, sp = 0.0;
    for (int i = 0; i < 5; i++) {
        const double q = q5[i], eps = sqrt(q * q + x * x), w = k5[i] * (1.0 + exp(-q));
        sr += w * eps / (q * q);
        sp += w / eps;
    }
    *rho = c.ncdm_pref * sr / a4;
    *p = c.ncdm_pref * sp / (3.0 * a4);
}

ABCMB_HD Cosmo load_cosmo(const double *rec)
{
    Cosmo c;
    c.H0 = rec[ABCMB_S_H0];
    c.Om_b = rec[ABCMB_S_OMB];
    c.Om_c = rec[ABCMB_S_OMC];
    c.Om_g = rec[ABCMB_S_OMG];
    c.Om_nu = rec[ABCMB_S_OMNU];
    c.Om_L = rec[ABCMB_S_OML];
    c.Om_r = c.Om_g + c.Om_nu;
    c.Om_m = c.Om_b + c.Om_c;
    c.R_nu = rec[ABCMB_S_RNU];
    c.f_He = rec[ABCMB_S_FHE];
    c.nH0 = rec[ABCMB_S_NH0];
    c.A_s = rec[ABCMB_S_AS];
    c.n_s = rec[ABCMB_S_NS];
    c.z_reion = rec[ABCMB_S_ZREION];
    c.lna_tc = rec[ABCMB_S_LNA_TC];
    c.lna_sw = rec[ABCMB_S_LNA_SW];
    c.tau0 = rec[ABCMB_S_TAU0];
    c.lna_He3 = rec[ABCMB_S_LNA_HE3];
    c.rho_g0 = 0.0;
    c.ncdm_pref = rec[ABCMB_S_NCDM_PREF];
    c.ncdm_x1 = rec[ABCMB_S_NCDM_X1];
    c.Om_ncdm_rel = rec[ABCMB_S_OMNCDM_REL];
    c.Om_r = c.Om_g + c.Om_nu + c.Om_ncdm_rel;
    return c;
}

// ---- closed-form background ----
struct BgClosed {
    double a, inv_a, Hc, fc, fb, fg, fnu, dlnHc; // dlnHc = d ln H_conf / d ln a
};

ABCMB_HD BgClosed closed_bg(const Cosmo &c, double lna)
{
    BgClosed b;
    b.a = exp(lna);
    b.inv_a = 1.0 / b.a;
    double ia = b.inv_a, ia3 = ia * ia * ia, ia4 = ia3 * ia;
    double rr = (c.Om_g + c.Om_nu) * ia4, rm = c.Om_m * ia3;
    double rn, pn;
    ncdm_rho_p(c, b.a, &rn, &pn);
    double e2 = rr + rm + c.Om_L + rn;
    double ie2 = 1.0 / e2;
    b.Hc = b.a * c.H0 * sqrt(e2);
    b.fc = c.Om_c * ia3 * ie2;
    b.fb = c.Om_b * ia3 * ie2;
    b.fg = c.Om_g * ia4 * ie2;
    b.fnu = c.Om_nu * ia4 * ie2;
    b.dlnHc = 1.0 - (2.0 * rr + 1.5 * rm + 1.5 * (rn + pn)) * ie2;
    return b;
}

ABCMB_HD double hconf(const Cosmo &c, double lna)
{
    double a = exp(lna), ia = 1.0 / a;
    double rn, pn;
    ncdm_rho_p(c, a, &rn, &pn);
    return a * c.H0 * sqrt((c.Om_g + c.Om_nu) * ia * ia * ia * ia + c.Om_m * ia * ia * ia + c.Om_L + rn);
}

// exact radiation+matter conformal time
ABCMB_HD double tau_rm(const Cosmo &c, double a)
{
    return 2.0 * a / (c.H0 * (sqrt(c.Om_r + c.Om_m * a) + sqrt(c.Om_r)));
}

// ---- cubic Hermite on the uniform table ----
struct Herm {
    int j;
    double h00, h10, h01, h11, d00, d10, d01, d11; // basis and d/du
};

ABCMB_HD Herm herm_at(double lna)
{
    Herm H;
    double t = (lna - kLna0) * ABCMB_BG_PER_UNIT;
    int j = (int)floor(t);
    if (j < 0) j = 0;
    if (j > kNlna - 2) j = kNlna - 2;
    double u = t - j, um = 1.0 - u;
    H.j = j;
    H.h00 = (1.0 + 2.0 * u) * um * um;
    H.h10 = u * um * um;
    H.h01 = u * u * (3.0 - 2.0 * u);
    H.h11 = u * u * (u - 1.0);
    H.d00 = 6.0 * u * (u - 1.0);
    H.d10 = um * (1.0 - 3.0 * u);
    H.d01 = -H.d00;
    H.d11 = u * (3.0 * u - 2.0);
    return H;
}

// value of column col with derivative column dcol (sign sgn applied to it)
ABCMB_HD double herm_val(const double *tab, const Herm &H, int col, int dcol, double sgn = 1.0)
{
    const double *r0 = tab + 8 * H.j, *r1 = r0 + 8;
    return H.h00 * r0[col] + H.h01 * r1[col] + sgn * kDlna * (H.h10 * r0[dcol] + H.h11 * r1[dcol]);
}

ABCMB_HD double herm_der(const double *tab, const Herm &H, int col, int dcol)
{
    const double *r0 = tab + 8 * H.j, *r1 = r0 + 8;
    return (H.d00 * r0[col] + H.d01 * r1[col]) * ABCMB_BG_PER_UNIT + H.d10 * r0[dcol] + H.d11 * r1[dcol];
}

// ---- thermal-history pieces ----
ABCMB_HD double saha_pref(double T, double mu)
{
    double v = 2.0 * kPi * mu * T / (kHc * kHc);
    return v * sqrt(v);
}
ABCMB_HD double mu_eH() { return kMe * kMH / (kMe + kMH); }
ABCMB_HD double mu_eHe() { return kMe * (kMHeOverMH * kMH) / (kMe + kMHeOverMH * kMH); }

// Stable root of x^2 + (b0 + s) x - s f = 0 and its ln a derivative, for a
// Saha ratio s whose log derivative is dls.
ABCMB_HD double saha_root(double s, double f, double b0, double dls, double *dx)
{
    double b = b0 + s, r = sqrt(b * b + 4.0 * s * f);
    double x = 2.0 * s * f / (b + r);
    *dx = s * (f - x) * dls / (2.0 * x + b);
    return x;
}

// Saha ratio S(T) e^{-E/T} / n_H with T = T0/a, n_H = nH0/a^3; its log
// derivative is 3/2 - E/T.
ABCMB_HD double saha_s(const Cosmo &c, double a, double E, double mu, double g, double *dls)
{
    double T = kTcmb0 / a;
    *dls = 1.5 - E / T;
    return g * saha_pref(T, mu) * exp(-E / T) * a * a * a / c.nH0;
}

ABCMB_HD double x_he(const Cosmo &c, double lna, double *dx)
{
    double a = exp(lna), dls;
    if (lna < c.lna_He3) {
        double s = saha_s(c, a, kEHe2, mu_eHe(), 1.0, &dls);
        return c.f_He + saha_root(s, c.f_He, 1.0 + c.f_He, dls, dx);
    }
    double s = saha_s(c, a, kEHe1, mu_eHe(), 4.0, &dls);
    return saha_root(s, c.f_He, 1.0, dls, dx);
}

ABCMB_HD double xp_saha(const Cosmo &c, double lna, double *dx)
{
    double dls;
    double s = saha_s(c, exp(lna), kEH, mu_eH(), 1.0, &dls);
    return saha_root(s, 1.0, 0.0, dls, dx);
}

ABCMB_HD double alpha_B(double T)
{
    double lt = log(T / kKB * 1.0e-4);
    return 4.309e-13 * exp(-0.6166 * lt) / (1.0 + 0.6703 * exp(0.5300 * lt));
}

ABCMB_HD double H_sec(const Cosmo &c, double lna) { return hconf(c, lna) * exp(-lna) * kC / kMpc; }

ABCMB_HD double gamma_C(const Cosmo &c, double a, double xe)
{
    double rho_g = c.rho_g0 / (a * a * a * a);
    return 8.0 * kSigmaT * kC * rho_g / (3.0 * kMe) * xe / (1.0 + c.f_He + xe);
}

// quasi-static matter temperature and d ln T_m / d ln a
ABCMB_HD double tm_qs(const Cosmo &c, double lna, double xe, double dxe, double *dlnTm)
{
    double a = exp(lna), T = kTcmb0 / a;
    BgClosed b = closed_bg(c, lna);
    double H = b.Hc * b.inv_a * kC / kMpc;
    double r = H / gamma_C(c, a, xe);
    double dlnH = b.dlnHc - 1.0;
    double dlnG = -4.0 + dxe * (1.0 + c.f_He) / (xe * (1.0 + c.f_He + xe));
    *dlnTm = -1.0 - r / (1.0 - r) * (dlnH - dlnG);
    return T * (1.0 - r);
}

// Peebles TLA for x_p (and T_m when two) in ln a
ABCMB_HD void tla_rhs(const Cosmo &c, double lna, double xp, double Tm_in, bool two,
                      double *dxp, double *dTm)
{
    double a = exp(lna), T = kTcmb0 / a, dum;
    double xe = xp + x_he(c, lna, &dum);
    double Tm = two ? Tm_in : T * (1.0 - H_sec(c, lna) / gamma_C(c, a, xe));
    double nH = c.nH0 / (a * a * a), H = H_sec(c, lna);
    double al = alpha_B(Tm);
    double be = alpha_B(T) * saha_pref(T, mu_eH()) * exp(-0.25 * kEH / T);
    double lam = kHc / (0.75 * kEH);
    double K = lam * lam * lam / (8.0 * kPi * H);
    double n1s = nH * (1.0 - xp);
    double C = (1.0 + K * kL2s1s * n1s) / (1.0 + K * (kL2s1s + be) * n1s);
    *dxp = -C * (al * nH * xe * xp - be * (1.0 - xp) * exp(-0.75 * kEH / T)) / H;
    *dTm = two ? (-2.0 * Tm + gamma_C(c, a, xe) / H * (T - Tm)) : 0.0;
}

// The parts of tla_rhs that depend on ln a alone, at one stage point.
struct TlaPt {
    double T, nH, H, K, be, bex, xhe, g0, e1, e2, iH;
};
constexpr int kTlaPtDoubles = 11;

ABCMB_HD TlaPt tla_point(const Cosmo &c, double lna)
{
    TlaPt P;
    const double a = exp(lna), dum0 = 0.0;
    (void)dum0;
    double dum;
    P.T = kTcmb0 / a;
    P.nH = c.nH0 / (a * a * a);
    P.H = H_sec(c, lna);
    const double lam = kHc / (0.75 * kEH);
    P.K = lam * lam * lam / (8.0 * kPi * P.H);
    P.be = alpha_B(P.T) * saha_pref(P.T, mu_eH()) * exp(-0.25 * kEH / P.T);
    P.bex = P.be * exp(-0.75 * kEH / P.T);
    P.xhe = x_he(c, lna, &dum);
    P.g0 = 8.0 * kSigmaT * kC * (c.rho_g0 / (a * a * a * a)) / (3.0 * kMe);
    const double lt0 = log(P.T / kKB * 1.0e-4);
    P.e1 = exp(-0.6166 * lt0);
    P.e2 = exp(0.5300 * lt0);
    P.iH = 1.0 / P.H;
    return P;
}

// tla_rhs from a stage point's ln a-only parts.  Above z = 700 T_m = T (1 - r),
// r = H / Gamma_C, and alpha_B(T_m) = alpha_B(T) scaled through (1 - r)^p, taken
// from the series of log(1 - r) and exp while r < 0.02 (both truncated below
// 1e-17); otherwise, and below z = 700, the rates are evaluated afresh.
ABCMB_HD void tla_rhs_pt(const Cosmo &c, const TlaPt &P, double xp, double Tm_in, bool two, double *dxp,
                         double *dTm)
{
    // The right-hand side is evaluated sequentially, one stage after another,
    // so its chain of dependent instructions sets the builder's time: the
    // series below run in Horner form on constant coefficients, and 1/H is
    // tabulated, which leaves two divisions.
    const double xe = xp + P.xhe;
    const double gam = P.g0 * xe / (1.0 + c.f_He + xe);
    double Tm, al;
    if (!two) {
        const double r = P.H / gam;
        Tm = P.T * (1.0 - r);
        if (r < 0.02) {
            // L = log(1 - r) = -sum_{n=1}^{12} r^n / n
            double L = 1.0 / 12.0;
#pragma unroll
            for (int n = 11; n >= 1; n--) L = fma(r, L, 1.0 / n);
            L *= -r;
            // f = exp(q) = sum_{n=0}^{8} q^n / n!, q1 = -0.6166 L, q2 = 0.53 L
            const double q1 = -0.6166 * L, q2 = 0.5300 * L;
            double f1 = 1.0, f2 = 1.0;
#pragma unroll
            for (int n = 8; n >= 1; n--) {
                f1 = fma(q1 * (1.0 / n), f1, 1.0);
                f2 = fma(q2 * (1.0 / n), f2, 1.0);
            }
            al = 4.309e-13 * P.e1 * f1 / (1.0 + 0.6703 * P.e2 * f2);
        } else {
            al = alpha_B(Tm);
        }
    } else {
        Tm = Tm_in;
        al = alpha_B(Tm);
    }
    const double n1s = P.nH * (1.0 - xp);
    const double C = (1.0 + P.K * kL2s1s * n1s) / (1.0 + P.K * (kL2s1s + P.be) * n1s);
    *dxp = -C * (al * P.nH * xe * xp - P.bex * (1.0 - xp)) * P.iH;
    *dTm = two ? (-2.0 * Tm + gam * P.iH * (P.T - Tm)) : 0.0;
}

ABCMB_HD double nuT_closed(const Cosmo &c, double lna, double xe)
{
    double a = exp(lna);
    return xe * c.nH0 * kSigmaT * kMpc / (a * a * hconf(c, lna));
}

// optical depth of the reionization electrons alone for a trial z_reion
ABCMB_HD double tau_reion_trial(const Cosmo &c, double zre)
{
    double dy = kBetaRe * kDzRe * pow(1.0 + zre, kBetaRe - 1.0);
    double yre = pow(1.0 + zre, kBetaRe);
    double zmax = pow(yre + 25.0 * dy, 1.0 / kBetaRe) - 1.0;
    double zhe = kZreHe + 25.0 * kDzReHe;
    if (zhe > zmax) zmax = zhe;
    double lo = -log(1.0 + zmax);
    const int np = 800;
    double hp = -lo / np, acc = 0.0;
    for (int p = 0; p < np; p++)
        for (int q = 0; q < 4; q++) {
            double lna = lo + hp * (p + 0.5 * (1.0 + gl4_x(q)));
            double z = exp(-lna) - 1.0;
            double S1 = 0.5 * (1.0 + tanh((yre - pow(1.0 + z, kBetaRe)) / dy));
            double S2 = 0.5 * (1.0 + tanh((kZreHe - z) / kDzReHe));
            acc += 0.5 * hp * gl4_w(q) * ((1.0 + c.f_He) * S1 + c.f_He * S2) * nuT_closed(c, lna, 1.0);
        }
    return acc;
}

// ---- point evaluation used by the ODE and the sources ----
struct BgPt {
    double Hc, inv_Hc, fc, fb, fg, fnu, nuT, Rinv, cs2, tau;
};

ABCMB_HD BgPt bg_point(const Cosmo &c, const double *tab, double lna)
{
    BgPt p;
    BgClosed b = closed_bg(c, lna);
    p.Hc = b.Hc;
    p.inv_Hc = 1.0 / b.Hc;
    p.fc = b.fc; p.fb = b.fb; p.fg = b.fg; p.fnu = b.fnu;
    p.Rinv = (4.0 / 3.0) * (c.Om_g / c.Om_b) * b.inv_a;
    Herm H = herm_at(lna);
    p.nuT = herm_val(tab, H, C_NUT, C_DNUT);
    p.cs2 = herm_val(tab, H, C_CS2, C_DCS2);
    p.tau = herm_val(tab, H, C_TAU, C_DTAU);
    return p;
}

// bisection for a root of f(x) - target on [lo, hi]; f monotone
template <class F>
ABCMB_HD double bisect(F f, double target, double lo, double hi, bool *ok)
{
    double flo = f(lo) - target, fhi = f(hi) - target;
    *ok = (flo < 0.0) != (fhi < 0.0);
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = f(mid) - target;
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; }
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}


// ---- lane helpers: on the device the builder runs on one warp per cosmology,
// on a host on one thread, or on an emulated warp where the host build
// defines ABCMB_HOST_WARPS (the CPU tests) ----
ABCMB_HD double lane_sum(double v)
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
#endif
    return v;
}

// sum of v over lanes below (dir > 0) or above (dir < 0) this one, in lane order
ABCMB_HD double lane_scan_excl(double v, int lane, int dir)
{
    double acc = 0.0;
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    for (int s = 0; s < 32; s++) {
        const int src = dir > 0 ? s : 31 - s;
        const double t = __shfl_sync(0xffffffffu, v, src);
        if (dir > 0 ? src < lane : src > lane) acc += t;
    }
#else
    (void)v; (void)lane; (void)dir;
#endif
    return acc;
}

ABCMB_HD void lane_sync()
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    __syncwarp();
#endif
}

// optical depth of the reionization electrons alone for a trial z_reion,
// composite Gauss-Legendre split over the lanes
ABCMB_HD double tau_reion_par(const Cosmo &c, double zre, int lane, int nl)
{
    const double dy = kBetaRe * kDzRe * pow(1.0 + zre, kBetaRe - 1.0);
    const double yre = pow(1.0 + zre, kBetaRe);
    double zmax = pow(yre + 25.0 * dy, 1.0 / kBetaRe) - 1.0;
    const double zhe = kZreHe + 25.0 * kDzReHe;
    if (zhe > zmax) zmax = zhe;
    const double lo = -log(1.0 + zmax);
    const int np = 800;
    const double hp = -lo / np;
    double acc = 0.0;
    for (int pnl = lane; pnl < np; pnl += nl)
        for (int q = 0; q < 4; q++) {
            const double lna = lo + hp * (pnl + 0.5 * (1.0 + gl4_x(q)));
            const double z = exp(-lna) - 1.0;
            const double S1 = 0.5 * (1.0 + tanh((yre - pow(1.0 + z, kBetaRe)) / dy));
            const double S2 = 0.5 * (1.0 + tanh((kZreHe - z) / kDzReHe));
            acc += 0.5 * hp * gl4_w(q) * ((1.0 + c.f_He) * S1 + c.f_He * S2) * nuT_closed(c, lna, 1.0);
        }
    return lane_sum(acc);
}

// ---- the builder (lane = 0..nl-1 of the warp that owns this cosmology) ----
ABCMB_HD void build_background(const double *p, double *rec, int n_tau, int lane, int nl, double m_ncdm = 0.0,
                               int node_recipe = 0)
{
    double *tab = rec + ABCMB_BG_TABLE;
    double *otab = rec + ABCMB_BG_ODETAB;
    double *nodes = rec + ABCMB_BG_NODES;
    int status = ABCMB_OK;
    bool ok = true;

    // derived parameters (every lane, identically)
    Cosmo c;
    const double h = p[2], h2 = h * h;
    c.H0 = h * 1.0e7 / kC;
    const double H100 = 1.0e7 / kMpc;
    const double rho_crit100 = 3.0 * H100 * H100 / (8.0 * kPi * kG) * kC * kC / kEvErg;
    const double T0 = kTcmb0, Tn = kTnuRatio * kTcmb0;
    const double hbc3 = kHbarC * kHbarC * kHbarC;
    c.rho_g0 = kPi * kPi / 15.0 * T0 * T0 * T0 * T0 / hbc3;
    // one massive neutrino: two massless species remain (App. A.1 example)
    const double n_massless = m_ncdm > 0.0 ? 2.0 : kNnu;
    const double rho_nu0 = n_massless * 7.0 * kPi * kPi / 120.0 * Tn * Tn * Tn * Tn / hbc3;
    c.Om_b = p[0] / h2;
    c.Om_c = p[1] / h2;
    c.Om_g = c.rho_g0 / (rho_crit100 * h2);
    c.Om_nu = rho_nu0 / (rho_crit100 * h2);
    c.ncdm_pref = c.ncdm_x1 = c.Om_ncdm_rel = 0.0;
    double Om_ncdm = 0.0;
    if (m_ncdm > 0.0) {
        const double Tm = kTncdmRatio * kTcmb0, Tm4 = Tm * Tm * Tm * Tm / hbc3;
        c.ncdm_x1 = m_ncdm / Tm;
        c.ncdm_pref = 4.0 / (kPi * kPi) * Tm4 / (rho_crit100 * h2);
        c.Om_ncdm_rel = 7.0 * kPi * kPi / 120.0 * Tm4 / (rho_crit100 * h2);
        double pn;
        ncdm_rho_p(c, 1.0, &Om_ncdm, &pn);
    }
    c.Om_r = c.Om_g + c.Om_nu + c.Om_ncdm_rel; // everything relativistic early on
    c.Om_m = c.Om_b + c.Om_c;
    c.Om_L = 1.0 - c.Om_m - (c.Om_g + c.Om_nu) - Om_ncdm;
    c.R_nu = (c.Om_nu + c.Om_ncdm_rel) / c.Om_r;
    c.f_He = kYHe / (kMHeOverMH * (1.0 - kYHe));
    c.nH0 = (1.0 - kYHe) * p[0] * rho_crit100 / kMH;
    c.A_s = exp(p[4]) * 1.0e-10;
    c.n_s = p[3];

    // helium and hydrogen phase switches
    c.lna_He3 = bisect([&](double l) { double d, dls;
                           double s = saha_s(c, exp(l), kEHe2, mu_eHe(), 1.0, &dls);
                           return saha_root(s, c.f_He, 1.0 + c.f_He, dls, &d); },
                       1e-9, -12.0, -5.0, &ok);
    if (!ok) status = ABCMB_E_BACKGROUND;
    c.lna_sw = bisect([&](double l) { double d; return xp_saha(c, l, &d); }, 0.99, -9.0, -6.0, &ok);
    if (!ok) status = ABCMB_E_BACKGROUND;

    // reionization redshift from tau_reion (lane-parallel quadrature, every
    // lane takes the same bisection path)
    // tau_reion(z) is smooth and increasing: regula falsi with the Illinois
    // modification (the retained end's value halved when the same end is
    // kept twice) converges superlinearly inside the bracket [0, 60], in about
    // a tenth of the evaluations bisection needs to reach rounding
    {
        double lo = 0.0, hi = 60.0;
        double flo = tau_reion_par(c, lo, lane, nl) - p[5], fhi = tau_reion_par(c, hi, lane, nl) - p[5];
        if (!(fhi >= 0.0) || !(flo <= 0.0)) status = ABCMB_E_BACKGROUND;
        double z = 0.5 * (lo + hi);
        int side = 0;
        for (int it = 0; it < 100 && status == ABCMB_OK; it++) {
            z = (fhi - flo) > 0.0 ? (lo * fhi - hi * flo) / (fhi - flo) : 0.5 * (lo + hi);
            if (!(z > lo && z < hi)) z = 0.5 * (lo + hi);
            if (hi - lo <= 1e-13 * (1.0 + hi)) break;
            const double f = tau_reion_par(c, z, lane, nl) - p[5];
            if (f == 0.0) break;
            if (f < 0.0) {
                lo = z;
                flo = f;
                if (side < 0) fhi *= 0.5;
                side = -1;
            } else {
                hi = z;
                fhi = f;
                if (side > 0) flo *= 0.5;
                side = 1;
            }
            if (fabs(f) <= 1e-15 * p[5]) break;
        }
        c.z_reion = z;
    }

    // Peebles TLA (x_p, then also T_m below z = 700), RK4, stored at the table
    // nodes at and after lna_sw.  The ln a-only parts of the right-hand side
    // at the stage points of the one-step-per-cell stretch (cell starts and
    // midpoints from node jc on) are tabulated by all lanes first, in the ODE
    // table's space (filled only later); the integration itself is
    // sequential, on lane 0: fine steps through the stiff transient after
    // lna_sw, then one RK4 step per table cell, each cell's first stage being
    // the previous node's stored derivative.
    {
        const int j0 = (int)ceil((c.lna_sw - kLna0) * ABCMB_BG_PER_UNIT);
        const int jc = (int)ceil((c.lna_sw + kTlaFineSpan - kLna0) * ABCMB_BG_PER_UNIT);
        double *pts = otab; // [2 (kNlna - jc) - 1][kTlaPtDoubles]
        for (int i = lane; i < 2 * (kNlna - jc) - 1; i += nl) {
            const TlaPt P = tla_point(c, kLna0 + (jc + 0.5 * i) * kDlna);
            double *d = pts + kTlaPtDoubles * i;
            d[0] = P.T; d[1] = P.nH; d[2] = P.H; d[3] = P.K; d[4] = P.be;
            d[5] = P.bex; d[6] = P.xhe; d[7] = P.g0; d[8] = P.e1; d[9] = P.e2; d[10] = P.iH;
        }
        lane_sync();
        if (lane == 0) {
            auto ptat = [&](int i) {
                const double *d = pts + kTlaPtDoubles * i;
                TlaPt P;
                P.T = d[0]; P.nH = d[1]; P.H = d[2]; P.K = d[3]; P.be = d[4];
                P.bex = d[5]; P.xhe = d[6]; P.g0 = d[7]; P.e1 = d[8]; P.e2 = d[9]; P.iH = d[10];
                return P;
            };
            double dum;
            double x = c.lna_sw;
            double y0 = xp_saha(c, x, &dum), y1 = 0.0;
            bool two = false;
            double dxp = 0.0, dTm = 0.0;
            for (int j = j0; j < kNlna; j++) {
                const double target = kLna0 + j * kDlna;
                if (j > jc && !(two == false && x < kLna700 && target >= kLna700)) {
                    // one RK4 step over the cell [j - 1, j] from tabulated stage points
                    const double hs = target - x;
                    const int i = 2 * (j - 1 - jc);
                    const TlaPt Pm = ptat(i + 1), Pe = ptat(i + 2);
                    double k2a, k2b, k3a, k3b, k4a, k4b;
                    const double k1a = dxp, k1b = dTm;
                    tla_rhs_pt(c, Pm, y0 + 0.5 * hs * k1a, y1 + 0.5 * hs * k1b, two, &k2a, &k2b);
                    tla_rhs_pt(c, Pm, y0 + 0.5 * hs * k2a, y1 + 0.5 * hs * k2b, two, &k3a, &k3b);
                    tla_rhs_pt(c, Pe, y0 + hs * k3a, y1 + hs * k3b, two, &k4a, &k4b);
                    y0 += hs / 6.0 * (k1a + 2.0 * k2a + 2.0 * k3a + k4a);
                    y1 += hs / 6.0 * (k1b + 2.0 * k2b + 2.0 * k3b + k4b);
                    x = target;
                    tla_rhs_pt(c, Pe, y0, y1, two, &dxp, &dTm);
                } else {
                    while (x < target) {
                        double hs = (x - c.lna_sw < kTlaFineSpan) ? kTlaFine : kDlna;
                        if (target - x < hs * (1.0 + 1e-9)) hs = target - x;
                        bool hit700 = false;
                        if (!two && x < kLna700 && x + hs >= kLna700) { hs = kLna700 - x; hit700 = true; }
                        double k1a, k1b, k2a, k2b, k3a, k3b, k4a, k4b;
                        tla_rhs(c, x, y0, y1, two, &k1a, &k1b);
                        tla_rhs(c, x + 0.5 * hs, y0 + 0.5 * hs * k1a, y1 + 0.5 * hs * k1b, two, &k2a, &k2b);
                        tla_rhs(c, x + 0.5 * hs, y0 + 0.5 * hs * k2a, y1 + 0.5 * hs * k2b, two, &k3a, &k3b);
                        tla_rhs(c, x + hs, y0 + hs * k3a, y1 + hs * k3b, two, &k4a, &k4b);
                        y0 += hs / 6.0 * (k1a + 2.0 * k2a + 2.0 * k3a + k4a);
                        y1 += hs / 6.0 * (k1b + 2.0 * k2b + 2.0 * k3b + k4b);
                        if (hit700) {
                            x = kLna700;
                            two = true;
                            const double xe = y0 + x_he(c, x, &dum);
                            y1 = kTcmb0 * exp(-x) * (1.0 - H_sec(c, x) / gamma_C(c, exp(x), xe));
                        } else {
                            x += hs;
                        }
                        if (x > target - 1e-14) x = target;
                    }
                    if (j >= jc) tla_rhs_pt(c, ptat(2 * (j - jc)), y0, y1, two, &dxp, &dTm);
                    else tla_rhs(c, target, y0, y1, two, &dxp, &dTm);
                }
                double *r = tab + 8 * j;
                r[C_XE] = y0;     // temporarily x_p
                r[C_KAPPA] = dxp; // temporarily dx_p/dln a
                r[C_CS2] = y1;    // temporarily T_m (z < 700)
                r[C_DCS2] = dTm;  // temporarily dT_m/dln a
            }
        }
        lane_sync();
    }

    // table: x_e, 1/(H tau_c), c_s^2, 1/H (lane-parallel)
    {
        const double yre = pow(1.0 + c.z_reion, kBetaRe);
        const double dyre = kBetaRe * kDzRe * pow(1.0 + c.z_reion, kBetaRe - 1.0);
        for (int j = lane; j < kNlna; j += nl) {
            const double lna = kLna0 + j * kDlna;
            double *r = tab + 8 * j;
            const BgClosed b = closed_bg(c, lna);
            double xp, dxp, dxh;
            if (lna < c.lna_sw) xp = xp_saha(c, lna, &dxp);
            else { xp = r[C_XE]; dxp = r[C_KAPPA]; }
            const double xh = x_he(c, lna, &dxh);
            const double xr = xp + xh, dxr = dxp + dxh;
            double Tm, dlnTm;
            if (lna < kLna700) Tm = tm_qs(c, lna, xr, dxr, &dlnTm);
            else { Tm = r[C_CS2]; dlnTm = r[C_DCS2] / Tm; }
            const double z = b.inv_a - 1.0;
            const double y = pow(1.0 + z, kBetaRe);
            const double t1 = tanh((yre - y) / dyre), t2 = tanh((kZreHe - z) / kDzReHe);
            const double S1 = 0.5 * (1.0 + t1), S2 = 0.5 * (1.0 + t2);
            const double dS1 = 0.5 * (1.0 - t1 * t1) * kBetaRe * y / dyre;
            const double dS2 = 0.5 * (1.0 - t2 * t2) * (1.0 + z) / kDzReHe;
            const double xe = xr + (1.0 + c.f_He - xr) * S1 + c.f_He * S2;
            const double dxe = dxr * (1.0 - S1) + (1.0 + c.f_He - xr) * dS1 + c.f_He * dS2;
            const double nuT = xe * c.nH0 * kSigmaT * kMpc * b.inv_a * b.inv_a / b.Hc;
            const double mub = kMH / ((1.0 + xe) * (1.0 - kYHe) + kYHe / kMHeOverMH);
            r[C_NUT] = nuT;
            r[C_DNUT] = nuT * (dxe / xe - 2.0 - b.dlnHc);
            r[C_CS2] = Tm / mub * (1.0 - dlnTm / 3.0);
            r[C_DTAU] = 1.0 / b.Hc;
            r[C_XE] = xe;
        }
    }
    lane_sync();
    for (int j = lane; j < kNlna; j += nl) {
        const int jl = j > 0 ? j - 1 : j, jh = j < kNlna - 1 ? j + 1 : j;
        tab[8 * j + C_DCS2] = (tab[8 * jh + C_CS2] - tab[8 * jl + C_CS2]) / ((jh - jl) * kDlna);
    }

    // conformal time: closed radiation+matter part plus the cumulative Lambda
    // correction; kappa: suffix sums of the exact cell integrals of the cubic
    // Hermite interpolant of 1/(H tau_c).  Cells are split into one
    // contiguous chunk per lane, chunk totals combined in lane order.
    {
        const int ncell = kNlna - 1;
        const int chunk = (ncell + nl - 1) / nl;
        const int c0 = lane * chunk, c1 = c0 + chunk < ncell ? c0 + chunk : ncell;
        double run = 0.0;
        for (int cell = c0; cell < c1; cell++) {
            const double l0 = kLna0 + cell * kDlna;
            for (int q = 0; q < 4; q++) {
                const double l = l0 + 0.5 * kDlna * (1.0 + gl4_x(q));
                const double a = exp(l);
                const double hrm = c.H0 * sqrt(c.Om_r / (a * a) + c.Om_m / a);
                run += 0.5 * kDlna * gl4_w(q) * (1.0 / hconf(c, l) - 1.0 / hrm);
            }
            tab[8 * (cell + 1) + C_TAU] = run; // partial, within the chunk
        }
        const double off = lane_scan_excl(run, lane, +1);
        lane_sync();
        for (int cell = c0; cell < c1; cell++) {
            const double lna = kLna0 + (cell + 1) * kDlna;
            tab[8 * (cell + 1) + C_TAU] += off + tau_rm(c, exp(lna));
        }
        if (lane == 0) tab[C_TAU] = tau_rm(c, exp(kLna0));
        lane_sync();
        // kappa
        double srun = 0.0;
        for (int cell = c1 - 1; cell >= c0; cell--) {
            const double *r0 = tab + 8 * cell, *r1 = r0 + 8;
            srun += 0.5 * kDlna * (r0[C_NUT] + r1[C_NUT]) + kDlna * kDlna / 12.0 * (r0[C_DNUT] - r1[C_DNUT]);
            tab[8 * cell + C_KAPPA] = srun; // partial, within the chunk
        }
        const double soff = lane_scan_excl(srun, lane, -1);
        lane_sync();
        for (int cell = c0; cell < c1; cell++) tab[8 * cell + C_KAPPA] += soff;
        if (lane == 0) tab[8 * (kNlna - 1) + C_KAPPA] = 0.0;
        lane_sync();
    }
    c.tau0 = tab[8 * (kNlna - 1) + C_TAU];

    // ODE table: (value, d/dln a) pairs of 1/H, 1/(H tau), f_c, f_b, f_g,
    // f_nu, 1/(H tau_c), R^-1/(H tau_c), c_s^2, H
    for (int j = lane; j < kNlna; j += nl) {
        const double lna = kLna0 + j * kDlna;
        const BgClosed b = closed_bg(c, lna);
        const double *r = tab + 8 * j;
        double *o = otab + 20 * j;
        const double ih = 1.0 / b.Hc, iht = ih / r[C_TAU];
        const double dlnE2 = 2.0 * (b.dlnHc - 1.0);
        const double Rinv = (4.0 / 3.0) * (c.Om_g / c.Om_b) * b.inv_a;
        o[0] = ih;
        o[1] = -ih * b.dlnHc;
        o[2] = iht;
        o[3] = iht * (-b.dlnHc - iht);
        o[4] = b.fc;
        o[5] = b.fc * (-3.0 - dlnE2);
        o[6] = b.fb;
        o[7] = b.fb * (-3.0 - dlnE2);
        o[8] = b.fg;
        o[9] = b.fg * (-4.0 - dlnE2);
        o[10] = b.fnu;
        o[11] = b.fnu * (-4.0 - dlnE2);
        o[12] = r[C_NUT];
        o[13] = r[C_DNUT];
        o[14] = Rinv * r[C_NUT];
        o[15] = Rinv * (r[C_DNUT] - r[C_NUT]);
        o[16] = r[C_CS2];
        o[17] = r[C_DCS2];
        o[18] = b.Hc;
        o[19] = b.Hc * b.dlnHc;
    }
    lane_sync();
    // the same table as one cubic per interval: the Hermite cubic of values
    // v0, v1 and slopes (per interval) d0, d1 is v0 + u (d0 + u (3 (v1 - v0)
    // - 2 d0 - d1 + u (d0 + d1 - 2 (v1 - v0))))
    double *opoly = rec + ABCMB_BG_ODEPOLY(n_tau);
    for (int j = lane; j < kNlna - 1; j += nl) {
        const double *o0 = otab + 20 * j, *o1 = o0 + 20;
        double *pc = opoly + 40 * j;
        for (int q = 0; q < 10; q++) {
            const double v0 = o0[2 * q], v1 = o1[2 * q];
            const double d0 = kDlna * o0[2 * q + 1], d1 = kDlna * o1[2 * q + 1], dv = v1 - v0;
            pc[4 * q] = v0;
            pc[4 * q + 1] = d0;
            pc[4 * q + 2] = 3.0 * dv - 2.0 * d0 - d1;
            pc[4 * q + 3] = d0 + d1 - 2.0 * dv;
        }
    }

    // tight-coupling start: H tau_c = R_tc (every lane, identically)
    c.lna_tc = bisect([&](double l) { Herm H = herm_at(l); return -herm_val(tab, H, C_NUT, C_DNUT); },
                      -1.0 / kRtc, kLna0 + 1.0, -3.0, &ok);
    if (!ok) status = ABCMB_E_BACKGROUND;

    // tau nodes (lane-parallel)
    double node_fail = 0.0;
    if (n_tau >= 8) {
        // recipe 0: 1/4 uniform in ln a to z = 1300, 1/2 uniform in z over
        // [1300, 900), the rest uniform in tau from z = 900 to today; recipe 1
        // (refined tail): 1/5, 2/5 over [1300, 900), 1/5 uniform in z over
        // [900, 300), the rest uniform in tau from z = 300
        const int nA = node_recipe ? n_tau / 5 : n_tau / 4, nB = node_recipe ? 2 * n_tau / 5 : n_tau / 2;
        const int nD = node_recipe ? n_tau / 5 : 0, nC = n_tau - nA - nB - nD;
        const double l1300 = -log(1301.0), lC = -log(1.0 + (node_recipe ? 300.0 : 900.0));
        const Herm HC = herm_at(lC);
        const double tC = herm_val(tab, HC, C_TAU, C_DTAU);
        for (int i = lane; i < n_tau; i += nl) {
            double lna;
            if (i < nA) lna = c.lna_tc + (l1300 - c.lna_tc) * i / nA;
            else if (i < nA + nB) lna = -log(1.0 + 1300.0 - 400.0 * (i - nA) / nB);
            else if (i < nA + nB + nD) lna = -log(1.0 + 900.0 - 600.0 * (i - nA - nB) / nD);
            else {
                const int jc = i - nA - nB - nD;
                const double tt = tC + (c.tau0 - tC) * jc / nC;
                bool ok2 = true;
                lna = jc == 0 ? lC
                    : bisect([&](double l) { Herm H = herm_at(l); return herm_val(tab, H, C_TAU, C_DTAU); },
                             tt, lC, 0.0, &ok2);
                if (!ok2) node_fail = 1.0;
            }
            const Herm H = herm_at(lna);
            const BgClosed b = closed_bg(c, lna);
            const double nu = herm_val(tab, H, C_NUT, C_DNUT);
            const double dnu = herm_der(tab, H, C_NUT, C_DNUT);
            const double kap = herm_val(tab, H, C_KAPPA, C_NUT, -1.0);
            const double emk = exp(-kap);
            const double g = b.Hc * nu * emk;
            double *nd = nodes + 8 * i;
            nd[N_LNA] = lna;
            nd[N_TAU] = herm_val(tab, H, C_TAU, C_DTAU);
            nd[N_G] = g;
            nd[N_DG] = g * (dnu / nu + b.dlnHc + nu);
            nd[N_EXPMK] = emk;
            nd[N_HC] = b.Hc;
            nd[N_DHC] = b.Hc * b.dlnHc;
        }
        lane_sync();
        for (int i = lane; i < n_tau; i += nl) {
            const double lo = nodes[8 * (i > 0 ? i - 1 : i) + N_TAU];
            const double hi = nodes[8 * (i < n_tau - 1 ? i + 1 : i) + N_TAU];
            nodes[8 * i + N_W] = 0.5 * (hi - lo);
        }
    }
    if (lane_sum(node_fail) > 0.0 && status == ABCMB_OK) status = ABCMB_E_BACKGROUND;

    if (!(c.tau0 > 0.0 && c.tau0 < 1e6) || !(c.lna_tc < 0.0)) {
        if (status == ABCMB_OK) status = ABCMB_E_NONFINITE;
    }
    if (lane == 0) {
        for (int i = ABCMB_S_COUNT; i < ABCMB_BG_NSCALAR; i++) rec[i] = 0.0;
        rec[ABCMB_S_STATUS] = status;
        rec[ABCMB_S_H0] = c.H0;
        rec[ABCMB_S_OMB] = c.Om_b;
        rec[ABCMB_S_OMC] = c.Om_c;
        rec[ABCMB_S_OMG] = c.Om_g;
        rec[ABCMB_S_OMNU] = c.Om_nu;
        rec[ABCMB_S_OML] = c.Om_L;
        rec[ABCMB_S_RNU] = c.R_nu;
        rec[ABCMB_S_FHE] = c.f_He;
        rec[ABCMB_S_NH0] = c.nH0;
        rec[ABCMB_S_AS] = c.A_s;
        rec[ABCMB_S_NS] = c.n_s;
        rec[ABCMB_S_ZREION] = c.z_reion;
        rec[ABCMB_S_LNA_TC] = c.lna_tc;
        rec[ABCMB_S_LNA_SW] = c.lna_sw;
        rec[ABCMB_S_TAU0] = c.tau0;
        rec[ABCMB_S_LNA_HE3] = c.lna_He3;
        rec[ABCMB_S_LNA_700] = kLna700;
        rec[ABCMB_S_NTAU] = n_tau;
        rec[ABCMB_S_NCDM_PREF] = c.ncdm_pref;
        rec[ABCMB_S_NCDM_X1] = c.ncdm_x1;
        rec[ABCMB_S_OMNCDM_REL] = c.Om_ncdm_rel;
    }
}

} // namespace abcmb
