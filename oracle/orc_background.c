/*
 * ORACLE (test infrastructure only; see orc.h).
 *
 * Background, thermal history and tau nodes of one flat-LCDM cosmology.
 *
 *  - densities: photons rho = pi^2/15 T^4 (App. C.4), massless neutrinos
 *    N 7 pi^2/120 T_nu^4 (App. C.5, Sec. 2.4 "Neutrino parameters"), baryons
 *    and CDM ~ a^-3 (App. C.2-C.3), Lambda fixed by flatness (App. A.2,
 *    derived omega_Lambda);
 *  - conformal time tau = int dln a / (a H), written as the exact
 *    radiation+matter closed form plus a quadrature of the Lambda correction;
 *  - helium: Saha HeIII/HeII until x_HeIII < 1e-9, then Saha HeII/HeI
 *    (App. B.1.1; the post-Saha correction and the helium ODE are not taken,
 *    a reading);
 *  - hydrogen: Saha (App. B.1.2, eq. SahaH) while x_p > 0.99, then a Peebles
 *    three-level atom (the TLA the paper cites in App. B.1.2).  Its rates are
 *    not printed in the paper and are taken from the literature: case-B
 *    recombination fit of Pequignot, Petitjean & Boisson (1991),
 *    photo-ionisation by detailed balance at the radiation temperature,
 *    Lambda_2s1s = 8.2245809 /s, Lyman-alpha escape through
 *    K = lambda_alpha^3 / (8 pi H).  Not compared with an external
 *    recombination code (none is available here); pinned by its Saha limit,
 *    its freeze-out range, the case-B coefficient against a textbook table
 *    and the visibility peak at the paper's fiducial recombination time;
 *  - matter temperature: T_m = T_CMB (1 - H/Gamma_C) for z > 700, then
 *    dT_m/dln a = (-2 H T_m + Gamma_C (T_CMB - T_m)) / H (App. B.1.2);
 *  - reionization: tanh steps (App. B.2, eqs. h_reion, y_reio, he_reion),
 *    patched as x_e = x_rec + (1 + f_He - x_rec) S_H + f_He S_He (a reading);
 *    z_reion from tau_reion by bisection (App. A.2, eq. tau_reion: only the
 *    reionization electrons count);
 *  - 1/tau_c = a n_e sigma_T, kappa, g, g' (App. B.4), baryon sound speed and
 *    mean mass (App. C.3);
 *  - start of tight coupling a_tc: H tau_c = R_tc (App. A.1, eq.
 *    k_start_small); start of each mode a_i(k) = min(a_tc, a_k) with
 *    k / H(a_k) = R_large (eq. k_start_large);
 *  - tau nodes: 1/4 uniform in ln a on [ln a_tc, ln a(z=1300)), 1/2 uniform in
 *    z on [1300, 900), 1/4 uniform in tau on [tau(z=900), tau_0); trapezoid
 *    weights in tau (App. B.6: trapezoid rules, no time cut).  Option
 *    node_recipe = 1: 1/5 in ln a, 2/5 over [1300, 900), 1/5 uniform in z
 *    over [900, 300), the rest uniform in tau from z = 300.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "orc.h"

/* ---- physical constants (CODATA 2018 / PDG) ---- */
#define O_PI 3.14159265358979323846
#define O_C_CMS 2.99792458e10
#define O_MPC_CM 3.0856775814913673e24
#define O_SIGMA_T 6.6524587321e-25     /* cm^2                              */
#define O_HC 1.239841984e-4            /* h c [eV cm]                       */
#define O_HBARC 1.973269804e-5         /* hbar c [eV cm]                    */
#define O_KB 8.617333262e-5            /* eV / K                            */
#define O_ME 510998.95                 /* m_e c^2 [eV]                      */
#define O_MH 938783073.6               /* m_H c^2 [eV]                      */
#define O_MHE_MH 3.971480              /* m(4He atom) / m(H atom)           */
#define O_EH 13.598434005              /* H ionization energy [eV]          */
#define O_EHE1 24.587387               /* He I ionization energy [eV]       */
#define O_EHE2 54.417760               /* He II ionization energy [eV]      */
#define O_L2S1S 8.2245809              /* 2s -> 1s two-photon rate [1/s]    */
#define O_G 6.67430e-8                 /* cm^3 / (g s^2)                    */
#define O_EV_ERG 1.602176634e-12

#define TH_PER_UNIT 2048  /* TLA table nodes per unit ln a */
#define KP_PER_UNIT 1024  /* kappa table nodes per unit ln a */
#define CT_PER_UNIT 128   /* conformal-time correction table */
#define LNA_MIN (-20.0)

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n.          */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; i++) {
        double z = cos(O_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; j++) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z; x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

#define GL_N 8
typedef struct { double x[GL_N], w[GL_N]; } gl_rule;
static gl_rule gl_make(void)
{
    gl_rule r;
    gauss_legendre(GL_N, r.x, r.w);
    return r;
}

static void hermite_basis(real_t u, real_t *h00, real_t *h10, real_t *h01, real_t *h11)
{
    *h00 = (1 + 2 * u) * (1 - u) * (1 - u);
    *h10 = u * (1 - u) * (1 - u);
    *h01 = u * u * (3 - 2 * u);
    *h11 = u * u * (u - 1);
}

/* ------------------------------------------------------------------ */
/* background                                                          */
/* One massive neutrino (App. B.3 "Massive neutrinos"): energy density and
   pressure in units of today's critical density by the 5-point Gauss-Laguerre
   rule the paper gives for the background,
     rho = (4/pi^2) T^4 a^-4 sum_i K_i (1 + e^-q_i) eps_i / q_i^2,
     p   = (4/(3 pi^2)) T^4 a^-4 sum_i K_i (1 + e^-q_i) / eps_i,
   eps_i = sqrt(q_i^2 + x^2), x = a m / T (the distribution is Fermi-Dirac in
   q: the e^eps of the printed f_0 is read as e^q, which the quadrature
   weights' q^4 e^q / (1 + e^q)^2 presuppose). */
static const real_t NCDM_Q5[5] = {0.583165, 2.0, 4.0, 7.26582, 13.0};
static const real_t NCDM_K5[5] = {0.0081201, 0.689407, 2.8063, 2.05156, 0.12681};

static void ncdm_rho_p(const orc_cosmo *c, real_t a, real_t *rho, real_t *p)
{
    *rho = *p = 0.0;
    if (c->ncdm_pref == 0.0) return;
    const real_t x = a * c->ncdm_x1, a4 = a * a * a * a;
    real_t sr = 0.0, sp = 0.0;
    for (int i = 0; i < 5; i++) {
        const real_t q = NCDM_Q5[i], eps = sqrt(q * q + x * x), w = NCDM_K5[i] * (1.0 + exp(-q));
        sr += w * eps / (q * q);
        sp += w / eps;
    }
    *rho = c->ncdm_pref * sr / a4;
    *p = c->ncdm_pref * sp / (3.0 * a4);
}

static real_t E2(const orc_cosmo *c, real_t a)
{
    real_t rn = 0.0, pn = 0.0;
    ncdm_rho_p(c, a, &rn, &pn);
    return (c->Om_g + c->Om_nu) / (a * a * a * a) + c->Om_m / (a * a * a) + c->Om_L + rn;
}

real_t orc_Hconf(const orc_cosmo *c, real_t lna)
{
    real_t a = exp(lna);
    return a * c->H0 * sqrt(E2(c, a));
}

/* radiation+matter conformal time, exact: 2a / (H0 (sqrt(Om_r+Om_m a)+sqrt(Om_r))) */
static real_t tau_rm(const orc_cosmo *c, real_t a)
{
    return 2.0 * a / (c->H0 * (sqrt(c->Om_r + c->Om_m * a) + sqrt(c->Om_r)));
}

static real_t tau_corr_integrand(const orc_cosmo *c, real_t lna)
{
    real_t a = exp(lna);
    real_t hc = a * c->H0 * sqrt(E2(c, a));
    real_t hrm = c->H0 * sqrt(c->Om_r / (a * a) + c->Om_m / a);
    return 1.0 / hc - 1.0 / hrm;
}

real_t orc_tau_of_lna(const orc_cosmo *c, real_t lna)
{
    real_t a = exp(lna);
    real_t t = (lna - c->ct_lna0) / c->ct_dlna;
    int i = (int)floor(RE(t));
    if (i < 0) return tau_rm(c, a);
    if (i > c->n_ct - 2) i = c->n_ct - 2;
    real_t u = t - i, h = c->ct_dlna, l0 = c->ct_lna0 + i * h;
    real_t d0 = tau_corr_integrand(c, l0), d1 = tau_corr_integrand(c, l0 + h);
    real_t h00, h10, h01, h11;
    hermite_basis(u, &h00, &h10, &h01, &h11);
    real_t corr = h00 * c->ct_tau[i] + h10 * h * d0 + h01 * c->ct_tau[i + 1] + h11 * h * d1;
    return tau_rm(c, a) + corr;
}

/* ------------------------------------------------------------------ */
/* recombination pieces                                                */
static real_t saha_pref(real_t T, real_t mu) /* (2 pi mu T / (hc)^2)^{3/2} [cm^-3] */
{
    real_t v = 2.0 * O_PI * mu * T / (O_HC * O_HC);
    return v * sqrt(v);
}

static real_t nH_of(const orc_cosmo *c, real_t a) { return c->nH0 / (a * a * a); }
static real_t Tg_of(const orc_cosmo *c, real_t a) { return c->TCMB0 / a; }
static real_t mu_eHe(void) { return O_ME * (O_MHE_MH * O_MH) / (O_ME + O_MHE_MH * O_MH); }
static real_t mu_eH(void) { return O_ME * O_MH / (O_ME + O_MH); }

static real_t x_heIII_saha(const orc_cosmo *c, real_t a)
{
    real_t T = Tg_of(c, a), f = c->f_He;
    real_t s = saha_pref(T, mu_eHe()) * exp(-O_EHE2 / T) / nH_of(c, a);
    real_t b = 1.0 + f + s;
    return 2.0 * s * f / (b + sqrt(b * b + 4.0 * s * f));
}

static real_t x_heII_saha(const orc_cosmo *c, real_t a)
{
    real_t T = Tg_of(c, a), f = c->f_He;
    real_t s = 4.0 * saha_pref(T, mu_eHe()) * exp(-O_EHE1 / T) / nH_of(c, a);
    real_t b = 1.0 + s;
    return 2.0 * s * f / (b + sqrt(b * b + 4.0 * s * f));
}

static real_t x_he(const orc_cosmo *c, real_t lna)
{
    real_t a = exp(lna);
    if (RE(lna) < RE(c->lna_He3)) return c->f_He + x_heIII_saha(c, a);
    return x_heII_saha(c, a);
}

static real_t xp_saha(const orc_cosmo *c, real_t a)
{
    real_t T = Tg_of(c, a);
    real_t s = saha_pref(T, mu_eH()) * exp(-O_EH / T) / nH_of(c, a);
    return 2.0 / (1.0 + sqrt(1.0 + 4.0 / s));
}

static real_t alpha_B(real_t T_eV) /* cm^3/s, Pequignot et al. (1991) case-B fit */
{
    real_t t = T_eV / O_KB / 1.0e4;
    return 1.0e-13 * 4.309 * pow(t, -0.6166) / (1.0 + 0.6703 * pow(t, 0.5300));
}

/* the case-B coefficient, for the oracle's own pins */
real_t orc_alpha_B_at(real_t T_eV) { return alpha_B(T_eV); }

static real_t H_sec(const orc_cosmo *c, real_t a) /* H [1/s] */
{
    return c->H0 * sqrt(E2(c, a)) * O_C_CMS / O_MPC_CM;
}

/* Compton rate Gamma_C [1/s] (App. B.1.2) for recombination x_e */
static real_t gamma_C(const orc_cosmo *c, real_t a, real_t xe)
{
    real_t rho_g = c->rho_g0 / (a * a * a * a);
    return 8.0 * O_SIGMA_T * O_C_CMS * rho_g / (3.0 * O_ME) * xe / (1.0 + c->f_He + xe);
}

static real_t Tm_quasistatic(const orc_cosmo *c, real_t a, real_t xe)
{
    return Tg_of(c, a) * (1.0 - H_sec(c, a) / gamma_C(c, a, xe));
}

/* Peebles TLA (+ T_m ODE when with_Tm) right-hand side in ln a. */
static void tla_rhs(const orc_cosmo *c, real_t lna, const real_t *y, int with_Tm, real_t *dy)
{
    real_t a = exp(lna);
    real_t xp = y[0];
    real_t xe = xp + x_he(c, lna);
    real_t Tg = Tg_of(c, a);
    real_t Tm = with_Tm ? y[1] : Tm_quasistatic(c, a, xe);
    real_t nH = nH_of(c, a), H = H_sec(c, a);
    real_t alpha = alpha_B(Tm);
    real_t beta = alpha_B(Tg) * saha_pref(Tg, mu_eH()) * exp(-0.25 * O_EH / Tg);
    real_t lam = O_HC / (0.75 * O_EH);
    real_t K = lam * lam * lam / (8.0 * O_PI * H);
    real_t n1s = nH * (1.0 - xp);
    real_t C = (1.0 + K * O_L2S1S * n1s) / (1.0 + K * (O_L2S1S + beta) * n1s);
    real_t dxdt = -C * (alpha * nH * xe * xp - beta * (1.0 - xp) * exp(-0.75 * O_EH / Tg));
    dy[0] = dxdt / H;
    if (with_Tm) dy[1] = -2.0 * Tm + gamma_C(c, a, xe) / H * (Tg - Tm);
}

/* 3-stage Radau IIA coefficients (Hairer & Wanner, order 5). */
static void radau_tableau(real_t A[3][3], real_t cc[3])
{
    real_t s6 = sqrt(6.0);
    A[0][0] = (88.0 - 7.0 * s6) / 360.0;
    A[0][1] = (296.0 - 169.0 * s6) / 1800.0;
    A[0][2] = (-2.0 + 3.0 * s6) / 225.0;
    A[1][0] = (296.0 + 169.0 * s6) / 1800.0;
    A[1][1] = (88.0 + 7.0 * s6) / 360.0;
    A[1][2] = (-2.0 - 3.0 * s6) / 225.0;
    A[2][0] = (16.0 - s6) / 36.0;
    A[2][1] = (16.0 + s6) / 36.0;
    A[2][2] = 1.0 / 9.0;
    cc[0] = (4.0 - s6) / 10.0;
    cc[1] = (4.0 + s6) / 10.0;
    cc[2] = 1.0;
}

/* Exposed for the order-condition pin. */
void orc_radau_tableau(real_t *out12)
{
    real_t A[3][3], cc[3];
    radau_tableau(A, cc);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) out12[3 * i + j] = A[i][j];
    for (int i = 0; i < 3; i++) out12[9 + i] = cc[i];
}

/* One Radau IIA step of the (n <= 2)-dimensional TLA system; simplified
   Newton with a finite-difference Jacobian, iterated to convergence. */
static int tla_radau_step(const orc_cosmo *c, real_t x, real_t h, real_t *y, int n)
{
    real_t A[3][3], cc[3];
    radau_tableau(A, cc);
    real_t J[2][2], f0[2], f1[2], yp[2];
    tla_rhs(c, x, y, n == 2, f0);
    for (int j = 0; j < n; j++) {
        real_t d = 1e-7 * (ABS(y[j]) + 1e-12);
        memcpy(yp, y, sizeof(real_t) * n);
        yp[j] += d;
        tla_rhs(c, x, yp, n == 2, f1);
        memcpy(yp, y, sizeof(real_t) * n);
        yp[j] -= d;
        real_t fm[2];
        tla_rhs(c, x, yp, n == 2, fm);
        for (int i = 0; i < n; i++) J[i][j] = (f1[i] - fm[i]) / (2.0 * d);
    }
    int m = 3 * n;
    real_t M[36], Z[6] = {0}, R[6];
    int piv[6], ext[12];
    for (int si = 0; si < 3; si++)
        for (int sj = 0; sj < 3; sj++)
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++)
                    M[(si * n + i) * m + sj * n + j] = (si == sj && i == j ? 1.0 : 0.0) - h * A[si][sj] * J[i][j];
    if (orc_lu_factor(M, m, piv, ext)) return -1;
    int extra = 0;
    for (int it = 0; it < 60; it++) {
        real_t F[3][2];
        for (int s = 0; s < 3; s++) {
            real_t ys[2];
            for (int i = 0; i < n; i++) ys[i] = y[i] + Z[s * n + i];
            tla_rhs(c, x + cc[s] * h, ys, n == 2, F[s]);
        }
        for (int s = 0; s < 3; s++)
            for (int i = 0; i < n; i++) {
                real_t acc = 0.0;
                for (int t = 0; t < 3; t++) acc += A[s][t] * F[t][i];
                R[s * n + i] = -(Z[s * n + i] - h * acc);
            }
        orc_lu_solve(M, m, piv, ext, R);
        real_t dmax = 0.0;
        for (int i = 0; i < m; i++) {
            Z[i] += R[i];
            real_t sc = ABS(R[i]) / (ABS(y[i % n]) + 1e-300);
            if (RE(sc) > RE(dmax)) dmax = sc;
        }
        /* the complex build iterates twice more, so that the imaginary parts
           (contracted by the same iteration) are converged as well */
        if (RE(dmax) < 1e-15 && ++extra > ORC_CS_EXTRA) break;
    }
    for (int i = 0; i < n; i++) y[i] += Z[2 * n + i];
    return 0;
}

/* locate ln a in the two-segment TLA table: returns interval index, u in [0,1] */
static int th_locate(const orc_cosmo *c, real_t lna, real_t *u, real_t *h)
{
    int n1 = c->n_th1, n = c->n_th1 + c->n_th2;
    int i;
    if (RE(lna) <= RE(c->lna_700)) {
        real_t dl = (c->lna_700 - c->lna_sw) / n1;
        i = (int)floor(RE((lna - c->lna_sw) / dl));
        if (i < 0) i = 0;
        if (i > n1 - 1) i = n1 - 1;
    } else {
        real_t dl = (0.0 - c->lna_700) / c->n_th2;
        i = n1 + (int)floor(RE((lna - c->lna_700) / dl));
        if (i < n1) i = n1;
        if (i > n - 1) i = n - 1;
    }
    *h = c->th_lna[i + 1] - c->th_lna[i];
    *u = (lna - c->th_lna[i]) / *h;
    return i;
}

static real_t th_interp(const orc_cosmo *c, const real_t *v, const real_t *dv, real_t lna)
{
    real_t u, h, h00, h10, h01, h11;
    int i = th_locate(c, lna, &u, &h);
    hermite_basis(u, &h00, &h10, &h01, &h11);
    return h00 * v[i] + h10 * h * dv[i] + h01 * v[i + 1] + h11 * h * dv[i + 1];
}

/* recombination-only electron fraction (no reionization) */
static real_t xe_rec(const orc_cosmo *c, real_t lna)
{
    real_t xp;
    if (RE(lna) < RE(c->lna_sw)) xp = xp_saha(c, exp(lna));
    else xp = th_interp(c, c->th_xp, c->th_dxp, lna);
    return xp + x_he(c, lna);
}

static real_t tanh_step(real_t u) { return 0.5 * (1.0 + tanh(u)); }

real_t orc_xe_of_lna(const orc_cosmo *c, real_t lna, real_t *dxe)
{
    if (c->hooks & ORC_HOOK_EDS_CDM) { if (dxe) *dxe = 0.0; return 0.0; }
    real_t z = exp(-lna) - 1.0;
    real_t beta = c->beta_re;
    real_t y = pow(1.0 + z, beta), yre = pow(1.0 + c->z_reion, beta);
    real_t dy = beta * c->dz_re * pow(1.0 + c->z_reion, beta - 1.0);
    real_t u1 = (yre - y) / dy, u2 = (c->z_re_He - z) / c->dz_re_He;
    real_t S1 = tanh_step(u1), S2 = tanh_step(u2);
    real_t xr = xe_rec(c, lna);
    real_t xe = xr + (1.0 + c->f_He - xr) * S1 + c->f_He * S2;
    if (dxe) {
        const real_t d = 1e-5;
        real_t dxr = (xe_rec(c, lna + d) - xe_rec(c, lna - d)) / (2.0 * d);
        real_t t1 = tanh(u1), t2 = tanh(u2);
        real_t dS1 = 0.5 * (1.0 - t1 * t1) * beta * y / dy;      /* dy/dlna = -beta y */
        real_t dS2 = 0.5 * (1.0 - t2 * t2) * (1.0 + z) / c->dz_re_He;
        *dxe = dxr * (1.0 - S1) + (1.0 + c->f_He - xr) * dS1 + c->f_He * dS2;
    }
    return xe;
}

/* matter temperature [eV] and its logarithmic derivative */
real_t orc_Tm_of_lna(const orc_cosmo *c, real_t lna, real_t *dlnTm)
{
    real_t a = exp(lna);
    if (RE(lna) < RE(c->lna_700)) {
        real_t Tm = Tm_quasistatic(c, a, xe_rec(c, lna));
        if (dlnTm) {
            const real_t d = 1e-5;
            real_t tp = Tm_quasistatic(c, exp(lna + d), xe_rec(c, lna + d));
            real_t tm = Tm_quasistatic(c, exp(lna - d), xe_rec(c, lna - d));
            *dlnTm = (log(tp) - log(tm)) / (2.0 * d);
        }
        return Tm;
    }
    real_t Tm = th_interp(c, c->th_Tm, c->th_dTm, lna);
    if (dlnTm) {
        real_t y[2] = {th_interp(c, c->th_xp, c->th_dxp, lna), Tm}, dy[2];
        tla_rhs(c, lna, y, 1, dy);
        *dlnTm = dy[1] / Tm;
    }
    return Tm;
}

static real_t nuT_of(const orc_cosmo *c, real_t lna, real_t xe)
{
    real_t a = exp(lna);
    return xe * c->nH0 * O_SIGMA_T * O_MPC_CM / (a * a * orc_Hconf(c, lna));
}

static real_t kappa_of(const orc_cosmo *c, real_t lna)
{
    real_t t = (lna - c->kp_lna0) / c->kp_dlna;
    int i = (int)floor(RE(t));
    if (i < 0) i = 0;
    if (i > c->n_kp - 2) i = c->n_kp - 2;
    real_t u = t - i, h = c->kp_dlna, l0 = c->kp_lna0 + i * h;
    real_t d0 = -nuT_of(c, l0, orc_xe_of_lna(c, l0, NULL));
    real_t d1 = -nuT_of(c, l0 + h, orc_xe_of_lna(c, l0 + h, NULL));
    real_t h00, h10, h01, h11;
    hermite_basis(u, &h00, &h10, &h01, &h11);
    return h00 * c->kp_kappa[i] + h10 * h * d0 + h01 * c->kp_kappa[i + 1] + h11 * h * d1;
}

void orc_bg_eval(const orc_cosmo *c, real_t lna, orc_bg *o, int with_thermo)
{
    real_t a = exp(lna);
    real_t e2 = E2(c, a);
    o->a = a;
    o->Hc = a * c->H0 * sqrt(e2);
    real_t rg = c->Om_g / (a * a * a * a), rn = c->Om_nu / (a * a * a * a);
    real_t rb = c->Om_b / (a * a * a), rc = c->Om_c / (a * a * a);
    real_t rm = 0.0, pm = 0.0;
    ncdm_rho_p(c, a, &rm, &pm);
    o->fc = rc / e2; o->fb = rb / e2; o->fg = rg / e2; o->fnu = rn / e2;
    o->fncdm = rm / e2;
    o->wncdm = RE(rm) > 0.0 ? pm / rm : 0.0;
    o->ncdm_x = a * c->ncdm_x1;
    o->ncdm_n = c->ncdm_pref / (a * a * a * a * e2);
    /* d ln H_conf / d ln a = 1 + (1/2) d ln E^2 / d ln a, d rho_ncdm / d ln a = -3 (rho + p) */
    o->dHc = o->Hc * (1.0 + 0.5 * (-4.0 * (rg + rn) - 3.0 * (rb + rc) - 3.0 * (rm + pm)) / e2);
    o->tau = orc_tau_of_lna(c, lna);
    o->Rinv = RE(c->Om_b) > 0.0 ? (4.0 / 3.0) * c->Om_g / (c->Om_b * a) : 0.0;
    if (!with_thermo || (c->hooks & ORC_HOOK_EDS_CDM)) {
        o->xe = o->dxe = o->nuT = o->cs2 = 0.0;
        o->kappa = 0.0; o->expmk = 1.0; o->g = o->dg = 0.0;
        return;
    }
    real_t dxe = 0.0;
    o->xe = orc_xe_of_lna(c, lna, with_thermo >= 2 ? &dxe : NULL);
    o->dxe = dxe;
    o->nuT = nuT_of(c, lna, o->xe);
    real_t dlnTm;
    real_t Tm = orc_Tm_of_lna(c, lna, &dlnTm);
    real_t mub = O_MH / ((1.0 + o->xe) * (1.0 - c->YHe) + c->YHe / O_MHE_MH);
    o->cs2 = Tm / mub * (1.0 - dlnTm / 3.0);
    if (with_thermo < 2) {
        o->kappa = 0.0; o->expmk = 1.0; o->g = o->dg = 0.0;
        return;
    }
    o->kappa = kappa_of(c, lna);
    o->expmk = exp(-o->kappa);
    o->g = o->Hc * o->nuT * o->expmk;
    o->dg = o->g * (dxe / o->xe - 2.0 + o->nuT);
}

/* ------------------------------------------------------------------ */
/* Root of f(c, x, arg) = 0 in [lo, hi] by bisection on the real parts.  The
   complex build then adds the root's imaginary part to first order: f(r +
   i s) = 0 gives s = -Im f(r) / f'(r), f' by a central difference of the
   real part (relative accuracy ~1e-10, far below what the tests resolve). */
static real_t root_im(real_t (*f)(const orc_cosmo *, real_t, real_t), const orc_cosmo *c, real_t arg, double r)
{
#ifdef ORC_CS
    const double d = 1e-6 * (fabs(r) + 1e-3);
    const double fp = (RE(f(c, r + d, arg)) - RE(f(c, r - d, arg))) / (2.0 * d);
    return r - I * (IM(f(c, r, arg)) / fp);
#else
    (void)f; (void)c; (void)arg;
    return r;
#endif
}

static real_t bisect(real_t (*f)(const orc_cosmo *, real_t, real_t), const orc_cosmo *c,
                     real_t arg, double lo, double hi)
{
    real_t flo = f(c, lo, arg);
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        real_t fm = f(c, mid, arg);
        if ((RE(fm) < 0.0) == (RE(flo) < 0.0)) { lo = mid; flo = fm; }
        else hi = mid;
    }
    return root_im(f, c, arg, 0.5 * (lo + hi));
}

static real_t f_he3(const orc_cosmo *c, real_t lna, real_t arg)
{ return x_heIII_saha(c, exp(lna)) - arg; }
static real_t f_hsw(const orc_cosmo *c, real_t lna, real_t arg)
{ return xp_saha(c, exp(lna)) - arg; }
static real_t f_tc(const orc_cosmo *c, real_t lna, real_t arg)
{ return nuT_of(c, lna, orc_xe_of_lna(c, lna, NULL)) - arg; }
static real_t f_Hk(const orc_cosmo *c, real_t lna, real_t arg)
{ return orc_Hconf(c, lna) - arg; }
static real_t f_tau(const orc_cosmo *c, real_t lna, real_t arg)
{ return orc_tau_of_lna(c, lna) - arg; }

/* optical depth from the reionization electrons alone, for a trial z_reion */
static real_t tau_reion_of(const orc_cosmo *c, real_t zre, const gl_rule *gl)
{
    real_t beta = c->beta_re;
    real_t dy = beta * c->dz_re * pow(1.0 + zre, beta - 1.0);
    real_t ymax = pow(1.0 + zre, beta) + 25.0 * dy;
    real_t zmax = pow(ymax, 1.0 / beta) - 1.0;
    real_t zhe = c->z_re_He + 25.0 * c->dz_re_He;
    if (RE(zhe) > RE(zmax)) zmax = zhe;
    real_t lo = -log(1.0 + zmax);
    int np = 400;
    real_t hp = (0.0 - lo) / np, acc = 0.0;
    for (int p = 0; p < np; p++) {
        for (int q = 0; q < GL_N; q++) {
            real_t lna = lo + hp * (p + 0.5 * (1.0 + gl->x[q]));
            real_t a = exp(lna), z = 1.0 / a - 1.0;
            real_t S1 = tanh_step((pow(1.0 + zre, beta) - pow(1.0 + z, beta)) / dy);
            real_t S2 = tanh_step((c->z_re_He - z) / c->dz_re_He);
            real_t xre = (1.0 + c->f_He) * S1 + c->f_He * S2;
            acc += 0.5 * hp * gl->w[q] * xre * nuT_of(c, lna, 1.0);
        }
    }
    return acc;
}

int orc_cosmo_init(orc_cosmo *c, const real_t p[6], int n_tau, int hooks, double m_ncdm, int node_recipe)
{
    memset(c, 0, sizeof(*c));
    gl_rule gl = gl_make();
    c->omega_b = p[0]; c->omega_cdm = p[1]; c->h = p[2];
    c->n_s = p[3]; c->ln10As = p[4]; c->tau_reio = p[5];
    c->hooks = hooks;
    c->YHe = 0.245; c->TCMB0 = 2.34865418e-4; c->Tnu_ratio = 0.71636856; c->N_nu = 3.0;
    c->m_ncdm = m_ncdm > 0.0 ? m_ncdm : 0.0;
    c->T_ncdm_ratio = 0.71611;
    if (RE(c->m_ncdm) > 0.0) c->N_nu = 2.0; /* App. A.1 example: two massless + one massive */
    c->z_re_He = 3.5; c->dz_re_He = 0.5; c->dz_re = 0.5; c->beta_re = 1.5;
    c->R_tc = 1.5e-3; c->R_large = 7e-2; c->k_pivot = 0.05;
    c->A_s = exp(c->ln10As) * 1e-10;
    c->H0 = c->h * 1.0e7 / O_C_CMS; /* 100 h km/s/Mpc divided by c, in 1/Mpc */
    real_t H100 = 1.0e7 / O_MPC_CM;  /* s^-1 */
    real_t rho_crit100 = 3.0 * H100 * H100 / (8.0 * O_PI * O_G) * O_C_CMS * O_C_CMS / O_EV_ERG; /* eV/cm^3 */
    real_t T = c->TCMB0;
    c->rho_g0 = O_PI * O_PI / 15.0 * T * T * T * T / (O_HBARC * O_HBARC * O_HBARC);
    real_t Tn = c->Tnu_ratio * T;
    real_t rho_nu0 = c->N_nu * 7.0 * O_PI * O_PI / 120.0 * Tn * Tn * Tn * Tn / (O_HBARC * O_HBARC * O_HBARC);
    real_t h2 = c->h * c->h;
    if (hooks & ORC_HOOK_EDS_CDM) {
        c->Om_c = 1.0; c->Om_m = 1.0;
    } else {
        c->Om_b = c->omega_b / h2;
        c->Om_c = c->omega_cdm / h2;
        c->Om_g = c->rho_g0 / (rho_crit100 * h2);
        c->Om_nu = rho_nu0 / (rho_crit100 * h2);
        if (RE(c->m_ncdm) > 0.0) {
            const real_t Tm = c->T_ncdm_ratio * T, Tm4 = Tm * Tm * Tm * Tm / (O_HBARC * O_HBARC * O_HBARC);
            c->ncdm_x1 = c->m_ncdm / Tm;
            c->ncdm_pref = 4.0 / (O_PI * O_PI) * Tm4 / (rho_crit100 * h2);
            c->Om_ncdm_rel = 7.0 * O_PI * O_PI / 120.0 * Tm4 / (rho_crit100 * h2);
            real_t pm;
            ncdm_rho_p(c, 1.0, &c->Om_ncdm, &pm);
        }
        /* Om_r: everything relativistic early on (the base of the conformal-time integral) */
        c->Om_r = c->Om_g + c->Om_nu + c->Om_ncdm_rel;
        c->Om_m = c->Om_b + c->Om_c;
        c->Om_L = 1.0 - c->Om_m - (c->Om_g + c->Om_nu) - c->Om_ncdm;
        c->R_nu = (c->Om_nu + c->Om_ncdm_rel) / c->Om_r;
    }
    c->f_He = c->YHe / (O_MHE_MH * (1.0 - c->YHe));
    c->nH0 = (1.0 - c->YHe) * c->omega_b * rho_crit100 / O_MH;

    /* conformal-time correction table */
    c->ct_lna0 = LNA_MIN;
    c->ct_dlna = 1.0 / CT_PER_UNIT;
    c->n_ct = (int)(-LNA_MIN * CT_PER_UNIT) + 1;
    c->ct_tau = (real_t *)calloc(c->n_ct, sizeof(real_t));
    for (int i = 1; i < c->n_ct; i++) {
        real_t l0 = c->ct_lna0 + (i - 1) * c->ct_dlna, acc = 0.0;
        for (int q = 0; q < GL_N; q++)
            acc += 0.5 * c->ct_dlna * gl.w[q] * tau_corr_integrand(c, l0 + 0.5 * c->ct_dlna * (1.0 + gl.x[q]));
        c->ct_tau[i] = c->ct_tau[i - 1] + acc;
    }
    c->tau0 = orc_tau_of_lna(c, 0.0);
    if (hooks & ORC_HOOK_EDS_CDM) return 0;

    /* helium HeIII -> HeII switch, hydrogen Saha -> TLA switch */
    c->lna_He3 = bisect(f_he3, c, 1e-9, -12.0, -5.0);
    c->lna_sw = bisect(f_hsw, c, 0.99, -9.0, -6.0);
    c->lna_700 = -log(701.0);

    /* TLA table */
    c->n_th1 = (int)ceil(RE(c->lna_700 - c->lna_sw) * TH_PER_UNIT);
    c->n_th2 = (int)ceil(RE(0.0 - c->lna_700) * TH_PER_UNIT);
    int nth = c->n_th1 + c->n_th2 + 1;
    c->th_lna = (real_t *)malloc(sizeof(real_t) * nth);
    c->th_xp = (real_t *)malloc(sizeof(real_t) * nth);
    c->th_dxp = (real_t *)malloc(sizeof(real_t) * nth);
    c->th_Tm = (real_t *)malloc(sizeof(real_t) * nth);
    c->th_dTm = (real_t *)malloc(sizeof(real_t) * nth);
    for (int i = 0; i <= c->n_th1; i++)
        c->th_lna[i] = c->lna_sw + (c->lna_700 - c->lna_sw) * i / c->n_th1;
    for (int i = 1; i <= c->n_th2; i++)
        c->th_lna[c->n_th1 + i] = c->lna_700 + (0.0 - c->lna_700) * i / c->n_th2;
    c->th_lna[nth - 1] = 0.0;
    real_t y[2] = {xp_saha(c, exp(c->lna_sw)), 0.0}, dy[2];
    for (int i = 0; i < nth; i++) {
        real_t lna = c->th_lna[i];
        int two = (i >= c->n_th1);
        if (i == c->n_th1)
            y[1] = Tm_quasistatic(c, exp(lna), y[0] + x_he(c, lna));
        tla_rhs(c, lna, y, two, dy);
        c->th_xp[i] = y[0];
        c->th_dxp[i] = dy[0];
        if (two) { c->th_Tm[i] = y[1]; c->th_dTm[i] = dy[1]; }
        else { c->th_Tm[i] = Tm_quasistatic(c, exp(lna), y[0] + x_he(c, lna)); c->th_dTm[i] = 0.0; }
        if (i + 1 < nth) {
            real_t h = c->th_lna[i + 1] - lna;
            if (tla_radau_step(c, lna, h, y, two ? 2 : 1)) return -1;
        }
    }

    /* reionization redshift from tau_reion */
    {
        double lo = 0.0, hi = 60.0;
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (RE(tau_reion_of(c, mid, &gl)) < RE(c->tau_reio)) lo = mid; else hi = mid;
        }
        c->z_reion = 0.5 * (lo + hi);
#ifdef ORC_CS
        /* the root's imaginary part, as in root_im */
        const double zr = RE(c->z_reion), d = 1e-6 * (zr + 1.0);
        const double fp = (RE(tau_reion_of(c, zr + d, &gl)) - RE(tau_reion_of(c, zr - d, &gl))) / (2.0 * d);
        c->z_reion = zr - I * (IM(tau_reion_of(c, zr, &gl) - c->tau_reio) / fp);
#endif
    }

    /* optical depth table, integrated from today backwards */
    c->kp_lna0 = LNA_MIN;
    c->kp_dlna = 1.0 / KP_PER_UNIT;
    c->n_kp = (int)(-LNA_MIN * KP_PER_UNIT) + 1;
    c->kp_kappa = (real_t *)calloc(c->n_kp, sizeof(real_t));
    for (int i = c->n_kp - 2; i >= 0; i--) {
        real_t l0 = c->kp_lna0 + i * c->kp_dlna, acc = 0.0;
        for (int q = 0; q < GL_N; q++) {
            real_t lna = l0 + 0.5 * c->kp_dlna * (1.0 + gl.x[q]);
            acc += 0.5 * c->kp_dlna * gl.w[q] * nuT_of(c, lna, orc_xe_of_lna(c, lna, NULL));
        }
        c->kp_kappa[i] = c->kp_kappa[i + 1] + acc;
    }

    /* tight-coupling start */
    c->lna_tc = bisect(f_tc, c, 1.0 / c->R_tc, LNA_MIN + 1.0, -3.0);

    /* tau nodes */
    if (n_tau >= 4) {
        /* recipe 0: 1/4 uniform in ln a to z = 1300, 1/2 uniform in z over
           [1300, 900), the rest uniform in tau from z = 900 to today; recipe 1:
           1/5, 2/5 over [1300, 900), 1/5 uniform in z over [900, 300), the rest
           uniform in tau from z = 300 (resolves the visibility's tail) */
        int nA = node_recipe ? n_tau / 5 : n_tau / 4, nB = node_recipe ? 2 * n_tau / 5 : n_tau / 2;
        int nD = node_recipe ? n_tau / 5 : 0, nC = n_tau - nA - nB - nD;
        c->n_tau = n_tau;
        c->node_lna = (real_t *)malloc(sizeof(real_t) * n_tau);
        c->node_tau = (real_t *)malloc(sizeof(real_t) * n_tau);
        c->node_w = (real_t *)malloc(sizeof(real_t) * n_tau);
        real_t l1300 = -log(1301.0), l900 = -log(901.0);
        for (int j = 0; j < nA; j++)
            c->node_lna[j] = c->lna_tc + (l1300 - c->lna_tc) * j / nA;
        for (int j = 0; j < nB; j++)
            c->node_lna[nA + j] = -log(1.0 + 1300.0 - 400.0 * j / nB);
        for (int j = 0; j < nD; j++)
            c->node_lna[nA + nB + j] = -log(1.0 + 900.0 - 600.0 * j / nD);
        real_t lC = node_recipe ? -log(301.0) : l900;
        real_t tC = orc_tau_of_lna(c, lC);
        for (int j = 0; j < nC; j++) {
            real_t tt = tC + (c->tau0 - tC) * j / nC;
            c->node_lna[nA + nB + nD + j] = j == 0 ? lC : bisect(f_tau, c, tt, lC, 0.0);
        }
        for (int j = 0; j < n_tau; j++) c->node_tau[j] = orc_tau_of_lna(c, c->node_lna[j]);
        for (int j = 0; j < n_tau; j++) {
            real_t lo = j > 0 ? c->node_tau[j - 1] : c->node_tau[j];
            real_t hi = j < n_tau - 1 ? c->node_tau[j + 1] : c->node_tau[j];
            c->node_w[j] = 0.5 * (hi - lo);
        }
    }
    return 0;
}

void orc_cosmo_free(orc_cosmo *c)
{
    free(c->ct_tau); free(c->th_lna); free(c->th_xp); free(c->th_dxp);
    free(c->th_Tm); free(c->th_dTm); free(c->kp_kappa);
    free(c->node_lna); free(c->node_tau); free(c->node_w);
    memset(c, 0, sizeof(*c));
}

real_t orc_lna_start(const orc_cosmo *c, real_t k)
{
    real_t target = k / c->R_large;
    if (RE(orc_Hconf(c, c->lna_tc)) >= RE(target)) return c->lna_tc;
    return bisect(f_Hk, c, target, LNA_MIN, RE(c->lna_tc));
}

/* Massive-neutrino energy density and pressure at a, in units of today's
   critical density (for the oracle's pins). */
int orc_ncdm_density(const real_t *p, real_t m_ncdm, real_t a, real_t *out)
{
    orc_cosmo c;
    if (orc_cosmo_init(&c, p, 0, 0, m_ncdm, 0)) return -1;
    ncdm_rho_p(&c, a, &out[0], &out[1]);
    out[2] = c.Om_ncdm_rel;
    out[3] = c.ncdm_x1;
    out[4] = c.h;
    orc_cosmo_free(&c);
    return 0;
}
