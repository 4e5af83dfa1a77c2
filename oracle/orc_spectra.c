/*
 * ORACLE (test infrastructure only; see orc.h).
 *
 * Spherical Bessel functions, line-of-sight projection and C_ell, plus the
 * flat C entry points the Python test wrapper calls.
 *
 * j_l(x), exact to rounding (the paper's tabulated/Debye scheme of App. B.4 is
 * an approximation of this): for x > l_max, upward recurrence from
 * j_0 = sin x / x, j_1 = sin x / x^2 - cos x / x (stable while l < x); else
 * Miller's downward recurrence started where j_l is below 1e-40 of its peak
 * and normalised to j_0 (or j_1 near a zero of j_0), with series for j_1 at
 * small x.  Derivatives from the recurrence and the Bessel equation:
 *   j_l' = j_{l-1} - (l+1) j_l / x,
 *   j_l'' = -(2/x) j_l' - (1 - l(l+1)/x^2) j_l.
 *
 * Projection (App. B.4): Delta_T = sum_i w_i [S_T0 j + S_T1 j' +
 * scale_pol S_P (3 j'' + j)/2], Delta_E = sum_i w_i sqrt(6) S_P
 * sqrt(3 (l+2)! / (8 (l-2)!)) j / x^2, x = k (tau_0 - tau_i), w_i the
 * trapezoid weights in tau; sums compensated (Neumaier).
 *
 * C_ell (eq. c_ell_def, eq. PK_pivot): 4 pi sum_k w_k A_s (k/k_pivot)^(n_s-1)
 * Delta_X Delta_Y, w_k the trapezoid weights in ln k; C_ell, not D_ell.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "orc.h"

#define S_PI 3.14159265358979323846

static real_t j1_of(real_t x)
{
    if (RE(x) < 0.5) { /* Taylor series; term ratio -x^2 / ((2n+2)(2n+5)) */
        real_t x2 = x * x;
        return x / 3.0 * (1.0 - x2 / 10.0 * (1.0 - x2 / 28.0 * (1.0 - x2 / 54.0 * (1.0 - x2 / 88.0 * (1.0 - x2 / 130.0 * (1.0 - x2 / 180.0))))));
    }
    return sin(x) / (x * x) - cos(x) / x;
}

static real_t j0_of(real_t x)
{
    if (RE(x) < 1e-4) return 1.0 - x * x / 6.0;
    return sin(x) / x;
}

void orc_bessel_all(int lmax, real_t x, real_t *j)
{
    memset(j, 0, sizeof(real_t) * (lmax + 1));
    if (x == 0.0) { j[0] = 1.0; return; }
    real_t j0 = j0_of(x), j1 = j1_of(x);
    if (RE(x) > lmax) {
        j[0] = j0;
        if (lmax >= 1) j[1] = j1;
        for (int l = 1; l < lmax; l++) j[l + 1] = (2.0 * l + 1.0) / x * j[l] - j[l - 1];
        return;
    }
    int ls = (int)ceil(RE(x) + 20.0 + 15.0 * cbrt(RE(x)));
    int lcap = lmax + 30 + (int)sqrt(40.0 * lmax);
    if (ls > lcap) ls = lcap;
    real_t jp = 0.0, jc = 1e-250;
    for (int l = ls; l >= 1; l--) {
        /* jc = j_l (unnormalised), jp = j_{l+1} */
        if (l <= lmax) j[l] = jc;
        real_t jm = (2.0 * l + 1.0) / x * jc - jp;
        jp = jc;
        jc = jm;
        if (RE(ABS(jc)) > 1e200) {
            jc *= 1e-200; jp *= 1e-200;
            int top = ls < lmax ? ls : lmax;
            for (int m = l; m <= top; m++) j[m] *= 1e-200;
        }
    }
    j[0] = jc;
    real_t scale = (RE(ABS(j0)) >= RE(ABS(j1))) ? j0 / j[0] : j1 / j[1];
    for (int l = 0; l <= lmax; l++) j[l] *= scale;
}

/* ------------------------------------------------------------------ */
static void neumaier_add(real_t *sum, real_t *comp, real_t v)
{
    real_t t = *sum + v;
    if (RE(ABS(*sum)) >= RE(ABS(v))) *comp += (*sum - t) + v;
    else *comp += (v - t) + *sum;
    *sum = t;
}

/* Project one k mode: S [n_tau][3] -> Delta [lmax-1][2] (l = 2..lmax). */
static void project_mode(int n_tau, const real_t *tau, const real_t *w, real_t tau0,
                         real_t k, const real_t *S, int lmax, real_t scale_pol,
                         real_t *Delta, real_t *jbuf, real_t *acc)
{
    int nl = lmax - 1;
    memset(acc, 0, sizeof(real_t) * 4 * nl);
    for (int i = 0; i < n_tau; i++) {
        real_t x = k * (tau0 - tau[i]);
        orc_bessel_all(lmax, x, jbuf);
        real_t s0 = S[3 * i], s1 = S[3 * i + 1], sp = S[3 * i + 2];
        for (int l = 2; l <= lmax; l++) {
            real_t jl = jbuf[l];
            real_t jp = jbuf[l - 1] - (l + 1.0) * jl / x;
            real_t jpp = -2.0 / x * jp - (1.0 - l * (l + 1.0) / (x * x)) * jl;
            real_t dT = w[i] * (s0 * jl + s1 * jp + scale_pol * sp * 0.5 * (3.0 * jpp + jl));
            real_t cE = sqrt(3.0 * (l + 2.0) * (l + 1.0) * l * (l - 1.0) / 8.0);
            real_t dE = w[i] * sqrt(6.0) * sp * cE * jl / (x * x);
            int q = l - 2;
            neumaier_add(&acc[4 * q], &acc[4 * q + 1], dT);
            neumaier_add(&acc[4 * q + 2], &acc[4 * q + 3], dE);
        }
    }
    for (int q = 0; q < nl; q++) {
        Delta[2 * q] = acc[4 * q] + acc[4 * q + 1];
        Delta[2 * q + 1] = acc[4 * q + 2] + acc[4 * q + 3];
    }
}

static void opts_from(const double *oa, orc_opts *o)
{
    o->lmax_g = (int)oa[0]; o->lmax_pol = (int)oa[1]; o->lmax_nu = (int)oa[2];
    o->scale_sw = oa[3]; o->scale_isw = oa[4]; o->scale_dop = oa[5]; o->scale_pol = oa[6];
    o->step_c = oa[7]; o->step_cap = oa[8]; o->hooks = (int)oa[9]; o->max_steps = (long)oa[10];
    o->lmax_ncdm = (int)oa[11]; o->m_ncdm = oa[12]; o->node_recipe = (int)oa[13];
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ---------------- C entry points for the Python test wrapper ---------------- */

/* Scalars: [H0, Om_b, Om_c, Om_g, Om_nu, Om_L, R_nu, f_He, nH0, A_s, z_reion,
             lna_tc, lna_sw, tau0, lna_He3, n_s, Om_ncdm] */
int orc_scalars(const real_t *p, int hooks, double m_ncdm, real_t *out)
{
    orc_cosmo c;
    if (orc_cosmo_init(&c, p, 0, hooks, m_ncdm, 0)) return -1;
    real_t v[17] = {c.H0, c.Om_b, c.Om_c, c.Om_g, c.Om_nu, c.Om_L, c.R_nu, c.f_He,
                    c.nH0, c.A_s, c.z_reion, c.lna_tc, c.lna_sw, c.tau0, c.lna_He3, c.n_s, c.Om_ncdm};
    memcpy(out, v, sizeof(v));
    orc_cosmo_free(&c);
    return 0;
}

/* Background at points: out[n][18] = [a, Hc, dHc, fc, fb, fg, fnu, tau, xe,
   dxe, nuT, Rinv, cs2, kappa, g, dg, fncdm, wncdm] */
int orc_background(const real_t *p, int hooks, double m_ncdm, const real_t *lna, int n, real_t *out)
{
    orc_cosmo c;
    if (orc_cosmo_init(&c, p, 0, hooks, m_ncdm, 0)) return -1;
    for (int i = 0; i < n; i++) {
        orc_bg b;
        orc_bg_eval(&c, lna[i], &b, 2);
        real_t v[18] = {b.a, b.Hc, b.dHc, b.fc, b.fb, b.fg, b.fnu, b.tau, b.xe, b.dxe,
                        b.nuT, b.Rinv, b.cs2, b.kappa, b.g, b.dg, b.fncdm, b.wncdm};
        memcpy(out + 18 * i, v, sizeof(v));
    }
    orc_cosmo_free(&c);
    return 0;
}

/* tau nodes: out[3][n_tau] = lna, tau, w */
/* Thermal history at ln a[n]: out[n][4] = matter temperature T_m [eV],
   d ln T_m / d ln a, x_e, baryon sound speed c_s^2 (App. B.1.2, App. C.3). */
int orc_thermo(const real_t *p, const real_t *lna, int n, real_t *out)
{
    orc_cosmo c;
    if (orc_cosmo_init(&c, p, 0, 0, 0.0, 0)) return -1;
    for (int i = 0; i < n; i++) {
        orc_bg b;
        orc_bg_eval(&c, lna[i], &b, 1);
        real_t dlnTm;
        out[4 * i] = orc_Tm_of_lna(&c, lna[i], &dlnTm);
        out[4 * i + 1] = dlnTm;
        out[4 * i + 2] = b.xe;
        out[4 * i + 3] = b.cs2;
    }
    orc_cosmo_free(&c);
    return 0;
}

int orc_nodes(const real_t *p, int n_tau, double m_ncdm, int node_recipe, real_t *out)
{
    orc_cosmo c;
    if (orc_cosmo_init(&c, p, n_tau, 0, m_ncdm, node_recipe)) return -1;
    memcpy(out, c.node_lna, sizeof(real_t) * n_tau);
    memcpy(out + n_tau, c.node_tau, sizeof(real_t) * n_tau);
    memcpy(out + 2 * n_tau, c.node_w, sizeof(real_t) * n_tau);
    orc_cosmo_free(&c);
    return 0;
}

int orc_nstate_of(const double *oa)
{
    orc_opts o;
    opts_from(oa, &o);
    return orc_nstate(&o);
}

real_t orc_lna_start_of(const real_t *p, real_t k, double m_ncdm)
{
    orc_cosmo c;
    if (orc_cosmo_init(&c, p, 0, 0, m_ncdm, 0)) return NAN;
    real_t v = orc_lna_start(&c, k);
    orc_cosmo_free(&c);
    return v;
}

/* Trajectory of one mode at ascending ln a points (y_init may be NULL). */
int orc_trajectory(const real_t *p, const double *oa, real_t k, const real_t *lna_out,
                   int n, real_t *y_out, const real_t *y_init, real_t lna_init, long *steps)
{
    orc_cosmo c;
    orc_opts o;
    opts_from(oa, &o);
    if (orc_cosmo_init(&c, p, 0, o.hooks & ORC_HOOK_EDS_CDM, o.m_ncdm, 0)) return -1;
    int rc = orc_solve_mode(&c, &o, k, lna_out, n, y_out, y_init, lna_init, steps);
    orc_cosmo_free(&c);
    return rc;
}

/* Right-hand side at one point (for consistency pins). */
int orc_rhs_at(const real_t *p, const double *oa, real_t k, real_t lna, const real_t *y, real_t *dy)
{
    orc_cosmo c;
    orc_opts o;
    opts_from(oa, &o);
    if (orc_cosmo_init(&c, p, 0, o.hooks & ORC_HOOK_EDS_CDM, o.m_ncdm, 0)) return -1;
    orc_rhs(&c, &o, k, lna, y, dy);
    orc_cosmo_free(&c);
    return 0;
}

void orc_bessel(int lmax, real_t x, real_t *out) { orc_bessel_all(lmax, x, out); }

/* Project given sources (synthetic ones in the pins) on given nodes. */
int orc_project(int n_tau, const real_t *tau, const real_t *w, real_t tau0,
                const real_t *k, int nk, const real_t *S, int lmax, real_t scale_pol,
                real_t *Delta, int nthreads)
{
    set_threads(nthreads);
    int nl = lmax - 1;
#pragma omp parallel
    {
        real_t *jbuf = (real_t *)malloc(sizeof(real_t) * (lmax + 1));
        real_t *acc = (real_t *)malloc(sizeof(real_t) * 4 * nl);
#pragma omp for schedule(dynamic, 1)
        for (int ik = 0; ik < nk; ik++)
            project_mode(n_tau, tau, w, tau0, k[ik], S + (size_t)ik * n_tau * 3, lmax,
                         scale_pol, Delta + (size_t)ik * nl * 2, jbuf, acc);
        free(jbuf);
        free(acc);
    }
    return 0;
}

/* C_ell from Delta[nk][lmax-1][2]: Cl[3][lmax-1] = TT, TE, EE */
int orc_cl(const real_t *k, int nk, const real_t *Delta, int lmax, real_t A_s, real_t n_s,
           real_t k_pivot, real_t *Cl)
{
    int nl = lmax - 1;
    real_t *wk = (real_t *)malloc(sizeof(real_t) * nk);
    for (int i = 0; i < nk; i++) {
        real_t lo = i > 0 ? log(k[i - 1]) : log(k[i]);
        real_t hi = i < nk - 1 ? log(k[i + 1]) : log(k[i]);
        wk[i] = 0.5 * (hi - lo);
    }
    for (int q = 0; q < nl; q++) {
        real_t s[3] = {0, 0, 0}, cmp[3] = {0, 0, 0};
        for (int i = 0; i < nk; i++) {
            real_t P = A_s * pow(k[i] / k_pivot, n_s - 1.0);
            real_t dT = Delta[((size_t)i * nl + q) * 2], dE = Delta[((size_t)i * nl + q) * 2 + 1];
            real_t f = 4.0 * S_PI * wk[i] * P;
            neumaier_add(&s[0], &cmp[0], f * dT * dT);
            neumaier_add(&s[1], &cmp[1], f * dT * dE);
            neumaier_add(&s[2], &cmp[2], f * dE * dE);
        }
        for (int t = 0; t < 3; t++) Cl[t * nl + q] = s[t] + cmp[t];
    }
    free(wk);
    return 0;
}

/* Whole path for one cosmology. Any output pointer may be NULL.
   S_out [nk][n_tau][3], Delta_out [nk][lmax-1][2], Cl_out [3][lmax-1],
   steps_out [nk]. */
int orc_run(const real_t *p, int n_tau, const double *oa, const real_t *k, int nk,
            int lmax_cl, real_t *S_out, real_t *Delta_out, real_t *Cl_out,
            long *steps_out, int nthreads)
{
    orc_cosmo c;
    orc_opts o;
    opts_from(oa, &o);
    if (orc_cosmo_init(&c, p, n_tau, o.hooks & ORC_HOOK_EDS_CDM, o.m_ncdm, o.node_recipe)) return -1;
    set_threads(nthreads);
    real_t *S = S_out ? S_out : (real_t *)malloc(sizeof(real_t) * (size_t)nk * n_tau * 3);
    int rc = 0;
    /* highest k first: the most expensive modes start earliest */
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
    for (int t = 0; t < nk; t++) {
        int ik = nk - 1 - t;
        long st = 0;
        rc |= orc_sources_mode(&c, &o, k[ik], S + (size_t)ik * n_tau * 3, &st);
        if (steps_out) steps_out[ik] = st;
    }
    if (rc == 0 && (Delta_out || Cl_out)) {
        int nl = lmax_cl - 1;
        real_t *D = Delta_out ? Delta_out : (real_t *)malloc(sizeof(real_t) * (size_t)nk * nl * 2);
        orc_project(n_tau, c.node_tau, c.node_w, c.tau0, k, nk, S, lmax_cl, o.scale_pol, D, nthreads);
        if (Cl_out) orc_cl(k, nk, D, lmax_cl, c.A_s, c.n_s, c.k_pivot, Cl_out);
        if (!Delta_out) free(D);
    }
    if (!S_out) free(S);
    orc_cosmo_free(&c);
    return rc;
}

/* Handle-based access for tests that call the right-hand side many times. */
void *orc_create(const real_t *p, int n_tau, int hooks, double m_ncdm)
{
    orc_cosmo *c = (orc_cosmo *)malloc(sizeof(orc_cosmo));
    if (orc_cosmo_init(c, p, n_tau, hooks, m_ncdm, 0)) { orc_cosmo_free(c); free(c); return NULL; }
    return c;
}

void orc_destroy(void *h)
{
    if (h) { orc_cosmo_free((orc_cosmo *)h); free(h); }
}

int orc_h_rhs(void *h, const double *oa, real_t k, real_t lna, const real_t *y, real_t *dy)
{
    orc_opts o;
    opts_from(oa, &o);
    orc_rhs((orc_cosmo *)h, &o, k, lna, y, dy);
    return 0;
}

/* dense A(ln a) [N][N] */
int orc_h_matrix(void *h, const double *oa, real_t k, real_t lna, real_t *A)
{
    orc_opts o;
    opts_from(oa, &o);
    int N = orc_nstate(&o);
    orc_bg b;
    orc_bg_eval((orc_cosmo *)h, lna, &b, 1);
    real_t *e = (real_t *)calloc(N, sizeof(real_t)), *col = (real_t *)malloc(sizeof(real_t) * N);
    for (int j = 0; j < N; j++) {
        e[j] = 1.0;
        orc_rhs_bg(&o, &b, k, e, col);
        for (int i = 0; i < N; i++) A[i * N + j] = col[i];
        e[j] = 0.0;
    }
    free(e);
    free(col);
    return 0;
}

/* LU solve of a dense system (pins the factorisation against a library solve) */
int orc_dense_solve(real_t *A, int n, real_t *b)
{
    int *piv = (int *)malloc(sizeof(int) * n), *ext = (int *)malloc(sizeof(int) * 2 * n);
    int rc = orc_lu_factor(A, n, piv, ext);
    if (!rc) orc_lu_solve(A, n, piv, ext, b);
    free(piv);
    free(ext);
    return rc;
}

/* Adiabatic initial state of the oracle at a given ln a. */
int orc_initial_at(const real_t *p, const double *oa, real_t k, real_t lna, real_t *y)
{
    orc_cosmo c;
    orc_opts o;
    opts_from(oa, &o);
    if (orc_cosmo_init(&c, p, 0, 0, o.m_ncdm, 0)) return -1;
    orc_initial(&c, &o, k, lna, y);
    orc_cosmo_free(&c);
    return 0;
}

/* Steps the oracle's schedule takes for each k mode over the tau nodes. */
int orc_count_steps(const real_t *p, int n_tau, const double *oa, const real_t *k, int nk, long *out)
{
    orc_cosmo c;
    orc_opts o;
    opts_from(oa, &o);
    if (orc_cosmo_init(&c, p, n_tau, 0, o.m_ncdm, o.node_recipe)) return -1;
    for (int i = 0; i < nk; i++) {
        real_t x = orc_lna_start(&c, k[i]);
        long n = 0;
        for (int j = 0; j < n_tau; j++) {
            if (RE(c.node_lna[j]) > RE(x)) { n += orc_schedule_count(&c, &o, k[i], x, c.node_lna[j]); x = c.node_lna[j]; }
        }
        out[i] = n;
    }
    orc_cosmo_free(&c);
    return 0;
}

/* Matter power spectrum at redshift z (App. B.4, eq. PK):
     P(k, z) = (2 pi^2 / k^3) A_s (k / k_pivot)^(n_s - 1) delta_m^2,
     delta_m = (rho_c delta_c + rho_b delta_b) / (rho_c + rho_b),
   the density-weighted contrast of the non-relativistic species (CDM and
   baryons here; photons and massless neutrinos are relativistic), with
   delta_c, delta_b (state entries 1 and 2) from the mode integrated from its
   adiabatic start to ln a = -ln(1 + z) on the oracle's step schedule. */
int orc_pk(const real_t *p, const double *oa, const real_t *k, int nk, double z, real_t *Pk, int nthreads)
{
    orc_cosmo c;
    orc_opts o;
    opts_from(oa, &o);
    if (orc_cosmo_init(&c, p, 0, o.hooks & ORC_HOOK_EDS_CDM, o.m_ncdm, 0)) return -1;
    set_threads(nthreads);
    const real_t lna = -log1p(z);
    orc_bg b;
    orc_bg_eval(&c, lna, &b, 0);
    const int N = orc_nstate(&o);
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
    for (int t = 0; t < nk; t++) {
        int ik = nk - 1 - t;
        real_t *y = (real_t *)malloc(sizeof(real_t) * N);
        long st = 0;
        if (RE(orc_lna_start(&c, k[ik])) >= RE(lna)) {
            rc |= 2; /* the mode starts after the requested time */
            Pk[ik] = NAN;
        } else {
            rc |= orc_solve_mode(&c, &o, k[ik], &lna, 1, y, NULL, 0.0, &st);
            const real_t dm = (b.fc * y[1] + b.fb * y[2]) / (b.fc + b.fb);
            const real_t kk = k[ik];
            Pk[ik] = 2.0 * S_PI * S_PI / (kk * kk * kk) * c.A_s * pow(kk / c.k_pivot, c.n_s - 1.0) * dm * dm;
        }
        free(y);
    }
    orc_cosmo_free(&c);
    return rc;
}

/* Density-weighted matter contrast delta_m = sum_i rho_i delta_i / sum_i rho_i
   over CDM, baryons and (when present) the massive neutrino, at every tau
   node, for each k: out[nk][n_tau] (App. B.4 eq. PK's bracket; inputs of the
   lensing potential, App. B.5). */
int orc_delta_m_nodes(const real_t *p, int n_tau, const double *oa, const real_t *k, int nk, real_t *out,
                      int nthreads)
{
    orc_cosmo c;
    orc_opts o;
    opts_from(oa, &o);
    if (orc_cosmo_init(&c, p, n_tau, o.hooks & ORC_HOOK_EDS_CDM, o.m_ncdm, o.node_recipe)) return -1;
    set_threads(nthreads);
    const int N = orc_nstate(&o);
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
    for (int t = 0; t < nk; t++) {
        int ik = nk - 1 - t;
        real_t *Y = (real_t *)malloc(sizeof(real_t) * (size_t)n_tau * N);
        long st = 0;
        rc |= orc_solve_mode(&c, &o, k[ik], c.node_lna, n_tau, Y, NULL, 0.0, &st);
        for (int i = 0; i < n_tau; i++) {
            orc_bg b;
            orc_bg_eval(&c, c.node_lna[i], &b, 0);
            const real_t *y = Y + (size_t)i * N;
            real_t num = b.fc * y[1] + b.fb * y[2], den = b.fc + b.fb;
            if (o.lmax_ncdm > 0) {
                /* the massive neutrino's delta rho / rho_tot from its momentum bins */
                const real_t q[3] = {0.913201, 3.37517, 7.79184}, K[3] = {0.0687359, 3.31435, 2.29911};
                const int i0 = orc_nstate(&o) - 3 * (o.lmax_ncdm + 1);
                real_t drho = 0.0;
                for (int j = 0; j < 3; j++) {
                    const real_t eps = sqrt(q[j] * q[j] + b.ncdm_x * b.ncdm_x);
                    drho += K[j] * (1.0 + exp(-q[j])) * eps / (q[j] * q[j]) * y[i0 + j * (o.lmax_ncdm + 1)];
                }
                num += b.ncdm_n * drho;
                den += b.fncdm;
            }
            out[(size_t)ik * n_tau + i] = num / den;
        }
        free(Y);
    }
    orc_cosmo_free(&c);
    return rc;
}
