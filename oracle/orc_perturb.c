/*
 * ORACLE (test infrastructure only; see orc.h).
 *
 * Synchronous-gauge linear perturbations of one k mode in x = ln a, and the
 * CMB sources at the tau nodes.
 *
 * State vector (fixed order):
 *   [eta, delta_c, delta_b, theta_b,
 *    delta_g, theta_g, sigma_g, F_g3 .. F_gL,     (photon temperature, L = lmax_g)
 *    G_0 .. G_Lp,                                  (photon polarization)
 *    delta_nu, theta_nu, sigma_nu, F_nu3 .. F_nuLn] (massless neutrinos)
 * with F_1 = 4 theta / (3k) and F_2 = 2 sigma (App. C.4).
 *
 * Equations (derivatives in ln a):
 *   metric       h' = 2 k^2 eta / H^2 + 3 sum_i f_i delta_i          (eq. hprime)
 *                eta' = 3 H / (2 k^2) sum_i f_i (1 + w_i) theta_i   (eq. etaprime)
 *                with 8 pi G a^2 rho_i = 3 H^2 f_i, f_i = rho_i / rho_tot;
 *   CDM          App. C.2;  baryons App. C.3;
 *   photons      App. C.4, with two readings: the -(9/10) term of sigma_g'
 *                multiplies sigma_g, and the polarization source is
 *                (1/2)(1/(H tau_c)) Pi (delta_l0 + delta_l2 / 5), Pi = 2 sigma_g
 *                + G_0 + G_2 (both follow from the Thomson collision term of
 *                the cited Ma & Bertschinger hierarchy, which also gives the
 *                (1/20)(G_0+G_2) of sigma_g');
 *                truncation (l_max+1)/(H tau) uses conformal time tau;
 *   neutrinos    App. C.5.
 * No tight-coupling, ultra-relativistic-fluid or radiation-streaming switch
 * (App. B.6).
 *
 * Initial conditions (not printed in the paper; the cited Ma & Bertschinger
 * 1995 adiabatic growing mode at leading order in k tau, normalised to
 * curvature R = 1, i.e. C = 1/2):
 *   delta_g = delta_nu = -(2/3) C (k tau)^2,  delta_b = delta_c = 3/4 delta_g,
 *   theta_g = theta_b = -C k^4 tau^3 / 18,
 *   theta_nu = theta_g (23 + 4 R_nu) / (15 + 4 R_nu),
 *   sigma_nu = 4 C (k tau)^2 / (3 (15 + 4 R_nu)),
 *   eta = 2C - C (k tau)^2 (5 + 4 R_nu) / (6 (15 + 4 R_nu)), all others 0.
 *
 * Integrator: 3-stage Radau IIA collocation (order 5, L-stable).  The system
 * is linear, dy/dx = A(x) y, so each step solves the 3N x 3N collocation
 * system (I - h a_ij A(x_n + c_j h)) Y = (y_n, y_n, y_n) by LU with partial
 * pivoting (unknowns ordered by multipole, exact zeros skipped: see
 * orc_linalg.c); A(x) is built column by column from the right-hand side.  Steps follow a fixed
 * schedule h <= step_c / (1 + k/H) (the fastest oscillation of the hierarchy
 * has phase rate k/H per unit ln a) and land on every tau node; convergence
 * of this schedule is pinned by a step-halving test.
 *
 * Sources (App. B.4, eq. source_functions) with
 *   alpha = H (h' + 6 eta') / (2 k^2),
 *   H alpha' = -2 H alpha + eta - (9/2) (H/k)^2 sum_i f_i (1 + w_i) sigma_i
 * (the traceless Einstein equation of the cited formalism, not printed in
 * the paper).  The switches group as: SW = g (delta_g/4 + H alpha');
 * ISW = g (eta - H alpha' - 2 H alpha) + 2 H e^-kappa (eta' - H' alpha - H alpha')
 * and all of S_T1; Doppler = the H [ ... ] bracket.  Stored per node:
 * (S_T0, S_T1, S_P) with S_P = g Pi / 8 unscaled; scale_pol is applied to
 * the temperature use of S_P in the projection and S_E = sqrt(6) S_P.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "orc.h"

#define I_ETA 0
#define I_DC 1
#define I_DB 2
#define I_TB 3
#define I_G0 4

static int i_pol(const orc_opts *o) { return I_G0 + o->lmax_g + 1; }
static int i_nu(const orc_opts *o) { return i_pol(o) + o->lmax_pol + 1; }
/* massive neutrinos: bins b = 0..2, Psi_0..Psi_L of bin b at i_ncdm + b (L + 1) */
static int i_ncdm(const orc_opts *o) { return i_nu(o) + o->lmax_nu + 1; }
static int n_ncdm(const orc_opts *o) { return o->lmax_ncdm > 0 ? 3 * (o->lmax_ncdm + 1) : 0; }
int orc_nstate(const orc_opts *o) { return i_ncdm(o) + n_ncdm(o); }

/* Momentum bins of the perturbed massive-neutrino integrals (App. B.3,
   3-point rule of the paper: int dq q^4 e^q/(1+e^q)^2 (q/eps)^w Psi ~
   4 sum K_i (q_i/eps_i)^w Psi(q_i)), and d ln f_0 / d ln q = -q / (1 + e^-q). */
static const real_t NCDM_Q3[3] = {0.913201, 3.37517, 7.79184};
static const real_t NCDM_K3[3] = {0.0687359, 3.31435, 2.29911};

/* delta rho, (rho + p) theta and (rho + p) sigma of the massive neutrinos as
   fractions of rho_tot (eq. mnu_sum) */
static void ncdm_sums(const orc_opts *o, const orc_bg *b, real_t k, const real_t *y,
                      real_t *drho, real_t *rpth, real_t *rpsig)
{
    *drho = *rpth = *rpsig = 0.0;
    if (o->lmax_ncdm <= 0) return;
    const int L = o->lmax_ncdm, i0 = i_ncdm(o);
    for (int j = 0; j < 3; j++) {
        const real_t q = NCDM_Q3[j], eps = sqrt(q * q + b->ncdm_x * b->ncdm_x);
        const real_t w = NCDM_K3[j] * (1.0 + exp(-q));
        const real_t *Ps = y + i0 + j * (L + 1);
        *drho += w * eps / (q * q) * Ps[0];
        *rpth += w / q * k * Ps[1];
        *rpsig += (2.0 / 3.0) * w / eps * Ps[2];
    }
    *drho *= b->ncdm_n;
    *rpth *= b->ncdm_n;
    *rpsig *= b->ncdm_n;
}

static void metric(const orc_opts *o, const orc_bg *b, real_t k, const real_t *y,
                   real_t *hp, real_t *etap)
{
    const int P = i_pol(o), Nn = i_nu(o);
    (void)P;
    real_t kH = k / b->Hc;
    *hp = 2.0 * kH * kH * y[I_ETA]
        + 3.0 * (b->fc * y[I_DC] + b->fb * y[I_DB] + b->fg * y[I_G0] + b->fnu * y[Nn]);
    *etap = 1.5 * b->Hc / (k * k)
        * (b->fb * y[I_TB] + (4.0 / 3.0) * b->fg * y[I_G0 + 1] + (4.0 / 3.0) * b->fnu * y[Nn + 1]);
    real_t drho, rpth, rpsig;
    ncdm_sums(o, b, k, y, &drho, &rpth, &rpsig);
    *hp += 3.0 * drho;
    *etap += 1.5 * b->Hc / (k * k) * rpth;
    if (o->hooks & ORC_HOOK_FREEZE_METRIC) { *hp = 0.0; *etap = 0.0; }
}

/* free-streaming hierarchy part of one chain starting at y[s] (l = 0..L),
   with first three entries (delta, theta, sigma); adds scattering -nu F_l
   for l >= 3 (nu = 0 for neutrinos) */
static void chain_tail(real_t kH, real_t Hc, real_t tau, real_t nu, int L,
                       const real_t *yc, real_t *dyc)
{
    for (int l = 3; l <= L; l++) {
        real_t Flm1 = (l == 3) ? 2.0 * yc[2] : yc[l - 1];
        if (l < L)
            dyc[l] = kH / (2.0 * l + 1.0) * (l * Flm1 - (l + 1.0) * yc[l + 1]) - nu * yc[l];
        else
            dyc[l] = kH * Flm1 - (L + 1.0) / (Hc * tau) * yc[l] - nu * yc[l];
    }
}

void orc_rhs_bg(const orc_opts *o, const orc_bg *b, real_t k, const real_t *y, real_t *dy)
{
    const int P = i_pol(o), Nn = i_nu(o);
    const int Lg = o->lmax_g, Lp = o->lmax_pol, Ln = o->lmax_nu;
    real_t hp, etap;
    metric(o, b, k, y, &hp, &etap);
    real_t Hc = b->Hc, kH = k / Hc;
    real_t nu = (o->hooks & ORC_HOOK_NO_THOMSON) ? 0.0 : b->nuT;

    dy[I_ETA] = etap;
    dy[I_DC] = -0.5 * hp;
    dy[I_DB] = -y[I_TB] / Hc - 0.5 * hp;
    dy[I_TB] = -y[I_TB] + b->cs2 * k * k * y[I_DB] / Hc + b->Rinv * nu * (y[I_G0 + 1] - y[I_TB]);

    /* photon temperature */
    const real_t *F = y + I_G0;
    real_t *dF = dy + I_G0;
    const real_t *G = y + P;
    real_t *dG = dy + P;
    dF[0] = -(4.0 / 3.0) * F[1] / Hc - (2.0 / 3.0) * hp;
    dF[1] = k * k / Hc * (0.25 * F[0] - F[2]) + nu * (y[I_TB] - F[1]);
    dF[2] = (4.0 / 15.0) * F[1] / Hc - 0.3 * kH * F[3] + (2.0 / 15.0) * hp + 0.8 * etap
          - 0.9 * nu * F[2] + 0.05 * nu * (G[0] + G[2]);
    chain_tail(kH, Hc, b->tau, nu, Lg, F, dF);

    /* photon polarization */
    real_t Pi = 2.0 * F[2] + G[0] + G[2];
    for (int l = 0; l <= Lp; l++) {
        real_t Glm1 = l > 0 ? G[l - 1] : 0.0;
        if (l < Lp)
            dG[l] = kH / (2.0 * l + 1.0) * (l * Glm1 - (l + 1.0) * G[l + 1]) - nu * G[l];
        else
            dG[l] = kH * Glm1 - (Lp + 1.0) / (Hc * b->tau) * G[l] - nu * G[l];
        if (l == 0) dG[l] += 0.5 * nu * Pi;
        if (l == 2) dG[l] += 0.1 * nu * Pi;
    }

    /* massless neutrinos */
    const real_t *Fn = y + Nn;
    real_t *dFn = dy + Nn;
    dFn[0] = -(4.0 / 3.0) * Fn[1] / Hc - (2.0 / 3.0) * hp;
    dFn[1] = k * k / Hc * (0.25 * Fn[0] - Fn[2]);
    dFn[2] = (4.0 / 15.0) * Fn[1] / Hc - 0.3 * kH * Fn[3] + (2.0 / 15.0) * hp + 0.8 * etap;
    chain_tail(kH, Hc, b->tau, 0.0, Ln, Fn, dFn);

    /* massive neutrinos (App. C.6), one hierarchy per momentum bin */
    if (o->lmax_ncdm > 0) {
        const int L = o->lmax_ncdm, i0 = i_ncdm(o);
        for (int j = 0; j < 3; j++) {
            const real_t q = NCDM_Q3[j], eps = sqrt(q * q + b->ncdm_x * b->ncdm_x);
            const real_t v = q * k / (eps * Hc), dlnf = -q / (1.0 + exp(-q));
            const real_t *Ps = y + i0 + j * (L + 1);
            real_t *dPs = dy + i0 + j * (L + 1);
            dPs[0] = -v * Ps[1] + hp / 6.0 * dlnf;
            dPs[1] = v / 3.0 * (Ps[0] - 2.0 * Ps[2]);
            dPs[2] = v / 5.0 * (2.0 * Ps[1] - 3.0 * Ps[3]) - (hp / 15.0 + 0.4 * etap) * dlnf;
            for (int l = 3; l < L; l++) dPs[l] = v / (2.0 * l + 1.0) * (l * Ps[l - 1] - (l + 1.0) * Ps[l + 1]);
            dPs[L] = v * Ps[L - 1] - (L + 1.0) / (Hc * b->tau) * Ps[L];
        }
    }
}

void orc_rhs(const orc_cosmo *c, const orc_opts *o, real_t k, real_t lna,
             const real_t *y, real_t *dy)
{
    orc_bg b;
    orc_bg_eval(c, lna, &b, 1);
    orc_rhs_bg(o, &b, k, y, dy);
}

void orc_initial(const orc_cosmo *c, const orc_opts *o, real_t k, real_t lna_i, real_t *y)
{
    int N = orc_nstate(o), Nn = i_nu(o);
    memset(y, 0, sizeof(real_t) * N);
    real_t tau = orc_tau_of_lna(c, lna_i), C = 0.5, Rn = c->R_nu;
    real_t kt = k * tau;
    real_t dg = -(2.0 / 3.0) * C * kt * kt;
    real_t tg = -C * k * kt * kt * kt / 18.0;
    y[I_ETA] = 2.0 * C - C * kt * kt * (5.0 + 4.0 * Rn) / (6.0 * (15.0 + 4.0 * Rn));
    y[I_DC] = 0.75 * dg;
    y[I_DB] = 0.75 * dg;
    y[I_TB] = tg;
    y[I_G0] = dg;
    y[I_G0 + 1] = tg;
    y[Nn] = dg;
    y[Nn + 1] = tg * (23.0 + 4.0 * Rn) / (15.0 + 4.0 * Rn);
    y[Nn + 2] = 4.0 * C * kt * kt / (3.0 * (15.0 + 4.0 * Rn));
    /* massive neutrinos, relativistic at the start: the massless neutrinos'
       delta, theta, sigma carried by each momentum bin (the cited Ma &
       Bertschinger adiabatic mode) */
    if (o->lmax_ncdm > 0) {
        const int L = o->lmax_ncdm, i0 = i_ncdm(o);
        const real_t x = exp(lna_i) * c->ncdm_x1;
        for (int j = 0; j < 3; j++) {
            const real_t q = NCDM_Q3[j], eps = sqrt(q * q + x * x), dlnf = -q / (1.0 + exp(-q));
            real_t *Ps = y + i0 + j * (L + 1);
            Ps[0] = -0.25 * y[Nn] * dlnf;
            Ps[1] = -eps / (3.0 * q * k) * y[Nn + 1] * dlnf;
            Ps[2] = -0.5 * y[Nn + 2] * dlnf;
        }
    }
}

/* dense A(x): column j = rhs(e_j) */
static void build_A(const orc_opts *o, const orc_bg *b, real_t k, int N, real_t *A, real_t *e, real_t *col)
{
    memset(e, 0, sizeof(real_t) * N);
    for (int j = 0; j < N; j++) {
        e[j] = 1.0;
        orc_rhs_bg(o, b, k, e, col);
        for (int i = 0; i < N; i++) A[i * N + j] = col[i];
        e[j] = 0.0;
    }
}

typedef struct {
    int N;
    real_t *M, *Mc, *A, *rhs, *rhs0, *res, *e, *col;
    int *piv, *ext, *pos, *mlo, *mhi;
} radau_ws;

/* Multipole index of state element i (the four scalars count as l = 0). */
static int multipole_of(const orc_opts *o, int i)
{
    if (i < I_G0) return 0;
    const int P = i_pol(o), Nn = i_nu(o), Nc = i_ncdm(o);
    if (i < P) return i - I_G0;
    if (i < Nn) return i - P;
    if (i < Nc) return i - Nn;
    return (i - Nc) % (o->lmax_ncdm + 1);
}

static void ws_alloc(radau_ws *w, const orc_opts *o, int N)
{
    w->N = N;
    w->M = (real_t *)malloc(sizeof(real_t) * 9 * N * N);
    w->Mc = (real_t *)malloc(sizeof(real_t) * 9 * N * N);
    w->res = (real_t *)malloc(sizeof(real_t) * 3 * N);
    w->A = (real_t *)malloc(sizeof(real_t) * 3 * N * N);
    w->rhs = (real_t *)malloc(sizeof(real_t) * 3 * N);
    w->rhs0 = (real_t *)malloc(sizeof(real_t) * 3 * N);
    w->e = (real_t *)malloc(sizeof(real_t) * N);
    w->col = (real_t *)malloc(sizeof(real_t) * N);
    w->piv = (int *)malloc(sizeof(int) * 3 * N);
    w->ext = (int *)malloc(sizeof(int) * 6 * N);
    w->pos = (int *)malloc(sizeof(int) * N);
    w->mlo = (int *)malloc(sizeof(int) * 3 * N);
    w->mhi = (int *)malloc(sizeof(int) * 3 * N);
    /* unknown ordering of the collocation system: by multipole, then element,
       then stage; the couplings of the hierarchies (l to l +- 1, the scalars
       to l <= 2) then stay near the diagonal */
    int p = 0, lmax = 0;
    for (int i = 0; i < N; i++) lmax = multipole_of(o, i) > lmax ? multipole_of(o, i) : lmax;
    for (int l = 0; l <= lmax; l++)
        for (int i = 0; i < N; i++)
            if (multipole_of(o, i) == l) w->pos[i] = p++;
}
static void ws_free(radau_ws *w)
{
    free(w->M); free(w->Mc); free(w->res); free(w->A); free(w->rhs); free(w->rhs0); free(w->e); free(w->col);
    free(w->piv); free(w->ext); free(w->pos); free(w->mlo); free(w->mhi);
}

void orc_radau_tableau(real_t *out12);

/* One step of the 3-stage Radau IIA collocation method for dy/dx = A(x) y:
   the stage values Y_s = y + h sum_t a_st A(x + c_t h) Y_t solve one linear
   system of 3N unknowns (stage s of element i is unknown 3 pos[i] + s); the
   step's result is the last stage (c_3 = 1). */
static int radau_linear_step(const orc_cosmo *c, const orc_opts *o, real_t k,
                             real_t x, real_t h, real_t *y, radau_ws *w)
{
    int N = w->N, M3 = 3 * N;
    const int *pos = w->pos;
    real_t t[12];
    orc_radau_tableau(t);
    for (int s = 0; s < 3; s++) {
        orc_bg b;
        orc_bg_eval(c, x + t[9 + s] * h, &b, 1);
        build_A(o, &b, k, N, w->A + (size_t)s * N * N, w->e, w->col);
    }
    for (int si = 0; si < 3; si++)
        for (int i = 0; i < N; i++) {
            const int r = 3 * pos[i] + si;
            real_t *row = w->M + (size_t)r * M3;
            int lo = M3, hi = -1;
            memset(row, 0, sizeof(real_t) * M3);
            for (int sj = 0; sj < 3; sj++) {
                real_t coef = h * t[3 * si + sj];
                const real_t *Aj = w->A + (size_t)sj * N * N + (size_t)i * N;
                for (int j = 0; j < N; j++) {
                    if (Aj[j] == 0.0) continue;
                    const int cidx = 3 * pos[j] + sj;
                    row[cidx] = -coef * Aj[j];
                    if (cidx < lo) lo = cidx;
                    if (cidx > hi) hi = cidx;
                }
            }
            row[r] += 1.0;
            w->mlo[r] = lo < r ? lo : r;
            w->mhi[r] = hi > r ? hi : r;
            w->rhs0[r] = y[i];
        }
    memcpy(w->Mc, w->M, sizeof(real_t) * (size_t)M3 * M3);
    if (orc_lu_factor(w->M, M3, w->piv, w->ext)) return -1;
    memcpy(w->rhs, w->rhs0, sizeof(real_t) * M3);
    orc_lu_solve(w->M, M3, w->piv, w->ext, w->rhs);
    /* iterative refinement: the state mixes O(1) and ~1e-15 components, and
       a single partial-pivoting solve is accurate only normwise */
    for (int it = 0; it < 3; it++) {
        for (int i = 0; i < M3; i++) {
            real_t r = w->rhs0[i];
            const real_t *row = w->Mc + (size_t)i * M3;
            for (int j = w->mlo[i]; j <= w->mhi[i]; j++) r -= row[j] * w->rhs[j];
            w->res[i] = r;
        }
        orc_lu_solve(w->M, M3, w->piv, w->ext, w->res);
        for (int i = 0; i < M3; i++) w->rhs[i] += w->res[i];
    }
    for (int i = 0; i < N; i++) y[i] = w->rhs[3 * pos[i] + 2];
    return 0;
}

static double hmax_at(const orc_cosmo *c, const orc_opts *o, real_t k, real_t lna)
{
    double h = o->step_c / (1.0 + RE(k) / RE(orc_Hconf(c, lna)));
    return h < o->step_cap ? h : o->step_cap;
}

/* number of equal steps the schedule takes between x0 and x1 */
int orc_schedule_count(const orc_cosmo *c, const orc_opts *o, real_t k, real_t x0, real_t x1)
{
    double h0 = hmax_at(c, o, k, x0), h1 = hmax_at(c, o, k, x1);
    double hm = h0 < h1 ? h0 : h1;
    int m = (int)ceil(RE(x1 - x0) / hm);
    return m < 1 ? 1 : m;
}

/* Integrate from (lna_init, y_init) -- or from the adiabatic initial
   condition at a_i(k) when y_init is NULL -- through the ascending output
   points, writing y at each into y_out[n_out][N]. */
int orc_solve_mode(const orc_cosmo *c, const orc_opts *o, real_t k,
                   const real_t *lna_out, int n_out, real_t *y_out,
                   const real_t *y_init, real_t lna_init, long *n_steps)
{
    int N = orc_nstate(o);
    real_t *y = (real_t *)malloc(sizeof(real_t) * N);
    real_t x;
    if (y_init) { memcpy(y, y_init, sizeof(real_t) * N); x = lna_init; }
    else { x = orc_lna_start(c, k); orc_initial(c, o, k, x, y); }
    radau_ws w;
    ws_alloc(&w, o, N);
    long steps = 0;
    int rc = 0;
    for (int n = 0; n < n_out && rc == 0; n++) {
        real_t x1 = lna_out[n];
        if (RE(x1) > RE(x)) {
            int m = orc_schedule_count(c, o, k, x, x1);
            real_t h = (x1 - x) / m;
            for (int s = 0; s < m && rc == 0; s++) {
                real_t xs = x + s * h;
                real_t hs = (s == m - 1) ? (x1 - xs) : h;
                if (o->max_steps > 0 && steps >= o->max_steps) { rc = 1; break; }
                rc = radau_linear_step(c, o, k, xs, hs, y, &w);
                steps++;
            }
            x = x1;
        }
        memcpy(y_out + (size_t)n * N, y, sizeof(real_t) * N);
    }
    if (rc == 1 && o->max_steps > 0) rc = 0; /* budget reached: timing sample only */
    ws_free(&w);
    free(y);
    if (n_steps) *n_steps = steps;
    return rc;
}

static void sources_at(const orc_cosmo *c, const orc_opts *o, real_t k, real_t lna,
                       const real_t *y, real_t *S, real_t *scratch)
{
    orc_bg b;
    orc_bg_eval(c, lna, &b, 2);
    const int Nn = i_nu(o), P = i_pol(o);
    real_t hp, etap;
    metric(o, &b, k, y, &hp, &etap);
    real_t *dy = scratch;
    orc_rhs_bg(o, &b, k, y, dy);
    real_t Hc = b.Hc, k2 = k * k;
    real_t alpha = Hc * (hp + 6.0 * etap) / (2.0 * k2);
    real_t drho, rpth, rpsig;
    ncdm_sums(o, &b, k, y, &drho, &rpth, &rpsig);
    real_t shear = (4.0 / 3.0) * (b.fg * y[I_G0 + 2] + b.fnu * y[Nn + 2]) + rpsig;
    real_t Ha_p = -2.0 * Hc * alpha + y[I_ETA] - 4.5 * Hc * Hc / k2 * shear; /* H alpha' */
    real_t alpha_p = Ha_p / Hc;
    real_t thb = y[I_TB], thb_p = dy[I_TB];
    real_t eta = y[I_ETA];
    real_t sw = b.g * (0.25 * y[I_G0] + Ha_p);
    real_t isw = b.g * (eta - Ha_p - 2.0 * Hc * alpha)
               + 2.0 * Hc * b.expmk * (etap - b.dHc * alpha - Ha_p);
    real_t dop = Hc * (b.g * (thb_p / k2 + alpha_p) + b.dg * (thb / k2 + alpha));
    S[0] = o->scale_sw * sw + o->scale_isw * isw + o->scale_dop * dop;
    S[1] = o->scale_isw * b.expmk * k * (Ha_p + 2.0 * Hc * alpha - eta);
    S[2] = b.g * (2.0 * y[I_G0 + 2] + y[P] + y[P + 2]) / 8.0;
}

int orc_sources_mode(const orc_cosmo *c, const orc_opts *o, real_t k, real_t *S, long *n_steps)
{
    int N = orc_nstate(o), nt = c->n_tau;
    real_t *Y = (real_t *)malloc(sizeof(real_t) * (size_t)nt * N);
    real_t *scratch = (real_t *)malloc(sizeof(real_t) * N);
    int rc = orc_solve_mode(c, o, k, c->node_lna, nt, Y, NULL, 0.0, n_steps);
    for (int i = 0; i < nt && rc == 0; i++)
        sources_at(c, o, k, c->node_lna[i], Y + (size_t)i * N, S + 3 * i, scratch);
    free(Y);
    free(scratch);
    return rc;
}
