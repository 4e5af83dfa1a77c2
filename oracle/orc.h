/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow FP64 CPU restatement of the ABCMB linear Einstein-Boltzmann hot
 * path (arXiv 2602.15104), used to check the CUDA library.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may load
 * it.  It shares no code, header, constant or table with the CUDA path.
 *
 * What it computes, per cosmology (each step cites the passage it follows):
 *   background        flat LCDM closed form (App. C.1-C.5), conformal time by
 *                     quadrature (Sec. 2.4 "Background")
 *   recombination     Saha helium (App. B.1.1), Saha hydrogen (App. B.1.2,
 *                     eq. SahaH) then a Peebles three-level atom (the TLA the
 *                     paper cites in App. B.1.2; rates from the literature),
 *                     matter temperature (App. B.1.2), tanh reionization
 *                     (App. B.2, eqs. h_reion, he_reion, y_reio), tau_reion root
 *                     (App. A.2, eq. tau_reion)
 *   perturbations     synchronous-gauge hierarchies in x = ln a (App. B.3.1,
 *                     App. C), start time a_i(k) (App. A.1, eqs. k_start_small
 *                     and k_start_large), adiabatic initial conditions, no
 *                     tight-coupling switch (App. B.6); solved by a 3-stage
 *                     Radau IIA collocation step on a fixed step schedule
 *                     landing on every tau node
 *   sources           S_T0, S_T1, S_T2 (App. B.4, eq. source_functions)
 *   projection        Delta_T, Delta_E by the trapezoid rule in tau (App. B.4,
 *                     App. B.6) with exact spherical Bessel functions
 *   C_ell             4 pi int dk/k P(k) Delta_X Delta_Y (App. B.4, eq.
 *                     c_ell_def, eq. PK_pivot), trapezoid in ln k
 *
 * Every part is pinned by tests/test_oracle_pins.py (closed forms, textbook
 * tables, the paper's printed values, defining equations), each pin checked
 * against a planted mistake.  What no test here can fix is the physical
 * accuracy against an external Boltzmann or recombination code (none is
 * available); orc_background.c says where that touches the thermal history.
 *
 * The arithmetic is written once over the scalar type real_t (orc_real.h):
 * double in liborc.so, double complex in liborc_cs.so, which gives the
 * forward sensitivities of every output to one parameter by the complex
 * step (see orc_real.h).
 */
#ifndef ORC_H
#define ORC_H

#include <stddef.h>

#include "orc_real.h"

#define ORC_MAX_L 64

/* Test hooks (bit flags) used only by the oracle's own pins. */
enum {
    ORC_HOOK_FREEZE_METRIC = 1, /* h' = eta' = 0 in every equation          */
    ORC_HOOK_NO_THOMSON = 2,    /* 1/(H tau_c) = 0                           */
    ORC_HOOK_EDS_CDM = 4,       /* Einstein-de Sitter background, CDM only   */
};

typedef struct {
    int lmax_g, lmax_pol, lmax_nu;
    double scale_sw, scale_isw, scale_dop, scale_pol;
    double step_c;   /* step schedule: h <= step_c / (1 + k/H)          */
    double step_cap; /* absolute cap on a step in ln a                  */
    int hooks;
    long max_steps;  /* 0 = unlimited; > 0 stops each mode early (timing samples) */
    int lmax_ncdm;   /* massive-neutrino hierarchies' truncation (0: none)      */
    double m_ncdm;   /* one massive neutrino of this mass [eV] (0: none); the
                        massless species then number two (App. A.1 example)   */
    int node_recipe; /* tau nodes: 0 the default placement, 1 the refined tail */
} orc_opts;

/* Per-cosmology state: derived parameters, thermal-history tables, tau nodes. */
typedef struct orc_cosmo orc_cosmo;

struct orc_cosmo {
    /* inputs */
    real_t omega_b, omega_cdm, h, n_s, ln10As, tau_reio;
    /* fixed parameters (App. A.2 defaults) */
    real_t YHe, TCMB0, Tnu_ratio, N_nu;
    real_t z_re_He, dz_re_He, dz_re, beta_re;
    real_t R_tc, R_large, k_pivot;
    /* derived */
    real_t H0;                         /* [1/Mpc]                           */
    real_t Om_b, Om_c, Om_g, Om_nu, Om_r, Om_m, Om_L;
    real_t R_nu, f_He, nH0, A_s;
    real_t rho_g0;                     /* photon energy density today [eV/cm^3] */
    real_t z_reion;
    real_t lna_tc, lna_He3, lna_sw, lna_700;
    real_t tau0;
    int hooks;
    /* one massive neutrino (App. B.3 "Massive neutrinos", App. C.6): mass,
       temperature today T_ncdm = 0.71611 T_gamma, x = a m / T_ncdm at a = 1,
       and rho_ncdm / rho_crit = ncdm_pref a^-4 sum_i K_i (1 + e^-q_i) eps_i / q_i^2 */
    real_t m_ncdm, T_ncdm_ratio, ncdm_x1, ncdm_pref, Om_ncdm_rel, Om_ncdm;
    /* conformal-time table, uniform in ln a */
    int n_ct; real_t ct_lna0, ct_dlna; real_t *ct_tau;
    /* TLA table (x_p, T_m and their ln a derivatives) on two uniform ln a
       segments: [lna_sw, lna_700] (n_th1 intervals) and [lna_700, 0]
       (n_th2 intervals); node i at th_lna[i] */
    int n_th1, n_th2; real_t *th_lna;
    real_t *th_xp, *th_dxp, *th_Tm, *th_dTm;
    /* optical depth table kappa(ln a), uniform grid from ct_lna0 to 0 */
    int n_kp; real_t kp_lna0, kp_dlna; real_t *kp_kappa;
    /* tau nodes */
    int n_tau; real_t *node_lna, *node_tau, *node_w;
};

/* background point evaluation */
typedef struct {
    real_t a, Hc, dHc;            /* conformal Hubble [1/Mpc] and d/dln a */
    real_t fc, fb, fg, fnu;       /* rho_i / rho_tot                      */
    real_t fncdm, wncdm;          /* massive neutrinos: rho / rho_tot, p / rho */
    real_t ncdm_x;                /* a m / T_ncdm                          */
    real_t ncdm_n;                /* ncdm_pref a^-4 / (rho_tot / rho_crit): turns the
                                     momentum sums into fractions of rho_tot */
    real_t tau;                   /* conformal time [Mpc]                 */
    real_t xe, dxe;               /* free-electron fraction and d/dln a   */
    real_t nuT;                   /* 1/(H tau_c) = a n_e sigma_T / H      */
    real_t Rinv;                  /* 4 rho_g / (3 rho_b)                  */
    real_t cs2;                   /* baryon sound speed squared           */
    real_t kappa, expmk, g, dg;   /* optical depth, e^-kappa, visibility  */
} orc_bg;

/* orc_background.c */
int orc_cosmo_init(orc_cosmo *c, const real_t p[6], int n_tau, int hooks, double m_ncdm, int node_recipe);
void orc_cosmo_free(orc_cosmo *c);
/* with_thermo: 0 background only, 1 + what the ODE needs, 2 + kappa, g, g' */
void orc_bg_eval(const orc_cosmo *c, real_t lna, orc_bg *out, int with_thermo);
real_t orc_Hconf(const orc_cosmo *c, real_t lna);
real_t orc_tau_of_lna(const orc_cosmo *c, real_t lna);
real_t orc_xe_of_lna(const orc_cosmo *c, real_t lna, real_t *dxe);
real_t orc_Tm_of_lna(const orc_cosmo *c, real_t lna, real_t *dlnTm);
real_t orc_lna_start(const orc_cosmo *c, real_t k);

/* orc_linalg.c */
int orc_lu_factor(real_t *A, int n, int *piv, int *ext /* [2n] */);
void orc_lu_solve(const real_t *A, int n, const int *piv, const int *ext, real_t *b);

/* orc_perturb.c */
int orc_nstate(const orc_opts *o);
int orc_schedule_count(const orc_cosmo *c, const orc_opts *o, real_t k, real_t x0, real_t x1);
void orc_rhs_bg(const orc_opts *o, const orc_bg *b, real_t k, const real_t *y,
                real_t *dy);
void orc_rhs(const orc_cosmo *c, const orc_opts *o, real_t k, real_t lna,
             const real_t *y, real_t *dy);
void orc_initial(const orc_cosmo *c, const orc_opts *o, real_t k, real_t lna_i,
                 real_t *y);
int orc_solve_mode(const orc_cosmo *c, const orc_opts *o, real_t k,
                   const real_t *lna_out, int n_out, real_t *y_out,
                   const real_t *y_init, real_t lna_init, long *n_steps);
int orc_sources_mode(const orc_cosmo *c, const orc_opts *o, real_t k,
                     real_t *S /* [n_tau][3] */, long *n_steps);

/* orc_spectra.c */
void orc_bessel_all(int lmax, real_t x, real_t *j /* [lmax+1] */);

#endif
