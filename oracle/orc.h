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
 * Parity-unpinned parts are listed in the file headers that implement them.
 */
#ifndef ORC_H
#define ORC_H

#include <stddef.h>

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
    double omega_b, omega_cdm, h, n_s, ln10As, tau_reio;
    /* fixed parameters (App. A.2 defaults) */
    double YHe, TCMB0, Tnu_ratio, N_nu;
    double z_re_He, dz_re_He, dz_re, beta_re;
    double R_tc, R_large, k_pivot;
    /* derived */
    double H0;                         /* [1/Mpc]                           */
    double Om_b, Om_c, Om_g, Om_nu, Om_r, Om_m, Om_L;
    double R_nu, f_He, nH0, A_s;
    double rho_g0;                     /* photon energy density today [eV/cm^3] */
    double z_reion;
    double lna_tc, lna_He3, lna_sw, lna_700;
    double tau0;
    int hooks;
    /* one massive neutrino (App. B.3 "Massive neutrinos", App. C.6): mass,
       temperature today T_ncdm = 0.71611 T_gamma, x = a m / T_ncdm at a = 1,
       and rho_ncdm / rho_crit = ncdm_pref a^-4 sum_i K_i (1 + e^-q_i) eps_i / q_i^2 */
    double m_ncdm, T_ncdm_ratio, ncdm_x1, ncdm_pref, Om_ncdm_rel, Om_ncdm;
    /* conformal-time table, uniform in ln a */
    int n_ct; double ct_lna0, ct_dlna; double *ct_tau;
    /* TLA table (x_p, T_m and their ln a derivatives) on two uniform ln a
       segments: [lna_sw, lna_700] (n_th1 intervals) and [lna_700, 0]
       (n_th2 intervals); node i at th_lna[i] */
    int n_th1, n_th2; double *th_lna;
    double *th_xp, *th_dxp, *th_Tm, *th_dTm;
    /* optical depth table kappa(ln a), uniform grid from ct_lna0 to 0 */
    int n_kp; double kp_lna0, kp_dlna; double *kp_kappa;
    /* tau nodes */
    int n_tau; double *node_lna, *node_tau, *node_w;
};

/* background point evaluation */
typedef struct {
    double a, Hc, dHc;            /* conformal Hubble [1/Mpc] and d/dln a */
    double fc, fb, fg, fnu;       /* rho_i / rho_tot                      */
    double fncdm, wncdm;          /* massive neutrinos: rho / rho_tot, p / rho */
    double ncdm_x;                /* a m / T_ncdm                          */
    double ncdm_n;                /* ncdm_pref a^-4 / (rho_tot / rho_crit): turns the
                                     momentum sums into fractions of rho_tot */
    double tau;                   /* conformal time [Mpc]                 */
    double xe, dxe;               /* free-electron fraction and d/dln a   */
    double nuT;                   /* 1/(H tau_c) = a n_e sigma_T / H      */
    double Rinv;                  /* 4 rho_g / (3 rho_b)                  */
    double cs2;                   /* baryon sound speed squared           */
    double kappa, expmk, g, dg;   /* optical depth, e^-kappa, visibility  */
} orc_bg;

/* orc_background.c */
int orc_cosmo_init(orc_cosmo *c, const double p[6], int n_tau, int hooks, double m_ncdm, int node_recipe);
void orc_cosmo_free(orc_cosmo *c);
/* with_thermo: 0 background only, 1 + what the ODE needs, 2 + kappa, g, g' */
void orc_bg_eval(const orc_cosmo *c, double lna, orc_bg *out, int with_thermo);
double orc_Hconf(const orc_cosmo *c, double lna);
double orc_tau_of_lna(const orc_cosmo *c, double lna);
double orc_xe_of_lna(const orc_cosmo *c, double lna, double *dxe);
double orc_Tm_of_lna(const orc_cosmo *c, double lna, double *dlnTm);
double orc_lna_start(const orc_cosmo *c, double k);

/* orc_linalg.c */
int orc_lu_factor(double *A, int n, int *piv, int *ext /* [2n] */);
void orc_lu_solve(const double *A, int n, const int *piv, const int *ext, double *b);

/* orc_perturb.c */
int orc_nstate(const orc_opts *o);
int orc_schedule_count(const orc_cosmo *c, const orc_opts *o, double k, double x0, double x1);
void orc_rhs_bg(const orc_opts *o, const orc_bg *b, double k, const double *y,
                double *dy);
void orc_rhs(const orc_cosmo *c, const orc_opts *o, double k, double lna,
             const double *y, double *dy);
void orc_initial(const orc_cosmo *c, const orc_opts *o, double k, double lna_i,
                 double *y);
int orc_solve_mode(const orc_cosmo *c, const orc_opts *o, double k,
                   const double *lna_out, int n_out, double *y_out,
                   const double *y_init, double lna_init, long *n_steps);
int orc_sources_mode(const orc_cosmo *c, const orc_opts *o, double k,
                     double *S /* [n_tau][3] */, long *n_steps);

/* orc_spectra.c */
void orc_bessel_all(int lmax, double x, double *j /* [lmax+1] */);

#endif
