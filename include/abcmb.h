/*
 * abcmb.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of the ABCMB linear Einstein-Boltzmann method (arXiv 2602.15104):
 *
 *   abcmb_background_tables   thermal history + tau nodes per cosmology
 *   abcmb_perturb             per-k stiff linear perturbation ODEs -> CMB sources
 *                             (abcmb_perturb_noalloc: the same with fixed scratch)
 *   abcmb_project             line-of-sight projection -> transfer functions
 *   abcmb_cl                  k-quadrature -> C_ell^{TT,TE,EE}
 *   abcmb_project_mixed, abcmb_cl_mixed   the same two steps in FP32
 * and around them
 *   abcmb_project_interp, abcmb_transfer_k_grid   projection on the transfer k grid
 *   abcmb_matter_pk           matter power spectrum P(k, z)
 *   abcmb_delta_m_nodes, abcmb_cl_psi, abcmb_lens  lensing potential (Limber)
 *                             and lensed spectra
 *   abcmb_perturb_taped, abcmb_perturb_adjoint, abcmb_project_adjoint,
 *   abcmb_cl_adjoint, abcmb_param_stencil, abcmb_record_vjp  reverse-mode gradients
 *   abcmb_server_*            a request server over one device arena
 *
 * Conventions shared by every entry point
 *   - Every pointer argument is a DEVICE pointer allocated by the caller
 *     (the library allocates no device memory; a server allocates its
 *     handle, streams, events and pinned host staging when it is created;
 *     apart from a server and the static scratch of abcmb_perturb_noalloc
 *     it keeps no state between calls), unless its name ends in _host.  Every array is C-contiguous
 *     float64 (int32 for status/step arrays, float32 where a name ends in 32)
 *     in the layout stated at each argument, and must hold at least the
 *     elements that layout gives: a plain pointer carries no extent, so the
 *     library cannot check it (the Python binding does, before each call).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls only enqueue work on it; results are valid once the
 *     stream has been synchronised.
 *   - Return value: ABCMB_OK, or an error code.  Arguments are validated on
 *     the host before anything is enqueued (ABCMB_E_INVALID_ARG); launch
 *     failures return ABCMB_E_CUDA.  Numerical failures found on the device
 *     are reported in the status words named at each call, never by aborting.
 *   - Units: Mpc for lengths and conformal time, 1/Mpc for k; C_ell is the
 *     dimensionless angular power for primordial curvature amplitude A_s
 *     (C_ell, not D_ell; paper Sec. 2.3 footnote).
 */
#ifndef ABCMB_H
#define ABCMB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ABCMB_OK = 0,
    ABCMB_E_INVALID_ARG = 1, /* host-side validation failed; nothing enqueued   */
    ABCMB_E_CUDA = 2,        /* a kernel launch or CUDA call failed             */
    ABCMB_E_MAX_STEPS = 3,   /* status word: a mode hit its step budget         */
    ABCMB_E_NONFINITE = 4,   /* status word: a non-finite value was produced    */
    ABCMB_E_BACKGROUND = 5,  /* status word: a background root was not found    */
    ABCMB_E_SCRATCH_TOO_SMALL = 6, /* abcmb_perturb_noalloc: problem needs more
                                      than ABCMB_NOALLOC_SCRATCH_BYTES     */
};

/* Number of doubles per cosmology in params: omega_b, omega_cdm, h, n_s,
   ln(1e10 A_s), tau_reion (paper App. A.2).  The other cosmological inputs
   are the paper's defaults: Y_He = 0.245, T_CMB0 = 2.34865418e-4 eV, three
   massless neutrinos with T_nu/T_gamma = 0.71636856 (N_eff = 3.044),
   reionization widths Delta z = 0.5, z_He = 3.5, Delta z_He = 0.5,
   beta = 1.5, k_pivot = 0.05/Mpc, R_tc = 1.5e-3, R_large = 7e-2. */
#define ABCMB_NPARAM 6

typedef struct {
    int lmax_g;      /* photon temperature hierarchy truncation, 4..128 (App. A.1 l_max_g) */
    int lmax_pol;    /* photon polarization hierarchy truncation, 4..128 (l_max_pol_g)     */
    int lmax_nu;     /* massless-neutrino hierarchy truncation, 4..128 (l_max_massless_nu) */
    int lmax_cl;     /* C_ell computed for every ell in [2, lmax_cl]; 2..5000 (App. A.1)   */
    int n_tau;       /* number of tau nodes of the line-of-sight integral, 8..65536        */
    int max_steps;   /* accepted+rejected ODE step budget per k mode, >= 1                 */
    double rtol;     /* ODE relative tolerance, (0, 1)                                     */
    double atol;     /* ODE absolute tolerance floor, >= 0                                 */
    double scale_sw, scale_isw, scale_dop, scale_pol; /* source switches (App. A.1)       */
    double m_ncdm;   /* one massive neutrino of this mass [eV] (App. B.3, App. C.6); 0: all
                        three neutrinos massless.  With a mass the massless species number
                        two and the massive one has T = 0.71611 T_gamma (App. A.1 example) */
    int lmax_ncdm;   /* its momentum-bin hierarchies' truncation: 0 when m_ncdm = 0, else
                        3..63 (App. A.1 l_max_massive_nu, default 17)                      */
    int node_recipe; /* tau nodes: 0 = 1/4 uniform in ln a from a_tc to z = 1300, 1/2 uniform
                        in z over [1300, 900), the rest uniform in tau to today (default);
                        1 = 1/5, 2/5 over [1300, 900), 1/5 uniform in z over [900, 300),
                        the rest uniform in tau from z = 300, which resolves the tail of
                        the visibility function (low-l TT converges with ~10x fewer nodes) */
    int n_wide;      /* abcmb_perturb with hierarchies 16..63: the modes of the n_wide largest k
                        (k ascending in the array) run on eight lanes each instead of four: the
                        same arithmetic per mode, a shorter chain of work per step for the most
                        expensive modes (a mode's result depends on its warp-mates only through
                        the warp-wide switch to the explicit regime, within the ODE tolerance);
                        0: none (the default: on the 64-cosmology, 400 k workload 12, 25 and
                        50 wide k gave no gain); must be >= 0                              */
    double err_floor; /* the four-lane kernel's error norm: component i is measured against
                        atol + rtol max(|y_i|, err_floor m_g), m_g the largest magnitude in its
                        group (eta/delta_c/delta_b, theta_b, photons, neutrinos), so components
                        below err_floor of their group are held to rtol of that level; in
                        (0, 1], default 1e-4 (the thread-per-mode and adjoint solvers keep
                        1e-4)                                                             */
} abcmb_options;

/* Fill *o with the defaults used by the library's tests: hierarchies 12,
   lmax_cl 2500, 6000 tau nodes, rtol 1e-6, atol 1e-12, switches 1.  At rtol
   1e-6 the ODE moves C_l by <= 5e-7 relative against the converged solution
   (measured on the 64-cosmology, l <= 2500 workload). */
void abcmb_default_options(abcmb_options *o);

/* ABCMB_OK if every field of *o is in its stated range (o may be NULL:
   ABCMB_E_INVALID_ARG).  Every entry point below applies this check first. */
int abcmb_validate_options(const abcmb_options *o);

/* Length, in doubles, of one cosmology's background record for these
   options (ABCMB_BG_* offsets below address it).  Returns 0 if invalid. */
size_t abcmb_bg_doubles(const abcmb_options *o);

/* Layout of one background record (doubles):
     [0, ABCMB_BG_NSCALAR)                 scalars, ABCMB_S_* indices
     [ABCMB_BG_TABLE, + 8 * ABCMB_BG_NLNA) table on the uniform ln a grid
            ln a_j = ABCMB_BG_LNA0 + j / ABCMB_BG_PER_UNIT, 8 columns per node:
            1/(H tau_c), d/dln a of it, tau, dtau/dln a = 1/H, c_s^2,
            d c_s^2/dln a, kappa, x_e
     [ABCMB_BG_ODETAB, + 20 * ABCMB_BG_NLNA) on the same grid, 10 (value,
            d/dln a) pairs per node read by the ODE kernel: 1/H, 1/(H tau),
            f_c, f_b, f_gamma, f_nu (rho_i / rho_tot), 1/(H tau_c),
            (4 rho_g / 3 rho_b) / (H tau_c), c_s^2, H (all conformal)
     [ABCMB_BG_NODES, + 8 * n_tau) 8 columns per tau node: ln a, tau,
            trapezoid weight, g, dg/dln a, e^-kappa, conformal H, dH/dln a
     [ABCMB_BG_NODES + 8 * n_tau, + ABCMB_BG_ODEPOLY_DOUBLES) the ODE table
            again, as the cubic Hermite polynomial of each interval: for
            interval j (ln a_j to ln a_j+1) and each of its 10 quantities in
            the order above, c0..c3 of c0 + u (c1 + u (c2 + u c3)), u the
            fraction of the interval (the form the four-lane ODE kernel reads)
   The whole record is ABCMB_BG_LEN(n_tau) doubles (abcmb_bg_doubles).      */
#define ABCMB_BG_NSCALAR 64
#define ABCMB_BG_PER_UNIT 1024
#define ABCMB_BG_LNA0 (-18.0)
#define ABCMB_BG_NLNA (18 * 1024 + 1)
#define ABCMB_BG_TABLE ABCMB_BG_NSCALAR
#define ABCMB_BG_ODETAB (ABCMB_BG_TABLE + 8 * ABCMB_BG_NLNA)
#define ABCMB_BG_NODES (ABCMB_BG_ODETAB + 20 * ABCMB_BG_NLNA)
#define ABCMB_BG_ODEPOLY_DOUBLES (40L * (ABCMB_BG_NLNA - 1))
#define ABCMB_BG_ODEPOLY(n_tau) (ABCMB_BG_NODES + 8L * (n_tau))
#define ABCMB_BG_LEN(n_tau) (ABCMB_BG_ODEPOLY(n_tau) + ABCMB_BG_ODEPOLY_DOUBLES)

enum {
    ABCMB_S_STATUS = 0, ABCMB_S_H0, ABCMB_S_OMB, ABCMB_S_OMC, ABCMB_S_OMG, ABCMB_S_OMNU,
    ABCMB_S_OML, ABCMB_S_RNU, ABCMB_S_FHE, ABCMB_S_NH0, ABCMB_S_AS, ABCMB_S_NS,
    ABCMB_S_ZREION, ABCMB_S_LNA_TC, ABCMB_S_LNA_SW, ABCMB_S_TAU0, ABCMB_S_LNA_HE3,
    ABCMB_S_LNA_700, ABCMB_S_NTAU,
    ABCMB_S_NCDM_PREF, /* massive neutrino: rho / rho_crit = PREF a^-4 sum_i K_i (1 + e^-q_i) eps_i / q_i^2 */
    ABCMB_S_NCDM_X1,   /* m / T_ncdm (eps_i = sqrt(q_i^2 + (a X1)^2))                             */
    ABCMB_S_OMNCDM_REL, /* its relativistic-limit density parameter                               */
    ABCMB_S_COUNT
};

/*
 * Background and thermal history of B cosmologies (paper Sec. 2.4
 * "Background", App. B.1-B.2, App. B.4 kappa and g, App. C.1-C.5 densities):
 * flat LCDM closed form, conformal time, Saha helium and hydrogen then a
 * Peebles three-level atom, matter temperature, tanh reionization with
 * z_reion solved from tau_reion, the tight-coupling start a_tc
 * (H tau_c = R_tc, App. A.1), and the n_tau tau nodes with trapezoid
 * weights (1/4 uniform in ln a from a_tc to z = 1300, 1/2 uniform in z on
 * [1300, 900), 1/4 uniform in tau from z = 900 to tau_0 exclusive).
 *
 *   params  [B][ABCMB_NPARAM]            device, read
 *   bg      [B][abcmb_bg_doubles(o)]     device, written
 * Device-side failure (a root not bracketed, a non-finite value) sets
 * bg[b*len + ABCMB_S_STATUS] to ABCMB_E_BACKGROUND / ABCMB_E_NONFINITE.
 */
int abcmb_background_tables(int B, const double *params, const abcmb_options *o,
                            double *bg, void *stream);

/*
 * Linear synchronous-gauge perturbations (App. B.3.1, App. C: metric eqs.
 * hprime/etaprime, CDM, baryons, photon temperature and polarization and
 * massless-neutrino hierarchies, no tight-coupling switch, App. B.6) for
 * every (cosmology, k) mode, from a_i(k) = min(a_tc, a_k), k/H(a_k) =
 * R_large (App. A.1), with adiabatic initial conditions, to the last tau
 * node, landing on every tau node and writing the CMB sources there
 * (App. B.4, eq. source_functions).
 *
 *   bg           [B][abcmb_bg_doubles(o)]  device, read (from abcmb_background_tables)
 *   k            [Nk]                      device, read, 1/Mpc, each > 0
 *   S            [B][Nk][n_tau][3]         device, written: S_T0, S_T1 and
 *                S_P = g Pi / 8 (S_T2 before scale_pol; S_E = sqrt(6) S_P)
 *   mode_status  [B][Nk] int32             device, written: ABCMB_OK,
 *                ABCMB_E_MAX_STEPS or ABCMB_E_NONFINITE per mode
 *   steps        [B][Nk][2] int32 or NULL  device, written: ODE steps taken
 *                (accepted and rejected) and linearly implicit substeps
 *   workspace    >= abcmb_perturb_workspace_bytes(B, Nk, o) bytes, device,
 *                256-byte aligned; returns ABCMB_E_INVALID_ARG if smaller.
 *                That size is 0, and workspace may be NULL, while every
 *                hierarchy truncation is <= 63: the state then lives on chip
 *                (four lanes per mode).  Deeper hierarchies (64..128) run one
 *                thread per mode with the state in this workspace.
 */
int abcmb_perturb(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                  double *S, int *mode_status, int *steps, void *workspace,
                  size_t workspace_bytes, void *stream);

/* Bytes of device workspace abcmb_perturb needs for B cosmologies and Nk
   modes: 0 when every hierarchy truncation is <= 63 (no workspace needed)
   or the options are invalid, else 64 (Lg + Lp + Ln + 7) bytes per mode.  The
   caller allocates it; its contents need no initialisation and are scratch
   after the call. */
size_t abcmb_perturb_workspace_bytes(int B, int Nk, const abcmb_options *o);

/*
 * abcmb_perturb for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a service of the library, not a step of the method.
 *
 * Some callers must not call cudaMalloc at all: an application whose device
 * memory is entirely owned by another runtime's caching pool (a stray
 * allocation outside the pool can fail or fragment it), or a latency-bound
 * loop in which an allocation's implicit device synchronisation is not
 * acceptable.  This entry point computes exactly what abcmb_perturb computes
 * (same kernels, same arguments except the workspace).  Hierarchies <= 63
 * need no scratch at all; deeper ones keep the working vectors in a static
 * device array of ABCMB_NOALLOC_SCRATCH_BYTES that the library owns.  It
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *
 *   - Size limit: abcmb_perturb_workspace_bytes(B, Nk, o) must not exceed
 *     ABCMB_NOALLOC_SCRATCH_BYTES (64 MiB: e.g. 4 245 modes at hierarchy 80,
 *     2 681 at hierarchy 128); larger problems return
 *     ABCMB_E_SCRATCH_TOO_SMALL and enqueue nothing.  Every GPU that loads the
 *     library reserves the array until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and so does the first
 *     call after the device's context was replaced (cudaDeviceReset): the
 *     address is cached per device together with the context's unique id.
 *     Make that first call before any stream capture begins.
 *   - Every call shares the one array, which keeps the last call's contents;
 *     the kernel overwrites every element it reads, so nothing needs
 *     clearing.  Calls whose kernels overlap on the GPU (different streams,
 *     no ordering between them) race on the array: order them.
 *   - Arguments, outputs and status words as abcmb_perturb.
 */
#define ABCMB_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int abcmb_perturb_noalloc(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                          double *S, int *mode_status, int *steps, void *stream);

/*
 * Matter power spectrum (App. B.4, eq. PK) at redshift z:
 *   P(k, z) = (2 pi^2 / k^3) A_s (k/k_pivot)^(n_s-1) delta_m(k, z)^2,
 *   delta_m = (rho_c delta_c + rho_b delta_b) / (rho_c + rho_b)
 * (the non-relativistic species), from the same perturbation equations and
 * integrator as abcmb_perturb, run from a_i(k) to a = 1/(1+z) with no tau
 * nodes to land on.
 *
 *   bg, k        as abcmb_perturb
 *   z            0 <= z <= 1000
 *   Pk           [B][Nk]       device, written, Mpc^3 (NaN for a failed mode)
 *   mode_status  [B][Nk] int32 device, written as abcmb_perturb
 * Hierarchies up to 63 (ABCMB_E_INVALID_ARG above).
 */
int abcmb_matter_pk(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double z,
                    double *Pk, int *mode_status, void *stream);

/*
 * Line-of-sight projection (App. B.4): for every ell in [2, lmax_cl],
 *   Delta_T = sum_i w_i [S_T0 j_l + S_T1 j_l' + scale_pol S_P (3 j_l'' + j_l)/2]
 *   Delta_E = sqrt(3 (l+2)! / (8 (l-2)!)) sum_i w_i sqrt(6) S_P j_l / x^2
 * with x = k (tau_0 - tau_i) and trapezoid weights w_i in tau (App. B.6).
 *
 *   bg     [B][abcmb_bg_doubles(o)]   device, read
 *   S      [B][Nk][n_tau][3]          device, read
 *   k      [Nk]                       device, read
 *   Delta  [B][Nk][lmax_cl-1][2]      device, written (Delta_T, Delta_E)
 */
int abcmb_project(int B, const double *bg, const double *S, const double *k, int Nk,
                  const abcmb_options *o, double *Delta, void *stream);

/*
 * k-quadrature (App. B.4 eq. c_ell_def, eq. PK_pivot):
 *   C_l^{XY} = 4 pi sum_k w_k A_s (k/0.05)^(n_s-1) Delta_X Delta_Y,
 * w_k the trapezoid weights in ln k over the given (ascending) k nodes.
 *
 *   bg     [B][abcmb_bg_doubles(o)]   device, read (A_s, n_s)
 *   Delta  [B][Nk][lmax_cl-1][2]      device, read
 *   k      [Nk]                       device, read, strictly ascending
 *   Cl     [B][3][lmax_cl-1]          device, written: TT, TE, EE for l = 2..lmax_cl
 */
int abcmb_cl(int B, const double *bg, const double *Delta, const double *k, int Nk,
             const abcmb_options *o, double *Cl, void *stream);

/*
 * Projection onto another k grid (App. A.1 transfer grid, eq.
 * k_transfer_spacing): abcmb_project at the wavenumbers kt, with each
 * tau node's sources interpolated from the ODE nodes k by piecewise cubic
 * Hermite polynomials in ln k whose slopes are three-point derivatives
 * (centred, one-sided at the ends; exact for quadratics in ln k; outside
 * [k_0, k_{Nk-1}] the end intervals' cubics extend).
 *
 *   S      [B][Nk][n_tau][3]        device, read (sources at k, as from abcmb_perturb)
 *   k      [Nk], Nk >= 4            device, read, strictly ascending
 *   kt     [Nkt]                    device, read
 *   Delta  [B][Nkt][lmax_cl-1][2]   device, written
 * abcmb_cl on (Delta, kt) then gives C_l on the transfer grid.
 */
int abcmb_project_interp(int B, const double *bg, const double *S, const double *k, int Nk, const double *kt,
                         int Nkt, const abcmb_options *o, double *Delta, void *stream);

/* The transfer grid for lmax_cl (host function; the paper's defaults):
   from 0.1 / tau0_fid while k tau0_fid <= 1.8 lmax_cl,
   k_{n+1} = k_n + k_period 0.45 k_n / (k_n + 0.45 / 170),
   k_period = 2 pi / (tau0_fid - tau_rec_fid), tau0_fid = 14186.68 Mpc,
   tau_rec_fid = 281.040565 Mpc.  Writes min(count, cap) nodes to k_host (may
   be NULL) and returns the count; -1 for lmax_cl outside 2..5000. */
int abcmb_transfer_k_grid(int lmax_cl, double *k_host, int cap);

/*
 * CMB lensing of the spectra (App. B.5): the all-sky correlation-function
 * method the paper cites (Challinor & Lewis 2005), integrated over all of
 * mu in [-1, 1] on n_mu Gauss-Legendre nodes (the paper rejects the restricted
 * "fast" range).  The lensed-minus-unlensed correlation functions are built at
 * each node to second order in C_gl,2 and transformed back with d^l_00,
 * d^l_22, d^l_2-2 and d^l_20.
 *
 *   Cl         [B][3][L-1]          device, read: unlensed TT, TE, EE, l = 2..L
 *                                   (as abcmb_cl writes them with lmax_cl = L)
 *   Cpsi       [B][L-1]             device, read: lensing potential C_l^psi, l = 2..L
 *   lmax_out   2..L (lensing moves power from above lmax_out, so L should exceed it)
 *   n_mu       L + 1 .. 20000 Gauss-Legendre nodes
 *   Cl_lensed  [B][4][lmax_out-1]   device, written: lensed TT, TE, EE, BB
 */
int abcmb_lens(int B, const double *Cl, int L, const double *Cpsi, int lmax_out, int n_mu, double *Cl_lensed,
               void *stream);

/*
 * Matter density contrast at the tau nodes (App. B.4, eq. PK, for the
 * lensing potential of App. B.5):
 *   delta_m(k, tau_i) = (rho_c delta_c + rho_b delta_b) / (rho_c + rho_b)
 * from the same perturbation equations, integrator and node landing as
 * abcmb_perturb (which writes the CMB sources at the same nodes).
 *
 *   bg, k, o, mode_status   as abcmb_perturb (massless neutrinos only:
 *                           m_ncdm > 0 is ABCMB_E_INVALID_ARG)
 *   Dm    [B][Nk][n_tau]    device, written (NaN rows for a failed mode)
 */
int abcmb_delta_m_nodes(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *Dm,
                        int *mode_status, void *stream);

/*
 * Lensing potential spectrum in the Limber approximation (App. B.5):
 *   C_l^psi = 8 pi^2 / (l+1/2)^3 int_0^chi* dchi/chi P_psi((l+1/2)/chi, tau0 - chi) ((chi* - chi)/chi*)^2,
 *   P_psi(k, tau) = 9 Omega_m(tau)^2 H(tau)^4 / (8 pi^2 k) P(k, tau),
 *   P(k, tau) = (2 pi^2 / k^3) A_s (k/0.05)^(n_s-1) delta_m(k, tau)^2,
 * with chi* = tau0 - tau at the node of largest visibility, the trapezoid
 * rule in chi over the nodes from there to tau0 (chi = 0), H the conformal
 * Hubble rate, and delta_m taken between the k nodes by cubic Hermite
 * interpolation in ln k (zero outside [k_0, k_{Nk-1}]).
 *
 *   bg    [B][abcmb_bg_doubles(o)]  device, read
 *   Dm    [B][Nk][n_tau]            device, read (abcmb_delta_m_nodes)
 *   k     [Nk]                      device, read, strictly ascending, Nk >= 4
 *   lmax  2..6000
 *   Cpsi  [B][lmax-1]               device, written: l = 2..lmax, the layout abcmb_lens reads
 */
int abcmb_cl_psi(int B, const double *bg, const double *Dm, const double *k, int Nk, const abcmb_options *o,
                 int lmax, double *Cpsi, void *stream);

/*
 * Mixed precision (the FP32 form of the two calls above; the sources stay
 * FP64): same projection and k-quadrature, with every (node, l) product and
 * the in-warp sums in FP32 and the sums over tau-node groups and over k
 * Kahan-compensated in FP32.  x, 1/x, sin x and cos x are formed in FP64 per
 * node; the Bessel recurrence runs in double-float (pairs of floats,
 * ~2^-44 relative), since plain FP32 rounding would be amplified past the
 * turning point.  Expected error against the FP64 path ~1e-5 of each
 * spectrum's largest value (the projection's FP32 products do not
 * compensate).
 *
 *   Delta32 [B][Nk][lmax_cl-1][2] float32, device (written by
 *           abcmb_project_mixed, read by abcmb_cl_mixed)
 *   other arguments as abcmb_project / abcmb_cl; Cl is float64.
 */
int abcmb_project_mixed(int B, const double *bg, const double *S, const double *k, int Nk,
                        const abcmb_options *o, float *Delta32, void *stream);
int abcmb_cl_mixed(int B, const double *bg, const float *Delta32, const double *k, int Nk,
                   const abcmb_options *o, double *Cl, void *stream);

/*
 * Gradients of C_l with respect to the six parameters (sec. "Gradients of
 * ABCMB outputs", and the gradient timings of sec. 5).  The paper takes them
 * by automatic differentiation; here the perturbation ODE, the projection and
 * the k-quadrature have hand-written discrete adjoints (reverse mode, one
 * contraction Cbar . dC/dtheta per call chain), and the background record's
 * parameter Jacobian is taken by central differences of
 * abcmb_background_tables (relative step 1e-4), contracted on the device.
 * Call order for one vector-Jacobian product:
 *
 *   [abcmb_grad_count_steps, abcmb_grad_plan   optional: tapes sized per mode]
 *   abcmb_perturb_taped   -> S (as abcmb_perturb) and the tape in workspace
 *   abcmb_project, abcmb_cl  (forward, unchanged)
 *   abcmb_cl_adjoint      Clbar   -> Deltabar, recbar += d/d(A_s, n_s)
 *   abcmb_project_adjoint Deltabar -> Sbar, recbar += d/d(node tau, w), d/d tau_0
 *   abcmb_perturb_adjoint Sbar    -> recbar += d/d(ODE table, conformal-time
 *                                    table, node data, R_nu)
 *   abcmb_param_stencil   theta -> h and the rows theta +- h e_j
 *   abcmb_record_vjp      recbar, records at theta +- h e_j -> grad
 *
 * recbar [B][abcmb_bg_doubles(o)] device, float64, zeroed by the caller
 * before the first adjoint call; the adjoint calls add into it (atomically).
 * Without a plan each mode may take up to 65536 accepted steps (more sets
 * its status to ABCMB_E_MAX_STEPS); with one (abcmb_grad_plan) each mode's
 * tape is as long as a first pass found it needs.  Errors as abcmb_perturb: ABCMB_E_INVALID_ARG for bad
 * sizes, pointers or options (nothing launched), ABCMB_E_CUDA for a failed
 * launch; per-mode status in mode_status.
 */

/* Bytes of device workspace abcmb_perturb_taped and abcmb_perturb_adjoint
   need for B cosmologies x Nk modes without a plan (each mode's tape then
   holds 65536 accepted steps; checkpoints every 64 accepted steps, replay
   segment, work vectors); 0 for invalid arguments. */
size_t abcmb_grad_workspace_bytes(int B, int Nk, const abcmb_options *o);

/*
 * Sizing a gradient run to its modes (a plan).  A mode's tape length is its
 * number of accepted steps, which grows with k and with a tighter rtol; a
 * first pass counts them, and the tapes are then laid out back to back:
 *
 *   abcmb_grad_count_steps   the forward of abcmb_perturb_taped without the
 *                            tape: writes S, mode_status and accepted [B][Nk]
 *                            int32 (device); workspace >=
 *                            abcmb_grad_count_workspace_bytes(B, Nk, o) bytes,
 *                            256-byte aligned
 *   abcmb_grad_plan          host function: from accepted (copied to the host)
 *                            fills plan_host [2 B Nk + 2] (prefix sums of tape
 *                            steps and checkpoint states per mode) and returns
 *                            the workspace bytes the planned calls need (0 for
 *                            invalid arguments)
 *   abcmb_perturb_taped / abcmb_perturb_adjoint with plan_host: that plan (the
 *                            same array for both calls; the calls copy it into
 *                            the workspace, so it may be freed after each call
 *                            returns)
 *
 * The taped forward repeats the counting pass's arithmetic exactly, so each
 * mode records as many steps as were counted.
 */
size_t abcmb_grad_count_workspace_bytes(int B, int Nk, const abcmb_options *o);
int abcmb_grad_count_steps(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *S,
                           int *mode_status, int *accepted, void *workspace, size_t workspace_bytes, void *stream);
size_t abcmb_grad_plan(int B, int Nk, const abcmb_options *o, const int *accepted_host, long long *plan_host);

/*
 * Forward ODE of abcmb_perturb (one warp per mode), recording each mode's
 * accepted steps.
 *   bg, k, S, mode_status   as abcmb_perturb
 *   workspace  device, 256-byte aligned, owned by the caller: >=
 *              abcmb_grad_workspace_bytes(B, Nk, o) bytes when plan_host is
 *              NULL, else >= the bytes abcmb_grad_plan returned for plan_host;
 *              written here, read by abcmb_perturb_adjoint (keep it unchanged
 *              in between)
 *   plan_host  NULL (65536 accepted steps per mode; more sets the mode's status
 *              to ABCMB_E_MAX_STEPS) or a plan from abcmb_grad_plan (host)
 */
int abcmb_perturb_taped(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *S,
                        int *mode_status, void *workspace, size_t workspace_bytes, const long long *plan_host,
                        void *stream);

/*
 * Reverse sweep of the ODE: replays each mode's steps from its checkpoints
 * and pulls Sbar [B][Nk][n_tau][3] (device, read) back to recbar.  Modes
 * whose forward status was not ABCMB_OK contribute nothing.  workspace and
 * plan_host as given to abcmb_perturb_taped.
 */
int abcmb_perturb_adjoint(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                          const double *Sbar, void *workspace, size_t workspace_bytes, const long long *plan_host,
                          double *recbar, void *stream);

/*
 * Adjoint of abcmb_cl.
 *   Delta    [B][Nk][lmax_cl-1][2]  device, read (the forward's)
 *   Clbar    [B][3][lmax_cl-1]      device, read
 *   Deltabar [B][Nk][lmax_cl-1][2]  device, written
 *   recbar   device, entries ABCMB_S_AS and ABCMB_S_NS added to
 */
int abcmb_cl_adjoint(int B, const double *bg, const double *Delta, const double *k, int Nk,
                     const abcmb_options *o, const double *Clbar, double *Deltabar, double *recbar, void *stream);

/*
 * Adjoint of abcmb_project.
 *   S        [B][Nk][n_tau][3]      device, read (the forward's)
 *   Deltabar [B][Nk][lmax_cl-1][2]  device, read
 *   Sbar     [B][Nk][n_tau][3]      device, written
 *   recbar   device, node tau and weight entries and ABCMB_S_TAU0 added to
 */
int abcmb_project_adjoint(int B, const double *bg, const double *S, const double *k, int Nk,
                          const abcmb_options *o, const double *Deltabar, double *Sbar, double *recbar,
                          void *stream);

/*
 * The central-difference stencil of the background record's parameter
 * Jacobian: for each cosmology b and parameter j,
 *   h[b][j] = rel_step * max(|params[b][j]|, floor_abs),
 *   params_plus[b][j]  = params[b] + h[b][j] e_j,
 *   params_minus[b][j] = params[b] - h[b][j] e_j
 * (the rows abcmb_background_tables turns into rec_plus / rec_minus below).
 *   params                     [B][ABCMB_NPARAM]                 device, read
 *   h                          [B][ABCMB_NPARAM]                 device, written
 *   params_plus, params_minus  [B][ABCMB_NPARAM][ABCMB_NPARAM]   device, written
 * rel_step > 0 and floor_abs > 0, else ABCMB_E_INVALID_ARG.
 */
int abcmb_param_stencil(int B, const double *params, double rel_step, double floor_abs, double *h,
                        double *params_plus, double *params_minus, void *stream);

/*
 * grad[b][j] = sum_e recbar[b][e] (rec_plus[b][j][e] - rec_minus[b][j][e]) / (2 h[b][j])
 *   recbar            [B][len]                 device, read
 *   rec_plus/minus    [B][ABCMB_NPARAM][len]   device, read: background
 *                     records at params[b] +- h[b][j] e_j
 *   h                 [B][ABCMB_NPARAM]        device, read, nonzero
 *   grad              [B][ABCMB_NPARAM]        device, written
 */
int abcmb_record_vjp(int B, const abcmb_options *o, const double *recbar, const double *rec_plus,
                     const double *rec_minus, const double *h, double *grad, void *stream);

/*
 * Continuous-batching spectrum server.  A host runtime over the calls above
 * (no counterpart in the paper, which evaluates one cosmology per call):
 * requests of different lmax_cl and k-grid size queue on the host and are
 * admitted as soon as a stream slot is free and the caller's device arena
 * holds their buffers (abcmb_server_request_bytes per request: background
 * record, k, sources, FP32 transfer functions, C_l).  The request at the head
 * of the queue is admitted first, together with up to seven later requests of
 * the same lmax_cl and k grid (as many as the arena then holds): a slot runs
 * them as one batch of cosmologies, one k per warp across them, on its
 * stream -- background tables, FP64 perturbations, FP32 projection and
 * k-quadrature (abcmb_project_mixed / abcmb_cl_mixed), C_l copied back --
 * and slots in flight overlap on the GPU.  A request's result does not
 * depend on the others beyond the ODE tolerance (the integrator's switch
 * from implicit to explicit steps is taken per warp).
 *
 * The server object, its streams, events and pinned host staging buffers are
 * created by abcmb_server_create and released by abcmb_server_destroy; all
 * device memory comes from the caller's arena (256-byte aligned, owned by
 * the caller, outliving the server).  Not thread-safe: one host thread drives
 * a server.  Hierarchy truncations must be <= 63 (on-chip ODE state).
 *
 *   abcmb_server_create   n_slots in 1..256 streams; requests up to
 *                         max_lmax_cl and max_n_k; o gives the hierarchies,
 *                         n_tau, tolerances and switches of every request
 *   abcmb_server_submit   queue one request: params_host[6] (as
 *                         abcmb_background_tables), lmax_cl, n_k log-spaced
 *                         k in [k_min, k_max]; ABCMB_E_SCRATCH_TOO_SMALL if it
 *                         could never fit the arena
 *   abcmb_server_progress admit, launch and retire without blocking; returns
 *                         the number of requests in flight (all slots'
 *                         batches), or a negated error code
 *   abcmb_server_queued   requests waiting for admission
 *   abcmb_server_poll     pop one finished request: returns 1 (tag, status --
 *                         ABCMB_OK or the first failing status --, lmax_cl,
 *                         C_l [3][lmax_cl - 1] into cl_host), 0 if none is
 *                         ready, or a negated error code
 */
typedef struct abcmb_server abcmb_server;
size_t abcmb_server_request_bytes(const abcmb_options *o, int lmax_cl, int n_k);
int abcmb_server_create(void *arena, size_t arena_bytes, int n_slots, int max_lmax_cl, int max_n_k,
                        const abcmb_options *o, abcmb_server **out);
int abcmb_server_destroy(abcmb_server *s);
int abcmb_server_submit(abcmb_server *s, long long tag, const double *params_host, int lmax_cl, int n_k,
                        double k_min, double k_max);
int abcmb_server_progress(abcmb_server *s);
int abcmb_server_queued(const abcmb_server *s);
int abcmb_server_poll(abcmb_server *s, long long *tag, int *status, int *lmax_cl, double *cl_host,
                      size_t cl_capacity);

#ifdef __cplusplus
}
#endif

#endif /* ABCMB_H */
