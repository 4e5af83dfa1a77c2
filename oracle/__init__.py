"""ORACLE -- test infrastructure only.

A plain, slow FP64 CPU restatement of the ABCMB hot path (arXiv 2602.15104)
used to check the CUDA library.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference legs may import it; the library in
paper_2602_15104_gb300/ never does.  The C sources next to this file cite the
paper passage each step follows.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

HOOK_FREEZE_METRIC = 1
HOOK_NO_THOMSON = 2
HOOK_EDS_CDM = 4

BG_FIELDS = ("a", "Hc", "dHc", "fc", "fb", "fg", "fnu", "tau", "xe", "dxe",
             "nuT", "Rinv", "cs2", "kappa", "g", "dg", "fncdm", "wncdm")
SCALAR_FIELDS = ("H0", "Om_b", "Om_c", "Om_g", "Om_nu", "Om_L", "R_nu", "f_He",
                 "nH0", "A_s", "z_reion", "lna_tc", "lna_sw", "tau0", "lna_He3", "n_s", "Om_ncdm")

_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_scalars.argtypes = [_D, ctypes.c_int, ctypes.c_double, _D]
        L.orc_background.argtypes = [_D, ctypes.c_int, ctypes.c_double, _D, ctypes.c_int, _D]
        L.orc_nodes.argtypes = [_D, ctypes.c_int, ctypes.c_double, ctypes.c_int, _D]
        L.orc_nstate_of.argtypes = [_D]
        L.orc_lna_start_of.argtypes = [_D, ctypes.c_double, ctypes.c_double]
        L.orc_lna_start_of.restype = ctypes.c_double
        L.orc_trajectory.argtypes = [_D, _D, ctypes.c_double, _D, ctypes.c_int, _D, _D,
                                     ctypes.c_double, _L]
        L.orc_rhs_at.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        L.orc_bessel.argtypes = [ctypes.c_int, ctypes.c_double, _D]
        L.orc_project.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, _D, ctypes.c_int, _D,
                                  ctypes.c_int, ctypes.c_double, _D, ctypes.c_int]
        L.orc_cl.argtypes = [_D, ctypes.c_int, _D, ctypes.c_int, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, _D]
        L.orc_run.argtypes = [_D, ctypes.c_int, _D, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D,
                              _L, ctypes.c_int]
        L.orc_radau_tableau.argtypes = [_D]
        L.orc_pk.argtypes = [_D, _D, _D, ctypes.c_int, ctypes.c_double, _D, ctypes.c_int]
        L.orc_ncdm_density.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D]
        L.orc_delta_m_nodes.argtypes = [_D, ctypes.c_int, _D, _D, ctypes.c_int, _D, ctypes.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


_lib_cs = None
_V = ctypes.c_void_p


def lib_cs():
    """The oracle built over double complex (orc_real.h): complex-step forward
    sensitivities."""
    global _lib_cs
    if _lib_cs is None:
        L = ctypes.CDLL(_build.build_cs())
        L.orc_run.argtypes = [_V, ctypes.c_int, _D, _V, ctypes.c_int, ctypes.c_int, _V, _V, _V, _L, ctypes.c_int]
        L.orc_scalars.argtypes = [_V, ctypes.c_int, ctypes.c_double, _V]
        L.orc_nodes.argtypes = [_V, ctypes.c_int, ctypes.c_double, ctypes.c_int, _V]
        L.orc_background.argtypes = [_V, ctypes.c_int, ctypes.c_double, _V, ctypes.c_int, _V]
        _lib_cs = L
    return _lib_cs


CS_STEP = 1e-20  # imaginary step: the O(h^2) term is ~1e-40 of the value


def _cs_params(params, j):
    p = np.ascontiguousarray(np.asarray(params, dtype=np.complex128))
    p[j] += 1j * CS_STEP
    return p


def _cv(a):
    return a.ctypes.data_as(_V) if a is not None else None


def _arr(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def opts(lmax=12, lmax_g=None, lmax_pol=None, lmax_nu=None, scale_sw=1.0, scale_isw=1.0,
         scale_dop=1.0, scale_pol=1.0, step_c=0.05, step_cap=0.05, hooks=0, max_steps=0,
         m_ncdm=0.0, lmax_ncdm=17, node_recipe=0):
    """Options vector: hierarchy truncations, source switches (App. A.1), the
    step schedule of the oracle's integrator, test hooks, and one massive
    neutrino of mass m_ncdm [eV] with hierarchies to lmax_ncdm (m_ncdm = 0:
    three massless neutrinos only), and the tau-node recipe (0 the default
    placement, 1 the refined tail)."""
    lg = lmax if lmax_g is None else lmax_g
    lp = lmax if lmax_pol is None else lmax_pol
    ln = lmax if lmax_nu is None else lmax_nu
    lm = lmax_ncdm if m_ncdm > 0.0 else 0
    return np.array([lg, lp, ln, scale_sw, scale_isw, scale_dop, scale_pol, step_c, step_cap,
                     hooks, max_steps, lm, m_ncdm, node_recipe], dtype=np.float64)


def nstate(o):
    return lib().orc_nstate_of(_p(_arr(o)))


def scalars(params, hooks=0, m_ncdm=0.0):
    out = np.zeros(17)
    rc = lib().orc_scalars(_p(_arr(params)), hooks, float(m_ncdm), _p(out))
    if rc:
        raise RuntimeError("oracle background failed")
    return dict(zip(SCALAR_FIELDS, out))


def background(params, lna, hooks=0, m_ncdm=0.0):
    lna = _arr(np.atleast_1d(lna))
    out = np.zeros((lna.size, 18))
    rc = lib().orc_background(_p(_arr(params)), hooks, float(m_ncdm), _p(lna), lna.size, _p(out))
    if rc:
        raise RuntimeError("oracle background failed")
    return {f: out[:, i] for i, f in enumerate(BG_FIELDS)}


def thermo(params, lna):
    """Thermal history at ln a: dict of T_m [eV], dlnTm (d ln T_m / d ln a),
    x_e and the baryon sound speed squared cs2 (App. B.1.2, App. C.3)."""
    lna = _arr(np.atleast_1d(lna))
    out = np.zeros((lna.size, 4))
    L = lib()
    L.orc_thermo.argtypes = [_D, _D, ctypes.c_int, _D]
    if L.orc_thermo(_p(_arr(params)), _p(lna), lna.size, _p(out)):
        raise RuntimeError("oracle background failed")
    return dict(Tm=out[:, 0], dlnTm=out[:, 1], xe=out[:, 2], cs2=out[:, 3])


def alpha_B(T_eV):
    """The Peebles atom's case-B recombination coefficient [cm^3/s] at T [eV]."""
    L = lib()
    L.orc_alpha_B_at.argtypes = [ctypes.c_double]
    L.orc_alpha_B_at.restype = ctypes.c_double
    return L.orc_alpha_B_at(float(T_eV))


def nodes(params, n_tau, m_ncdm=0.0, node_recipe=0):
    out = np.zeros((3, n_tau))
    if lib().orc_nodes(_p(_arr(params)), n_tau, float(m_ncdm), int(node_recipe), _p(out)):
        raise RuntimeError("oracle nodes failed")
    return out[0], out[1], out[2]


def lna_start(params, k, m_ncdm=0.0):
    return lib().orc_lna_start_of(_p(_arr(params)), float(k), float(m_ncdm))


def trajectory(params, o, k, lna_out, y_init=None, lna_init=0.0):
    o = _arr(o)
    lna_out = _arr(lna_out)
    n = nstate(o)
    y = np.zeros((lna_out.size, n))
    steps = ctypes.c_long(0)
    yi = _arr(y_init) if y_init is not None else None
    rc = lib().orc_trajectory(_p(_arr(params)), _p(o), float(k), _p(lna_out), lna_out.size,
                              _p(y), _p(yi), float(lna_init), ctypes.byref(steps))
    if rc:
        raise RuntimeError("oracle trajectory failed")
    return y, steps.value


def rhs(params, o, k, lna, y):
    o = _arr(o)
    dy = np.zeros(nstate(o))
    lib().orc_rhs_at(_p(_arr(params)), _p(o), float(k), float(lna), _p(_arr(y)), _p(dy))
    return dy


def bessel(lmax, x):
    out = np.zeros(lmax + 1)
    lib().orc_bessel(int(lmax), float(x), _p(out))
    return out


def project(tau, w, tau0, k, S, lmax, scale_pol=1.0, nthreads=0):
    tau, w, k, S = _arr(tau), _arr(w), _arr(k), _arr(S)
    D = np.zeros((k.size, lmax - 1, 2))
    lib().orc_project(tau.size, _p(tau), _p(w), float(tau0), _p(k), k.size, _p(S), int(lmax),
                      float(scale_pol), _p(D), int(nthreads))
    return D


def cl(k, Delta, lmax, A_s, n_s, k_pivot=0.05):
    k, Delta = _arr(k), _arr(Delta)
    out = np.zeros((3, lmax - 1))
    lib().orc_cl(_p(k), k.size, _p(Delta), int(lmax), float(A_s), float(n_s), float(k_pivot),
                 _p(out))
    return out


def radau_tableau():
    out = np.zeros(12)
    lib().orc_radau_tableau(_p(out))
    return out[:9].reshape(3, 3), out[9:]


def run(params, k, n_tau, lmax_cl, o, want=("S", "Delta", "Cl"), nthreads=0):
    """Whole path for one cosmology; returns a dict with the requested arrays
    plus per-mode step counts."""
    k = _arr(k)
    o = _arr(o)
    nk = k.size
    S = np.zeros((nk, n_tau, 3)) if "S" in want else None
    D = np.zeros((nk, lmax_cl - 1, 2)) if "Delta" in want else None
    C = np.zeros((3, lmax_cl - 1)) if "Cl" in want else None
    steps = np.zeros(nk, dtype=np.int64)
    rc = lib().orc_run(_p(_arr(params)), int(n_tau), _p(o), _p(k), nk, int(lmax_cl), _p(S),
                       _p(D), _p(C), steps.ctypes.data_as(_L), int(nthreads))
    if rc:
        raise RuntimeError(f"oracle run failed ({rc})")
    return {"S": S, "Delta": D, "Cl": C, "steps": steps}


def sensitivity(params, j, k, n_tau, lmax_cl, o, want=("Cl",), nthreads=0):
    """Forward sensitivity of the whole path to parameter j (0..5: omega_b,
    omega_cdm, h, n_s, ln 10^10 A_s, tau_reio) by the complex step: returns
    {name: (value, d value / d theta_j)} for the requested arrays, exact to
    rounding (no difference quotient; orc_real.h)."""
    k = np.ascontiguousarray(np.asarray(k, dtype=np.complex128))
    o = _arr(o)
    nk = k.size
    S = np.zeros((nk, n_tau, 3), dtype=np.complex128) if "S" in want else None
    D = np.zeros((nk, lmax_cl - 1, 2), dtype=np.complex128) if "Delta" in want else None
    C = np.zeros((3, lmax_cl - 1), dtype=np.complex128) if "Cl" in want else None
    steps = np.zeros(nk, dtype=np.int64)
    rc = lib_cs().orc_run(_cv(_cs_params(params, j)), int(n_tau), _p(o), _cv(k), nk, int(lmax_cl), _cv(S),
                          _cv(D), _cv(C), steps.ctypes.data_as(_L), int(nthreads))
    if rc:
        raise RuntimeError(f"oracle run failed ({rc})")
    out = {}
    for name, a in (("S", S), ("Delta", D), ("Cl", C)):
        if a is not None:
            out[name] = (a.real.copy(), a.imag / CS_STEP)
    return out


def scalars_sensitivity(params, j, m_ncdm=0.0):
    """Derived scalars (SCALAR_FIELDS) and their derivatives by theta_j."""
    out = np.zeros(17, dtype=np.complex128)
    if lib_cs().orc_scalars(_cv(_cs_params(params, j)), 0, float(m_ncdm), _cv(out)):
        raise RuntimeError("oracle background failed")
    return {f: (v.real, v.imag / CS_STEP) for f, v in zip(SCALAR_FIELDS, out)}


def nodes_sensitivity(params, j, n_tau, node_recipe=0):
    """tau nodes (ln a, tau, w) and their derivatives by theta_j."""
    out = np.zeros((3, n_tau), dtype=np.complex128)
    if lib_cs().orc_nodes(_cv(_cs_params(params, j)), n_tau, 0.0, int(node_recipe), _cv(out)):
        raise RuntimeError("oracle nodes failed")
    return out.real.copy(), out.imag / CS_STEP


def background_sensitivity(params, j, lna):
    """Background fields (BG_FIELDS) at fixed ln a and their derivatives by theta_j."""
    lna = np.ascontiguousarray(np.atleast_1d(lna).astype(np.complex128))
    out = np.zeros((lna.size, 18), dtype=np.complex128)
    if lib_cs().orc_background(_cv(_cs_params(params, j)), 0, 0.0, _cv(lna), lna.size, _cv(out)):
        raise RuntimeError("oracle background failed")
    return {f: (out[:, i].real.copy(), out[:, i].imag / CS_STEP) for i, f in enumerate(BG_FIELDS)}


def ncdm_density(params, m_ncdm, a):
    """One massive neutrino: (rho, p) / rho_crit today at scale factor a, its
    relativistic-limit Omega (rho a^4 / rho_crit as a -> 0) and m / T_ncdm."""
    out = np.zeros(5)
    if lib().orc_ncdm_density(_p(_arr(params)), float(m_ncdm), float(a), _p(out)):
        raise RuntimeError("oracle background failed")
    return dict(rho=out[0], p=out[1], Om_rel=out[2], x1=out[3])


def delta_m_nodes(params, k, n_tau, o, nthreads=0):
    """delta_m(k, tau_i) [n_k, n_tau]: the density-weighted CDM + baryon (+ massive
    neutrino) contrast at every tau node."""
    k = _arr(k)
    out = np.zeros((k.size, n_tau))
    rc = lib().orc_delta_m_nodes(_p(_arr(params)), int(n_tau), _p(_arr(o)), _p(k), k.size, _p(out), int(nthreads))
    if rc:
        raise RuntimeError(f"oracle delta_m failed ({rc})")
    return out


def pk(params, k, z, o, nthreads=0):
    """Matter power spectrum P(k, z) [Mpc^3] (App. B.4 eq. PK) of one cosmology."""
    k = _arr(k)
    out = np.zeros(k.size)
    rc = lib().orc_pk(_p(_arr(params)), _p(_arr(o)), _p(k), k.size, float(z), _p(out), int(nthreads))
    if rc:
        raise RuntimeError(f"oracle P(k) failed ({rc})")
    return out


# Transfer-function k grid (App. A.1, eq. k_transfer_spacing and eq. defkperiod)
# with the paper's default parameters.
TRANSFER_GRID = dict(tau0_fid=1.418668e4, tau_rec_fid=281.040565, linstep=0.45, logstep=170.0,
                     kmin_tau0=0.1, kmax_tau0_over_lmax=1.8)


def transfer_k_grid(lmax_cl, tau0_fid=1.418668e4, tau_rec_fid=281.040565, linstep=0.45, logstep=170.0,
                    kmin_tau0=0.1, kmax_tau0_over_lmax=1.8):
    """k~ nodes from k_min = kmin_tau0 / tau0_fid up to the last node not above
    k_max = kmax_tau0_over_lmax * lmax_cl / tau0_fid (reading of eq. kmax_grid:
    k_max tau0 / lmax = 1.8), each step
    k_{n+1} = k_n + k_period linstep k_n / (k_n + linstep / logstep),
    k_period = 2 pi / (tau0_fid - tau_rec_fid)."""
    kp = 2.0 * np.pi / (tau0_fid - tau_rec_fid)
    k = kmin_tau0 / tau0_fid
    kmax = kmax_tau0_over_lmax * lmax_cl / tau0_fid
    out = []
    while k <= kmax:
        out.append(k)
        k = k + kp * linstep * k / (k + linstep / logstep)
    return np.array(out)


def interp_sources(S, k, kt):
    """Sources S[..., n_k, n_tau, 3] on the ascending nodes k, interpolated in
    ln k onto kt (within [k_0, k_last]) by piecewise cubic Hermite
    polynomials whose slopes at the nodes are the three-point derivatives
    (centred, one-sided at the ends) -- exact for quadratics in ln k.  The
    paper interpolates the sources onto its transfer grid without naming the
    scheme; this is the reading taken."""
    S = np.asarray(S, dtype=np.float64)
    x = np.log(np.asarray(k, dtype=np.float64))
    xt = np.log(np.asarray(kt, dtype=np.float64))
    n = x.size
    ax = S.ndim - 3  # the k axis
    Sk = np.moveaxis(S, ax, 0)
    slope = np.empty_like(Sk)
    for i in range(n):
        if i == 0:
            a, b, c = 0, 1, 2
        elif i == n - 1:
            a, b, c = n - 3, n - 2, n - 1
        else:
            a, b, c = i - 1, i, i + 1
        # derivative at x_i of the parabola through (x_a, x_b, x_c)
        xa, xb, xc, xi = x[a], x[b], x[c], x[i]
        la = ((xi - xb) + (xi - xc)) / ((xa - xb) * (xa - xc))
        lb = ((xi - xa) + (xi - xc)) / ((xb - xa) * (xb - xc))
        lc = ((xi - xa) + (xi - xb)) / ((xc - xa) * (xc - xb))
        slope[i] = la * Sk[a] + lb * Sk[b] + lc * Sk[c]
    out = np.empty((xt.size,) + Sk.shape[1:])
    for j, xv in enumerate(xt):
        i = min(max(np.searchsorted(x, xv, side="right") - 1, 0), n - 2)
        h = x[i + 1] - x[i]
        t = (xv - x[i]) / h
        h00, h10 = (1 + 2 * t) * (1 - t) ** 2, t * (1 - t) ** 2
        h01, h11 = t * t * (3 - 2 * t), t * t * (t - 1)
        out[j] = h00 * Sk[i] + h10 * h * slope[i] + h01 * Sk[i + 1] + h11 * h * slope[i + 1]
    return np.moveaxis(out, 0, ax)


class Cosmo:
    """Handle on one oracle cosmology (background built once)."""

    def __init__(self, params, n_tau=0, hooks=0, m_ncdm=0.0):
        L = lib()
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_h_rhs.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        L.orc_h_matrix.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_double, _D]
        self._h = L.orc_create(_p(_arr(params)), int(n_tau), int(hooks), float(m_ncdm))
        if not self._h:
            raise RuntimeError("oracle background failed")

    def rhs(self, o, k, lna, y):
        o = _arr(o)
        dy = np.zeros(nstate(o))
        lib().orc_h_rhs(self._h, _p(o), float(k), float(lna), _p(_arr(y)), _p(dy))
        return dy

    def matrix(self, o, k, lna):
        o = _arr(o)
        n = nstate(o)
        A = np.zeros((n, n))
        lib().orc_h_matrix(self._h, _p(o), float(k), float(lna), _p(A))
        return A

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None


def dense_solve(A, b):
    A = _arr(A).copy()
    b = _arr(b).copy()
    L = lib()
    L.orc_dense_solve.argtypes = [_D, ctypes.c_int, _D]
    if L.orc_dense_solve(_p(A), b.size, _p(b)):
        raise RuntimeError("singular")
    return b


def count_steps(params, k, n_tau, o):
    """Radau steps the oracle's fixed schedule takes per k mode (no solve)."""
    k = _arr(k)
    out = np.zeros(k.size, dtype=np.int64)
    L = lib()
    L.orc_count_steps.argtypes = [_D, ctypes.c_int, _D, _D, ctypes.c_int, _L]
    if L.orc_count_steps(_p(_arr(params)), int(n_tau), _p(_arr(o)), _p(k), k.size, out.ctypes.data_as(_L)):
        raise RuntimeError("oracle background failed")
    return out
