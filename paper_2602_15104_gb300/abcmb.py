"""Thin Python binding of libabcmb.so (C ABI: include/abcmb.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels; torch supplies device memory and the current stream.  The
functions carry the C entry points' names.  If the library has not been built
(``__graft_entry__.build()`` or ``python -m paper_2602_15104_gb300.build``)
every call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libabcmb.so")

OK, E_INVALID_ARG, E_CUDA, E_MAX_STEPS, E_NONFINITE, E_BACKGROUND, E_SCRATCH_TOO_SMALL = range(7)
ERRORS = {1: "invalid argument", 2: "CUDA error", 3: "step budget exhausted",
          4: "non-finite value", 5: "background root not found",
          6: "problem larger than the library's static scratch"}
NOALLOC_SCRATCH_BYTES = 64 << 20

NPARAM = 6
BG_NSCALAR = 64
BG_PER_UNIT = 1024
BG_LNA0 = -18.0
BG_NLNA = 18 * 1024 + 1
BG_TABLE = BG_NSCALAR
BG_ODETAB = BG_TABLE + 8 * BG_NLNA
BG_NODES = BG_ODETAB + 20 * BG_NLNA
BG_ODEPOLY_DOUBLES = 40 * (BG_NLNA - 1)  # the ODE table as per-interval cubics, after the nodes
S_INDEX = dict(STATUS=0, H0=1, OMB=2, OMC=3, OMG=4, OMNU=5, OML=6, RNU=7, FHE=8, NH0=9, AS=10,
               NS=11, ZREION=12, LNA_TC=13, LNA_SW=14, TAU0=15, LNA_HE3=16, LNA_700=17, NTAU=18)
TABLE_COLUMNS = ("nuT", "dnuT", "tau", "dtau", "cs2", "dcs2", "kappa", "xe")
NODE_COLUMNS = ("lna", "tau", "w", "g", "dg", "expmk", "Hc", "dHc")


class Options(ctypes.Structure):
    """Mirror of abcmb_options."""

    _fields_ = [("lmax_g", ctypes.c_int), ("lmax_pol", ctypes.c_int), ("lmax_nu", ctypes.c_int),
                ("lmax_cl", ctypes.c_int), ("n_tau", ctypes.c_int), ("max_steps", ctypes.c_int),
                ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("scale_sw", ctypes.c_double), ("scale_isw", ctypes.c_double),
                ("scale_dop", ctypes.c_double), ("scale_pol", ctypes.c_double),
                ("m_ncdm", ctypes.c_double), ("lmax_ncdm", ctypes.c_int), ("node_recipe", ctypes.c_int),
                ("n_wide", ctypes.c_int), ("err_floor", ctypes.c_double)]


def options(lmax_hier=12, lmax_cl=2500, n_tau=6000, rtol=1e-6, atol=1e-12, max_steps=2_000_000,
            scale_sw=1.0, scale_isw=1.0, scale_dop=1.0, scale_pol=1.0, lmax_g=None, lmax_pol=None,
            lmax_nu=None, m_ncdm=0.0, lmax_ncdm=17, node_recipe=0, n_wide=0, err_floor=1e-4) -> Options:
    """m_ncdm > 0: one massive neutrino of that mass [eV] (two massless ones
    remain), its hierarchies to lmax_ncdm; abcmb_perturb then runs one warp
    per mode and needs a workspace.  node_recipe 1 places the tau nodes so
    that the tail of the visibility function is resolved (abcmb.h)."""
    o = Options()
    o.m_ncdm = float(m_ncdm)
    o.lmax_ncdm = int(lmax_ncdm) if m_ncdm > 0.0 else 0
    o.node_recipe = int(node_recipe)
    o.n_wide = int(n_wide)
    o.err_floor = float(err_floor)
    o.lmax_g = lmax_hier if lmax_g is None else lmax_g
    o.lmax_pol = lmax_hier if lmax_pol is None else lmax_pol
    o.lmax_nu = lmax_hier if lmax_nu is None else lmax_nu
    o.lmax_cl, o.n_tau, o.max_steps = lmax_cl, n_tau, max_steps
    o.rtol, o.atol = rtol, atol
    o.scale_sw, o.scale_isw, o.scale_dop, o.scale_pol = scale_sw, scale_isw, scale_dop, scale_pol
    return o


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libabcmb.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        O = ctypes.POINTER(Options)
        L.abcmb_default_options.argtypes = [O]
        L.abcmb_validate_options.argtypes = [O]
        L.abcmb_bg_doubles.argtypes = [O]
        L.abcmb_bg_doubles.restype = ctypes.c_size_t
        L.abcmb_perturb_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, O]
        L.abcmb_perturb_workspace_bytes.restype = ctypes.c_size_t
        L.abcmb_background_tables.argtypes = [ctypes.c_int, _P, O, _P, _P]
        L.abcmb_perturb.argtypes = [ctypes.c_int, _P, _P, ctypes.c_int, O, _P, _P, _P, _P,
                                    ctypes.c_size_t, _P]
        L.abcmb_perturb_noalloc.argtypes = [ctypes.c_int, _P, _P, ctypes.c_int, O, _P, _P, _P, _P]
        L.abcmb_matter_pk.argtypes = [ctypes.c_int, _P, _P, ctypes.c_int, O, ctypes.c_double, _P, _P, _P]
        L.abcmb_project.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, O, _P, _P]
        L.abcmb_project_interp.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, ctypes.c_int, O, _P, _P]
        L.abcmb_transfer_k_grid.argtypes = [ctypes.c_int, _P, ctypes.c_int]
        L.abcmb_lens.argtypes = [ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P, _P]
        L.abcmb_delta_m_nodes.argtypes = [ctypes.c_int, _P, _P, ctypes.c_int, O, _P, _P, _P]
        L.abcmb_cl_psi.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, O, ctypes.c_int, _P, _P]
        L.abcmb_cl.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, O, _P, _P]
        L.abcmb_project_mixed.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, O, _P, _P]
        L.abcmb_cl_mixed.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, O, _P, _P]
        L.abcmb_grad_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, O]
        L.abcmb_grad_workspace_bytes.restype = ctypes.c_size_t
        L.abcmb_perturb_taped.argtypes = [ctypes.c_int, _P, _P, ctypes.c_int, O, _P, _P, _P, ctypes.c_size_t, _P,
                                          _P]
        L.abcmb_perturb_adjoint.argtypes = [ctypes.c_int, _P, _P, ctypes.c_int, O, _P, _P, ctypes.c_size_t, _P,
                                            _P, _P]
        L.abcmb_grad_count_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, O]
        L.abcmb_grad_count_workspace_bytes.restype = ctypes.c_size_t
        L.abcmb_grad_count_steps.argtypes = [ctypes.c_int, _P, _P, ctypes.c_int, O, _P, _P, _P, _P, ctypes.c_size_t,
                                             _P]
        L.abcmb_grad_plan.argtypes = [ctypes.c_int, ctypes.c_int, O, _P, _P]
        L.abcmb_grad_plan.restype = ctypes.c_size_t
        L.abcmb_cl_adjoint.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, O, _P, _P, _P, _P]
        L.abcmb_project_adjoint.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, O, _P, _P, _P, _P]
        L.abcmb_record_vjp.argtypes = [ctypes.c_int, O, _P, _P, _P, _P, _P, _P]
        L.abcmb_param_stencil.argtypes = [ctypes.c_int, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P, _P]
        L.abcmb_server_request_bytes.argtypes = [O, ctypes.c_int, ctypes.c_int]
        L.abcmb_server_request_bytes.restype = ctypes.c_size_t
        L.abcmb_server_create.argtypes = [_P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, O,
                                          ctypes.POINTER(_P)]
        L.abcmb_server_destroy.argtypes = [_P]
        L.abcmb_server_submit.argtypes = [_P, ctypes.c_longlong, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double]
        L.abcmb_server_progress.argtypes = [_P]
        L.abcmb_server_queued.argtypes = [_P]
        L.abcmb_server_poll.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), _P, ctypes.c_size_t]
        _lib = L
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc, what):
    if rc != OK:
        raise RuntimeError(f"{what}: {ERRORS.get(rc, rc)}")


def _on_gpu(t):
    return isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()


def _dev(t, dtype=torch.float64):
    if not (_on_gpu(t) and t.dtype == dtype):
        raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
    return t


def _fits(t, n, what, dtype=torch.float64):
    """t as a buffer the library reads or writes n elements of through its
    pointer (the extent include/abcmb.h gives): a contiguous CUDA tensor of
    dtype with at least n elements, else the call is refused before it is
    made."""
    _dev(t, dtype)
    if t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the call needs {n}")
    return t


def _bytes(t, what):
    """A workspace of any dtype -> its size in bytes."""
    if not _on_gpu(t):
        raise TypeError(f"{what}: expected a contiguous CUDA tensor")
    return t.numel() * t.element_size()


def bg_doubles(o: Options) -> int:
    n = lib().abcmb_bg_doubles(ctypes.byref(o))
    if n == 0:
        raise ValueError("invalid options")
    return n


def perturb_workspace_bytes(B: int, Nk: int, o: Options) -> int:
    return lib().abcmb_perturb_workspace_bytes(B, Nk, ctypes.byref(o))


def abcmb_background_tables(params: torch.Tensor, o: Options, out: torch.Tensor | None = None):
    """params [B, 6] (omega_b, omega_cdm, h, n_s, ln(1e10 A_s), tau_reion) -> bg [B, bg_doubles]."""
    _dev(params)
    if params.dim() != 2 or params.shape[1] != NPARAM:
        raise ValueError(f"params: expected [B, {NPARAM}], got {list(params.shape)}")
    B, n = params.shape[0], bg_doubles(o)
    bg = out if out is not None else torch.empty((B, n), dtype=torch.float64, device=params.device)
    _fits(bg, B * n, "bg")
    _check(lib().abcmb_background_tables(B, _ptr(params), ctypes.byref(o), _ptr(bg), _stream()),
           "abcmb_background_tables")
    return bg


def abcmb_perturb(bg: torch.Tensor, k: torch.Tensor, o: Options, S=None, status=None, steps=None,
                  workspace=None):
    """-> S [B, Nk, n_tau, 3], mode status [B, Nk] int32, steps [B, Nk, 2] int32
    (steps taken, IMEX substeps)."""
    _dev(bg), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    dev = bg.device
    if S is None:
        S = torch.empty((B, Nk, o.n_tau, 3), dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty((B, Nk), dtype=torch.int32, device=dev)
    if steps is None:
        steps = torch.empty((B, Nk, 2), dtype=torch.int32, device=dev)
    _fits(S, B * Nk * o.n_tau * 3, "S")
    _fits(status, B * Nk, "mode_status", torch.int32)
    _fits(steps, B * Nk * 2, "steps", torch.int32)
    nbytes = perturb_workspace_bytes(B, Nk, o)
    if workspace is None and nbytes > 0:  # hierarchies > 63 and massive neutrinos
        workspace = torch.empty(nbytes // 8, dtype=torch.float64, device=dev)
    wbytes = 0 if workspace is None else _bytes(workspace, "workspace")
    _check(lib().abcmb_perturb(B, _ptr(bg), _ptr(k), Nk, ctypes.byref(o), _ptr(S), _ptr(status),
                               _ptr(steps), _ptr(workspace), wbytes, _stream()),
           "abcmb_perturb")
    return S, status, steps


def abcmb_perturb_noalloc(bg: torch.Tensor, k: torch.Tensor, o: Options, S, status, steps=None):
    """abcmb_perturb without a workspace, for callers that cannot allocate
    device memory: hierarchies > 63 keep their working vectors in the
    library's static scratch.  Outputs must be preallocated by the caller
    ([B, Nk, n_tau, 3], [B, Nk] and [B, Nk, 2] as abcmb_perturb; their
    sizes are not checked here, since a problem beyond the scratch is
    refused before they are touched); returns the C status code."""
    _dev(bg), _dev(k), _dev(S), _dev(status, torch.int32)
    if steps is not None:
        _dev(steps, torch.int32)
    B, Nk = bg.shape[0], k.shape[0]
    return lib().abcmb_perturb_noalloc(B, _ptr(bg), _ptr(k), Nk, ctypes.byref(o), _ptr(S), _ptr(status),
                                       _ptr(steps), _stream())


def abcmb_matter_pk(bg: torch.Tensor, k: torch.Tensor, o: Options, z: float = 0.0, out=None, status=None):
    """-> P(k, z) [B, Nk] in Mpc^3, mode status [B, Nk] int32."""
    _dev(bg), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    Pk = out if out is not None else torch.empty((B, Nk), dtype=torch.float64, device=bg.device)
    if status is None:
        status = torch.empty((B, Nk), dtype=torch.int32, device=bg.device)
    _fits(Pk, B * Nk, "Pk")
    _fits(status, B * Nk, "mode_status", torch.int32)
    _check(lib().abcmb_matter_pk(B, _ptr(bg), _ptr(k), Nk, ctypes.byref(o), float(z), _ptr(Pk), _ptr(status),
                                 _stream()),
           "abcmb_matter_pk")
    return Pk, status


def abcmb_project(bg: torch.Tensor, S: torch.Tensor, k: torch.Tensor, o: Options, out=None):
    """-> Delta [B, Nk, lmax_cl - 1, 2] (T, E) for l = 2..lmax_cl."""
    _dev(bg), _dev(S), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    _fits(S, B * Nk * o.n_tau * 3, "S")
    D = out if out is not None else torch.empty((B, Nk, o.lmax_cl - 1, 2), dtype=torch.float64,
                                                device=bg.device)
    _fits(D, B * Nk * (o.lmax_cl - 1) * 2, "Delta")
    _check(lib().abcmb_project(B, _ptr(bg), _ptr(S), _ptr(k), Nk, ctypes.byref(o), _ptr(D), _stream()),
           "abcmb_project")
    return D


def abcmb_project_interp(bg: torch.Tensor, S: torch.Tensor, k: torch.Tensor, kt: torch.Tensor, o: Options,
                         out=None):
    """Sources S at the ODE nodes k -> Delta [B, len(kt), lmax_cl - 1, 2] at kt."""
    _dev(bg), _dev(S), _dev(k), _dev(kt)
    B, Nk, Nkt = bg.shape[0], k.shape[0], kt.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    _fits(S, B * Nk * o.n_tau * 3, "S")
    D = out if out is not None else torch.empty((B, Nkt, o.lmax_cl - 1, 2), dtype=torch.float64,
                                                device=bg.device)
    _fits(D, B * Nkt * (o.lmax_cl - 1) * 2, "Delta")
    _check(lib().abcmb_project_interp(B, _ptr(bg), _ptr(S), _ptr(k), Nk, _ptr(kt), Nkt, ctypes.byref(o), _ptr(D),
                                      _stream()),
           "abcmb_project_interp")
    return D


def abcmb_lens(Cl: torch.Tensor, Cpsi: torch.Tensor, lmax_out: int, n_mu: int | None = None, out=None):
    """Cl [B, 3, L - 1] (TT, TE, EE for l = 2..L, as abcmb_cl writes them), Cpsi [B, L - 1] ->
    lensed [B, 4, lmax_out - 1] (TT, TE, EE, BB)."""
    _dev(Cl), _dev(Cpsi)
    if Cl.dim() != 3 or Cl.shape[1] != 3:
        raise ValueError(f"Cl: expected [B, 3, L - 1], got {list(Cl.shape)}")
    B, L = Cl.shape[0], Cl.shape[2] + 1
    _fits(Cpsi, B * (L - 1), "Cpsi")
    n_mu = n_mu or L + 100
    D = out if out is not None else torch.empty((B, 4, max(lmax_out - 1, 0)), dtype=torch.float64,
                                                device=Cl.device)
    _fits(D, B * 4 * max(lmax_out - 1, 0), "Cl_lensed")
    _check(lib().abcmb_lens(B, _ptr(Cl), L, _ptr(Cpsi), int(lmax_out), int(n_mu), _ptr(D), _stream()),
           "abcmb_lens")
    return D


def abcmb_delta_m_nodes(bg: torch.Tensor, k: torch.Tensor, o: Options, out=None, status=None):
    """-> (delta_m [B, Nk, n_tau] at the tau nodes, mode_status [B, Nk])."""
    _dev(bg), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    D = out if out is not None else torch.empty((B, Nk, o.n_tau), dtype=torch.float64, device=bg.device)
    st = status if status is not None else torch.empty((B, Nk), dtype=torch.int32, device=bg.device)
    _fits(D, B * Nk * o.n_tau, "Dm")
    _fits(st, B * Nk, "mode_status", torch.int32)
    _check(lib().abcmb_delta_m_nodes(B, _ptr(bg), _ptr(k), Nk, ctypes.byref(o), _ptr(D), _ptr(st), _stream()),
           "abcmb_delta_m_nodes")
    return D, st


def abcmb_cl_psi(bg: torch.Tensor, Dm: torch.Tensor, k: torch.Tensor, o: Options, lmax: int, out=None):
    """Limber C_l^psi [B, lmax - 1] for l = 2..lmax from delta_m at the nodes."""
    _dev(bg), _dev(Dm), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    _fits(Dm, B * Nk * o.n_tau, "Dm")
    C = out if out is not None else torch.empty((B, max(lmax - 1, 0)), dtype=torch.float64, device=bg.device)
    _fits(C, B * max(lmax - 1, 0), "Cpsi")
    _check(lib().abcmb_cl_psi(B, _ptr(bg), _ptr(Dm), _ptr(k), Nk, ctypes.byref(o), int(lmax), _ptr(C),
                              _stream()), "abcmb_cl_psi")
    return C


def transfer_k_grid(lmax_cl: int) -> np.ndarray:
    """The transfer-function k grid for lmax_cl (host)."""
    n = lib().abcmb_transfer_k_grid(int(lmax_cl), None, 0)
    if n < 0:
        raise ValueError("lmax_cl out of range")
    out = np.empty(n)
    lib().abcmb_transfer_k_grid(int(lmax_cl), out.ctypes.data_as(ctypes.c_void_p), n)
    return out


def abcmb_cl(bg: torch.Tensor, Delta: torch.Tensor, k: torch.Tensor, o: Options, out=None):
    """-> C_l [B, 3, lmax_cl - 1] (TT, TE, EE) for l = 2..lmax_cl."""
    _dev(bg), _dev(Delta), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    _fits(Delta, B * Nk * (o.lmax_cl - 1) * 2, "Delta")
    C = out if out is not None else torch.empty((B, 3, o.lmax_cl - 1), dtype=torch.float64,
                                                device=bg.device)
    _fits(C, B * 3 * (o.lmax_cl - 1), "Cl")
    _check(lib().abcmb_cl(B, _ptr(bg), _ptr(Delta), _ptr(k), Nk, ctypes.byref(o), _ptr(C), _stream()),
           "abcmb_cl")
    return C


def abcmb_project_mixed(bg: torch.Tensor, S: torch.Tensor, k: torch.Tensor, o: Options, out=None):
    """FP32 projection -> Delta32 [B, Nk, lmax_cl - 1, 2] float32 (T, E)."""
    _dev(bg), _dev(S), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    _fits(S, B * Nk * o.n_tau * 3, "S")
    D = out if out is not None else torch.empty((B, Nk, o.lmax_cl - 1, 2), dtype=torch.float32,
                                                device=bg.device)
    _fits(D, B * Nk * (o.lmax_cl - 1) * 2, "Delta32", torch.float32)
    _check(lib().abcmb_project_mixed(B, _ptr(bg), _ptr(S), _ptr(k), Nk, ctypes.byref(o), _ptr(D), _stream()),
           "abcmb_project_mixed")
    return D


def abcmb_cl_mixed(bg: torch.Tensor, Delta32: torch.Tensor, k: torch.Tensor, o: Options, out=None):
    """FP32 k-quadrature with Kahan sums -> C_l [B, 3, lmax_cl - 1] float64."""
    _dev(bg), _dev(Delta32, torch.float32), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    _fits(Delta32, B * Nk * (o.lmax_cl - 1) * 2, "Delta32", torch.float32)
    C = out if out is not None else torch.empty((B, 3, o.lmax_cl - 1), dtype=torch.float64,
                                                device=bg.device)
    _fits(C, B * 3 * (o.lmax_cl - 1), "Cl")
    _check(lib().abcmb_cl_mixed(B, _ptr(bg), _ptr(Delta32), _ptr(k), Nk, ctypes.byref(o), _ptr(C), _stream()),
           "abcmb_cl_mixed")
    return C


def grad_workspace_bytes(B: int, Nk: int, o: Options) -> int:
    n = lib().abcmb_grad_workspace_bytes(B, Nk, ctypes.byref(o))
    if n == 0:
        raise ValueError("invalid arguments")
    return n


def _plan_ptr(plan, B, Nk):
    if plan is None:
        return None
    if not (isinstance(plan, np.ndarray) and plan.dtype == np.int64 and plan.flags.c_contiguous):
        raise TypeError("plan: a contiguous int64 numpy array from grad_plan")
    if plan.size < 2 * B * Nk + 2:
        raise ValueError(f"plan: {plan.size} entries, a plan of {B} x {Nk} modes has {2 * B * Nk + 2}")
    return plan.ctypes.data_as(ctypes.c_void_p)


def abcmb_grad_count_steps(bg: torch.Tensor, k: torch.Tensor, o: Options, S=None, status=None):
    """First pass of a gradient run: the taped forward without the tape.
    -> S, mode status, accepted steps per mode [B, Nk] (device, int32)."""
    _dev(bg), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    dev = bg.device
    if S is None:
        S = torch.empty((B, Nk, o.n_tau, 3), dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty((B, Nk), dtype=torch.int32, device=dev)
    _fits(S, B * Nk * o.n_tau * 3, "S")
    _fits(status, B * Nk, "mode_status", torch.int32)
    acc = torch.empty((B, Nk), dtype=torch.int32, device=dev)
    nb = lib().abcmb_grad_count_workspace_bytes(B, Nk, ctypes.byref(o))
    if nb == 0:
        raise ValueError("invalid arguments")
    ws = torch.empty(nb // 8 + 1, dtype=torch.float64, device=dev)
    _check(lib().abcmb_grad_count_steps(B, _ptr(bg), _ptr(k), Nk, ctypes.byref(o), _ptr(S), _ptr(status), _ptr(acc),
                                        _ptr(ws), ws.numel() * 8, _stream()), "abcmb_grad_count_steps")
    return S, status, acc


def grad_plan(o: Options, accepted: torch.Tensor):
    """Host plan of per-mode tapes from the counted accepted steps [B, Nk]
    -> (plan int64 array, workspace bytes)."""
    acc = np.ascontiguousarray(accepted.detach().cpu().numpy(), dtype=np.int32)
    B, Nk = acc.shape
    plan = np.empty(2 * B * Nk + 2, dtype=np.int64)
    nb = lib().abcmb_grad_plan(B, Nk, ctypes.byref(o), acc.ctypes.data_as(ctypes.c_void_p),
                               plan.ctypes.data_as(ctypes.c_void_p))
    if nb == 0:
        raise ValueError("invalid arguments")
    return plan, nb


def abcmb_perturb_taped(bg: torch.Tensor, k: torch.Tensor, o: Options, workspace: torch.Tensor, S=None,
                        status=None, plan=None):
    """Forward ODE recording the tape for abcmb_perturb_adjoint in workspace
    (a CUDA tensor of >= grad_workspace_bytes bytes, or of the bytes
    grad_plan returned with plan).  -> S, mode status."""
    _dev(bg), _dev(k)
    B, Nk = bg.shape[0], k.shape[0]
    _fits(bg, B * bg_doubles(o), "bg")
    dev = bg.device
    if S is None:
        S = torch.empty((B, Nk, o.n_tau, 3), dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty((B, Nk), dtype=torch.int32, device=dev)
    _fits(S, B * Nk * o.n_tau * 3, "S")
    _fits(status, B * Nk, "mode_status", torch.int32)
    _check(lib().abcmb_perturb_taped(B, _ptr(bg), _ptr(k), Nk, ctypes.byref(o), _ptr(S), _ptr(status),
                                     _ptr(workspace), _bytes(workspace, "workspace"), _plan_ptr(plan, B, Nk),
                                     _stream()),
           "abcmb_perturb_taped")
    return S, status


def abcmb_perturb_adjoint(bg, k, o: Options, Sbar, workspace, recbar, plan=None):
    _dev(bg), _dev(k)
    B, Nk, n = bg.shape[0], k.shape[0], bg_doubles(o)
    _fits(bg, B * n, "bg"), _fits(Sbar, B * Nk * o.n_tau * 3, "Sbar"), _fits(recbar, B * n, "recbar")
    _check(lib().abcmb_perturb_adjoint(B, _ptr(bg), _ptr(k), Nk, ctypes.byref(o), _ptr(Sbar),
                                       _ptr(workspace), _bytes(workspace, "workspace"),
                                       _plan_ptr(plan, B, Nk), _ptr(recbar), _stream()),
           "abcmb_perturb_adjoint")
    return recbar


def abcmb_cl_adjoint(bg, Delta, k, o: Options, Clbar, recbar, Deltabar=None):
    _dev(bg), _dev(k)
    B, Nk, n = bg.shape[0], k.shape[0], bg_doubles(o)
    nD = B * Nk * (o.lmax_cl - 1) * 2
    _fits(bg, B * n, "bg"), _fits(Delta, nD, "Delta"), _fits(recbar, B * n, "recbar")
    _fits(Clbar, B * 3 * (o.lmax_cl - 1), "Clbar")
    if Deltabar is None:
        Deltabar = torch.empty_like(Delta)
    _fits(Deltabar, nD, "Deltabar")
    _check(lib().abcmb_cl_adjoint(B, _ptr(bg), _ptr(Delta), _ptr(k), Nk, ctypes.byref(o),
                                  _ptr(Clbar), _ptr(Deltabar), _ptr(recbar), _stream()),
           "abcmb_cl_adjoint")
    return Deltabar


def abcmb_project_adjoint(bg, S, k, o: Options, Deltabar, recbar, Sbar=None):
    _dev(bg), _dev(k)
    B, Nk, n = bg.shape[0], k.shape[0], bg_doubles(o)
    nS = B * Nk * o.n_tau * 3
    _fits(bg, B * n, "bg"), _fits(S, nS, "S"), _fits(recbar, B * n, "recbar")
    _fits(Deltabar, B * Nk * (o.lmax_cl - 1) * 2, "Deltabar")
    if Sbar is None:
        Sbar = torch.empty_like(S)
    _fits(Sbar, nS, "Sbar")
    _check(lib().abcmb_project_adjoint(B, _ptr(bg), _ptr(S), _ptr(k), Nk, ctypes.byref(o),
                                       _ptr(Deltabar), _ptr(Sbar), _ptr(recbar), _stream()),
           "abcmb_project_adjoint")
    return Sbar


def abcmb_param_stencil(params, rel_step: float, floor_abs: float):
    """-> h [B, 6], params_plus [B * 6, 6], params_minus [B * 6, 6] (abcmb.h)."""
    _dev(params)
    if params.dim() != 2 or params.shape[1] != NPARAM:
        raise ValueError(f"params: expected [B, {NPARAM}], got {list(params.shape)}")
    B = params.shape[0]
    h = torch.empty((B, NPARAM), dtype=torch.float64, device=params.device)
    pp = torch.empty((B * NPARAM, NPARAM), dtype=torch.float64, device=params.device)
    pm = torch.empty_like(pp)
    _check(lib().abcmb_param_stencil(B, _ptr(params), float(rel_step), float(floor_abs), _ptr(h), _ptr(pp),
                                     _ptr(pm), _stream()), "abcmb_param_stencil")
    return h, pp, pm


def abcmb_record_vjp(o: Options, recbar, rec_plus, rec_minus, h, grad=None):
    _dev(recbar)
    B, n = recbar.shape[0], bg_doubles(o)
    _fits(recbar, B * n, "recbar"), _fits(h, B * NPARAM, "h")
    _fits(rec_plus, B * NPARAM * n, "rec_plus"), _fits(rec_minus, B * NPARAM * n, "rec_minus")
    if grad is None:
        grad = torch.empty((B, NPARAM), dtype=torch.float64, device=recbar.device)
    _fits(grad, B * NPARAM, "grad")
    _check(lib().abcmb_record_vjp(B, ctypes.byref(o), _ptr(recbar), _ptr(rec_plus), _ptr(rec_minus), _ptr(h),
                                  _ptr(grad), _stream()),
           "abcmb_record_vjp")
    return grad


# relative step of the central differences that give the background record's
# parameter Jacobian (the record is smooth in the parameters: fixed-step
# thermal history, converged root finds), floor 1e-3 in absolute terms
FD_REL_STEP = 1e-4
FD_ABS_FLOOR = 1e-3


class ClWithGradient(torch.autograd.Function):
    """C_l [B, 3, lmax_cl - 1] (FP64 path) of params [B, 6], differentiable
    in params by the library's adjoint calls.  forward counts each mode's
    accepted steps (abcmb_grad_count_steps), sizes the tapes to them
    (abcmb_grad_plan) and runs the taped forward; backward runs
    abcmb_cl_adjoint, abcmb_project_adjoint and abcmb_perturb_adjoint (the
    tape of abcmb_perturb_taped), then contracts the adjoint of the
    background record with its parameter Jacobian (abcmb_record_vjp)."""

    @staticmethod
    def forward(ctx, params, k, o):
        _dev(params), _dev(k)
        bg = abcmb_background_tables(params, o)
        # first pass: count each mode's accepted steps, then size its tape
        S, status, acc = abcmb_grad_count_steps(bg, k, o)
        plan, nbytes = grad_plan(o, acc)
        ws = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device=params.device)
        S, status = abcmb_perturb_taped(bg, k, o, ws, S=S, status=status, plan=plan)
        D = abcmb_project(bg, S, k, o)
        C = abcmb_cl(bg, D, k, o)
        if bool((bg[:, S_INDEX["STATUS"]] != 0).any()) or bool((status != 0).any()):
            raise RuntimeError("forward pass failed (background or mode status set)")
        ctx.state = (params.detach(), k, o, bg, ws, plan, S, D)
        return C

    @staticmethod
    def backward(ctx, Cbar):
        params, k, o, bg, ws, plan, S, D = ctx.state
        recbar = torch.zeros_like(bg)
        Cbar = Cbar.contiguous().to(torch.float64)
        Dbar = abcmb_cl_adjoint(bg, D, k, o, Cbar, recbar)
        Sbar = abcmb_project_adjoint(bg, S, k, o, Dbar, recbar)
        abcmb_perturb_adjoint(bg, k, o, Sbar, ws, recbar, plan=plan)
        h, pp, pm = abcmb_param_stencil(params.contiguous(), FD_REL_STEP, FD_ABS_FLOOR)
        rp = abcmb_background_tables(pp, o)
        rm = abcmb_background_tables(pm, o)
        grad = abcmb_record_vjp(o, recbar, rp, rm, h)
        return grad, None, None


def cl_with_gradient(params: torch.Tensor, k: torch.Tensor, o: Options) -> torch.Tensor:
    """C_l of params with torch.autograd support (see ClWithGradient)."""
    return ClWithGradient.apply(params, k, o)


def server_request_bytes(o: Options, lmax_cl: int, n_k: int) -> int:
    return lib().abcmb_server_request_bytes(ctypes.byref(o), lmax_cl, n_k)


class Server:
    """Continuous-batching spectrum server (abcmb_server_*): requests of any
    lmax_cl / k-grid size queue here and run, overlapped on the GPU, as stream
    slots and arena memory free up.  The device arena is a torch tensor owned
    by this object."""

    def __init__(self, arena_bytes: int, n_slots: int, max_lmax_cl: int, max_n_k: int, o: Options,
                 device="cuda"):
        self.o = o
        self.max_lmax_cl = max_lmax_cl
        self.arena = torch.empty(arena_bytes // 8, dtype=torch.float64, device=device)
        h = ctypes.c_void_p()
        _check(lib().abcmb_server_create(_ptr(self.arena), self.arena.numel() * 8, n_slots, max_lmax_cl,
                                         max_n_k, ctypes.byref(o), ctypes.byref(h)), "abcmb_server_create")
        self._h = h
        self._buf = np.empty(3 * (max_lmax_cl - 1), dtype=np.float64)

    def submit(self, tag: int, params, lmax_cl: int, n_k: int, k_min: float, k_max: float) -> int:
        """Queue one cosmology (params: its 6 parameters, host) -> the C status code."""
        p = np.ascontiguousarray(params, dtype=np.float64)
        if p.size != NPARAM:
            raise ValueError(f"params: {NPARAM} values, got {p.size}")  # the library copies exactly 6
        return lib().abcmb_server_submit(self._h, tag, p.ctypes.data_as(ctypes.c_void_p), lmax_cl, n_k,
                                         k_min, k_max)

    def progress(self) -> int:
        n = lib().abcmb_server_progress(self._h)
        if n < 0:
            raise RuntimeError(f"abcmb_server_progress: {ERRORS.get(-n, -n)}")
        return n

    def queued(self) -> int:
        return lib().abcmb_server_queued(self._h)

    def poll(self):
        """-> (tag, status, C_l [3, lmax_cl - 1]) or None."""
        tag, st, lm = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        r = lib().abcmb_server_poll(self._h, ctypes.byref(tag), ctypes.byref(st), ctypes.byref(lm),
                                    self._buf.ctypes.data_as(ctypes.c_void_p), self._buf.size)
        if r < 0:
            raise RuntimeError(f"abcmb_server_poll: {ERRORS.get(-r, -r)}")
        if r == 0:
            return None
        n = lm.value - 1
        return tag.value, st.value, self._buf[:3 * n].reshape(3, n).copy()

    def close(self):
        if self._h:
            lib().abcmb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """Preallocated buffers for repeated whole-path calls of one shape."""

    def __init__(self, B: int, k, o: Options, device="cuda", mixed: bool = False):
        """mixed: FP32 projection and k-quadrature (abcmb_project_mixed /
        abcmb_cl_mixed) after the FP64 ODE."""
        self.o, self.B, self.mixed = o, B, mixed
        self.k = torch.as_tensor(np.asarray(k, dtype=np.float64), device=device).contiguous()
        Nk = self.k.shape[0]
        dev = self.k.device
        self.bg = torch.empty((B, bg_doubles(o)), dtype=torch.float64, device=dev)
        self.S = torch.empty((B, Nk, o.n_tau, 3), dtype=torch.float64, device=dev)
        self.status = torch.empty((B, Nk), dtype=torch.int32, device=dev)
        self.steps = torch.empty((B, Nk, 2), dtype=torch.int32, device=dev)
        nbytes = perturb_workspace_bytes(B, Nk, o)
        self.ws = torch.empty(nbytes // 8, dtype=torch.float64, device=dev) if nbytes else None
        self.D = torch.empty((B, Nk, o.lmax_cl - 1, 2), dtype=torch.float32 if mixed else torch.float64,
                             device=dev)
        self.C = torch.empty((B, 3, o.lmax_cl - 1), dtype=torch.float64, device=dev)
        self.params = torch.empty((B, NPARAM), dtype=torch.float64, device=dev)

    def run(self, params: torch.Tensor | None = None):
        """Whole path on device-resident params; returns the C_l tensor."""
        p = self.params if params is None else params
        abcmb_background_tables(p, self.o, out=self.bg)
        abcmb_perturb(self.bg, self.k, self.o, S=self.S, status=self.status, steps=self.steps,
                      workspace=self.ws)
        if self.mixed:
            abcmb_project_mixed(self.bg, self.S, self.k, self.o, out=self.D)
            abcmb_cl_mixed(self.bg, self.D, self.k, self.o, out=self.C)
        else:
            abcmb_project(self.bg, self.S, self.k, self.o, out=self.D)
            abcmb_cl(self.bg, self.D, self.k, self.o, out=self.C)
        return self.C

    def run_host(self, params_host: np.ndarray, cl_host: torch.Tensor | None = None):
        """End to end from host parameters (pinned copy in, C_l copy out into a
        pinned host tensor).  Asynchronous like every call here: synchronise
        the current stream before reading the returned tensor."""
        src = torch.from_numpy(np.ascontiguousarray(params_host, dtype=np.float64))
        if not src.is_pinned():
            src = src.pin_memory()
        self.params.copy_(src, non_blocking=True)
        C = self.run()
        out = cl_host if cl_host is not None else torch.empty(C.shape, dtype=C.dtype, pin_memory=True)
        out.copy_(C, non_blocking=True)
        return out

    def check_status(self):
        """Raise if any background or mode status word is set (syncs)."""
        bad_bg = (self.bg[:, S_INDEX["STATUS"]] != 0).nonzero()
        if bad_bg.numel():
            raise RuntimeError(f"background failed for cosmologies {bad_bg.flatten().tolist()}")
        bad = (self.status != 0).nonzero()
        if bad.numel():
            code = int(self.status[tuple(bad[0])])
            raise RuntimeError(f"{bad.shape[0]} modes failed, first {bad[0].tolist()}: {ERRORS.get(code)}")


def bg_view(bg_row: torch.Tensor, n_tau: int):
    """Split one background record (on any device) into scalars, the 8-column
    ln a table and the tau nodes (the ODE table between them is skipped)."""
    r = bg_row.detach().cpu().numpy()
    scal = {k: r[i] for k, i in S_INDEX.items()}
    tab = r[BG_TABLE:BG_ODETAB].reshape(BG_NLNA, 8)
    nodes = r[BG_NODES:BG_NODES + 8 * n_tau].reshape(n_tau, 8)
    return scal, tab, nodes
