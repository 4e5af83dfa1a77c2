"""CPU checks of the projection and k-quadrature adjoint kernels
(abcmb_grad.cuh: project_adjoint_kernel and cl_adjoint_kernel, behind
abcmb_project_adjoint and abcmb_cl_adjoint), built for the host with every
CTA's threads run as host threads (tests/host/warp_emu.h), beside the forward
kernels built the same way (abcmb_spectra.cuh):

  * Sbar is the exact transpose of the projection, which is linear in S:
    <Dbar, P S> = <P^T Dbar, S>;
  * the node-weight adjoints satisfy Euler's identity for a map linear in
    the weights, sum_i w_i wbar_i = <Dbar, P S>;
  * the node-position and tau_0 adjoints equal Richardson differences of the
    oracle's exact-Bessel projection (App. B.4 transfer functions), and sum
    to zero (only tau_0 - tau_i enters);
  * Deltabar is the derivative of <Cbar, C> (App. B.4 eq. c_ell_def, quadratic
    in Delta: central differences are exact), and the A_s and n_s adjoints
    match differences of the forward quadrature;
  * the ODE passes over a batch of modes (taped_kernel, adjoint_kernel) in
    a workspace laid out from the library's own step-count plan
    (abcmb_grad_plan) reproduce the per-mode one-lane build: the counted
    steps, the sources bit for bit, and each cosmology's record adjoint as
    the sum of its modes'.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2602_15104_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
D = ctypes.c_double
I = ctypes.c_int
NODES = 64 + 28 * (18 * 1024 + 1)  # ABCMB_BG_NODES
S_AS, S_NS, S_TAU0 = 10, 11, 15  # ABCMB_S_AS, ABCMB_S_NS, ABCMB_S_TAU0
N_TAU, LMAX = 600, 400
K = np.array([3e-4, 0.004, 0.05, 0.15])


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("gradk") / "libgradk.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "grad_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_build_bg.argtypes = [P, I, P]
    L.h_project.argtypes = [I, P, P, P, I, I, D, P]
    L.h_cl.argtypes = [I, P, P, P, I, I, P]
    L.h_project_adjoint.argtypes = [I, P, P, P, I, I, D, P, P, P]
    L.h_cl_adjoint.argtypes = [I, P, P, P, I, I, P, P, P]
    L.h_record_vjp.argtypes = [I, ctypes.c_long, P, P, P, P, P]
    return L


def ptr(a):
    return a.ctypes.data_as(P)


@pytest.fixture(scope="module")
def case(H):
    p = W.BATCH64.params()[7]
    bg = np.zeros((1, H.h_bg_len(N_TAU)))
    H.h_build_bg(ptr(p), N_TAU, ptr(bg))
    S = W.synthetic_sources(K.size, N_TAU, 5)[None]
    Db = np.random.default_rng(1).normal(size=(1, K.size, LMAX - 1, 2))
    Sb, rb = np.zeros_like(S), np.zeros_like(bg)
    H.h_project_adjoint(1, ptr(bg), ptr(S), ptr(K), K.size, LMAX, 1.0, ptr(Db), ptr(Sb), ptr(rb))
    return dict(p=p, bg=bg, S=S, Db=Db, Sb=Sb, rb=rb)


def project(H, bg, S):
    Dl = np.zeros((1, K.size, LMAX - 1, 2))
    H.h_project(1, ptr(bg), ptr(S), ptr(K), K.size, LMAX, 1.0, ptr(Dl))
    return Dl


def richardson(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
    return (4 * d1 - d2) / 3


def test_projection_adjoint_is_the_transpose(H, case):
    bg, S, Db, Sb, rb = case["bg"], case["S"], case["Db"], case["Sb"], case["rb"]
    L0 = np.sum(Db * project(H, bg, S))
    assert abs(np.sum(Sb * S) / L0 - 1) < 1e-13
    w = bg[0, NODES + 2:NODES + 8 * N_TAU:8]
    wb = rb[0, NODES + 2:NODES + 8 * N_TAU:8]
    assert abs(np.sum(w * wb) / L0 - 1) < 1e-13
    taub = rb[0, NODES + 1:NODES + 8 * N_TAU:8]
    assert abs(taub.sum() + rb[0, S_TAU0]) < 1e-12 * abs(rb[0, S_TAU0])


def test_node_position_adjoints_against_oracle_differences(case):
    # measured 4e-11 (tau_0) and <= 3e-9 of the largest node adjoint
    p, S, Db, rb = case["p"], case["S"], case["Db"], case["rb"]
    lna, tau, w = O.nodes(p, N_TAU)
    t0 = O.scalars(p)["tau0"]

    def L(tau_, t0_):
        return np.sum(Db[0] * O.project(tau_, w, t0_, K, S[0], LMAX))

    g0 = richardson(lambda e: L(tau, t0 + e), 1e-2)
    assert abs(rb[0, S_TAU0] / g0 - 1) < 1e-8
    taub = rb[0, NODES + 1:NODES + 8 * N_TAU:8]
    for i in (150, 300, 420, 590):
        def f(e, i=i):
            tt = tau.copy()
            tt[i] += e
            return L(tt, t0)
        assert abs(taub[i] - richardson(f, 1e-2)) < 1e-7 * np.abs(taub).max(), i


def test_quadrature_adjoint(H, case):
    bg = case["bg"]
    Dl = project(H, bg, case["S"])
    rng = np.random.default_rng(2)
    Cb = rng.normal(size=(1, 3, LMAX - 1))

    def L(bg_, D_):
        C = np.zeros((1, 3, LMAX - 1))
        H.h_cl(1, ptr(bg_), ptr(D_), ptr(K), K.size, LMAX, ptr(C))
        return np.sum(Cb * C)

    Dbar, rb = np.zeros_like(Dl), np.zeros_like(bg)
    H.h_cl_adjoint(1, ptr(bg), ptr(Dl), ptr(K), K.size, LMAX, ptr(Cb), ptr(Dbar), ptr(rb))
    V = rng.normal(size=Dl.shape)
    fd = (L(bg, Dl + 1e-3 * V) - L(bg, Dl - 1e-3 * V)) / 2e-3  # exact for a quadratic
    assert abs(np.sum(Dbar * V) / fd - 1) < 1e-10  # measured 6e-13
    for idx in (S_AS, S_NS):
        h = 1e-5 * abs(bg[0, idx])

        def f(e, idx=idx):
            b2 = bg.copy()
            b2[0, idx] += e
            return L(b2, Dl)
        assert abs(rb[0, idx] / richardson(f, h) - 1) < 1e-8, idx


@pytest.fixture(scope="module")
def one_lane(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("adjone") / "libadjone.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "adjoint_mode_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_fwd.argtypes = [P, D, I, D, P, P]
    L.h_grad.argtypes = [P, D, I, D, P, P]
    return L


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="the library's host functions need nvcc to build")
def test_planned_batch_of_modes_matches_the_per_mode_adjoint(H, one_lane):
    from paper_2602_15104_gb300 import abcmb as A
    from paper_2602_15104_gb300 import build
    build.build()
    lib = A.lib()  # host functions only: the workspace sizes and the tape plan
    H.h_taped.argtypes = [I, P, P, I, I, D, D, I, P, P, P, P, P]
    H.h_adjoint.argtypes = [I, P, P, I, I, P, P, P, P]
    B, L, n_tau, rtol = 2, 8, 120, 1e-5
    k = np.array([0.02, 0.05])
    params = W.BATCH64.params()[[0, 9]]
    o = A.options(lmax_hier=L, n_tau=n_tau, lmax_cl=40, rtol=rtol, atol=1e-14)
    n = one_lane.h_bg_len(n_tau)
    bg = np.zeros((B, n))
    for b in range(B):
        one_lane.h_build_bg(ptr(np.ascontiguousarray(params[b])), n_tau, ptr(bg[b]))
    S = np.zeros((B, k.size, n_tau, 3))
    st = np.full((B, k.size), -1, np.int32)
    acc = np.zeros((B, k.size), np.int32)
    ws = np.zeros(lib.abcmb_grad_count_workspace_bytes(B, k.size, ctypes.byref(o)) // 8 + 1)
    H.h_taped(B, ptr(bg), ptr(k), k.size, L, rtol, 1e-14, 10_000_000, ptr(S), ptr(st), ptr(ws), None, ptr(acc))
    assert np.all(st == 0)
    plan = np.zeros(2 * B * k.size + 2, np.int64)
    nbytes = lib.abcmb_grad_plan(B, k.size, ctypes.byref(o), ptr(acc), ptr(plan))
    assert nbytes > 0
    ws = np.zeros(nbytes // 8 + 1)
    S2 = np.zeros_like(S)
    H.h_taped(B, ptr(bg), ptr(k), k.size, L, rtol, 1e-14, 10_000_000, ptr(S2), ptr(st), ptr(ws), ptr(plan), None)
    assert np.all(st == 0)
    np.testing.assert_array_equal(S2, S)
    Sb = np.random.default_rng(4).normal(size=S.shape) / np.abs(S).max()
    rb = np.zeros_like(bg)
    H.h_adjoint(B, ptr(bg), ptr(k), k.size, L, ptr(Sb), ptr(ws), ptr(plan), ptr(rb))
    for b in range(B):
        ref = np.zeros(n)
        for i in range(k.size):
            S1, sig, g = np.zeros((n_tau, 3)), np.zeros(3, np.int32), np.zeros(n)
            assert one_lane.h_fwd(ptr(bg[b]), k[i], L, rtol, ptr(S1), ptr(sig)) == 0
            assert sig[0] == acc[b, i]
            np.testing.assert_array_equal(S[b, i], S1)
            assert one_lane.h_grad(ptr(bg[b]), k[i], L, rtol, ptr(np.ascontiguousarray(Sb[b, i])), ptr(g)) == 0
            ref += g
        # measured 3e-17 of the largest entry
        assert np.abs(rb[b] - ref).max() <= 1e-12 * np.abs(ref).max(), b


@pytest.fixture(scope="module")
def ncdm_lane(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("ncdmone") / "libncdmone.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "ncdm_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_bg_len.restype = ctypes.c_long
    L.h_build_bg_m.argtypes = [P, I, D, P]
    L.h_fwd_m.argtypes = [P, D, I, I, D, P]
    return L


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="the library's host functions need nvcc to build")
def test_massive_neutrino_warps_equal_the_one_lane_forward(H, ncdm_lane):
    # plain_kernel, the massive-neutrino path of abcmb_perturb: its momentum-
    # bin sums split over the lanes; the one-lane build is held against the
    # oracle in tests/test_ncdm_host.py
    H.h_plain.argtypes = [I, P, P, I, I, I, D, D, I, P, P, P, P]
    p = np.ascontiguousarray(W.BATCH64.params()[7])
    m, n_tau, L, Lm, rtol = 0.1, 300, 8, 6, 1e-7
    k = np.array([0.01, 0.08])
    rec = np.zeros((1, ncdm_lane.h_bg_len(n_tau)))
    ncdm_lane.h_build_bg_m(ptr(p), n_tau, m, ptr(rec))
    from paper_2602_15104_gb300 import abcmb as A
    from paper_2602_15104_gb300 import build
    build.build()
    o = A.options(lmax_hier=L, n_tau=n_tau, lmax_cl=40, m_ncdm=m, lmax_ncdm=Lm)
    work = np.zeros(A.perturb_workspace_bytes(1, k.size, o) // 8)  # the library's own size for this path
    assert work.size > 0
    S = np.zeros((1, k.size, n_tau, 3))
    st = np.full((1, k.size), -1, np.int32)
    steps = np.zeros((1, k.size, 2), np.int32)
    H.h_plain(1, ptr(rec), ptr(k), k.size, L, Lm, rtol, 1e-15, 20_000_000, ptr(S), ptr(st), ptr(steps), ptr(work))
    assert np.all(st == 0)
    for i in range(k.size):
        S1 = np.zeros((n_tau, 3))
        assert ncdm_lane.h_fwd_m(ptr(rec[0]), k[i], L, Lm, rtol, ptr(S1)) == 0
        assert np.abs(S[0, i] - S1).max() <= 1e-12 * np.abs(S1).max(), i


def test_record_vector_jacobian_product(H):
    # grad[b][j] = sum_e recbar[b][e] (rp[b][j][e] - rm[b][j][e]) / (2 h[b][j])
    rng = np.random.default_rng(6)
    B, n = 2, 5000
    rb = rng.normal(size=(B, n))
    rb[:, ::7] = 0.0  # entries the kernel skips
    rp, rm = rng.normal(size=(B, 6, n)), rng.normal(size=(B, 6, n))
    h = rng.uniform(1e-4, 1e-2, size=(B, 6))
    grad = np.zeros((B, 6))
    H.h_record_vjp(B, n, ptr(rb), ptr(rp), ptr(rm), ptr(h), ptr(grad))
    ref = np.einsum("be,bje->bj", rb, rp - rm) / (2 * h)
    np.testing.assert_allclose(grad, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
