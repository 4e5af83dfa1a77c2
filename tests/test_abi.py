"""Host-side checks of the C ABI library (no GPU compute): it builds for
sm_103a, loads, exports every entry point include/abcmb.h declares, and
rejects invalid arguments on the host before enqueuing anything."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "abcmb.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def A():
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(abcmb_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(A):
    L = A.lib()
    syms = declared_symbols()
    assert len(syms) >= 8
    for s in syms:
        assert hasattr(L, s), s


def test_defaults_and_sizes(A):
    L = A.lib()
    o = A.Options()
    L.abcmb_default_options(ctypes.byref(o))
    assert (o.lmax_g, o.lmax_cl, o.n_tau, o.node_recipe, o.n_wide) == (12, 2500, 6000, 0, 0)
    assert o.err_floor == 1e-4
    assert L.abcmb_validate_options(ctypes.byref(A.options(node_recipe=1))) == A.OK
    assert A.bg_doubles(o) == A.BG_NODES + 8 * o.n_tau + A.BG_ODEPOLY_DOUBLES
    # hierarchies <= 63 keep the ODE state on chip: no workspace
    assert A.perturb_workspace_bytes(64, 400, o) == 0
    assert A.perturb_workspace_bytes(64, 400, A.options(lmax_hier=63)) == 0
    N = 4 + 3 * 81
    assert A.perturb_workspace_bytes(64, 400, A.options(lmax_hier=80)) == 8 * N * 64 * 400 * 8
    bad = A.options(lmax_hier=3)
    assert L.abcmb_bg_doubles(ctypes.byref(bad)) == 0
    assert L.abcmb_perturb_workspace_bytes(64, 400, ctypes.byref(bad)) == 0


@pytest.mark.parametrize("field,value", [("lmax_g", 3), ("lmax_nu", 129), ("lmax_cl", 1), ("lmax_cl", 5001),
                                         ("n_tau", 7), ("max_steps", 0), ("rtol", 0.0), ("rtol", 1.0),
                                         ("atol", -1.0), ("node_recipe", 2), ("node_recipe", -1),
                                         ("n_wide", -1), ("err_floor", 0.0), ("err_floor", 1.5)])
def test_invalid_options_rejected_on_host(A, field, value):
    L = A.lib()
    o = A.options()
    setattr(o, field, value)
    fake = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    assert L.abcmb_background_tables(1, fake, ctypes.byref(o), fake, None) == A.E_INVALID_ARG
    assert L.abcmb_perturb(1, fake, fake, 4, ctypes.byref(o), fake, fake, None, fake, 1 << 30,
                           None) == A.E_INVALID_ARG
    assert L.abcmb_project(1, fake, fake, fake, 4, ctypes.byref(o), fake, None) == A.E_INVALID_ARG
    assert L.abcmb_cl(1, fake, fake, fake, 4, ctypes.byref(o), fake, None) == A.E_INVALID_ARG


def test_invalid_shapes_and_pointers_rejected(A):
    L = A.lib()
    o = A.options()
    f = ctypes.c_void_p(256)
    assert L.abcmb_background_tables(0, f, ctypes.byref(o), f, None) == A.E_INVALID_ARG
    assert L.abcmb_background_tables(1, None, ctypes.byref(o), f, None) == A.E_INVALID_ARG
    assert L.abcmb_perturb(1, f, f, 0, ctypes.byref(o), f, f, None, f, 1 << 40, None) == A.E_INVALID_ARG
    # deep hierarchies need a workspace: missing, too small, or misaligned
    o80 = A.options(lmax_hier=80)
    assert L.abcmb_perturb(1, f, f, 4, ctypes.byref(o80), f, f, None, None, 1 << 40, None) == A.E_INVALID_ARG
    assert L.abcmb_perturb(1, f, f, 4, ctypes.byref(o80), f, f, None, f, 8, None) == A.E_INVALID_ARG
    assert L.abcmb_perturb(1, f, f, 4, ctypes.byref(o80), f, f, None, ctypes.c_void_p(264), 1 << 40,
                           None) == A.E_INVALID_ARG
    assert L.abcmb_project(1, f, None, f, 4, ctypes.byref(o), f, None) == A.E_INVALID_ARG
    assert L.abcmb_cl(1, f, f, f, 1, ctypes.byref(o), f, None) == A.E_INVALID_ARG  # one k: no quadrature
    assert L.abcmb_cl(1, f, f, f, 4, ctypes.byref(o), None, None) == A.E_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2602_15104_gb300 import abcmb
    monkeypatch.setattr(abcmb, "_lib", None)
    monkeypatch.setattr(abcmb, "LIB_PATH", "/nonexistent/libabcmb.so")
    with pytest.raises(RuntimeError, match="missing"):
        abcmb.lib()


def test_library_package_never_uses_the_oracle():
    pkg = os.path.join(ROOT, "paper_2602_15104_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "orc_" not in text, f


def test_workload_is_seeded():
    from paper_2602_15104_gb300 import workload as W
    a = W.draw_cosmologies(64, 20260102)
    b = W.draw_cosmologies(4, 20260102)
    np.testing.assert_array_equal(a[:4], b)
    for j, (lo, hi) in enumerate(W.PRIORS):
        assert np.all((a[:, j] >= lo) & (a[:, j] <= hi))
    k = W.BATCH64.k()
    assert k.size == 400 and abs(k[0] - 1e-5) < 1e-20 and abs(k[-1] - 0.5) < 1e-15
    np.testing.assert_allclose(np.diff(np.log(k)), np.log(0.5 / 1e-5) / 399, rtol=1e-10)
    S1 = W.synthetic_sources(3, 100, 5)
    S2 = W.synthetic_sources(3, 100, 5)
    np.testing.assert_array_equal(S1, S2)


def test_variant_entry_points_reject_on_host(A):
    # each of these returns before its first CUDA call (so it runs without a GPU)
    L = A.lib()
    o = A.options()
    f = ctypes.c_void_p(256)
    D = ctypes.c_double
    # P(k): redshift outside [0, 1000], a massive neutrino, hierarchies above 63
    assert L.abcmb_matter_pk(1, f, f, 4, ctypes.byref(o), D(-0.5), f, f, None) == A.E_INVALID_ARG
    assert L.abcmb_matter_pk(1, f, f, 4, ctypes.byref(o), D(2000.0), f, f, None) == A.E_INVALID_ARG
    assert L.abcmb_matter_pk(1, f, f, 4, ctypes.byref(A.options(m_ncdm=0.06)), D(0.0), f, f,
                             None) == A.E_INVALID_ARG
    assert L.abcmb_matter_pk(1, f, f, 4, ctypes.byref(A.options(lmax_hier=80)), D(0.0), f, f,
                             None) == A.E_INVALID_ARG
    # delta_m at the nodes: empty batch, missing output, massive neutrino, deep hierarchy
    assert L.abcmb_delta_m_nodes(0, f, f, 4, ctypes.byref(o), f, f, None) == A.E_INVALID_ARG
    assert L.abcmb_delta_m_nodes(1, f, f, 4, ctypes.byref(o), None, f, None) == A.E_INVALID_ARG
    assert L.abcmb_delta_m_nodes(1, f, f, 4, ctypes.byref(A.options(m_ncdm=0.06)), f, f, None) == A.E_INVALID_ARG
    assert L.abcmb_delta_m_nodes(1, f, f, 4, ctypes.byref(A.options(lmax_hier=80)), f, f, None) == A.E_INVALID_ARG
    # Limber: fewer than 4 k nodes (no Hermite interpolation), l range
    assert L.abcmb_cl_psi(1, f, f, f, 3, ctypes.byref(o), 100, f, None) == A.E_INVALID_ARG
    assert L.abcmb_cl_psi(1, f, f, f, 8, ctypes.byref(o), 1, f, None) == A.E_INVALID_ARG
    assert L.abcmb_cl_psi(1, f, f, f, 8, ctypes.byref(o), 6001, f, None) == A.E_INVALID_ARG
    # lensing: lmax_out above L, too few Gauss-Legendre nodes
    assert L.abcmb_lens(1, f, 100, f, 120, 200, f, None) == A.E_INVALID_ARG
    assert L.abcmb_lens(1, f, 100, f, 80, 100, f, None) == A.E_INVALID_ARG
    # transfer-grid projection: fewer than 4 ODE k nodes
    assert L.abcmb_project_interp(1, f, f, f, 3, f, 10, ctypes.byref(o), f, None) == A.E_INVALID_ARG
    # the transfer grid itself (host function): out-of-range lmax, and its size
    assert L.abcmb_transfer_k_grid(1, None, 0) == -1
    assert L.abcmb_transfer_k_grid(2500, None, 0) == 1703


def test_server_request_bytes(A):
    # host function: a request's arena footprint grows with lmax_cl and n_k, is
    # dominated by its FP64 sources (n_k x n_tau x 3 doubles), and invalid
    # requests need nothing
    o = A.options(lmax_hier=30, n_tau=6000)
    b = {(lm, nk): A.server_request_bytes(o, lm, nk) for lm in (500, 2500) for nk in (80, 400)}
    assert b[(500, 80)] < b[(500, 400)] and b[(500, 80)] < b[(2500, 80)] < b[(2500, 400)]
    assert b[(2500, 400)] >= 400 * 6000 * 3 * 8
    assert A.server_request_bytes(o, 1, 80) == 0 and A.server_request_bytes(o, 500, 1) == 0
    assert A.server_request_bytes(A.options(n_tau=4), 500, 80) == 0


def test_gradient_plan_host_function(A):
    """abcmb_grad_plan (host): per-mode tape and checkpoint prefix sums in the
    kernels' k-descending mode order, and the workspace they need, which grows
    with the counted steps and stays below the fixed-capacity workspace for
    modes shorter than 65536 steps."""
    o = A.options(lmax_hier=12, n_tau=600, lmax_cl=400)
    B, Nk = 2, 3
    acc = np.array([[10, 200, 70000], [0, 64, 129]], dtype=np.int32)
    acc_t = A.torch.tensor(acc)
    plan, nb = A.grad_plan(o, acc_t)
    M = B * Nk
    # mode m -> (b = m % B, kidx = Nk - 1 - m // B)
    order = [acc[m % B, Nk - 1 - m // B] for m in range(M)]
    assert plan[M] == sum(order)
    np.testing.assert_array_equal(plan[:M], np.concatenate([[0], np.cumsum(order)[:-1]]))
    ck = [a // 64 + 1 for a in order]
    assert plan[2 * M + 1] == sum(ck)
    np.testing.assert_array_equal(plan[M + 1:2 * M + 1], np.concatenate([[0], np.cumsum(ck)[:-1]]))
    plan2, nb2 = A.grad_plan(o, A.torch.tensor(acc * 2))
    assert nb2 > nb
    small, nbs = A.grad_plan(o, A.torch.tensor(np.full((B, Nk), 100, dtype=np.int32)))
    assert nbs < A.grad_workspace_bytes(B, Nk, o)
