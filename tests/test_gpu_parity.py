"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Tolerances (stated per test): background quantities 1e-9 (two independent
quadratures/integrators of the same definitions), sources 1e-6 of each
source's maximum (two independent adaptive/fixed-step ODE solvers converged
far below the target), projection 1e-6 of the transfer function's maximum
(the kernel's Bessel recurrence stops ~1e-7 below the turning-point value),
C_l 1e-5 relative (TT, EE: |dC|/|C|; TE: |dC|/sqrt(C_TT C_EE), since TE
crosses zero).
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_15104_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


def run_gpu(A, params, k, o, stages=("bg", "perturb", "project", "cl")):
    p = torch.tensor(np.atleast_2d(params), dtype=torch.float64, device="cuda")
    kk = torch.tensor(k, dtype=torch.float64, device="cuda") if k is not None else None
    out = {}
    bg = A.abcmb_background_tables(p, o)
    out["bg"] = bg
    if "perturb" in stages:
        S, st, steps = A.abcmb_perturb(bg, kk, o)
        out.update(S=S, status=st, steps=steps)
    if "project" in stages:
        out["Delta"] = A.abcmb_project(bg, out["S"], kk, o)
    if "cl" in stages:
        out["Cl"] = A.abcmb_cl(bg, out["Delta"], kk, o)
    torch.cuda.synchronize()
    return {n: v.cpu().numpy() for n, v in out.items()}


def cl_errors(C, ref):
    tt = np.abs(C[0] - ref[0]) / np.abs(ref[0])
    ee = np.abs(C[2] - ref[2]) / np.abs(ref[2])
    te = np.abs(C[1] - ref[1]) / np.sqrt(np.abs(ref[0] * ref[2]))
    return tt.max(), te.max(), ee.max()


def test_background_parity(A):
    params = np.vstack([W.SMALL_TT.params(), W.BATCH64.params()[[0, 31, 63]]])
    n_tau = 2000
    o = A.options(n_tau=n_tau)
    r = run_gpu(A, params, None, o, stages=("bg",))
    for b, p in enumerate(params):
        s = O.scalars(p)
        scal, tab, nodes = A.bg_view(torch.tensor(r["bg"][b]), n_tau)
        assert scal["STATUS"] == 0
        for gk, ok in [("H0", "H0"), ("OMB", "Om_b"), ("OMC", "Om_c"), ("OMG", "Om_g"), ("OML", "Om_L"),
                       ("RNU", "R_nu"), ("NH0", "nH0"), ("AS", "A_s"), ("TAU0", "tau0")]:
            assert abs(scal[gk] / s[ok] - 1) < 1e-12, gk
        for gk, ok in [("ZREION", "z_reion"), ("LNA_TC", "lna_tc"), ("LNA_SW", "lna_sw")]:
            assert abs(scal[gk] - s[ok]) < 1e-9 * abs(s[ok]), gk
        lna, tau, w = O.nodes(p, n_tau)
        np.testing.assert_allclose(nodes[:, 0], lna, rtol=0, atol=1e-9)
        np.testing.assert_allclose(nodes[:, 1], tau, rtol=1e-10)
        np.testing.assert_allclose(nodes[:, 2], w, rtol=1e-8)
        bg = O.background(p, lna)
        for c, name in [(3, "g"), (4, "dg"), (6, "Hc"), (7, "dHc")]:
            assert np.max(np.abs(nodes[:, c] - bg[name])) < 1e-8 * np.max(np.abs(bg[name])), name
        # e^-kappa: relative error = absolute error of kappa, which is ~1e-8 relative to
        # kappa (~400 at the earliest nodes); only values that reach the sources matter
        np.testing.assert_allclose(nodes[:, 5], np.exp(-bg["kappa"]), rtol=1e-8, atol=1e-14)
        lt = A.BG_LNA0 + np.arange(A.BG_NLNA) / A.BG_PER_UNIT
        sel = np.arange(500, A.BG_NLNA, 1013)
        ob = O.background(p, lt[sel])
        for c, name in [(0, "nuT"), (2, "tau"), (4, "cs2"), (7, "xe")]:
            np.testing.assert_allclose(tab[sel, c], ob[name], rtol=1e-9, err_msg=name)


def test_sources_parity(A):
    params = np.vstack([W.SMALL_TT.params(), W.BATCH64.params()[[5]]])
    k = np.array([1e-4, 1e-3, 5e-3, 0.02, 0.08, 0.3])
    n_tau, L = 2000, 12
    o = A.options(lmax_hier=L, n_tau=n_tau, lmax_cl=40)
    r = run_gpu(A, params, k, o, stages=("bg", "perturb"))
    assert np.all(r["status"] == 0)
    for b, p in enumerate(params):
        ref = O.run(p, k, n_tau, 40, O.opts(lmax=L), want=("S",))["S"]
        for i in range(k.size):
            err = np.abs(r["S"][b, i] - ref[i]).max(axis=0) / np.abs(ref[i]).max(axis=0)
            assert np.all(err < 1e-6), (b, k[i], err)


def test_hierarchy_paths_agree_where_truncation_is_negligible(A):
    """Hierarchies <= 15, <= 31 and <= 63 run the four-lanes-per-mode kernel with 4, 8
    and 16 moments per lane; 64..128 the one-thread-per-mode kernel.  For k tau_0 < 8
    the moments beyond l ~ 30 are below e^-30 of the low ones, so every truncation
    from 30 up must give the same sources to the ODE tolerance."""
    params = W.BATCH64.params()[[3, 40]]
    k = np.array([1e-4, 3e-4, 5e-4])
    n_tau = 400
    runs = {}
    for L in (30, 40, 63, 64, 100, 128):
        o = A.options(lmax_hier=L, n_tau=n_tau, lmax_cl=40)
        r = run_gpu(A, params, k, o, stages=("bg", "perturb"))
        assert np.all(r["status"] == 0), L
        runs[L] = r["S"]
    ref = runs[30]
    scale = np.abs(ref).max(axis=2, keepdims=True)
    for L, S in runs.items():
        assert np.all(np.abs(S - ref) <= 1e-6 * scale), L
    # and the L = 30 result against the oracle at the same truncation
    o = A.options(lmax_hier=30, n_tau=n_tau, lmax_cl=40)
    for b, p in enumerate(params):
        S_o = O.run(p, k, n_tau, 40, O.opts(lmax=30), want=("S",))["S"]
        err = np.abs(ref[b] - S_o).max(axis=1) / np.abs(S_o).max(axis=1)
        assert np.all(err < 1e-6), (b, err)


def test_projection_parity_synthetic_sources(A):
    params = W.BATCH64.params()[[0, 63]]
    k = np.array([1e-5, 3e-4, 0.004, 0.05, 0.18, 0.5])
    n_tau, lmax = 6000, 2500
    o = A.options(n_tau=n_tau, lmax_cl=lmax)
    S = np.stack([W.synthetic_sources(k.size, n_tau, 100 + b) for b in range(2)])
    p = torch.tensor(params, device="cuda")
    bg = A.abcmb_background_tables(p, o)
    D = A.abcmb_project(bg, torch.tensor(S, device="cuda"), torch.tensor(k, device="cuda"), o).cpu().numpy()
    for b in range(2):
        lna, tau, w = O.nodes(params[b], n_tau)
        ref = O.project(tau, w, O.scalars(params[b])["tau0"], k, S[b], lmax)
        for i in range(k.size):
            for c in range(2):
                scale = np.abs(ref[i, :, c]).max()
                assert np.max(np.abs(D[b, i, :, c] - ref[i, :, c])) < 1e-6 * scale, (b, k[i], c)


def test_cl_parity_synthetic_transfer(A):
    rng = np.random.default_rng(11)
    params = W.BATCH64.params()[:3]
    k = W.log_k_nodes(37, 1e-4, 0.3)
    lmax = 300
    o = A.options(lmax_cl=lmax, n_tau=64)
    D = rng.normal(size=(3, k.size, lmax - 1, 2))
    p = torch.tensor(params, device="cuda")
    bg = A.abcmb_background_tables(p, o)
    C = A.abcmb_cl(bg, torch.tensor(D, device="cuda"), torch.tensor(k, device="cuda"), o).cpu().numpy()
    for b in range(3):
        s = O.scalars(params[b])
        ref = O.cl(k, D[b], lmax, s["A_s"], params[b][3])
        np.testing.assert_allclose(C[b], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_end_to_end_small_tt_workload(A):
    wl = W.SMALL_TT
    p, k = wl.params(), wl.k()
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau)
    r = run_gpu(A, p, k, o)
    assert np.all(r["status"] == 0)
    ref = O.run(p[0], k, wl.n_tau, wl.l_max_cl, O.opts(lmax=wl.l_max_hier), want=("Cl",))["Cl"]
    tt, te, ee = cl_errors(r["Cl"][0], ref)
    assert tt < 1e-5 and te < 1e-5 and ee < 1e-5, (tt, te, ee)


def test_full_size_sampled_modes(A):
    # the throughput workload in the launch configuration the benchmark
    # times (64 cosmologies x 400 k, hierarchies 30, 6000 nodes, l <= 2500),
    # checked on sampled modes the oracle can afford and by properties
    wl = W.BATCH64
    params, k = wl.params(), wl.k()
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau)
    pipe = A.Pipeline(wl.n_cosmo, k, o)
    C = pipe.run(torch.tensor(params, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    pipe.check_status()
    assert np.all(np.isfinite(C))
    assert np.all(C[:, 0] > 0) and np.all(C[:, 2] > 0)
    assert np.all(C[:, 1] ** 2 <= C[:, 0] * C[:, 2] * (1 + 1e-12))
    samples = [(0, 0), (17, 150), (63, 230)]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(len(samples)) as ex:
        refs = list(ex.map(lambda s: O.run(params[s[0]], k[[s[1]]], wl.n_tau, wl.l_max_cl,
                                           O.opts(lmax=wl.l_max_hier), want=("S", "Delta"), nthreads=1),
                           samples))
    for (b, i), ref in zip(samples, refs):
        S = pipe.S[b, i].cpu().numpy()
        err = np.abs(S - ref["S"][0]).max(axis=0) / np.abs(ref["S"][0]).max(axis=0)
        assert np.all(err < 1e-6), (b, i, err)
        D = pipe.D[b, i].cpu().numpy()
        for c in range(2):
            scale = np.abs(ref["Delta"][0, :, c]).max()
            assert np.max(np.abs(D[:, c] - ref["Delta"][0, :, c])) < 1e-5 * scale, (b, i, c)


def test_default_tolerance_moves_cl_by_far_less_than_the_target(A):
    # the library's default rtol against a 1e-10 solution of the same
    # discretisation, at the full l <= 2500, 400 k, hierarchy 30, 6000-node size
    wl = W.BATCH64
    params, k = wl.params()[[7, 50]], wl.k()
    C = {}
    for rt in (None, 1e-10):
        kw = {} if rt is None else {"rtol": rt}
        o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau, **kw)
        pipe = A.Pipeline(len(params), k, o)
        C[rt] = pipe.run(torch.tensor(params, device="cuda")).cpu().numpy()
        pipe.check_status()
    for b in range(len(params)):
        tt, te, ee = cl_errors(C[None][b], C[1e-10][b])
        assert max(tt, te, ee) < 2e-6, (b, tt, te, ee)


def test_highest_k_self_convergence(A):
    # k = 0.5 is beyond what the oracle's dense solver affords at hierarchy 30;
    # the adaptive solver's sources must be converged well below the target
    p = W.BATCH64.params()[:2]
    k = np.array([0.35, 0.5])
    o1 = A.options(lmax_hier=30, n_tau=6000, lmax_cl=10, rtol=1e-8)
    o2 = A.options(lmax_hier=30, n_tau=6000, lmax_cl=10, rtol=1e-10)
    r1 = run_gpu(A, p, k, o1, stages=("bg", "perturb"))
    r2 = run_gpu(A, p, k, o2, stages=("bg", "perturb"))
    err = np.abs(r1["S"] - r2["S"]).max(axis=2) / np.abs(r2["S"]).max(axis=2)
    assert np.all(err < 1e-6), err


def test_minimal_and_ragged_shapes(A):
    params = W.BATCH64.params()[:3]
    k = np.array([2e-4, 1e-3, 3e-3, 7e-3, 1.2e-2])
    n_tau, lmax, L = 8, 2, 4
    o = A.options(lmax_hier=L, n_tau=n_tau, lmax_cl=lmax)
    r = run_gpu(A, params, k, o)
    assert np.all(r["status"] == 0)
    for b in range(3):
        ref = O.run(params[b], k, n_tau, lmax, O.opts(lmax=L), want=("S", "Cl"))
        err = np.abs(r["S"][b] - ref["S"]).max() / np.abs(ref["S"]).max()
        assert err < 1e-6
        tt, te, ee = cl_errors(r["Cl"][b], ref["Cl"])
        assert max(tt, te, ee) < 1e-5


def test_step_budget_reported(A):
    p = W.BATCH64.params()[:2]
    o = A.options(lmax_hier=8, n_tau=64, lmax_cl=10, max_steps=5)
    r = run_gpu(A, p, np.array([1e-3, 0.1]), o, stages=("bg", "perturb"))
    assert np.all(r["status"] == A.E_MAX_STEPS)
    assert np.all(r["steps"][..., 0] == 6)


def test_background_failure_reported(A):
    p = W.BATCH64.params()[:2].copy()
    p[1, 5] = 5.0  # optical depth no reionization redshift in range can give
    o = A.options(lmax_hier=8, n_tau=64, lmax_cl=10)
    r = run_gpu(A, p, np.array([1e-3, 0.01]), o, stages=("bg", "perturb"))
    assert r["bg"][0, A.S_INDEX["STATUS"]] == 0
    assert r["bg"][1, A.S_INDEX["STATUS"]] == A.E_BACKGROUND
    assert np.all(r["status"][0] == 0) and np.all(r["status"][1] == A.E_NONFINITE)


def test_repeatable(A):
    p = W.BATCH64.params()[:2]
    k = W.log_k_nodes(9, 1e-4, 0.1)
    o = A.options(lmax_hier=10, n_tau=500, lmax_cl=300)
    r1 = run_gpu(A, p, k, o)
    r2 = run_gpu(A, p, k, o)
    np.testing.assert_array_equal(r1["S"], r2["S"])
    np.testing.assert_allclose(r1["Cl"], r2["Cl"], rtol=1e-13)


@pytest.mark.parametrize("lmax_hier", [30, 40])
def test_eight_lane_layout_agrees_with_the_four_lane_one(A, lmax_hier):
    # abcmb_options.n_wide moves the modes of the highest k from four lanes per
    # mode to eight, with the same arithmetic per mode; a mode's result still
    # depends on its warp-mates through the warp-wide switch to the explicit
    # regime, so the layouts agree to the ODE tolerance, not bit for bit
    # (ragged: 5 cosmologies, so warps of the eight-lane layout mix k values)
    p = W.BATCH64.params()[:5]
    k = torch.tensor(W.log_k_nodes(23, 1e-4, 0.5), device="cuda")
    bg = A.abcmb_background_tables(torch.tensor(p, device="cuda"),
                                   A.options(lmax_hier=lmax_hier, n_tau=800, lmax_cl=300))
    out = []
    for n_wide in (0, 7, 23, 40):  # (steps returned for the record, not compared)
        o = A.options(lmax_hier=lmax_hier, n_tau=800, lmax_cl=300, n_wide=n_wide, rtol=1e-9)
        S, st, steps = A.abcmb_perturb(bg, k, o)
        out.append((S.cpu().numpy(), st.cpu().numpy(), steps.cpu().numpy()))
    S0 = out[0][0]
    peak = np.abs(S0).max(axis=2, keepdims=True)
    assert np.all(out[0][1] == 0)
    for S, st, steps in out[1:]:
        np.testing.assert_array_equal(st, out[0][1])
        assert np.all(np.abs(S - S0) <= 1e-7 * peak), np.abs((S - S0) / peak).max()
        # (step counts differ: a warp of mixed k keeps its modes in the
        # implicit regime until the last of them may leave it)
