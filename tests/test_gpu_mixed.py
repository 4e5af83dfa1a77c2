"""GPU parity of the mixed-precision path (FP64 ODE, FP32 projection and
k-quadrature) against the FP64 oracle and the FP64 path.

Tolerances: the FP32 products carry ~1e-7 relative rounding each and the sum
over ~6000 tau nodes grows it like sqrt(n) with cancellation between
oscillating terms, so the projection is held to 2e-5 of each transfer
function's largest value; C_l to 1e-4 relative per spectrum (TT, EE:
|dC|/|C|; TE: |dC|/sqrt(C_TT C_EE)), the bar stated for the mixed form.
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


def cl_errors(C, ref):
    tt = np.abs(C[0] - ref[0]) / np.abs(ref[0])
    ee = np.abs(C[2] - ref[2]) / np.abs(ref[2])
    te = np.abs(C[1] - ref[1]) / np.sqrt(np.abs(ref[0] * ref[2]))
    return tt.max(), te.max(), ee.max()


def test_mixed_projection_against_oracle_synthetic_sources(A):
    params = W.BATCH64.params()[[0, 63]]
    k = np.array([1e-5, 3e-4, 0.004, 0.05, 0.18, 0.5])
    n_tau, lmax = 6000, 2500
    o = A.options(n_tau=n_tau, lmax_cl=lmax)
    S = np.stack([W.synthetic_sources(k.size, n_tau, 100 + b) for b in range(2)])
    p = torch.tensor(params, device="cuda")
    bg = A.abcmb_background_tables(p, o)
    D = A.abcmb_project_mixed(bg, torch.tensor(S, device="cuda"), torch.tensor(k, device="cuda"), o)
    D = D.double().cpu().numpy()
    for b in range(2):
        lna, tau, w = O.nodes(params[b], n_tau)
        ref = O.project(tau, w, O.scalars(params[b])["tau0"], k, S[b], lmax)
        for i in range(k.size):
            for c in range(2):
                scale = np.abs(ref[i, :, c]).max()
                err = np.max(np.abs(D[b, i, :, c] - ref[i, :, c])) / scale
                assert err < 2e-5, (b, k[i], c, err)


def test_mixed_cl_small_tt_against_oracle(A):
    wl = W.SMALL_TT
    p, k = wl.params(), wl.k()
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau)
    pipe = A.Pipeline(1, k, o, mixed=True)
    C = pipe.run(torch.tensor(p, device="cuda")).cpu().numpy()[0]
    pipe.check_status()
    ref = O.run(p[0], k, wl.n_tau, wl.l_max_cl, O.opts(lmax=wl.l_max_hier), want=("Cl",))["Cl"]
    tt, te, ee = cl_errors(C, ref)
    assert tt < 1e-4 and te < 1e-4 and ee < 1e-4, (tt, te, ee)


def test_mixed_cl_full_size_against_fp64_path(A):
    # the mixed-precision configuration: BATCH64's shapes (l <= 2500, 400 k,
    # hierarchies 30, 6000 nodes) on 4 of its cosmologies; the FP64 path is
    # within 1e-5 of the oracle (test_gpu_parity), so this bounds the mixed
    # path's error against the oracle by 1e-4 + 1e-5
    wl = W.BATCH64
    params, k = wl.params()[[0, 21, 42, 63]], wl.k()
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau)
    pipe = A.Pipeline(len(params), k, o)
    C64 = pipe.run(torch.tensor(params, device="cuda")).cpu().numpy()
    pipe.check_status()
    D32 = A.abcmb_project_mixed(pipe.bg, pipe.S, pipe.k, o)
    C32 = A.abcmb_cl_mixed(pipe.bg, D32, pipe.k, o).cpu().numpy()
    for b in range(len(params)):
        tt, te, ee = cl_errors(C32[b], C64[b])
        assert tt < 1e-4 and te < 1e-4 and ee < 1e-4, (b, tt, te, ee)


def test_mixed_cl_quadrature_matches_fp64_quadrature(A):
    # same Delta in both precisions: the FP32 Kahan k-sum against the FP64 one
    rng = np.random.default_rng(12)
    params = W.BATCH64.params()[:2]
    k = W.log_k_nodes(400, 1e-5, 0.5)
    lmax = 300
    o = A.options(lmax_cl=lmax, n_tau=64)
    D = rng.normal(size=(2, k.size, lmax - 1, 2)).astype(np.float32)
    bg = A.abcmb_background_tables(torch.tensor(params, device="cuda"), o)
    kk = torch.tensor(k, device="cuda")
    C32 = A.abcmb_cl_mixed(bg, torch.tensor(D, device="cuda"), kk, o).cpu().numpy()
    C64 = A.abcmb_cl(bg, torch.tensor(D.astype(np.float64), device="cuda"), kk, o).cpu().numpy()
    # products of float inputs rounded once in FP32: 3 roundings per term, compensated sum
    assert np.all(np.abs(C32 - C64) <= 1e-6 * np.abs(C64).max(axis=2, keepdims=True))
