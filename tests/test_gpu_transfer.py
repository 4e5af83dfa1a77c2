"""The transfer-grid variant (App. A.1 eq. k_transfer_spacing): sources
computed on an ODE k grid, interpolated in ln k onto the transfer grid inside
the projection (abcmb_project_interp), then the k-quadrature on that grid --
against the oracle's interpolation, projection and quadrature."""
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


def test_interpolating_projection_against_oracle(A):
    # smooth synthetic sources on 60 ODE nodes, projected at 37 other k (some
    # outside the nodes, where the end cubics extend)
    params = W.BATCH64.params()[[4, 50]]
    n_tau, lmax = 3000, 1200
    k = np.exp(np.linspace(np.log(2e-4), np.log(0.1), 60))
    kt = np.exp(np.linspace(np.log(1.5e-4), np.log(0.11), 37))
    o = A.options(n_tau=n_tau, lmax_cl=lmax)
    S = np.stack([W.synthetic_sources_smooth(k, n_tau, 300 + b) for b in range(2)])
    bg = A.abcmb_background_tables(torch.tensor(params, device="cuda"), o)
    D = A.abcmb_project_interp(bg, torch.tensor(S, device="cuda"), torch.tensor(k, device="cuda"),
                               torch.tensor(kt, device="cuda"), o).cpu().numpy()
    for b in range(2):
        lna, tau, w = O.nodes(params[b], n_tau)
        St = O.interp_sources(S[b], k, kt)
        ref = O.project(tau, w, O.scalars(params[b])["tau0"], kt, St, lmax)
        for i in range(kt.size):
            for c in range(2):
                scale = np.abs(ref[i, :, c]).max()
                assert np.max(np.abs(D[b, i, :, c] - ref[i, :, c])) < 1e-6 * scale, (b, kt[i], c)


def test_transfer_grid_cl_against_oracle(A):
    lmax, n_tau, L = 300, 2000, 12
    kt = A.transfer_k_grid(lmax)
    k = np.exp(np.linspace(np.log(kt[0]), np.log(kt[-1]), 120))  # ODE nodes covering the grid
    p = W.SMALL_TT.params()
    o = A.options(lmax_hier=L, lmax_cl=lmax, n_tau=n_tau)
    bg = A.abcmb_background_tables(torch.tensor(p, device="cuda"), o)
    kk, ktt = torch.tensor(k, device="cuda"), torch.tensor(kt, device="cuda")
    S, st, _ = A.abcmb_perturb(bg, kk, o)
    D = A.abcmb_project_interp(bg, S, kk, ktt, o)
    C = A.abcmb_cl(bg, D, ktt, o).cpu().numpy()[0]
    assert bool((st == 0).all())
    r = O.run(p[0], k, n_tau, lmax, O.opts(lmax=L), want=("S",))
    lna, tau, w = O.nodes(p[0], n_tau)
    sc = O.scalars(p[0])
    Dref = O.project(tau, w, sc["tau0"], kt, O.interp_sources(r["S"], k, kt), lmax)
    ref = O.cl(kt, Dref, lmax, sc["A_s"], sc["n_s"])
    tt = np.abs(C[0] - ref[0]) / np.abs(ref[0])
    ee = np.abs(C[2] - ref[2]) / np.abs(ref[2])
    te = np.abs(C[1] - ref[1]) / np.sqrt(np.abs(ref[0] * ref[2]))
    assert tt.max() < 1e-5 and te.max() < 1e-5 and ee.max() < 1e-5, (tt.max(), te.max(), ee.max())
