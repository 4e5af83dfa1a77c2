"""GPU parity of the massive-neutrino path (one massive neutrino, App. B.3,
App. C.6): background, sources from abcmb_perturb (one warp per mode) and C_l,
against the oracle."""
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


def test_sources_and_cl_with_a_massive_neutrino(A):
    params = W.BATCH64.params()[[7, 30]]
    m, n_tau, L, Lm, lmax = 0.1, 300, 8, 6, 60
    k = np.array([3e-4, 2e-3, 0.01, 0.05])
    o = A.options(lmax_hier=L, n_tau=n_tau, lmax_cl=lmax, rtol=1e-9, m_ncdm=m, lmax_ncdm=Lm)
    bg = A.abcmb_background_tables(torch.tensor(params, device="cuda"), o)
    kk = torch.tensor(k, device="cuda")
    S, st, _ = A.abcmb_perturb(bg, kk, o)
    D = A.abcmb_project(bg, S, kk, o)
    C = A.abcmb_cl(bg, D, kk, o).cpu().numpy()
    S = S.cpu().numpy()
    assert bool((st == 0).all())
    for b in range(2):
        r = O.run(params[b], k, n_tau, lmax, O.opts(lmax=L, m_ncdm=m, lmax_ncdm=Lm))
        for i in range(k.size):
            err = np.abs(S[b, i] - r["S"][i]).max(axis=0) / np.abs(r["S"][i]).max(axis=0)
            assert np.all(err < 1e-6), (b, k[i], err)
        tt = np.abs(C[b, 0] - r["Cl"][0]) / np.abs(r["Cl"][0])
        ee = np.abs(C[b, 2] - r["Cl"][2]) / np.abs(r["Cl"][2])
        assert tt.max() < 1e-5 and ee.max() < 1e-5, (b, tt.max(), ee.max())


def test_massive_neutrino_rejected_where_unsupported(A):
    o = A.options(lmax_hier=8, n_tau=64, lmax_cl=40, m_ncdm=0.06, lmax_ncdm=6)
    bg = A.abcmb_background_tables(torch.tensor(W.BATCH64.params()[:1], device="cuda"), o)
    k = torch.tensor([1e-3, 1e-2], dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        A.abcmb_matter_pk(bg, k, o)
    ws = torch.empty(A.grad_workspace_bytes(1, 2, A.options(lmax_hier=8, n_tau=64, lmax_cl=40)) // 8 + 1,
                     dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        A.abcmb_perturb_taped(bg, k, o, ws)
