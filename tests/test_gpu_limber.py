"""GPU parity of the lensing potential's inputs (App. B.5): delta_m at the tau
nodes (abcmb_delta_m_nodes) and the Limber C_l^psi (abcmb_cl_psi) against the
oracle.  delta_m carries the ODE error of rtol 1e-6 relative to the mode's
largest value so far; C_l^psi is quadratic in it, so 2e-5 relative is the bar
for both."""
import numpy as np
import pytest

import oracle as O
from oracle import lensing as LZ
from paper_2602_15104_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_TAU = 400


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


def _setup(A, params, k, **kw):
    o = A.options(lmax_hier=12, n_tau=N_TAU, lmax_cl=40, **kw)
    bg = A.abcmb_background_tables(torch.tensor(np.atleast_2d(params), device="cuda"), o)
    return o, bg, torch.tensor(np.asarray(k, dtype=np.float64), device="cuda")


def test_delta_m_at_nodes_against_oracle(A):
    params = np.vstack([W.SMALL_TT.params(), W.BATCH64.params()[[17]]])
    k = np.array([1e-4, 1e-3, 0.01, 0.05])
    o, bg, kt = _setup(A, params, k)
    Dm, st = A.abcmb_delta_m_nodes(bg, kt, o)
    Dm, st = Dm.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0)
    for b in range(2):
        ref = O.delta_m_nodes(params[b], k, N_TAU, O.opts(lmax=12))
        scale = np.maximum.accumulate(np.abs(ref), axis=1)
        err = np.abs(Dm[b] - ref) / scale
        assert err.max() < 2e-5, (b, err.max(), np.unravel_index(err.argmax(), err.shape))


def test_limber_cl_psi_against_oracle(A):
    p = W.BATCH64.params()[17]
    k = np.exp(np.linspace(np.log(1e-4), np.log(0.08), 24))
    lmax = 120
    o, bg, kt = _setup(A, p, k)
    Dm, st = A.abcmb_delta_m_nodes(bg, kt, o)
    assert int(st.abs().sum()) == 0
    C = A.abcmb_cl_psi(bg, Dm, kt, o, lmax).cpu().numpy()[0]
    ref = LZ.cl_psi(p, k, N_TAU, lmax, O.opts(lmax=12))[2:]
    np.testing.assert_allclose(C, ref, rtol=2e-5)


def test_limber_rejects_bad_arguments(A):
    p = W.BATCH64.params()[17]
    o, bg, kt = _setup(A, p, [1e-3, 2e-3, 4e-3])
    Dm = torch.zeros((1, 3, N_TAU), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        A.abcmb_cl_psi(bg, Dm, kt, o, 50)  # fewer than 4 k nodes
    o2, bg2, kt2 = _setup(A, p, [1e-3], m_ncdm=0.06)
    with pytest.raises(RuntimeError):
        A.abcmb_delta_m_nodes(bg2, kt2, o2)  # massive neutrinos are not covered
