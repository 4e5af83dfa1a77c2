"""GPU parity of the matter power spectrum (abcmb_matter_pk, App. B.4 eq. PK)
against the oracle.  P is quadratic in delta_m, whose ODE error at the default
rtol 1e-6 is ~1e-6, so 1e-5 relative is the bar, as for C_l."""
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


def gpu_pk(A, params, k, z, L=12, **kw):
    o = A.options(lmax_hier=L, n_tau=400, lmax_cl=40, **kw)
    bg = A.abcmb_background_tables(torch.tensor(np.atleast_2d(params), device="cuda"), o)
    Pk, st = A.abcmb_matter_pk(bg, torch.tensor(k, device="cuda"), o, z)
    return Pk.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("z", [0.0, 2.0])
def test_pk_against_oracle(A, z):
    params = np.vstack([W.SMALL_TT.params(), W.BATCH64.params()[[17]]])
    k = np.array([1e-5, 1e-4, 1e-3, 6e-3, 0.02, 0.05])
    P, st = gpu_pk(A, params, k, z)
    assert np.all(st == 0)
    for b in range(2):
        ref = O.pk(params[b], k, z, O.opts(lmax=12))
        err = np.abs(P[b] / ref - 1.0)
        assert np.all(err < 1e-5), (b, err)


def test_pk_hierarchy_paths_agree_at_large_scales(A):
    # k <= 1e-3 is superhorizon through the radiation era, where the hierarchy
    # truncation could matter, so hierarchies 12 (4 moments per lane), 30 (8)
    # and 50 (16) give the same P(k)
    params = W.BATCH64.params()[[2, 9]]
    k = np.array([2e-5, 2e-4, 1e-3])
    ref, _ = gpu_pk(A, params, k, 0.0, L=12)
    for L in (30, 50):
        P, st = gpu_pk(A, params, k, 0.0, L=L)
        assert np.all(st == 0)
        np.testing.assert_allclose(P, ref, rtol=2e-6)


def test_pk_rejects_bad_arguments(A):
    params = W.BATCH64.params()[:1]
    k = np.array([1e-3])
    with pytest.raises(RuntimeError):
        gpu_pk(A, params, k, -0.5)
    with pytest.raises(RuntimeError):
        gpu_pk(A, params, k, 0.0, L=80)
