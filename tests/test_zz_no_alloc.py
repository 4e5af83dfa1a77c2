"""abcmb_perturb_noalloc: the perturbation step for callers that cannot
allocate device memory (an application whose device memory belongs to another
runtime's pool, or a loop that cannot afford an allocation's implicit
synchronisation).  It runs the same kernels on the same inputs as
abcmb_perturb, so its sources, status words and step counts must equal
abcmb_perturb's bit for bit, call after call: from the library's own static
scratch for hierarchies above 63 (the one-thread-per-mode kernel), with no
scratch at all below.  Before the compared calls another, larger problem runs
through the same scratch, so that a value read before it is written would
show.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest

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


def fill_scratch(A):
    """A different problem (deeper hierarchies, more modes) through the shared
    scratch: it leaves other values where the compared call works."""
    params = torch.tensor(W.BATCH64.params()[10:14], device="cuda")
    k = torch.tensor(W.log_k_nodes(20, 2e-4, 0.08), device="cuda")
    o = A.options(lmax_hier=128, n_tau=300, lmax_cl=10)
    bg = A.abcmb_background_tables(params, o)
    S = torch.empty((4, 20, 300, 3), dtype=torch.float64, device="cuda")
    st = torch.empty((4, 20), dtype=torch.int32, device="cuda")
    assert A.abcmb_perturb_noalloc(bg, k, o, S, st) == A.OK
    torch.cuda.synchronize()


@pytest.mark.parametrize("lmax_hier", [70, 12])
def test_noalloc_matches_workspace_entry_point_twice(A, lmax_hier):
    params = torch.tensor(W.BATCH64.params()[:3], device="cuda")
    k = torch.tensor(W.log_k_nodes(7, 1e-4, 0.05), device="cuda")
    o = A.options(lmax_hier=lmax_hier, n_tau=500, lmax_cl=10)
    assert (A.perturb_workspace_bytes(3, 7, o) > 0) == (lmax_hier > 63)
    bg = A.abcmb_background_tables(params, o)
    S_ref, st_ref, steps_ref = A.abcmb_perturb(bg, k, o)
    torch.cuda.synchronize()
    assert int(st_ref.abs().sum()) == 0
    fill_scratch(A)
    for _ in range(2):  # the scratch keeps the previous call's contents
        S = torch.full_like(S_ref, float("nan"))
        st = torch.full_like(st_ref, -1)
        steps = torch.full_like(steps_ref, -1)
        rc = A.abcmb_perturb_noalloc(bg, k, o, S, st, steps)
        torch.cuda.synchronize()
        assert rc == A.OK
        np.testing.assert_array_equal(st.cpu().numpy(), st_ref.cpu().numpy())
        np.testing.assert_array_equal(steps.cpu().numpy(), steps_ref.cpu().numpy())
        np.testing.assert_array_equal(S.cpu().numpy(), S_ref.cpu().numpy())


def test_noalloc_rejects_problems_beyond_its_scratch(A):
    o = A.options(lmax_hier=80, n_tau=6000, lmax_cl=2500)
    assert A.perturb_workspace_bytes(64, 400, o) > A.NOALLOC_SCRATCH_BYTES
    params = torch.tensor(W.BATCH64.params()[:1], device="cuda")
    bg = A.abcmb_background_tables(params, o)
    bg64 = bg.expand(64, -1).contiguous()
    k = torch.tensor(W.BATCH64.k(), device="cuda")
    S = torch.empty(1, dtype=torch.float64, device="cuda")  # never written: rejected on the host
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    assert A.abcmb_perturb_noalloc(bg64, k, o, S, st) == A.E_SCRATCH_TOO_SMALL
