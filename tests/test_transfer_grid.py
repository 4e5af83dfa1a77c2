"""The library's transfer-function k grid (host code, no GPU needed) against
the oracle's construction of App. A.1 eq. k_transfer_spacing."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def A():
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


@pytest.mark.parametrize("lmax", [2, 300, 2500, 5000])
def test_transfer_grid_matches_oracle(A, lmax):
    k = A.transfer_k_grid(lmax)
    ref = O.transfer_k_grid(lmax)
    assert k.size == ref.size
    np.testing.assert_allclose(k, ref, rtol=1e-14, atol=0)


def test_transfer_grid_rejects_bad_lmax(A):
    assert A.lib().abcmb_transfer_k_grid(1, None, 0) == -1
    assert A.lib().abcmb_transfer_k_grid(5001, None, 0) == -1
