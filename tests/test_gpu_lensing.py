"""GPU parity of abcmb_lens (App. B.5) against the oracle's lensed spectra."""
import os
import sys

import numpy as np
import pytest

from oracle import lensing as LZ

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


def test_lensed_spectra_against_oracle(A):
    from test_lensing_host import spectra
    L, lout = 400, 300
    sp = [spectra(L, 7 + b) for b in range(2)]
    Cl = np.stack([np.stack([s[0][2:], s[2][2:], s[1][2:]]) for s in sp])
    Cpsi = np.stack([s[3][2:] for s in sp])
    out = A.abcmb_lens(torch.tensor(Cl, device="cuda"), torch.tensor(Cpsi, device="cuda"), lout,
                       n_mu=L + 100).cpu().numpy()
    for b, (ctt, cee, cte, cpsi) in enumerate(sp):
        TT, EE, TE, BB = LZ.lensed_cls(ctt, cee, cte, cpsi, lout, n_mu=L + 100)
        for c, ref, scale in [(0, TT, ctt), (2, EE, cee), (1, TE, np.sqrt(ctt * cee)), (3, BB, cee)]:
            err = np.abs(out[b, c] - ref[2:]).max() / np.abs(scale).max()
            assert err < 1e-10, (b, c, err)


def test_lens_rejects_bad_arguments(A):
    Cl = torch.zeros((1, 3, 99), dtype=torch.float64, device="cuda")
    Cpsi = torch.zeros((1, 99), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        A.abcmb_lens(Cl, Cpsi, 200)  # lmax_out above L
    with pytest.raises(RuntimeError):
        A.abcmb_lens(Cl, Cpsi, 80, n_mu=50)  # too few nodes
