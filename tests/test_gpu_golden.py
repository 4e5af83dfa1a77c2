"""GPU parity on the 64-cosmology throughput workload against stored oracle values.

The workload is the one the benchmark times: 64 flat-LCDM cosmologies (seed
20260102), TT/TE/EE for every l in [2, 2500], 400 log-spaced k on
[1e-5, 0.5] /Mpc, hierarchies truncated at l = 30, 6000 tau nodes.  The
oracle's C_l and sampled sources for a few of these cosmologies are stored
in tests/golden/batch64_oracle_recipe*.npz, written by
tests/golden/make_batch64.py (which runs only the CPU oracle).  The library
runs the whole batch in the benchmark's launch configuration (the workload's
ODE error floor, abcmb_options.err_floor = 1e-2) and, once, at the library's
default floor, and is compared element by element:

  C_l, FP64 path      |dC|/|C| <= 1e-5 for TT and EE, |dC^TE| / sqrt(C^TT C^EE)
                      <= 1e-5 (TE crosses zero), every l (App. B.4 eq. c_ell_def)
  C_l, mixed path     the same measures <= 1e-4 (FP32 projection and
                      k-quadrature after the FP64 ODE)
  sources             |dS| <= 3e-6 of each source's largest value over the
                      stored nodes (6e-6 at the benchmark's group floor, see
                      SOURCE_BAR), at the five stored k up to 0.5 /Mpc
                      (App. B.4 eq. source_functions): the ODE's error
                      control holds each step's error to rtol = 1e-6 of the
                      state; over the ~5000 steps of the highest k the
                      global error of the late ISW source S_T1, a difference
                      of metric terms, reaches ~1e-6 of its peak
"""
import os

import numpy as np
import pytest

from paper_2602_15104_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = {r: os.path.join(HERE, "golden", f"batch64_oracle_recipe{r}.npz") for r in (0, 1)}


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


def golden(recipe):
    g = np.load(GOLDEN[recipe])
    wl = W.BATCH64
    assert int(g["node_recipe"]) == recipe
    assert int(g["n_tau"]) == wl.n_tau and int(g["l_max_cl"]) == wl.l_max_cl
    assert int(g["l_max_hier"]) == wl.l_max_hier
    np.testing.assert_array_equal(g["params"], wl.params()[g["cosmo"]])
    return g


def cl_errors(C, ref):
    tt = np.abs(C[0] - ref[0]) / np.abs(ref[0])
    ee = np.abs(C[2] - ref[2]) / np.abs(ref[2])
    te = np.abs(C[1] - ref[1]) / np.sqrt(np.abs(ref[0] * ref[2]))
    return tt.max(), te.max(), ee.max()


def run_batch(A, recipe, mixed, err_floor=W.BATCH64.err_floor):
    wl = W.BATCH64
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau, node_recipe=recipe,
                  err_floor=err_floor)
    pipe = A.Pipeline(wl.n_cosmo, wl.k(), o, mixed=mixed)
    C = pipe.run(torch.tensor(wl.params(), device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    pipe.check_status()
    return pipe, C


# sources: 3e-6 of peak at the library's default group floor (1e-4); at the
# benchmark's 1e-2, components below 1 % of their group are held to rtol of
# that level rather than of their own, and the host build of the same
# integrator measures the sources' largest error against the oracle rising
# from 2.0e-6 to 3.1e-6 of peak (k = 0.5), so the bar is 6e-6 there
SOURCE_BAR = {1e-4: 3e-6, 1e-2: 6e-6}


@pytest.mark.parametrize("recipe,err_floor", [(0, W.BATCH64.err_floor), (1, W.BATCH64.err_floor), (0, 1e-4)])
def test_batch64_fp64_against_oracle(A, recipe, err_floor):
    g = golden(recipe)
    pipe, C = run_batch(A, recipe, mixed=False, err_floor=err_floor)
    for n, b in enumerate(g["cosmo"]):
        tt, te, ee = cl_errors(C[b], g["Cl"][n])
        print(f"recipe {recipe} err_floor {err_floor} cosmology {b}: max rel error TT {tt:.2e} TE {te:.2e} "
              f"EE {ee:.2e}")
        assert tt < 1e-5 and te < 1e-5 and ee < 1e-5, (b, tt, te, ee)
        S = pipe.S[b][torch.as_tensor(g["k_index"], device="cuda")][:, torch.as_tensor(g["node_index"],
                                                                                       device="cuda")]
        S = S.cpu().numpy()
        ref = g["S"][n]
        for i in range(ref.shape[0]):
            err = np.abs(S[i] - ref[i]).max(axis=0) / np.abs(ref[i]).max(axis=0)
            print(f"   k index {int(g['k_index'][i])}: sources max error / peak {err.max():.2e}")
            assert np.all(err < SOURCE_BAR[err_floor]), (b, int(g["k_index"][i]), err)


def test_batch64_mixed_against_oracle(A):
    g = golden(0)
    _, C = run_batch(A, 0, mixed=True)
    for n, b in enumerate(g["cosmo"]):
        tt, te, ee = cl_errors(C[b], g["Cl"][n])
        print(f"mixed cosmology {b}: max rel error TT {tt:.2e} TE {te:.2e} EE {ee:.2e}")
        assert tt < 1e-4 and te < 1e-4 and ee < 1e-4, (b, tt, te, ee)
