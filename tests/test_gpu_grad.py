"""The hand-written adjoint (ClWithGradient): Cbar . dC_l/dtheta for the six
parameters, against central differences of the same forward (relative step
1e-4), against the oracle's forward sensitivities (tests/golden/
grad_forward_*.npz: the whole oracle run in complex arithmetic, one run per
parameter, exact to rounding) and its Richardson-extrapolated central
differences (tests/golden/grad_oracle_*.npz), both written by
tests/golden/make_grad_reference.py from the oracle alone, and the taped
forward against the plain pipeline.

The contraction weights are Cbar_l = z_l / |C_l| with z_l ~ N(0, 1), so every
l counts alike.  The ODE runs at rtol 1e-9: adaptive step decisions that flip
between theta +- h move C_l by ~rtol, which the differences divide by 2h ~
1e-4 theta; at 1e-9 that stays below 1e-5 of the gradient.  Each mode's tape
is sized by a first pass (abcmb_grad_count_steps / abcmb_grad_plan), so the
k range reaches 0.3 here and 0.5 at hierarchy 30 below.
"""
import os

import numpy as np
import pytest

from paper_2602_15104_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the oracle reference's "small" case
N_K, K_MIN, K_MAX, L_HIER, N_TAU, LMAX_CL = 40, 1e-4, 0.3, 12, 600, 400
REL_STEP = 1e-4


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


@pytest.fixture(scope="module")
def case(A):
    o = A.options(lmax_hier=L_HIER, n_tau=N_TAU, lmax_cl=LMAX_CL, rtol=1e-9, atol=1e-15)
    params = W.draw_cosmologies(2, 20260104)
    k = torch.tensor(W.log_k_nodes(N_K, K_MIN, K_MAX), device="cuda")
    p = torch.tensor(params, device="cuda", requires_grad=True)
    C = A.cl_with_gradient(p, k, o)
    rng = np.random.default_rng(5)
    Cbar = rng.normal(size=C.shape) / np.abs(C.detach().cpu().numpy())
    (C * torch.tensor(Cbar, device="cuda")).sum().backward()
    return dict(o=o, params=params, k=k, C=C.detach().cpu().numpy(), Cbar=Cbar, grad=p.grad.cpu().numpy())


def forward(A, params, k, o):
    with torch.no_grad():
        return A.cl_with_gradient(torch.tensor(params, device="cuda"), k, o).cpu().numpy()


def test_adjoint_against_differences_of_the_same_forward(A, case):
    # central differences at relative steps 2e-4 and 1e-4 combined by
    # Richardson extrapolation: a plain central difference errs by O(h^2),
    # up to ~2e-4 of the largest component for these weights at 1e-4
    params, Cbar, g = case["params"], case["Cbar"], case["grad"]
    for b in range(1):  # each difference is a full forward; one cosmology suffices
        fd = np.zeros(6)
        for j in range(6):
            est = []
            for rel in (2 * REL_STEP, REL_STEP):
                h = rel * max(abs(params[b, j]), 1e-3)
                pp, pm = params[b:b + 1].copy(), params[b:b + 1].copy()
                pp[0, j] += h
                pm[0, j] -= h
                Cp, Cm = forward(A, pp, case["k"], case["o"]), forward(A, pm, case["k"], case["o"])
                est.append(np.sum(Cbar[b] * (Cp[0] - Cm[0])) / (2 * h))
            fd[j] = (4.0 * est[1] - est[0]) / 3.0
        err = np.abs(g[b] - fd)
        assert np.all(err <= 1e-4 * np.abs(fd).max()), (b, g[b], fd, err)


def oracle_reference(case_name, forward=False):
    g = np.load(os.path.join(GOLDEN, f"grad_{'forward' if forward else 'oracle'}_{case_name}.npz"))
    np.testing.assert_array_equal(g["params"], W.BATCH16_GRAD.params()[0])
    return g


@pytest.mark.parametrize("forward", [True, False])
def test_adjoint_against_the_oracle_derivatives(A, case, forward):
    g = oracle_reference("small", forward)
    assert int(g["l_hier"]) == L_HIER and int(g["n_tau"]) == N_TAU and int(g["lmax_cl"]) == LMAX_CL
    np.testing.assert_allclose(g["k"], case["k"].cpu().numpy(), rtol=1e-15)
    Cbar, grad = case["Cbar"][0], case["grad"][0]
    ref = np.array([np.sum(Cbar * g["dCl"][j]) for j in range(6)])
    err = np.abs(grad - ref)
    assert np.all(err <= 1e-4 * np.abs(ref).max()), (grad, ref, err)


def test_adjoint_at_hierarchy_30_to_l_2500_and_k_0p5_against_the_oracle(A):
    """The differentiation workload's grids (hierarchies 30, 6000 tau nodes,
    l <= 2500) on 12 k reaching 0.5 /Mpc, one cosmology, against the oracle's
    forward sensitivities.  (Its Richardson differences are not used here:
    the oracle's fixed step schedule changes its step count between nodes as
    theta moves, and those jumps put the differences 1.13e-4 of the largest
    component off the forward sensitivity in the omega_cdm contraction.)"""
    g = oracle_reference("full", forward=True)
    o = A.options(lmax_hier=int(g["l_hier"]), n_tau=int(g["n_tau"]), lmax_cl=int(g["lmax_cl"]), rtol=1e-9,
                  atol=1e-15)
    k = torch.tensor(g["k"], device="cuda")
    p = torch.tensor(g["params"][None], device="cuda", requires_grad=True)
    C = A.cl_with_gradient(p, k, o)
    Cn = C.detach().cpu().numpy()[0]
    rng = np.random.default_rng(9)
    Cbar = rng.normal(size=Cn.shape) / np.abs(Cn)
    (C * torch.tensor(Cbar[None], device="cuda")).sum().backward()
    grad = p.grad.cpu().numpy()[0]
    ref = np.array([np.sum(Cbar * g["dCl"][j]) for j in range(6)])
    err = np.abs(grad - ref)
    assert np.all(err <= 1e-4 * np.abs(ref).max()), (grad, ref, err)
    # and the forward itself against the oracle's C_l
    assert np.max(np.abs(Cn[0] - g["Cl"][0]) / np.abs(g["Cl"][0])) < 1e-5


def test_taped_forward_matches_the_pipeline(A, case):
    o, params = case["o"], case["params"]
    pipe = A.Pipeline(len(params), case["k"].cpu().numpy(), o)
    C = pipe.run(torch.tensor(params, device="cuda")).cpu().numpy()
    pipe.check_status()
    assert np.all(np.abs(case["C"] - C) <= 1e-6 * np.abs(C).max(axis=2, keepdims=True))


def test_gradient_calls_reject_bad_arguments(A, case):
    o = case["o"]
    assert A.lib().abcmb_grad_workspace_bytes(0, 4, A.ctypes.byref(o)) == 0
    bg = torch.zeros((1, A.bg_doubles(o)), dtype=torch.float64, device="cuda")
    k = case["k"]
    small = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        A.abcmb_perturb_taped(bg, k, o, small)
    with pytest.raises(ValueError):  # a negative step count is no plan
        A.grad_plan(o, torch.full((1, k.shape[0]), -1, dtype=torch.int32))
    with pytest.raises(RuntimeError):
        A.abcmb_perturb_adjoint(bg, k, o, torch.zeros((1, k.shape[0], o.n_tau, 3), dtype=torch.float64,
                                                      device="cuda"), small, torch.zeros_like(bg))
