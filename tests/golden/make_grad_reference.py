"""Write the oracle's derivatives dC_l/dtheta for the gradient tests.

For one flat-LCDM cosmology of the differentiation workload (seed 20260104,
the first draw) and two discretisations this script runs only the CPU oracle
and stores C_l^{TT,TE,EE} and their derivatives with respect to the six
parameters (omega_b, omega_cdm, h, n_s, ln 1e10 A_s, tau_reion; the paper's
sec. "Gradients of ABCMB outputs"), taken by central differences at relative
steps 2e-4 and 1e-4 (floor 1e-3 in absolute terms) combined by Richardson
extrapolation, which removes the O(h^2) term.  The oracle's C_l is smooth in
the parameters only piecewise: its fixed step schedule changes its step
count between two nodes as the parameters move, and each such jump moves
C_l by the discretisation error (~1e-9), so per multipole the differences
agree with the exact derivative to ~1e-7 of its largest value, but weighted
sums that stress small C_l (near zeros of TE) can be off by ~1e-4 (the
forward sensitivities below have no such error):

  small   40 log-spaced k on [1e-4, 0.3] /Mpc, hierarchies 12, 600 tau nodes,
          l <= 400
  full    12 log-spaced k on [1e-4, 0.5] /Mpc, hierarchies 30, 6000 tau nodes,
          l <= 2500

Output: tests/golden/grad_oracle_<case>.npz (params, k, Cl [3][l_max - 1],
dCl [6][3][l_max - 1], and the grid sizes).

With --forward the script writes instead the oracle's forward sensitivities
(oracle.sensitivity: the whole path run in complex arithmetic with the
parameter's imaginary part set, one run per parameter, exact to rounding;
the forward mode of the paper's gradients, Sec. 3) to
tests/golden/grad_forward_<case>.npz, same fields, no step sizes.

Usage:  python tests/golden/make_grad_reference.py [--forward] small full
(the full case takes about half an hour on 8 host cores, a quarter of an
hour with --forward).
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2602_15104_gb300 import workload as W  # noqa: E402

CASES = {
    "small": dict(n_k=40, k_min=1e-4, k_max=0.3, l_hier=12, n_tau=600, lmax_cl=400),
    "full": dict(n_k=12, k_min=1e-4, k_max=0.5, l_hier=30, n_tau=6000, lmax_cl=2500),
}
REL_STEPS = (2e-4, 1e-4)
ABS_FLOOR = 1e-3


def path_for(case: str, forward: bool = False) -> str:
    return os.path.join(HERE, f"grad_forward_{case}.npz" if forward else f"grad_oracle_{case}.npz")


def sensitivities(params, k, c, threads=0):
    """dC_l/dtheta_j by the oracle's complex-step forward mode."""
    o = O.opts(lmax=c["l_hier"])
    C, D = None, None
    for j in range(6):
        v, d = O.sensitivity(params, j, k, c["n_tau"], c["lmax_cl"], o, want=("Cl",), nthreads=threads)["Cl"]
        if C is None:
            C, D = v, np.zeros((6,) + v.shape)
        D[j] = d
        print(f"  parameter {j} done", flush=True)
    return C, D


def derivatives(params, k, c, threads=0):
    o = O.opts(lmax=c["l_hier"])

    def cl(p):
        return O.run(p, k, c["n_tau"], c["lmax_cl"], o, want=("Cl",), nthreads=threads)["Cl"]

    C = cl(params)
    D = np.zeros((6,) + C.shape)
    for j in range(6):
        est = []
        for rel in REL_STEPS:
            h = rel * max(abs(params[j]), ABS_FLOOR)
            pp, pm = params.copy(), params.copy()
            pp[j] += h
            pm[j] -= h
            est.append((cl(pp) - cl(pm)) / (2.0 * h))
        # central differences err by a h^2 + O(h^4): the steps halve, so the
        # combination (4 D(h) - D(2h)) / 3 cancels the h^2 term
        D[j] = (4.0 * est[1] - est[0]) / 3.0
        print(f"  parameter {j} done", flush=True)
    return C, D


def main() -> None:
    params = W.BATCH16_GRAD.params()[0]
    args = sys.argv[1:]
    forward = "--forward" in args
    cases = [a for a in args if a != "--forward"] or list(CASES)
    for case in cases:
        c = CASES[case]
        k = W.log_k_nodes(c["n_k"], c["k_min"], c["k_max"])
        print(case, flush=True)
        if forward:
            C, D = sensitivities(params, k, c)
            np.savez_compressed(path_for(case, True), params=params, k=k, Cl=C, dCl=D, l_hier=c["l_hier"],
                                n_tau=c["n_tau"], lmax_cl=c["lmax_cl"])
            continue
        C, D = derivatives(params, k, c)
        np.savez_compressed(path_for(case), params=params, k=k, Cl=C, dCl=D, l_hier=c["l_hier"],
                            n_tau=c["n_tau"], lmax_cl=c["lmax_cl"], rel_steps=np.array(REL_STEPS),
                            abs_floor=ABS_FLOOR)


if __name__ == "__main__":
    main()
