"""Write the oracle's reference values for the 64-cosmology throughput workload.

The workload: flat LCDM cosmologies drawn with seed 20260102, TT/TE/EE to
l = 2500, 400 log-spaced k on [1e-5, 0.5] /Mpc, photon temperature,
polarization and neutrino hierarchies truncated at l = 30, 6000 tau nodes
(App. A.1 truncation, App. B.4 projection and eq. c_ell_def).  For each chosen
cosmology this script runs the CPU oracle (and nothing else) over the whole
k grid and stores

  Cl[c][3][2499]        C_l^{TT,TE,EE}, l = 2..2500 (eq. c_ell_def)
  S[c][5][n_sub][3]     the sources S_T0, S_T1, S_P (App. B.4, eq.
                        source_functions) at the five k nodes nearest to
                        0.02, 0.08, 0.18, 0.35 and 0.5 /Mpc, on every
                        NODE_STRIDE-th tau node
  steps[c][400]         the oracle's Radau steps per mode

Usage (about 20 minutes per cosmology on 8 host cores):
  python tests/golden/make_batch64.py --cosmo 0 63 --node-recipe 0
  python tests/golden/make_batch64.py --cosmo 31 --node-recipe 1
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2602_15104_gb300 import workload as W  # noqa: E402

SAMPLE_K = (0.02, 0.08, 0.18, 0.35, 0.5)
NODE_STRIDE = 4


def path_for(node_recipe: int) -> str:
    return os.path.join(HERE, f"batch64_oracle_recipe{node_recipe}.npz")


def sample_k_indices(k: np.ndarray) -> np.ndarray:
    return np.array([int(np.argmin(np.abs(np.log(k / s)))) for s in SAMPLE_K])


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--cosmo", type=int, nargs="+", required=True)
    ap.add_argument("--node-recipe", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    wl = W.BATCH64
    params, k = wl.params(), wl.k()
    ik = sample_k_indices(k)
    nodes = np.arange(0, wl.n_tau, NODE_STRIDE)
    o = O.opts(lmax=wl.l_max_hier, node_recipe=a.node_recipe)
    Cl, S, steps = [], [], []
    for c in a.cosmo:
        t0 = time.time()
        r = O.run(params[c], k, wl.n_tau, wl.l_max_cl, o, want=("S", "Cl"), nthreads=a.threads)
        Cl.append(r["Cl"])
        S.append(r["S"][ik][:, nodes, :])
        steps.append(r["steps"])
        print(f"cosmology {c}: {time.time() - t0:.0f} s, {r['steps'].sum()} steps", flush=True)
    np.savez_compressed(path_for(a.node_recipe), cosmo=np.array(a.cosmo), params=params[a.cosmo],
                        k_index=ik, node_index=nodes, Cl=np.array(Cl), S=np.array(S),
                        steps=np.array(steps), node_recipe=a.node_recipe,
                        l_max_hier=wl.l_max_hier, n_tau=wl.n_tau, l_max_cl=wl.l_max_cl)


if __name__ == "__main__":
    main()
