"""Calls into AddressSanitizer / UndefinedBehaviorSanitizer builds of the
oracle's C sources (run by tests/test_oracle_sanitized.py in a subprocess
with the sanitizer runtimes preloaded): the double build through its whole
path (background and thermal history with both node recipes, perturbations
with and without a massive neutrino, projection, C_l, P(k), delta_m at the
nodes, Bessel functions) and the complex-step build's sensitivities, on small
and ragged sizes.  A read or write past a buffer, or undefined behaviour,
ends the process with the sanitizer's report.

usage: python sanitize_oracle.py <double .so> <complex .so>
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402
from oracle import build as B  # noqa: E402
from paper_2602_15104_gb300 import workload as W  # noqa: E402

B.build = lambda force=False: sys.argv[1]  # the instrumented builds in place of the plain ones
B.build_cs = lambda force=False: sys.argv[2]

p = W.BATCH64.params()[3]
o = O.opts(lmax=8)
k = np.array([1e-4, 0.01, 0.1])
r = O.run(p, k, 57, 70, o, want=("S", "Delta", "Cl"), nthreads=2)
assert np.isfinite(r["Cl"]).all()
assert np.isfinite(O.pk(p, k[:2], 0.5, o)).all()  # to a = 1/1.5: the low k keep it short
assert np.isfinite(O.delta_m_nodes(p, k[:2], 57, o)).all()
lna, tau, w = O.nodes(p, 23, node_recipe=1)
assert np.isfinite(O.background(p, lna)["g"]).all() and O.scalars(p)["tau0"] > 0
assert np.isfinite(O.bessel(300, 150.0)).all()
r2 = O.run(p, np.array([0.01, 0.02]), 31, 40, O.opts(lmax=6, m_ncdm=0.06, lmax_ncdm=4), want=("Cl",),
           nthreads=2)
assert np.isfinite(r2["Cl"]).all()
_, d = O.sensitivity(p, 5, k[1:], 23, 40, O.opts(lmax=6), nthreads=2)["Cl"]
assert np.isfinite(d).all()
print("ok")
