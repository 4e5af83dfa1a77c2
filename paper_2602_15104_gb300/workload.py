"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method itself: it only draws cosmological
parameters and lays out wavenumber nodes.  Everything downstream (background,
recombination, perturbations, sources, projection, C_ell) is computed
independently by the CUDA library and by the CPU oracle from these inputs.

Parameter priors follow the paper's validation protocol (Sec. 4: uniform draws
over the six LCDM parameters, ranges of the table in Sec. 4); the fixed
parameters are the paper's defaults (App. A.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Order of the six drawn parameters, per cosmology (one row of `params`).
PARAM_NAMES = ("omega_b", "omega_cdm", "h", "n_s", "ln10As", "tau_reio")

# Uniform priors, in PARAM_NAMES order.
PRIORS = (
    (0.020, 0.024),
    (0.11, 0.13),
    (0.64, 0.72),
    (0.94, 0.99),
    (2.9, 3.2),
    (0.04, 0.08),
)


def draw_cosmologies(n: int, seed: int) -> np.ndarray:
    """Return an (n, 6) float64 array of cosmologies drawn with numpy PCG64.

    Draws are taken cosmology by cosmology, parameter by parameter, in the
    PARAM_NAMES order, so that the first m rows of a larger draw equal a draw of
    m with the same seed.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n, 6), dtype=np.float64)
    for i in range(n):
        for j, (lo, hi) in enumerate(PRIORS):
            out[i, j] = rng.uniform(lo, hi)
    return out


def log_k_nodes(n: int, k_min: float, k_max: float) -> np.ndarray:
    """n wavenumbers [1/Mpc], log-spaced on [k_min, k_max] inclusive."""
    if n < 2:
        raise ValueError("need at least two k nodes")
    return np.exp(np.linspace(np.log(k_min), np.log(k_max), n))


def synthetic_sources(n_k: int, n_tau: int, seed: int) -> np.ndarray:
    """Seeded smooth source arrays S[n_k][n_tau][3] indexed by tau-node number,
    shaped like CMB sources on the standard node grid (a narrow peak where the
    recombination nodes sit, oscillating with a k-dependent phase, plus a weak
    late tail); used to feed identical sources to both projections."""
    rng = np.random.default_rng(seed)
    i = np.arange(n_tau) / n_tau
    out = np.empty((n_k, n_tau, 3))
    for m in range(n_k):
        for c in range(3):
            amp, ph, fr = rng.uniform(0.5, 1.5), rng.uniform(0, 2 * np.pi), rng.uniform(5, 60)
            peak = np.exp(-0.5 * ((i - 0.45) / 0.08) ** 2)
            tail = 0.05 * np.exp(-((i - 0.9) / 0.1) ** 2)
            out[m, :, c] = amp * (peak * np.cos(fr * i + ph) + tail) * 10.0 ** (-c)
    return out


def synthetic_sources_smooth(k: np.ndarray, n_tau: int, seed: int) -> np.ndarray:
    """Seeded source arrays S[len(k)][n_tau][3] that vary smoothly with k
    (a recombination-like peak in the node index with a phase k r, r drawn per
    component, plus a weak late tail): inputs for interpolation in k."""
    rng = np.random.default_rng(seed)
    i = np.arange(n_tau) / n_tau
    k = np.asarray(k, dtype=np.float64)
    out = np.empty((k.size, n_tau, 3))
    peak = np.exp(-0.5 * ((i - 0.45) / 0.08) ** 2)
    tail = 0.05 * np.exp(-((i - 0.9) / 0.1) ** 2)
    for c in range(3):
        amp, ph, r = rng.uniform(0.5, 1.5), rng.uniform(0, 2 * np.pi), rng.uniform(50.0, 150.0)
        out[:, :, c] = amp * (peak[None, :] * np.cos(k[:, None] * r * (1.0 + i[None, :]) + ph)
                              + tail[None, :]) * 10.0 ** (-c)
    return out


@dataclass(frozen=True)
class Workload:
    """One named configuration of the hot path."""

    name: str
    n_cosmo: int
    seed: int
    n_k: int
    k_min: float
    k_max: float
    l_max_cl: int
    l_max_hier: int  # photon T, photon polarization and neutrino hierarchies
    n_tau: int
    spectra: tuple = ("TT", "TE", "EE")
    extra: dict = field(default_factory=dict)
    # the ODE error norm's group floor the configuration is run with
    # (abcmb_options.err_floor; the library's default is 1e-4)
    err_floor: float = 1e-4

    def params(self) -> np.ndarray:
        return draw_cosmologies(self.n_cosmo, self.seed)

    def k(self) -> np.ndarray:
        return log_k_nodes(self.n_k, self.k_min, self.k_max)


# Single flat-LCDM cosmology, TT only, small enough for the oracle in seconds.
SMALL_TT = Workload("lcdm_tt_l500_k100_hier12_tau2000", 1, 20260101,
                    100, 1e-4, 0.3, 500, 12, 2000, spectra=("TT",))

# Batch of 64 cosmologies, TT/TE/EE to l=2500: the throughput workload.
BATCH64 = Workload("lcdm_batch64_l2500_k400_hier30_tau6000", 64, 20260102,
                   400, 1e-5, 0.5, 2500, 30, 6000, err_floor=1e-2)

# Batch of 16 used for the differentiation workload (same grids as BATCH64).
BATCH16_GRAD = Workload("lcdm_batch16_grad_l2500_k400_hier30_tau6000", 16,
                        20260104, 400, 1e-5, 0.5, 2500, 30, 6000)

WORKLOADS = {w.name: w for w in (SMALL_TT, BATCH64, BATCH16_GRAD)}
