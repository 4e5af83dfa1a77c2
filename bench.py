#!/usr/bin/env python
"""Throughput benchmark of the C_ell hot path on GB300.

One step = the whole path (background tables -> perturbation ODEs and CMB
sources -> line-of-sight projection -> k-quadrature) for one batch of 64
seeded flat-LCDM cosmologies: TT/TE/EE to l = 2500, 400 log-spaced k in
[1e-5, 0.5]/Mpc, hierarchies at l = 30, 6000 tau nodes, FP64.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own batch
(weak scaling; no collective on the data path -- cosmologies are independent).
`--impl reference` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_15104_gb300 import workload as W  # noqa: E402

METRIC = "C_ℓ spectra/s at ℓmax=2500 TT/TE/EE (≤1e-5 rel vs FP64 oracle); p50/p99 latency"
FP64_PEAK = 2 * 2 * 152 * 2.07e9  # FMA units/SM x flops/FMA x SMs x max SM clock (1.26 TFLOP/s)
FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per mode of the FP64 perturbation kernel, from an
# ncu capture of the kernel as built; traffic grows in proportion to the
# modes, since every mode reads its cosmology's tables and writes its own
# sources.  None: the kernel gained the err_floor argument and the benchmark
# runs it at 1e-2 after the last capture (1.75 MB per mode at 1e-4), which has
# not been repeated.
PERTURB_DRAM_BYTES_PER_MODE = None


def flops_per_step(N: int, stages: int = 6) -> float:
    """Algorithmic FP64 work of one ODE step of one mode: s stages x (a
    right-hand side, ~12 N flops, plus a structured solve of (I - gamma h A),
    ~20 N) plus the error estimate, ~35 N s flops with s = 6 stages; a dense LU
    (~2 N^3 / 3) is avoidable work and not counted.  The kernel's step count
    (accepted and rejected) is the number of steps."""
    return 35.0 * N * stages


def flops_per_substep(N: int) -> float:
    """Diagnostic only: FP64 flops the kernel spends per linearly implicit
    Euler / Gragg substep (~6N right-hand side, ~0.3N Thomson solve, ~3.3N
    tableau and error norm amortised, ~150 for the background point; FMA = 2).
    This counts the extrapolation scheme's extra substeps as work."""
    return 10.0 * N + 150.0


def rank_params(wl, B: int, rank: int) -> np.ndarray:
    """Cosmologies of one rank: each rank draws its own seeded batch (weak
    scaling over independent cosmologies; no data exchange between ranks)."""
    return W.draw_cosmologies(B, wl.seed + 1000 * rank)


def max_over_ranks(values, dist, device) -> list:
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    whole job's time); identity on one rank."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / (ms * 1e-3)


def bessel_cut(x: np.ndarray, lmax: int) -> np.ndarray:
    """Last l the projection kernel keeps at x: the smallest l > x whose Debye
    decay exponent nu (alpha - tanh alpha), cosh alpha = nu / x, nu = l + 1/2,
    reaches 16 + 2 ln(1/x) for x < 1 (the kernel's own rule, evaluated here
    in float64 to count work)."""
    x = np.asarray(x, dtype=np.float64)
    T = 16.0 + 2.0 * np.maximum(0.0, -np.log(np.maximum(x, 1e-300)))
    nu = x + 1.0 + 7.2 * np.cbrt(np.maximum(x, 1.0))
    for _ in range(8):
        r = np.maximum(nu / np.maximum(x, 1e-30), 1.0 + 1e-6)
        al = np.arccosh(r)
        f = nu * (al - np.tanh(al)) - T
        nu = np.maximum(nu - f / np.maximum(al, 1e-3), x + 0.5)
    lc = np.clip(np.ceil(nu - 0.5), 2, lmax)
    lc = np.where(x < 1.0, np.minimum(lc, 30), lc)
    return np.where(x > lmax + 200.0, lmax, lc)


def projection_points(tau_nodes: np.ndarray, tau0: float, k: np.ndarray, lmax: int) -> float:
    """(node, l) points the projection kernel evaluates: l = 2 .. bessel_cut(x)
    per node, x = k (tau_0 - tau)."""
    x = np.outer(k, tau0 - tau_nodes)
    return float(np.maximum(bessel_cut(x, lmax) - 1.0, 0.0).sum())


class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(wl, p, k, cores: int, modes_per_core: int = 1) -> dict:
    """Time the FP64 oracle on a bounded sample of one cosmology of wl and
    scale it to the whole spectrum.  ODE: cores x modes_per_core complete
    integrations of low-k modes, which all take the same number of Radau
    steps (the schedule's landings on the tau nodes), one per thread, so the
    threads stay balanced; every step solves one 3N x 3N collocation system,
    so the rate (steps per second on all cores) scales to the schedule's
    exact step count over all k.  Projection: `cores` k spread over the grid
    at every l and tau node, scaled by n_k / cores."""
    import oracle as O
    o = O.opts(lmax=wl.l_max_hier)
    sched = O.count_steps(p, k, wl.n_tau, o)
    n_ode = cores * modes_per_core
    base = int(sched.min())
    low = np.flatnonzero(sched == base)[:n_ode]
    if low.size < n_ode:
        low = np.argsort(sched, kind="stable")[:n_ode]
    t0 = time.perf_counter()
    O.scalars(p)
    t_bg = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = O.run(p, k[low], wl.n_tau, 2, o, want=("S",), nthreads=cores)
    t_ode = time.perf_counter() - t0
    run_steps = int(r["steps"].sum())
    assert run_steps == int(sched[low].sum())
    idx = np.linspace(0, len(k) - 1, cores).round().astype(int)
    lna, tau, w = O.nodes(p, wl.n_tau)
    tau0 = O.scalars(p)["tau0"]
    S = np.ones((cores, wl.n_tau, 3))
    t0 = time.perf_counter()
    O.project(tau, w, tau0, k[idx], S, wl.l_max_cl, nthreads=cores)
    t_proj = time.perf_counter() - t0
    measured = t_bg + t_ode + t_proj
    sec = t_bg + t_ode * sched.sum() / run_steps + t_proj * len(k) / cores
    return {"measured_s": measured, "seconds_per_spectrum": sec, "fraction": measured / sec,
            "sample": (f"one cosmology of {wl.name}: {low.size} complete k modes ({run_steps} Radau steps of the "
                       f"{int(sched.sum())} the schedule takes over all {len(k)} k) on {cores} threads, and "
                       f"{cores} k projected at l <= {wl.l_max_cl} on {wl.n_tau} nodes; timed {measured:.1f} s, "
                       f"scaled to the spectrum by step count and k count")}


def cpu_baseline(wl, params, k, nthreads=None) -> dict:
    """The FP64 oracle on the host cores: the 64-cosmology workload on a
    bounded sample scaled to spectra/s (oracle_sample), and the single-
    cosmology TT workload (l <= 500, 100 k, hierarchies 12, 2000 nodes) run
    in full and timed."""
    import oracle as O
    cores = nthreads or os.cpu_count()
    smp = oracle_sample(wl, params[0], k, cores, 2)
    s1 = W.SMALL_TT
    t0 = time.perf_counter()
    O.run(s1.params()[0], s1.k(), s1.n_tau, s1.l_max_cl, O.opts(lmax=s1.l_max_hier), want=("Cl",),
          nthreads=cores)
    t_small = time.perf_counter() - t0
    return {"value": 1.0 / smp["seconds_per_spectrum"], "unit": "spectra/s", "cores": cores, "kind": "oracle",
            "seconds_per_spectrum": smp["seconds_per_spectrum"], "sample": smp["sample"],
            "full_run": {"workload": s1.name, "seconds": t_small, "spectra_per_s": 1.0 / t_small,
                         "what": "the whole path for one cosmology, timed in full"}}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is a bounded sample of one
    cosmology of the workload (oracle_sample), timed; the value is that
    step's share of a spectrum per second of it."""
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    params, k = wl.params(), wl.k()
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_sample(wl, params[0], k, cores)
    ms, vals, smp = [], [], None
    for _ in range(args.steps):
        smp = oracle_sample(wl, params[0], k, cores)
        ms.append(1e3 * smp["measured_s"])
        vals.append(smp["fraction"] / smp["measured_s"])
    v = statistics.mean(vals)
    cb = {"value": v, "unit": "spectra/s", "cores": cores, "kind": "oracle", "sample": smp["sample"]}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "spectra/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": wl.name, "batch": wl.n_cosmo},
           "step": "a bounded sample of one cosmology, share of a spectrum "
                   f"{smp['fraction']:.2e}",
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_serving(args, A, torch):
    """Serving benchmark: requests arrive as a Poisson process (seeded), each a
    cosmology from the priors with lmax_cl uniform on {500, 1000, 2000, 2500,
    3500} and n_k = 0.16 lmax_cl log-spaced k in [1e-5, 0.5] (hierarchies 30,
    6000 tau nodes, FP64 ODE, FP32 projection), submitted to abcmb_server at
    their arrival times; latency = completion - arrival on the host clock."""
    rng = np.random.default_rng(20260106)
    n = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=n))
    lmaxes = rng.choice([500, 1000, 2000, 2500, 3500], size=n)
    nks = np.round(0.16 * lmaxes).astype(int)
    params = W.draw_cosmologies(n, 20260105)
    o = A.options(lmax_hier=30, n_tau=6000, rtol=args.rtol)
    srv = A.Server(int(args.arena_gb * (1 << 30)), args.slots, 3500, int(nks.max()), o)
    # warm-up: one request of each size, not timed
    for i, lm in enumerate([500, 1000, 2000, 2500, 3500]):
        srv.submit(-1 - i, params[i], lm, int(round(0.16 * lm)), 1e-5, 0.5)
    done = 0
    while done < 5:
        srv.progress()
        while srv.poll() is not None:
            done += 1
        time.sleep(0.001)
    clocks = ClockSampler()
    clocks.start()
    t0 = time.perf_counter()
    nxt, finished, lat, ok, in_flight = 0, 0, np.zeros(n), np.zeros(n, dtype=bool), []
    while finished < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            rc = srv.submit(nxt, params[nxt], int(lmaxes[nxt]), int(nks[nxt]), 1e-5, 0.5)
            if rc != A.OK:
                raise RuntimeError(f"submit failed: {rc}")
            nxt += 1
        in_flight.append(srv.progress())
        r = srv.poll()
        while r is not None:
            tag, st, _ = r
            lat[tag] = time.perf_counter() - t0 - arrivals[tag]
            ok[tag] = st == A.OK
            finished += 1
            r = srv.poll()
        time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    clk = clocks.stop()
    srv.close()
    bad = int(n - ok.sum())
    lat = lat[ok]  # failed requests count neither as served nor in the latencies
    # the plain batched form on the same GPU: one 64-cosmology step of the
    # throughput workload (l <= 2500, 400 k), FP64 and mixed, after a warm-up step
    batched = {}
    wl = W.BATCH64
    ob = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau, rtol=args.rtol)
    pb = torch.tensor(wl.params(), device="cuda")
    for name, mixed in (("fp64", False), ("mixed", True)):
        pipe = A.Pipeline(wl.n_cosmo, wl.k(), ob, mixed=mixed)
        pipe.run(pb)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pipe.run(pb)
        e1.record()
        torch.cuda.synchronize()
        pipe.check_status()
        batched[name] = wl.n_cosmo / (e0.elapsed_time(e1) * 1e-3)
        del pipe
    out = {"metric": "served C_l spectra/s (mixed precision), p50/p99 latency", "value": int(ok.sum()) / makespan,
           "unit": "spectra/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": "serving_poisson_lmax500-3500", "requests": n, "rate_per_s": args.rate,
                      "nk_per_lmax": 0.16, "hierarchy_lmax": 30, "n_tau": 6000, "slots": args.slots,
                      "arena_gb": args.arena_gb, "rtol": args.rtol},
           "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                         "mean": float(lat.mean())},
           "makespan_s": makespan, "failed": bad, "mean_in_flight": float(np.mean(in_flight)),
           "batched_spectra_per_s": {**batched, "workload": wl.name},
           "clocks": clk}
    print(json.dumps(out), flush=True)


def run_gradient(args, A, torch):
    """Gradient benchmark: Cbar . dC_l/dtheta for the six parameters of each
    cosmology of a batch (hand-written adjoint through ClWithGradient): one
    step = taped forward (background, ODE, projection, quadrature) + backward
    (quadrature, projection and ODE adjoints, the background record's
    parameter Jacobian by central differences, the contraction)."""
    wl = W.BATCH16_GRAD
    B = args.batch or wl.n_cosmo
    params = W.draw_cosmologies(B, wl.seed)
    k_np = W.log_k_nodes(args.n_k, wl.k_min, wl.k_max) if args.n_k else wl.k()
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau, rtol=args.rtol)
    k = torch.tensor(k_np, device="cuda")
    rng = np.random.default_rng(3)
    Cbar = torch.tensor(rng.normal(size=(B, 3, o.lmax_cl - 1)), device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(p_dev):
        p = p_dev.detach().requires_grad_(True)
        C = A.cl_with_gradient(p, k, o)
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        (C * Cbar).sum().backward()
        return p.grad, e

    p_dev = torch.tensor(params, device="cuda")
    for _ in range(args.warmup):
        step(p_dev)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    ms, fwd_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g, emid = step(p_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        fwd_ms.append(e0.elapsed_time(emid))
    clk = clocks.stop()
    assert bool(torch.isfinite(g).all())
    t = statistics.mean(ms)
    out = {"metric": "dC_l/dtheta (6 parameters) per second, hand-written adjoint", "value": B / (t * 1e-3),
           "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
           "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "batch": B, "n_k": len(k_np), "k_range": [wl.k_min, wl.k_max],
                      "lmax_cl": wl.l_max_cl, "hierarchy_lmax": wl.l_max_hier, "n_tau": wl.n_tau,
                      "rtol": args.rtol, "checkpoint_every": 64,
                      "l2": "flushed (512 MiB write) between timed steps"},
           "forward_ms": statistics.mean(fwd_ms), "backward_ms": t - statistics.mean(fwd_ms),
           "gpu_launches": 10 * args.steps, "clocks": clk}
    print(json.dumps(out), flush=True)


def run_variants(args, A, torch):
    """Timings of the variant paths on a batch of the 64-cosmology workload
    (TT/TE/EE to l = 2500, 400 k in [1e-5, 0.5], hierarchies 30, 6000 tau
    nodes): the transfer k grid (projection onto the 1703-node grid by
    interpolation in ln k, then the quadrature), P(k, z = 0), the lensing
    chain (delta_m at the nodes, Limber C_l^psi to l = 2500, lensed spectra
    to l = 2000 from L = 2500) and the massive-neutrino perturbation solve
    (m = 0.06 eV).  Each line: CUDA-event time per call on the current
    stream after the warm-up calls, L2 flushed before each timed call."""
    wl = W.BATCH64
    B = args.batch or 8
    params = W.draw_cosmologies(B, wl.seed)
    k_np = W.log_k_nodes(args.n_k, wl.k_min, wl.k_max) if args.n_k else wl.k()
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau, rtol=args.rtol)
    k = torch.tensor(k_np, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    p_dev = torch.tensor(params, device="cuda")

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms), r

    def line(name, units, unit, ms, extra):
        out = {"metric": f"{name} ({unit})", "value": units / (ms * 1e-3), "unit": unit, "n_gpus": 1,
               "steps": args.steps, "warmup": args.warmup, "ms_per_call": ms, "higher_is_better": True,
               "dtype": "f64", "data": "synthetic",
               "config": {"workload": f"{wl.name} first {B} cosmologies", "n_k": len(k_np), "rtol": args.rtol,
                          "l2": "flushed (512 MiB write) before each timed call", **extra}}
        print(json.dumps(out), flush=True)

    clocks = ClockSampler()
    clocks.start()
    bg = A.abcmb_background_tables(p_dev, o)
    ms, (S, st, _) = timed(lambda: A.abcmb_perturb(bg, k, o))
    assert int(st.abs().sum()) == 0
    line("perturbation solve + sources, massless neutrinos", B, "cosmologies/s", ms, {})
    kt = torch.tensor(A.transfer_k_grid(o.lmax_cl), device="cuda")

    def transfer():
        D = A.abcmb_project_interp(bg, S, k, kt, o)
        return A.abcmb_cl(bg, D, kt, o)
    ms, C = timed(transfer)
    assert bool(torch.isfinite(C).all())
    line("projection on the transfer k grid + quadrature", B, "spectra/s", ms, {"n_k_transfer": kt.numel()})
    del S
    ms, (P, st) = timed(lambda: A.abcmb_matter_pk(bg, k, o, 0.0))
    assert int(st.abs().sum()) == 0
    line("matter power spectrum P(k, z=0)", B * len(k_np), "modes/s", ms, {"z": 0.0})
    ms, (Dm, st) = timed(lambda: A.abcmb_delta_m_nodes(bg, k, o))
    assert int(st.abs().sum()) == 0
    line("delta_m at the tau nodes", B, "cosmologies/s", ms, {})
    ms, Cpsi = timed(lambda: A.abcmb_cl_psi(bg, Dm, k, o, o.lmax_cl))
    line("Limber C_l^psi to l = 2500", B, "cosmologies/s", ms, {})
    del Dm
    Bl = min(B, 4)
    ms, CL = timed(lambda: A.abcmb_lens(C[:Bl].contiguous(), Cpsi[:Bl].contiguous(), 2000, n_mu=2600))
    assert bool(torch.isfinite(CL).all())
    line("lensed TT/TE/EE/BB to l = 2000 from L = 2500", Bl, "spectra/s", ms, {"batch": Bl, "n_mu": 2600})
    Bn = min(B, 2)
    on = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau, rtol=args.rtol, m_ncdm=0.06)
    bgn = A.abcmb_background_tables(p_dev[:Bn].contiguous(), on)
    ms, (Sn, st, _) = timed(lambda: A.abcmb_perturb(bgn, k, on))
    assert int(st.abs().sum()) == 0
    line("perturbation solve + sources, one massive neutrino 0.06 eV", Bn, "cosmologies/s", ms,
         {"batch": Bn, "lmax_ncdm": on.lmax_ncdm})
    print(json.dumps({"clocks": clocks.stop()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=W.BATCH64.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=None,
                    help="cosmologies per step (default: the workload's); smaller cases are for profiling")
    ap.add_argument("--n-k", type=int, default=None,
                    help="k modes (default: the workload's), log-spaced over the workload's range")
    ap.add_argument("--k-range", type=float, nargs=2, default=None, metavar=("K_MIN", "K_MAX"),
                    help="override the workload's k range (profiling cases; with --n-k 1, k = K_MAX alone)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed: FP64 ODE, FP32 projection and k-quadrature with Kahan sums")
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark: Poisson arrivals of mixed-size requests through abcmb_server")
    ap.add_argument("--grad", action="store_true",
                    help="gradient benchmark: dC_l/dtheta of a batch through the hand-written adjoint")
    ap.add_argument("--err-floor", type=float, default=None,
                    help="ODE error norm's group floor (abcmb_options.err_floor; default: the workload's)")
    ap.add_argument("--n-wide", type=int, default=0,
                    help="modes of the n highest k on eight lanes (abcmb_options.n_wide)")
    ap.add_argument("--node-recipe", type=int, default=0, choices=[0, 1],
                    help="tau-node placement: 0 the default, 1 the refined visibility tail")
    ap.add_argument("--variants", action="store_true",
                    help="time the variant paths (transfer grid, P(k), lensing chain, massive neutrino)")
    ap.add_argument("--requests", type=int, default=4096)
    ap.add_argument("--rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--arena-gb", type=float, default=24.0)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    if args.serve:
        # one hardware work queue per server slot (the default 8 would alias the
        # slots' streams onto 8 queues and serialise their kernels); read once,
        # when the CUDA context is created
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_2602_15104_gb300 import abcmb as A

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.serve:
        if rank == 0:
            run_serving(args, A, torch)
        return
    if args.grad:
        if rank == 0:
            run_gradient(args, A, torch)
        return
    if args.variants:
        if rank == 0:
            run_variants(args, A, torch)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = W.WORKLOADS[args.workload]
    B = args.batch or wl.n_cosmo
    params = rank_params(wl, B, rank)
    k_min, k_max = args.k_range if args.k_range else (wl.k_min, wl.k_max)
    if args.n_k == 1:
        k = np.array([k_max])
    elif args.n_k or args.k_range:
        k = W.log_k_nodes(args.n_k or wl.n_k, k_min, k_max)
    else:
        k = wl.k()
    err_floor = wl.err_floor if args.err_floor is None else args.err_floor
    o = A.options(lmax_hier=wl.l_max_hier, lmax_cl=wl.l_max_cl, n_tau=wl.n_tau, rtol=args.rtol,
                  node_recipe=args.node_recipe, n_wide=args.n_wide, err_floor=err_floor)
    N = 4 + 3 * (wl.l_max_hier + 1)
    mixed = args.precision == "mixed"
    pipe = A.Pipeline(B, k, o, mixed=mixed)
    project = A.abcmb_project_mixed if mixed else A.abcmb_project
    quadrature = A.abcmb_cl_mixed if mixed else A.abcmb_cl
    p_dev = torch.tensor(params, dtype=torch.float64, device="cuda")
    p_host = torch.from_numpy(params).pin_memory()
    cl_host = torch.empty((B, 3, o.lmax_cl - 1), dtype=torch.float64, pin_memory=True)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        pipe.run(p_dev)
    torch.cuda.synchronize()
    pipe.check_status()

    # device-resident timed steps, per-kernel events on the launching stream
    names = ["background", "perturb", "project", "cl"]
    ktimes = {n: [] for n in names}
    step_ms = []
    clocks = ClockSampler()
    clocks.start()
    barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between timed iterations (outside the events)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        A.abcmb_background_tables(p_dev, o, out=pipe.bg)
        ev[1].record(stream)
        A.abcmb_perturb(pipe.bg, pipe.k, o, S=pipe.S, status=pipe.status, steps=pipe.steps,
                        workspace=pipe.ws)
        ev[2].record(stream)
        project(pipe.bg, pipe.S, pipe.k, o, out=pipe.D)
        ev[3].record(stream)
        quadrature(pipe.bg, pipe.D, pipe.k, o, out=pipe.C)
        ev[4].record(stream)
        torch.cuda.synchronize()
        for i, n in enumerate(names):
            ktimes[n].append(ev[i].elapsed_time(ev[i + 1]))
        step_ms.append(ev[0].elapsed_time(ev[4]))
    barrier()
    clk = clocks.stop()
    pipe.check_status()

    # end to end through the public API: host params in, host C_l out
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pipe.run_host(p_host, cl_host)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))

    t_step = statistics.mean(step_ms)
    t_e2e = statistics.mean(e2e_ms)
    t_step, t_e2e = max_over_ranks([t_step, t_e2e], dist, "cuda")
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (FP64 ALU bound), on the algorithmic work
    # count per ODE step; the per-substep count is reported beside it
    kavg = {n: statistics.mean(v) for n, v in ktimes.items()}
    steps_taken = float(pipe.steps[:, :, 0].double().sum().item())
    substeps = float(pipe.steps[:, :, 1].double().sum().item())
    flops = {"perturb": steps_taken * flops_per_step(N)}
    pts = 0.0
    for b in range(B):
        scal, _, nodes = A.bg_view(pipe.bg[b], o.n_tau)
        pts += projection_points(nodes[:, 1], scal["TAU0"], k, o.lmax_cl)
    flops["project"] = 13.0 * pts
    dom = max(kavg, key=kavg.get)
    if dom in flops:
        ach = flops[dom] / (kavg[dom] * 1e-3)
        traffic = (PERTURB_DRAM_BYTES_PER_MODE * B * len(k)
                   if dom == "perturb" and PERTURB_DRAM_BYTES_PER_MODE is not None else None)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach / 1e12, "peak": FP64_PEAK / 1e12,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK, "traffic": traffic,
                "peak_source": "FP64 pipe: 2 FMA/clk/SM x 152 SMs x 2070 MHz (nominal 1.26 TFLOP/s)",
                "work": ("35 N s flops per ODE step, s = 6, N = 97 (steps taken)" if dom == "perturb"
                         else "13 flops per evaluated (node, l) point")}
        if dom == "perturb":
            roof["substep_model_tflops"] = substeps * flops_per_substep(N) / (kavg[dom] * 1e-3) / 1e12
    else:
        roof = None
    kern = {n: {"ms": kavg[n], "share": kavg[n] / sum(kavg.values())} for n in names}
    for n in flops:
        kern[n]["tflops"] = flops[n] / (kavg[n] * 1e-3) / 1e12
    value = whole_job_rate(B, world, t_step)
    lat = sorted(e2e_ms)
    out = {
        "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": wl.name, "batch": B, "n_k": len(k), "k_range": [float(k[0]), float(k[-1])],
                   "lmax_cl": wl.l_max_cl, "hierarchy_lmax": wl.l_max_hier, "n_tau": wl.n_tau,
                   "rtol": args.rtol, "precision": args.precision, "node_recipe": args.node_recipe,
                   "n_wide": args.n_wide, "err_floor": err_floor,
                   "l2": "flushed (512 MiB write) between timed steps",
                   "parallelism": f"replicas x{world}"},
        "clocks": clk,
        "e2e": {"value": whole_job_rate(B, world, t_e2e), "unit": "spectra/s",
                "h2d_bytes_per_step": int(params.nbytes),
                "d2h_bytes_per_step": int(B * 3 * (o.lmax_cl - 1) * 8)},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "what": f"batch of {B} spectra, host params to host C_l"},
        "gpu_launches": 4 * args.steps,
        "roofline": roof,
        "kernels": kern,
        "ode": {"mean_steps_per_mode": steps_taken / (B * len(k)), "steps_total": steps_taken,
                "substeps_total": substeps},
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(wl, params, k)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
