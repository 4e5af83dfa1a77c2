"""The emulated kernels under the compilers' sanitizers: each host harness
built with -fsanitize=address,undefined, and the multi-threaded ones also with
-fsanitize=thread, driven by tests/host/sanitize_calls.py in a subprocess with
the sanitizer runtime preloaded, on small and ragged shapes (node counts and
l ranges that fill no tile evenly, one- and eight-lane layouts, hierarchies
up to 50, a step budget that runs out, the smallest shapes).

  * AddressSanitizer / UBSan: a read or write past any buffer the kernels
    index (the caller's arrays and the emulated shared memory), or undefined
    behaviour in their integer and floating-point arithmetic, fails the run.
  * ThreadSanitizer: the emulation runs a CTA's threads as host threads that
    synchronise only where the device code does (warp collectives,
    __syncwarp, __syncthreads, atomics), so two lanes touching the same
    memory without one of those between them -- a data race under the CUDA
    memory model, whether or not the lanes of a warp happen to stay in step
    on the GPU -- is reported.  It finds the race the adjoint had before the
    barriers that close op_E_bgrad and op_T_bgrad.

Also the thread-per-mode solver for deep hierarchies, the serving arena's
allocator and the serving runtime itself (over its stand-in CUDA runtime).
compute-sanitizer is not used here.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST = os.path.join(ROOT, "tests", "host")


def _runtime(name):
    try:
        path = subprocess.check_output(["gcc", f"-print-file-name={name}"], text=True).strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


ASAN, UBSAN, TSAN = _runtime("libasan.so"), _runtime("libubsan.so"), _runtime("libtsan.so")

HARNESSES = {"quad": "quad_harness.cpp", "spectra": "spectra_harness.cpp", "mixed": "spectra_mixed_harness.cpp",
             "grad": "grad_harness.cpp", "lens": "lens_kernels_harness.cpp", "bgwarp": "bg_warp_harness.cpp",
             "adjwarp": "adjoint_warp_harness.cpp", "ode": "ode_harness.cpp", "arena": "arena_harness.cpp",
             "server": "server_harness.cpp"}
THREADED = ["quad", "spectra", "mixed", "grad", "lens", "bgwarp", "adjwarp", "ode"]
CASES = [(n, "address") for n in HARNESSES] + [(n, "thread") for n in THREADED]


def _build(d, name, kind):
    so = str(d / f"{name}_{kind}.so")
    flags = ["-ffp-contract=off"] if name == "mixed" else []
    flags += ["-fsanitize=address,undefined", "-fno-omit-frame-pointer"] if kind == "address" else \
        ["-fsanitize=thread"]
    sources = [os.path.join(HOST, HARNESSES[name])]
    if name == "server":  # the runtime itself, over the stand-in CUDA runtime
        flags.append("-I" + os.path.join(HOST, "fake_cuda"))
        sources = ["-x", "c++", os.path.join(ROOT, "paper_2602_15104_gb300", "csrc", "abcmb_server.cu"),
                   "-x", "none", *sources]
    job = subprocess.Popen(["g++", "-O1", "-g", "-std=c++17", "-pthread", "-fPIC", "-shared", *flags,
                            "-I" + os.path.join(ROOT, "include"),
                            "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"), *sources, "-o", so])
    return so, job


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    d = tmp_path_factory.mktemp("sanitized")
    out, jobs = {}, []
    for name, kind in CASES:  # compiled side by side
        if (kind == "address" and ASAN and UBSAN) or (kind == "thread" and TSAN):
            out[name, kind], job = _build(d, name, kind)
            jobs.append(job)
    assert all(j.wait() == 0 for j in jobs)
    return out


@pytest.mark.parametrize("name,kind", CASES)
def test_kernels_run_clean_under_the_sanitizers(builds, name, kind):
    if (name, kind) not in builds:
        pytest.skip(f"no {kind} sanitizer runtime")
    if kind == "address":
        env = dict(os.environ, LD_PRELOAD=f"{ASAN}:{UBSAN}",
                   ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:abort_on_error=0",
                   UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    else:
        env = dict(os.environ, LD_PRELOAD=TSAN, TSAN_OPTIONS="halt_on_error=1 report_signal_unsafe=0",
                   SANITIZE_LIGHT="1")  # the same paths on fewer steps: every access is instrumented
    args = [sys.executable, os.path.join(HOST, "sanitize_calls.py"), name, builds[name, kind]]
    if name == "adjwarp":
        args.append(builds["bgwarp", kind])
    r = subprocess.run(args, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.returncode, r.stdout[-2000:], r.stderr[-4000:])
