"""The emulated kernels under AddressSanitizer and UndefinedBehaviorSanitizer:
each host harness built with -fsanitize=address,undefined and driven by
tests/host/sanitize_calls.py in a subprocess with the sanitizer runtimes
preloaded, on small and ragged shapes (node counts and l ranges that fill no
tile evenly, one- and eight-lane layouts, hierarchies up to 50, a step
budget that runs out).  A read or write past any buffer the kernels index
(the caller's arrays and the emulated shared memory), or undefined behaviour
in their integer and floating-point arithmetic, fails the run.  Also the
thread-per-mode solver for deep hierarchies, the serving arena's allocator
and the serving runtime itself (over its stand-in CUDA runtime).  On the device the same accesses are unchecked; compute-sanitizer
is not used here.
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


ASAN, UBSAN = _runtime("libasan.so"), _runtime("libubsan.so")
pytestmark = pytest.mark.skipif(ASAN is None or UBSAN is None, reason="no sanitizer runtimes")

HARNESSES = {"quad": "quad_harness.cpp", "spectra": "spectra_harness.cpp", "mixed": "spectra_mixed_harness.cpp",
             "grad": "grad_harness.cpp", "lens": "lens_kernels_harness.cpp", "bgwarp": "bg_warp_harness.cpp",
             "adjwarp": "adjoint_warp_harness.cpp", "ode": "ode_harness.cpp", "arena": "arena_harness.cpp",
             "server": "server_harness.cpp"}


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    d = tmp_path_factory.mktemp("sanitized")
    out, jobs = {}, []
    for name, src in HARNESSES.items():  # compiled side by side
        so = str(d / f"{name}.so")
        flags = ["-ffp-contract=off"] if name == "mixed" else []
        sources = [os.path.join(HOST, src)]
        if name == "server":  # the runtime itself, over the stand-in CUDA runtime
            flags.append("-I" + os.path.join(HOST, "fake_cuda"))
            sources = ["-x", "c++", os.path.join(ROOT, "paper_2602_15104_gb300", "csrc", "abcmb_server.cu"),
                       "-x", "none", *sources]
        jobs.append(subprocess.Popen(["g++", "-O1", "-g", "-std=c++17", "-pthread", "-fPIC", "-shared", *flags,
                                      "-fsanitize=address,undefined", "-fno-omit-frame-pointer",
                                      "-I" + os.path.join(ROOT, "include"),
                                      "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                                      *sources, "-o", so]))
        out[name] = so
    assert all(j.wait() == 0 for j in jobs)
    return out


@pytest.mark.parametrize("name", list(HARNESSES))
def test_kernels_run_clean_under_the_sanitizers(builds, name):
    env = dict(os.environ, LD_PRELOAD=f"{ASAN}:{UBSAN}",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    args = [sys.executable, os.path.join(HOST, "sanitize_calls.py"), name, builds[name]]
    if name == "adjwarp":
        args.append(builds["bgwarp"])
    r = subprocess.run(args, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.returncode, r.stdout[-2000:], r.stderr[-4000:])
