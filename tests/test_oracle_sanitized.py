"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: its C
sources built with -fsanitize=address,undefined (the double build and the
complex-step build) and driven through its whole path by
tests/host/sanitize_oracle.py in a subprocess with the sanitizer runtimes
preloaded.  The oracle is what every parity test trusts, so a read past one
of its buffers would corrupt references silently; here it ends the run."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")


def _runtime(name):
    try:
        path = subprocess.check_output(["gcc", f"-print-file-name={name}"], text=True).strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


ASAN, UBSAN = _runtime("libasan.so"), _runtime("libubsan.so")


@pytest.mark.skipif(ASAN is None or UBSAN is None, reason="no sanitizer runtimes")
def test_oracle_runs_clean_under_the_sanitizers(tmp_path):
    sys.path.insert(0, ROOT)
    from oracle import build as B
    sources = [os.path.join(ORACLE, s) for s in B.SOURCES]
    out = {}
    jobs = []
    for name, defines in (("double", []), ("complex", ["-DORC_CS"])):
        out[name] = str(tmp_path / f"liborc_{name}.so")
        jobs.append(subprocess.Popen(["gcc", "-O1", "-g", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                                      "-fsanitize=address,undefined", "-fno-omit-frame-pointer", *defines,
                                      "-o", out[name], *sources, "-lm"]))
    assert all(j.wait() == 0 for j in jobs)
    env = dict(os.environ, LD_PRELOAD=f"{ASAN}:{UBSAN}",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "host", "sanitize_oracle.py"), out["double"],
                        out["complex"]], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.returncode, r.stdout[-2000:], r.stderr[-4000:])
