"""Build the oracle's shared library (test infrastructure only).

Plain gcc, no architecture-specific flags, so that the same source builds on
x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_background.c", "orc_linalg.c", "orc_perturb.c", "orc_spectra.c"]
HEADERS = ["orc.h", "orc_real.h"]
OUT_DIR = os.path.join(HERE, "_lib")
OUT = os.path.join(OUT_DIR, "liborc.so")
# the same sources over double complex: complex-step forward sensitivities (orc_real.h)
OUT_CS = os.path.join(OUT_DIR, "liborc_cs.so")


def _build_one(out: str, defines: list, force: bool) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES + HEADERS]
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
           "-Wno-unused-variable"] + defines + ["-o", tmp] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Both oracle libraries; returns the path of the double one."""
    _build_one(OUT_CS, ["-DORC_CS"], force)
    return _build_one(OUT, [], force)


def build_cs(force: bool = False) -> str:
    return _build_one(OUT_CS, ["-DORC_CS"], force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
