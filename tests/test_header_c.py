"""The C ABI's header as a C program sees it: include/abcmb.h compiles as
strict ISO C (C99 and C11, -pedantic, warnings as errors) and as C++, and
every layout the Python binding mirrors in ctypes -- abcmb_options' size and
field offsets, the status codes, the background record's constants and its
scalar slots -- equals what the C compiler lays out (tests/host/abi_layout.c).
A field added to the header but not to the binding, or one reordered, shifts
an offset and fails here on the CPU, where on the GPU it would have passed
wrong options to every call."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
SOURCE = os.path.join(ROOT, "tests", "host", "abi_layout.c")

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")


def _compiled(tmp_path, std):
    exe = str(tmp_path / f"abi_layout_{std}")
    subprocess.check_call(["gcc", f"-std={std}", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I" + INCLUDE,
                           SOURCE, "-o", exe])
    out = subprocess.check_output([exe], text=True)
    return dict(line.split() for line in out.splitlines())


@pytest.fixture(scope="module")
def seen(tmp_path_factory):
    d = tmp_path_factory.mktemp("abi_layout")
    c99, c11 = _compiled(d, "c99"), _compiled(d, "c11")
    assert c99 == c11
    return c99


def test_the_header_builds_as_cxx(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "use.cpp"
    # every entry point keeps C linkage inside a C++ translation unit
    src.write_text('#include "abcmb.h"\nint main() { abcmb_options o; abcmb_default_options(&o); return 0; }\n')
    subprocess.check_call(["g++", "-std=c++17", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I" + INCLUDE,
                           "-c", str(src), "-o", str(tmp_path / "use.o")])
    syms = subprocess.check_output(["nm", str(tmp_path / "use.o")], text=True)
    assert " U abcmb_default_options" in syms  # unmangled


def test_options_layout_matches_the_binding(seen):
    from paper_2602_15104_gb300.abcmb import Options
    assert int(seen["sizeof.abcmb_options"]) == ctypes.sizeof(Options)
    names = [f for f, _ in Options._fields_]
    assert sorted(k[len("offset."):] for k in seen if k.startswith("offset.")) == sorted(names)
    for f in names:
        assert int(seen["offset." + f]) == getattr(Options, f).offset, f


def test_constants_match_the_binding(seen):
    from paper_2602_15104_gb300 import abcmb as A
    codes = dict(ABCMB_OK=A.OK, ABCMB_E_INVALID_ARG=A.E_INVALID_ARG, ABCMB_E_CUDA=A.E_CUDA,
                 ABCMB_E_MAX_STEPS=A.E_MAX_STEPS, ABCMB_E_NONFINITE=A.E_NONFINITE,
                 ABCMB_E_BACKGROUND=A.E_BACKGROUND, ABCMB_E_SCRATCH_TOO_SMALL=A.E_SCRATCH_TOO_SMALL,
                 ABCMB_NPARAM=A.NPARAM, ABCMB_NOALLOC_SCRATCH_BYTES=A.NOALLOC_SCRATCH_BYTES,
                 ABCMB_BG_NSCALAR=A.BG_NSCALAR, ABCMB_BG_PER_UNIT=A.BG_PER_UNIT, ABCMB_BG_NLNA=A.BG_NLNA,
                 ABCMB_BG_TABLE=A.BG_TABLE, ABCMB_BG_ODETAB=A.BG_ODETAB, ABCMB_BG_NODES=A.BG_NODES,
                 ABCMB_BG_ODEPOLY_DOUBLES=A.BG_ODEPOLY_DOUBLES)
    for name, value in codes.items():
        assert int(seen[name]) == value, name
    assert float(seen["ABCMB_BG_LNA0"]) == A.BG_LNA0
    assert int(seen["ABCMB_BG_LEN(6000)"]) == A.BG_NODES + 8 * 6000 + A.BG_ODEPOLY_DOUBLES
    for name, slot in A.S_INDEX.items():
        assert int(seen["ABCMB_S_" + name]) == slot, name
    # the scalar slots fit the record's scalar block
    assert int(seen["ABCMB_S_COUNT"]) <= A.BG_NSCALAR
    assert set(A.ERRORS) == set(range(1, A.E_SCRATCH_TOO_SMALL + 1))
