"""Every entry point include/abcmb.h declares is declared to ctypes by the
Python binding with the same parameters, in the same order and of matching
C types, and with the declared return type (CPU, no library needed: the
binding's loader runs against a stand-in that keeps what it is given).

ctypes trusts what it is told: a size_t passed where argtypes say int, or
an argument left out, reaches the entry point as garbage in a register
rather than as an error.  The header is parsed for its prototypes; each
parameter's C type is mapped to the ctypes types that carry it correctly --
a pointer may go as c_void_p or as a pointer to its pointee type, the
options always as a pointer to the binding's Options structure."""
import ctypes
import os
import re
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "abcmb.h")

SCALARS = {"int": ctypes.c_int, "size_t": ctypes.c_size_t, "double": ctypes.c_double,
           "long long": ctypes.c_longlong, "float": ctypes.c_float}


def prototypes():
    """name -> (return type, [(base type, pointer depth, parameter name)])"""
    src = re.sub(r"/\*.*?\*/", " ", open(HEADER).read(), flags=re.S)
    src = "\n".join(line for line in src.splitlines() if not line.lstrip().startswith("#"))
    src = src.replace('extern "C" {', " ")
    out = {}
    for chunk in src.split(";"):
        m = re.fullmatch(r"\s*([A-Za-z_][\w ]*?)\s*(\**)\s*\b(abcmb_\w+)\s*\(([^()]*)\)\s*", chunk, flags=re.S)
        if not m:
            continue
        ret, ret_ptr, name, args = m.groups()
        params = []
        for a in args.split(","):
            a = " ".join(a.split())
            if a in ("", "void"):
                continue
            depth = a.count("*")
            words = [w for w in a.replace("*", " ").split() if w != "const"]
            params.append((" ".join(words[:-1]), depth, words[-1]))
        out[name] = (ret + ret_ptr, params)
    return out


class FakeCDLL:
    """Keeps the argtypes and restype the binding assigns, per symbol."""

    def __init__(self, path):
        self.fns = {}

    def __getattr__(self, name):
        if name.startswith("__"):
            raise AttributeError(name)
        return self.fns.setdefault(name, types.SimpleNamespace(argtypes=None, restype=ctypes.c_int))


@pytest.fixture(scope="module")
def declared():
    protos = prototypes()
    assert len(protos) >= 30  # the parse found the header's entry points
    return protos


@pytest.fixture
def bound(monkeypatch):
    from paper_2602_15104_gb300 import abcmb
    monkeypatch.setattr(abcmb, "_lib", None)
    monkeypatch.setattr(abcmb, "LIB_PATH", HEADER)  # any file that exists
    monkeypatch.setattr(abcmb.ctypes, "CDLL", FakeCDLL)
    L = abcmb.lib()
    monkeypatch.setattr(abcmb, "_lib", None)  # the next real load starts afresh
    return L.fns, abcmb.Options


def carries(ct, base, depth, Options):
    """whether ctypes type ct passes a C parameter of this base type and
    pointer depth as the entry point expects it"""
    if depth == 0:
        return ct is SCALARS[base]
    if base == "abcmb_options":
        return depth == 1 and ct is ctypes.POINTER(Options)
    if depth == 1:
        return ct is ctypes.c_void_p or (base in SCALARS and ct is ctypes.POINTER(SCALARS[base]))
    return depth == 2 and ct is ctypes.POINTER(ctypes.c_void_p)


def test_the_header_parse_is_complete(declared):
    # every name the header writes as a call is a parsed prototype
    src = open(HEADER).read()
    named = set(re.findall(r"^\s*(?:const\s+)?\w[\w ]*?\**\s*\b(abcmb_[a-z_0-9]+)\s*\(", src, flags=re.M))
    assert named <= set(declared), named - set(declared)
    assert declared["abcmb_perturb"][1][9] == ("size_t", 0, "workspace_bytes")


def test_every_entry_point_is_declared_to_ctypes_as_in_the_header(declared, bound):
    fns, Options = bound
    for name, (ret, params) in declared.items():
        assert name in fns, f"{name}: not declared by the binding"
        f = fns[name]
        if params:
            assert f.argtypes is not None, f"{name}: no argtypes"
            assert len(f.argtypes) == len(params), (name, len(f.argtypes), len(params))
            for i, ((base, depth, pname), ct) in enumerate(zip(params, f.argtypes)):
                assert carries(ct, base, depth, Options), (name, i, pname, base, depth, ct)
        if ret == "size_t":
            assert f.restype is ctypes.c_size_t, name
        elif ret == "int":
            assert f.restype is ctypes.c_int, name
        else:
            assert ret == "void", (name, ret)
