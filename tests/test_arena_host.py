"""Host logic of the spectrum server: its first-fit arena allocator
(abcmb_arena.h, built for the host) against a plain model of the free list,
over seeded random admission/retirement sequences."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
S = ctypes.c_size_t


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("arena") / "libarena.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "arena_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_arena_init.argtypes = [S]
    L.h_arena_alloc.argtypes = [S, ctypes.POINTER(S)]
    L.h_arena_release.argtypes = [S, S]
    L.h_arena_largest.restype = S
    L.h_arena_size.restype = S
    return L


def gran(n):
    return (n + 255) // 256 * 256


class Model:
    """Free list as sorted (offset, length) pairs, coalesced."""

    def __init__(self, size):
        self.free = [(0, size)]

    def alloc(self, n):
        n = gran(n)
        for i, (o, l) in enumerate(self.free):
            if l >= n:
                self.free[i] = (o + n, l - n)
                if l == n:
                    del self.free[i]
                return o
        return None

    def release(self, off, n):
        self.free.append((off, gran(n)))
        self.free.sort()
        merged = [self.free[0]]
        for o, l in self.free[1:]:
            if merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((o, l))
        self.free = merged

    def largest(self):
        return max((l for _, l in self.free), default=0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_first_fit_with_coalescing_matches_the_model(H, seed):
    rng = np.random.default_rng(seed)
    size = 1 << 24
    H.h_arena_init(size + 100)  # rounded down to the 256-byte granule
    assert H.h_arena_size() == size
    m = Model(size)
    live = []
    for _ in range(3000):
        if live and (rng.random() < 0.45 or len(live) > 60):
            off, n = live.pop(int(rng.integers(len(live))))
            H.h_arena_release(off, n)
            m.release(off, n)
        else:
            n = int(rng.integers(1, 1 << 20))
            got = S(0)
            ok = H.h_arena_alloc(n, ctypes.byref(got))
            want = m.alloc(n)
            assert bool(ok) == (want is not None)
            if ok:
                assert got.value == want and got.value % 256 == 0 and got.value + gran(n) <= size
                live.append((got.value, n))
        assert H.h_arena_largest() == m.largest()
    # live blocks never overlap
    spans = sorted((o, o + gran(n)) for o, n in live)
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    for off, n in live:
        H.h_arena_release(off, n)
    assert H.h_arena_largest() == size  # everything coalesced back
