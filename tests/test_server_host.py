"""CPU tests of the spectrum server's runtime (abcmb_server.cu: queue,
same-shape batching, first-fit arena admission, slots retired by event query,
results by tag), built for the host over a stand-in CUDA runtime and stand-ins
for the compute calls (tests/host/server_harness.cpp): what the GPU test
tests/test_gpu_server.py cannot see -- which requests went into which batch,
and that no batch's arena span is handed out twice while it is in flight."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
I = ctypes.c_int
OK, E_INVALID_ARG, E_MAX_STEPS, E_BACKGROUND, E_SCRATCH_TOO_SMALL = 0, 1, 3, 5, 6


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("server") / "libserver.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "tests", "host", "fake_cuda"),
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2602_15104_gb300", "csrc"),
                           "-x", "c++", os.path.join(ROOT, "paper_2602_15104_gb300", "csrc", "abcmb_server.cu"),
                           "-x", "none", os.path.join(ROOT, "tests", "host", "server_harness.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    L.h_arena.restype = P
    L.h_arena.argtypes = [ctypes.c_size_t]
    L.h_free.argtypes = [P]
    L.h_reset.argtypes = [P, ctypes.c_size_t, I]
    L.h_launch.argtypes = [I, P, P]
    L.abcmb_server_request_bytes.restype = ctypes.c_size_t
    L.abcmb_server_create.argtypes = [P, ctypes.c_size_t, I, I, I, P, ctypes.POINTER(P)]
    L.abcmb_server_destroy.argtypes = [P]
    L.abcmb_server_submit.argtypes = [P, ctypes.c_longlong, P, I, I, ctypes.c_double, ctypes.c_double]
    L.abcmb_server_progress.argtypes = [P]
    L.abcmb_server_queued.argtypes = [P]
    L.abcmb_server_poll.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I), ctypes.POINTER(I), P,
                                    ctypes.c_size_t]
    return L


def opts(lmax_cl):
    from paper_2602_15104_gb300 import abcmb as A
    return A.options(lmax_hier=12, n_tau=16, lmax_cl=lmax_cl)


class Run:
    def __init__(self, H, arena_bytes, slots, max_lmax=400, max_nk=64, not_ready=2):
        self.H, self.o = H, opts(max_lmax)
        self.arena = H.h_arena(arena_bytes)
        H.h_reset(self.arena, arena_bytes, not_ready)
        self.h = P()
        assert H.abcmb_server_create(self.arena, arena_bytes, slots, max_lmax, max_nk, ctypes.byref(self.o),
                                     ctypes.byref(self.h)) == OK
        self.buf = np.zeros(3 * (max_lmax - 1))

    def submit(self, tag, params, lmax, nk, kmin=1e-5, kmax=0.5):
        p = np.ascontiguousarray(params, dtype=np.float64)
        return self.H.abcmb_server_submit(self.h, tag, p.ctypes.data_as(P), lmax, nk, kmin, kmax)

    def drain(self, n, limit=100000):
        out = {}
        for _ in range(limit):
            assert self.H.abcmb_server_progress(self.h) >= 0
            tag, st, lm = ctypes.c_longlong(), I(), I()
            while self.H.abcmb_server_poll(self.h, ctypes.byref(tag), ctypes.byref(st), ctypes.byref(lm),
                                           self.buf.ctypes.data_as(P), self.buf.size) == 1:
                assert tag.value not in out
                out[tag.value] = (st.value, lm.value, self.buf[:3 * (lm.value - 1)].reshape(3, -1).copy())
            if len(out) == n:
                return out
        raise AssertionError(f"{len(out)} of {n} results")

    def launches(self):
        res = []
        for i in range(self.H.h_launches()):
            info, tags = np.zeros(4, np.int32), np.zeros(8, np.int64)
            self.H.h_launch(i, info.ctypes.data_as(P), tags.ctypes.data_as(P))
            res.append((int(info[0]), int(info[1]), int(info[2]), tags[:info[0]].tolist()))
        return res

    def close(self):
        self.H.abcmb_server_destroy(self.h)
        self.H.h_free(self.arena)


def expected_cl(tag, lmax, nk, kmax):
    q = np.arange(lmax - 1)
    return np.stack([1000.0 * tag + 100.0 * t + q + 1e-3 * nk + 1e-6 * kmax for t in range(3)])


SHAPES = [(100, 16), (100, 32), (200, 32), (300, 8)]  # two share l_max, two share n_k


def test_mixed_requests_are_batched_by_shape_and_all_served(H):
    rng = np.random.default_rng(1)
    r = Run(H, 400 << 20, slots=3)
    reqs = {}
    for tag in range(40):
        lm, nk = SHAPES[rng.integers(len(SHAPES))]
        p = np.array([float(tag), 0.12, 0.7, 0.96, 3.0, 0.06])
        if tag == 7:
            p[5] = 2.0  # a mode runs out of steps
        if tag == 13:
            p[0] = -13.0  # no background
        assert r.submit(tag, p, lm, nk) == OK
        reqs[tag] = (lm, nk)
    out = r.drain(40)
    for tag, (lm, nk) in reqs.items():
        st, lm_got, cl = out[tag]
        assert lm_got == lm
        if tag == 7:
            assert st == E_MAX_STEPS
        elif tag == 13:
            assert st == E_BACKGROUND
        else:
            assert st == OK
            np.testing.assert_allclose(cl, expected_cl(tag, lm, nk, 0.5), rtol=1e-13)
    launches = r.launches()
    served = []
    for B, lm, nk, tags in launches:
        assert 1 <= B <= 8
        tags = [t if t >= 0 else -t for t in tags]  # tag 13 carries -13
        assert all(reqs[t] == (lm, nk) for t in tags)  # one shape per batch
        assert tags == sorted(tags)  # queue order within a batch
        served += tags
    assert sorted(served) == list(range(40))
    assert max(B for B, *_ in launches) == 8  # full batches where the queue allows
    assert H.h_max_inflight() >= 2  # slots overlapped
    assert H.h_violations() == 0  # every span in the arena, none handed out twice
    r.close()


def test_the_head_of_the_queue_waits_for_memory_and_keeps_its_place(H):
    # an arena that holds one large request or a few small ones: the large
    # head waits until the slots drain, then runs before the small ones behind it
    one_large = H.abcmb_server_request_bytes(ctypes.byref(opts(400)), 400, 64)
    r = Run(H, one_large + (1 << 20), slots=4)
    p = np.array([0.0, 0.12, 0.7, 0.96, 3.0, 0.06])
    assert r.submit(0, p, 100, 16) == OK
    big = p.copy()
    big[0] = 1
    assert r.submit(1, big, 400, 64) == OK
    for tag in range(2, 6):
        q = p.copy()
        q[0] = tag
        assert r.submit(tag, q, 100, 16) == OK
    out = r.drain(6)
    assert all(out[t][0] == OK for t in range(6))
    order = [tags for *_, tags in r.launches()]
    first_big = next(i for i, t in enumerate(order) if 1 in t)
    # nothing queued behind the large request ran before it
    assert all(t == 0 for batch in order[:first_big] for t in batch)
    assert H.h_violations() == 0
    r.close()


def test_requests_the_server_cannot_take_are_refused_at_submit(H):
    small = H.abcmb_server_request_bytes(ctypes.byref(opts(100)), 100, 16)
    r = Run(H, small + 4096, slots=2, max_lmax=400, max_nk=64)
    p = np.zeros(6)
    assert r.submit(0, p, 401, 16) == E_INVALID_ARG  # above max_lmax_cl
    assert r.submit(0, p, 100, 65) == E_INVALID_ARG  # above max_n_k
    assert r.submit(0, p, 100, 16, kmin=0.2, kmax=0.1) == E_INVALID_ARG
    assert r.submit(0, p, 400, 64) == E_SCRATCH_TOO_SMALL  # larger than the whole arena
    assert H.abcmb_server_queued(r.h) == 0
    assert r.submit(3, p, 100, 16) == OK
    assert r.drain(1)[3][0] == OK
    r.close()
