"""Calls into an AddressSanitizer / UndefinedBehaviorSanitizer build of one
host harness (run by tests/test_sanitized_kernels_host.py in a subprocess with
the sanitizer runtimes preloaded): the emulated kernels on small, ragged
shapes, every buffer its own allocation, so that a read or write past any
buffer the kernels index, or undefined behaviour in their arithmetic, ends
the process with the sanitizer's report.

usage: python sanitize_calls.py <harness> <path to the instrumented .so>
       [<path to the instrumented background harness, for adjwarp>]
"""
import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))
from paper_2602_15104_gb300 import workload as W  # noqa: E402

P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
# a lighter set of the same paths, for ThreadSanitizer (tens of times slower)
LIGHT = os.environ.get("SANITIZE_LIGHT") == "1"


def ptr(a):
    return a.ctypes.data_as(P)


def own(a):
    """a copy in a buffer of exactly its size"""
    return np.array(a, copy=True, order="C")


def records(H, params, n_tau, build):
    H.h_bg_len.restype = ctypes.c_long
    out = []
    for p in np.atleast_2d(params):
        r = np.zeros(H.h_bg_len(n_tau))
        build(own(p), r)
        out.append(r)
    return own(np.stack(out))


def quad(H):
    H.h_build_bg.argtypes = [P, I, P]
    H.h_quad.argtypes = [I, P, P, I, I, D, D, I, D, I, P, P, P]
    H.h_quad_pk.argtypes = [I, P, P, I, I, D, D, I, D, D, P, P, P]
    H.h_quad_dm.argtypes = [I, P, P, I, I, D, D, I, D, P, P]
    n_tau, rtol = (40, 1e-4) if LIGHT else (157, 1e-5)
    bg = records(H, W.BATCH64.params()[:3], n_tau, lambda p, r: H.h_build_bg(ptr(p), n_tau, ptr(r)))
    k = own([0.002, 0.03])
    cases = [(12, 0), (30, 1)] if LIGHT else [(12, 0), (30, 0), (30, 1), (50, 2)]
    for L, n_wide in cases:
        S, st, steps = np.zeros((3, 2, n_tau, 3)), np.zeros((3, 2), np.int32), np.zeros((3, 2, 2), np.int32)
        H.h_quad(3, ptr(bg), ptr(k), 2, L, rtol, 1e-12, 2_000_000, 1e-4, n_wide, ptr(S), ptr(st), ptr(steps))
        assert np.all(st == 0), (L, n_wide, st)
    Pk, st = np.zeros((3, 2)), np.zeros((3, 2), np.int32)
    H.h_quad_pk(3, ptr(bg), ptr(k), 2, 12, rtol, 1e-12, 2_000_000, 1e-4, 0.5, ptr(Pk), ptr(st), None)
    Dm = np.zeros((3, 2, n_tau))
    H.h_quad_dm(3, ptr(bg), ptr(k), 2, 12, rtol, 1e-12, 2_000_000, 1e-4, ptr(Dm), ptr(st))
    S, st, steps = np.zeros((1, 1, n_tau, 3)), np.zeros((1, 1), np.int32), np.zeros((1, 1, 2), np.int32)
    H.h_quad(1, ptr(own(bg[:1])), ptr(own([0.05])), 1, 12, 1e-6, 1e-12, 40, 1e-4, 0, ptr(S), ptr(st), ptr(steps))
    assert st[0, 0] == 3  # the step budget
    # the smallest shapes: one cosmology, one k, the minimum of 8 tau nodes, hierarchy 4
    bg8 = records(H, W.BATCH64.params()[5:6], 8, lambda p, r: H.h_build_bg(ptr(p), 8, ptr(r)))
    S = np.zeros((1, 1, 8, 3))
    H.h_quad(1, ptr(bg8), ptr(own([1e-3])), 1, 4, 1e-5, 1e-12, 2_000_000, 1e-4, 0, ptr(S), ptr(st), ptr(steps))
    assert st[0, 0] == 0


def spectra(H):
    H.h_build_bg.argtypes = [P, I, P]
    H.h_project.argtypes = [I, P, P, P, I, I, D, P]
    H.h_project_interp.argtypes = [I, P, P, P, I, P, I, I, D, P]
    H.h_cl.argtypes = [I, P, P, P, I, I, P]
    n_tau, lmax = 333, 257
    bg = records(H, W.BATCH64.params()[:2], n_tau, lambda p, r: H.h_build_bg(ptr(p), n_tau, ptr(r)))
    k = own([1e-5, 3e-4, 0.01, 0.2, 0.5])
    S = own(np.stack([W.synthetic_sources(k.size, n_tau, b) for b in range(2)]))
    Dl = np.zeros((2, k.size, lmax - 1, 2))
    H.h_project(2, ptr(bg), ptr(S), ptr(k), k.size, lmax, 1.0, ptr(Dl))
    kt = own([2e-5, 1e-3, 0.3])
    Dt = np.zeros((2, kt.size, lmax - 1, 2))
    H.h_project_interp(2, ptr(bg), ptr(S), ptr(k), k.size, ptr(kt), kt.size, lmax, 1.0, ptr(Dt))
    C = np.zeros((2, 3, lmax - 1))
    H.h_cl(2, ptr(bg), ptr(Dl), ptr(k), k.size, lmax, ptr(C))
    assert np.isfinite(C).all()
    # the smallest shapes: 8 nodes, l = 2 alone and l <= 3, two k, one below the series limit
    bg8 = records(H, W.BATCH64.params()[5:6], 8, lambda p, r: H.h_build_bg(ptr(p), 8, ptr(r)))
    k2 = own([1e-6, 0.4])
    S8 = own(W.synthetic_sources(2, 8, 9)[None])
    for lm in (2, 3):
        D8, C8 = np.zeros((1, 2, lm - 1, 2)), np.zeros((1, 3, lm - 1))
        H.h_project(1, ptr(bg8), ptr(S8), ptr(k2), 2, lm, 1.0, ptr(D8))
        H.h_cl(1, ptr(bg8), ptr(D8), ptr(k2), 2, lm, ptr(C8))
        assert np.isfinite(C8).all()


def mixed(H):
    H.h_build_bg.argtypes = [P, I, P]
    H.h_project_mixed.argtypes = [I, P, P, P, I, I, D, P]
    H.h_cl_mixed.argtypes = [I, P, P, P, I, I, P]
    n_tau, lmax = 333, 257
    bg = records(H, W.BATCH64.params()[:2], n_tau, lambda p, r: H.h_build_bg(ptr(p), n_tau, ptr(r)))
    k = own([1e-5, 0.01, 0.5])
    S = own(np.stack([W.synthetic_sources(k.size, n_tau, b) for b in range(2)]))
    Dl = np.zeros((2, k.size, lmax - 1, 2), np.float32)
    H.h_project_mixed(2, ptr(bg), ptr(S), ptr(k), k.size, lmax, 1.0, ptr(Dl))
    C = np.zeros((2, 3, lmax - 1))
    H.h_cl_mixed(2, ptr(bg), ptr(Dl), ptr(k), k.size, lmax, ptr(C))
    assert np.isfinite(C).all()
    bg8 = records(H, W.BATCH64.params()[5:6], 8, lambda p, r: H.h_build_bg(ptr(p), 8, ptr(r)))
    k2 = own([1e-6, 0.4])
    S8 = own(W.synthetic_sources(2, 8, 9)[None])
    for lm in (2, 3):
        D8, C8 = np.zeros((1, 2, lm - 1, 2), np.float32), np.zeros((1, 3, lm - 1))
        H.h_project_mixed(1, ptr(bg8), ptr(S8), ptr(k2), 2, lm, 1.0, ptr(D8))
        H.h_cl_mixed(1, ptr(bg8), ptr(D8), ptr(k2), 2, lm, ptr(C8))
        assert np.isfinite(C8).all()


def grad(H):
    H.h_build_bg.argtypes = [P, I, P]
    H.h_project_adjoint.argtypes = [I, P, P, P, I, I, D, P, P, P]
    H.h_cl_adjoint.argtypes = [I, P, P, P, I, I, P, P, P]
    H.h_record_vjp.argtypes = [I, ctypes.c_long, P, P, P, P, P]
    n_tau, lmax = 333, 257
    bg = records(H, W.BATCH64.params()[3:4], n_tau, lambda p, r: H.h_build_bg(ptr(p), n_tau, ptr(r)))
    k = own([1e-5, 0.01, 0.5])
    S = own(W.synthetic_sources(k.size, n_tau, 2)[None])
    rng = np.random.default_rng(0)
    Db, Sb, rb = rng.normal(size=(1, k.size, lmax - 1, 2)), np.zeros_like(S), np.zeros_like(bg)
    H.h_project_adjoint(1, ptr(bg), ptr(S), ptr(k), k.size, lmax, 1.0, ptr(Db), ptr(Sb), ptr(rb))
    Cb, Dbar = rng.normal(size=(1, 3, lmax - 1)), np.zeros_like(Db)
    H.h_cl_adjoint(1, ptr(bg), ptr(Db), ptr(k), k.size, lmax, ptr(Cb), ptr(Dbar), ptr(rb))
    n = 777
    g = np.zeros((2, 6))
    H.h_record_vjp(2, n, ptr(rng.normal(size=(2, n))), ptr(rng.normal(size=(2, 6, n))),
                   ptr(rng.normal(size=(2, 6, n))), ptr(rng.uniform(1e-3, 1e-2, size=(2, 6))), ptr(g))
    assert np.isfinite(rb).all() and np.isfinite(g).all()
    # the ODE passes of the gradient, two one-warp modes per CTA: the counting
    # pass of taped_kernel, and plain_kernel (the massive-neutrino forward,
    # here on a massless record)
    H.h_taped.argtypes = [I, P, P, I, I, D, D, I, P, P, P, P, P]
    H.h_plain.argtypes = [I, P, P, I, I, I, D, D, I, P, P, P, P]
    H.h_grad_layout_bytes.restype = ctypes.c_size_t
    H.h_grad_layout_bytes.argtypes = [I, I, I, ctypes.c_long, ctypes.c_long]
    n_tau = 40
    bg2 = records(H, W.BATCH64.params()[:2], n_tau, lambda p, r: H.h_build_bg(ptr(p), n_tau, ptr(r)))
    k2 = own([0.01, 0.05])
    S, st, acc = np.zeros((2, 2, n_tau, 3)), np.zeros((2, 2), np.int32), np.zeros((2, 2), np.int32)
    ws = np.zeros(H.h_grad_layout_bytes(2, 2, 8, 0, 0) // 8 + 1)
    H.h_taped(2, ptr(bg2), ptr(k2), 2, 8, 1e-4, 1e-14, 10_000_000, ptr(S), ptr(st), ptr(ws), None, ptr(acc))
    assert np.all(st == 0) and np.all(acc > 0)
    # then the recording pass and the reverse sweep in the planned workspace
    H.h_make_plan.restype = ctypes.c_size_t
    H.h_make_plan.argtypes = [I, I, I, P, P]
    H.h_adjoint.argtypes = [I, P, P, I, I, P, P, P, P]
    plan = np.zeros(2 * 4 + 2, np.int64)
    ws = np.zeros(H.h_make_plan(2, 2, 8, ptr(acc), ptr(plan)) // 8 + 1)
    H.h_taped(2, ptr(bg2), ptr(k2), 2, 8, 1e-4, 1e-14, 10_000_000, ptr(S), ptr(st), ptr(ws), ptr(plan), None)
    Sb2, rb2 = own(rng.normal(size=S.shape)), np.zeros_like(bg2)
    H.h_adjoint(2, ptr(bg2), ptr(k2), 2, 8, ptr(Sb2), ptr(ws), ptr(plan), ptr(rb2))
    assert np.all(st == 0) and np.isfinite(rb2).all()
    work = np.zeros(2 * 2 * 64 * (4 + 3 * 9))  # at least V_COUNT (32) vectors of N per mode
    steps = np.zeros((2, 2, 2), np.int32)
    H.h_plain(2, ptr(bg2), ptr(k2), 2, 8, 0, 1e-4, 1e-14, 10_000_000, ptr(S), ptr(st), ptr(steps), ptr(work))
    assert np.all(st == 0)


def lens(H):
    from test_lensing_host import spectra as synthetic_spectra
    H.h_lens.argtypes = [I, P, I, P, I, I, P]
    L, lout = 150, 100
    sp = [synthetic_spectra(L, 7 + b) for b in range(2)]
    Cl = own(np.stack([np.stack([s[0][2:], s[2][2:], s[1][2:]]) for s in sp]))
    Cpsi = own(np.stack([s[3][2:] for s in sp]))
    out = np.zeros((2, 4, lout - 1))
    H.h_lens(2, ptr(Cl), L, ptr(Cpsi), lout, L + 37, ptr(out))
    assert np.isfinite(out).all()


def bgwarp(H):
    H.h_bg_len.restype = ctypes.c_long
    H.h_build_bg_warp.argtypes = [P, I, D, I, P]
    for b, m, recipe, n_tau in [(0, 0.0, 0, 101), (17, 0.06, 1, 64)]:
        r = np.zeros(H.h_bg_len(n_tau))
        H.h_build_bg_warp(ptr(own(W.BATCH64.params()[b])), n_tau, m, recipe, ptr(r))
        assert r[0] == 0


def adjwarp(H):
    H.h_bg_len.restype = ctypes.c_long
    H.h_fwd_warp.argtypes = [P, D, I, D, P, P]
    H.h_grad_warp.argtypes = [P, D, I, D, P, P]
    # the adjoint harness has no background builder: the record comes from
    # the instrumented background harness, argv[3]
    lib = ctypes.CDLL(sys.argv[3])
    lib.h_bg_len.restype = ctypes.c_long
    lib.h_build_bg_warp.argtypes = [P, I, D, I, P]
    n_tau, rtol = (30, 1e-3) if LIGHT else (60, 1e-4)
    r = np.zeros(lib.h_bg_len(n_tau))
    lib.h_build_bg_warp(ptr(own(W.BATCH64.params()[0])), n_tau, 0.0, 0, ptr(r))
    S, sig = np.zeros((n_tau, 3)), np.zeros(3, np.int32)
    assert H.h_fwd_warp(ptr(r), 0.05, 8, rtol, ptr(S), ptr(sig)) == 0
    Sb, rb = own(np.random.default_rng(1).normal(size=(n_tau, 3))), np.zeros_like(r)
    assert H.h_grad_warp(ptr(r), 0.05, 8, rtol, ptr(Sb), ptr(rb)) == 0
    assert np.isfinite(rb).all()


def ode(H):
    # the thread-per-mode solver (hierarchies 64..128), one lane
    H.h_bg_len.restype = ctypes.c_long
    H.h_build_bg.argtypes = [P, I, P]
    H.h_integrate.argtypes = [P, D, I, D, P, P]
    n_tau = 77
    r = np.zeros(H.h_bg_len(n_tau))
    H.h_build_bg(ptr(own(W.BATCH64.params()[2])), n_tau, ptr(r))
    for k, L in [(3e-4, 64), (0.02, 90)]:
        S, steps = np.zeros((n_tau, 3)), np.zeros(2, np.int32)
        assert H.h_integrate(ptr(r), k, L, 1e-5, ptr(S), ptr(steps)) == 0
    H.h_integrate_batch.argtypes = [P, P, I, I, D, P, P]
    k = own([3e-4, 1e-3, 5e-3])  # three modes interleaved in one workspace, at once
    S, st = np.zeros((3, n_tau, 3)), np.zeros(3, np.int32)
    H.h_integrate_batch(ptr(r), ptr(k), 3, 66, 1e-5, ptr(S), ptr(st))
    assert np.all(st == 0)


def arena(H):
    # the serving arena's first-fit allocator under a seeded random workload
    H.h_arena_init.argtypes = [ctypes.c_size_t]
    H.h_arena_alloc.argtypes = [ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    H.h_arena_release.argtypes = [ctypes.c_size_t, ctypes.c_size_t]
    H.h_arena_largest.restype = H.h_arena_size.restype = ctypes.c_size_t
    rng = np.random.default_rng(3)
    H.h_arena_init(1 << 20)
    live = []
    for _ in range(4000):
        if live and rng.uniform() < 0.45:
            off, n = live.pop(rng.integers(len(live)))
            H.h_arena_release(off, n)
        else:
            n, got = int(rng.integers(1, 40000)), ctypes.c_size_t()
            if H.h_arena_alloc(n, ctypes.byref(got)):
                live.append((got.value, n))
    for off, n in live:
        H.h_arena_release(off, n)
    assert H.h_arena_largest() == H.h_arena_size()


def server(H):
    # the serving runtime over its stand-in CUDA runtime: mixed shapes queued,
    # batched, admitted to a small arena and retired until all are served
    from test_server_host import Run
    H.h_arena.restype = P
    H.h_arena.argtypes = [ctypes.c_size_t]
    H.h_free.argtypes = [P]
    H.h_reset.argtypes = [P, ctypes.c_size_t, I]
    H.h_launch.argtypes = [I, P, P]
    H.abcmb_server_request_bytes.restype = ctypes.c_size_t
    H.abcmb_server_create.argtypes = [P, ctypes.c_size_t, I, I, I, P, ctypes.POINTER(P)]
    H.abcmb_server_destroy.argtypes = [P]
    H.abcmb_server_submit.argtypes = [P, ctypes.c_longlong, P, I, I, D, D]
    H.abcmb_server_progress.argtypes = [P]
    H.abcmb_server_poll.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I), ctypes.POINTER(I), P,
                                    ctypes.c_size_t]
    rng = np.random.default_rng(2)
    r = Run(H, 120 << 20, slots=3)
    for tag in range(30):
        lm, nk = [(100, 16), (100, 32), (300, 8)][rng.integers(3)]
        assert r.submit(tag, own([float(tag), 0.12, 0.7, 0.96, 3.0, 0.06]), lm, nk) == 0
    assert len(r.drain(30)) == 30
    assert H.h_violations() == 0
    r.close()


if __name__ == "__main__":
    which, so = sys.argv[1], sys.argv[2]
    globals()[which](ctypes.CDLL(so))
    print("ok")
