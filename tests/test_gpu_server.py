"""The continuous-batching server (abcmb_server_*): every result is the same
alone and in a mix of requests of other sizes -- within the ODE tolerance,
since requests of one shape run as one batch and the integrator's switch
from implicit to explicit steps is taken per warp --, the mix is admitted by
the arena budget, results agree with the plain mixed-precision pipeline on
the same inputs, and a served request of the single-cosmology TT workload
agrees with the FP64 oracle within the mixed path's 1e-4."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2602_15104_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    abcmb.lib()
    return abcmb


def drain(srv, n, timeout=600.0):
    out, t0, peak = {}, time.time(), 0
    while len(out) < n:
        peak = max(peak, srv.progress())
        r = srv.poll()
        while r is not None:
            out[r[0]] = r
            r = srv.poll()
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(out)} of {n} results after {timeout} s")
        time.sleep(0.002)
    return out, peak


def cl_errors(C, ref):
    tt = np.abs(C[0] - ref[0]) / np.abs(ref[0])
    ee = np.abs(C[2] - ref[2]) / np.abs(ref[2])
    te = np.abs(C[1] - ref[1]) / np.sqrt(np.abs(ref[0] * ref[2]))
    return max(tt.max(), te.max(), ee.max())


def test_result_same_alone_and_in_a_mix(A):
    o = A.options(lmax_hier=30, n_tau=2000)
    params = W.draw_cosmologies(8, 20260105)
    sizes = [(500, 80), (1000, 160), (300, 48), (800, 120), (500, 80), (1200, 192), (400, 64), (700, 112)]
    arena = 8 * max(A.server_request_bytes(o, lm, nk) for lm, nk in sizes)
    srv = A.Server(arena, 8, 1200, 192, o)
    try:
        srv.submit(0, params[0], *sizes[0], 1e-5, 0.5)
        alone, _ = drain(srv, 1)
        for i in range(8):
            srv.submit(100 + i, params[i], *sizes[i], 1e-5, 0.5)
        mix, peak = drain(srv, 8)
    finally:
        srv.close()
    assert peak > 1  # requests really overlapped
    assert alone[0][1] == A.OK and all(r[1] == A.OK for r in mix.values())
    # request 100 ran in one batch with request 104 (same shape), request 0 alone
    assert cl_errors(mix[100][2], alone[0][2]) < 1e-5
    # request 4 repeats request 0's shape with another cosmology: a different result
    assert cl_errors(mix[104][2], mix[100][2]) > 1e-3
    # against the plain mixed-precision pipeline on the same cosmologies and grid
    # (the server lays out its k grid on the host, the pipeline takes numpy's:
    # last-bit differences in k can change an adaptive step, ~rtol in C_l)
    o500 = A.options(lmax_hier=30, n_tau=2000, lmax_cl=500)
    pipe = A.Pipeline(2, W.log_k_nodes(80, 1e-5, 0.5), o500, mixed=True)
    C = pipe.run(torch.tensor(params[[0, 4]], device="cuda")).cpu().numpy()
    assert cl_errors(mix[100][2], C[0]) < 1e-6
    assert cl_errors(mix[104][2], C[1]) < 1e-6


def test_requests_of_one_shape_run_as_a_batch(A):
    o = A.options(lmax_hier=30, n_tau=2000)
    params = W.draw_cosmologies(12, 31)
    srv = A.Server(16 * A.server_request_bytes(o, 400, 64), 4, 400, 64, o)
    try:
        for i in range(12):
            srv.submit(i, params[i], 400, 64, 1e-5, 0.5)
        n0 = srv.progress()  # one admission pass: a batch of eight, then the other four
        res, _ = drain(srv, 12)
    finally:
        srv.close()
    assert n0 == 12
    assert all(r[1] == A.OK for r in res.values())
    o400 = A.options(lmax_hier=30, n_tau=2000, lmax_cl=400)
    pipe = A.Pipeline(8, W.log_k_nodes(64, 1e-5, 0.5), o400, mixed=True)
    C = pipe.run(torch.tensor(params[:8], device="cuda")).cpu().numpy()
    for i in range(8):  # the first batch is the batched pipeline's, up to the k grids' last bits
        assert cl_errors(res[i][2], C[i]) < 1e-6


def test_served_small_tt_request_against_the_oracle(A):
    wl = W.SMALL_TT
    o = A.options(lmax_hier=wl.l_max_hier, n_tau=wl.n_tau)
    p = wl.params()[0]
    srv = A.Server(2 * A.server_request_bytes(o, wl.l_max_cl, wl.n_k), 2, wl.l_max_cl, wl.n_k, o)
    try:
        srv.submit(7, p, wl.l_max_cl, wl.n_k, wl.k_min, wl.k_max)
        res, _ = drain(srv, 1)
    finally:
        srv.close()
    assert res[7][1] == A.OK
    ref = O.run(p, wl.k(), wl.n_tau, wl.l_max_cl, O.opts(lmax=wl.l_max_hier), want=("Cl",))["Cl"]
    assert cl_errors(res[7][2], ref) < 1e-4


def test_admission_by_arena_budget(A):
    o = A.options(lmax_hier=30, n_tau=2000)
    req = A.server_request_bytes(o, 600, 96)
    srv = A.Server(2 * req + 4096, 6, 600, 96, o)  # room for two requests at a time
    params = W.draw_cosmologies(5, 7)
    try:
        for i in range(5):
            assert srv.submit(i, params[i], 600, 96, 1e-5, 0.5) == A.OK
        # a request that can never fit is refused at submission
        assert srv.submit(99, params[0], 600, 96 * 3, 1e-5, 0.5) in (A.E_INVALID_ARG, A.E_SCRATCH_TOO_SMALL)
        res, peak = drain(srv, 5)
    finally:
        srv.close()
    assert peak <= 2
    assert sorted(res) == list(range(5))
    assert all(r[1] == A.OK for r in res.values())


def test_a_failing_request_is_reported_and_leaves_the_others_intact(A):
    o = A.options(lmax_hier=30, n_tau=2000)
    params = W.draw_cosmologies(3, 11)
    bad = params[1].copy()
    bad[5] = 5.0  # tau_reio no reionization history can reach: the background fails
    srv = A.Server(4 * A.server_request_bytes(o, 400, 64), 3, 400, 64, o)
    try:
        srv.submit(0, params[0], 400, 64, 1e-5, 0.5)
        srv.submit(1, bad, 400, 64, 1e-5, 0.5)
        srv.submit(2, params[2], 400, 64, 1e-5, 0.5)
        res, _ = drain(srv, 3)
        srv.submit(10, params[0], 400, 64, 1e-5, 0.5)
        alone, _ = drain(srv, 1)
    finally:
        srv.close()
    assert res[0][1] == A.OK and res[2][1] == A.OK
    assert res[1][1] != A.OK
    assert cl_errors(res[0][2], alone[10][2]) < 1e-5
