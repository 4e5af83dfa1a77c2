"""CPU checks of the Python binding's marshalling (no GPU compute).

Every buffer a call hands the library is held against the extent that
include/abcmb.h gives it ([B][Nk][n_tau][3] sources, [B][abcmb_bg_doubles]
records, ...) before the C entry point is called, so a short tensor is
refused on the host instead of being read or written past its end; a
workspace goes over with its size in bytes whatever its dtype; each
buffer reaches the entry point; and Pipeline hands one set of buffers from
call to call (the background record to every step, the sources to the
projection, the transfer functions to the quadrature), and ClWithGradient
its forward and reverse calls (each adjoint to the next, the tape and its
plan from the taped forward to the reverse sweep).  The compute entry points are replaced by a
recorder and the device test by one that accepts host tensors; the size
queries (abcmb_bg_doubles, the workspace sizes, the gradient plan) are the
real library's host functions.
"""
import ctypes
import os
import shutil

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")

SIZE_QUERIES = {"abcmb_bg_doubles", "abcmb_perturb_workspace_bytes", "abcmb_grad_workspace_bytes",
                "abcmb_grad_count_workspace_bytes", "abcmb_grad_plan", "abcmb_default_options",
                "abcmb_validate_options", "abcmb_transfer_k_grid"}


class Recorder:
    """The library with every compute entry point replaced by a stub that
    records its arguments and returns ABCMB_OK."""

    def __init__(self, real):
        self.real, self.calls = real, []

    def __getattr__(self, name):
        if name in SIZE_QUERIES:
            return getattr(self.real, name)

        def call(*args):
            self.calls.append((name, args))
            return 0
        return call


@pytest.fixture(scope="module")
def real_lib():
    from paper_2602_15104_gb300 import abcmb, build
    build.build()
    return abcmb.lib()


@pytest.fixture
def AR(real_lib, monkeypatch):
    from paper_2602_15104_gb300 import abcmb
    rec = Recorder(real_lib)
    monkeypatch.setattr(abcmb, "lib", lambda: rec)
    monkeypatch.setattr(abcmb, "_stream", lambda: None)
    monkeypatch.setattr(abcmb, "_on_gpu", lambda t: isinstance(t, torch.Tensor) and t.is_contiguous())
    return abcmb, rec


B, NK, NKT, LMAX_PSI, LOUT = 2, 5, 7, 30, 20


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def i32(*shape):
    return torch.zeros(shape, dtype=torch.int32)


def cases(A):
    """name -> (call(buffers), buffers at the sizes abcmb.h gives)."""
    o = A.options(lmax_hier=12, lmax_cl=40, n_tau=64)
    n, nt, L = A.bg_doubles(o), o.n_tau, o.lmax_cl
    k, kt = f64(NK), f64(NKT)
    D = (B, NK, L - 1, 2)
    return {
        "abcmb_background_tables": (
            lambda b: A.abcmb_background_tables(b["params"], o, out=b["bg"]),
            dict(params=f64(B, 6), bg=f64(B, n))),
        "abcmb_perturb": (
            lambda b: A.abcmb_perturb(b["bg"], k, o, S=b["S"], status=b["status"], steps=b["steps"]),
            dict(bg=f64(B, n), S=f64(B, NK, nt, 3), status=i32(B, NK), steps=i32(B, NK, 2))),
        "abcmb_matter_pk": (
            lambda b: A.abcmb_matter_pk(b["bg"], k, o, 0.0, out=b["Pk"], status=b["status"]),
            dict(bg=f64(B, n), Pk=f64(B, NK), status=i32(B, NK))),
        "abcmb_project": (
            lambda b: A.abcmb_project(b["bg"], b["S"], k, o, out=b["Delta"]),
            dict(bg=f64(B, n), S=f64(B, NK, nt, 3), Delta=f64(*D))),
        "abcmb_project_interp": (
            lambda b: A.abcmb_project_interp(b["bg"], b["S"], k, kt, o, out=b["Delta"]),
            dict(bg=f64(B, n), S=f64(B, NK, nt, 3), Delta=f64(B, NKT, L - 1, 2))),
        "abcmb_cl": (
            lambda b: A.abcmb_cl(b["bg"], b["Delta"], k, o, out=b["Cl"]),
            dict(bg=f64(B, n), Delta=f64(*D), Cl=f64(B, 3, L - 1))),
        "abcmb_project_mixed": (
            lambda b: A.abcmb_project_mixed(b["bg"], b["S"], k, o, out=b["Delta32"]),
            dict(bg=f64(B, n), S=f64(B, NK, nt, 3), Delta32=torch.zeros(D, dtype=torch.float32))),
        "abcmb_cl_mixed": (
            lambda b: A.abcmb_cl_mixed(b["bg"], b["Delta32"], k, o, out=b["Cl"]),
            dict(bg=f64(B, n), Delta32=torch.zeros(D, dtype=torch.float32), Cl=f64(B, 3, L - 1))),
        "abcmb_delta_m_nodes": (
            lambda b: A.abcmb_delta_m_nodes(b["bg"], k, o, out=b["Dm"], status=b["status"]),
            dict(bg=f64(B, n), Dm=f64(B, NK, nt), status=i32(B, NK))),
        "abcmb_cl_psi": (
            lambda b: A.abcmb_cl_psi(b["bg"], b["Dm"], k, o, LMAX_PSI, out=b["Cpsi"]),
            dict(bg=f64(B, n), Dm=f64(B, NK, nt), Cpsi=f64(B, LMAX_PSI - 1))),
        "abcmb_lens": (
            lambda b: A.abcmb_lens(b["Cl"], b["Cpsi"], LOUT, out=b["lensed"]),
            dict(Cl=f64(B, 3, L - 1), Cpsi=f64(B, L - 1), lensed=f64(B, 4, LOUT - 1))),
        "abcmb_grad_count_steps": (
            lambda b: A.abcmb_grad_count_steps(b["bg"], k, o, S=b["S"], status=b["status"]),
            dict(bg=f64(B, n), S=f64(B, NK, nt, 3), status=i32(B, NK))),
        "abcmb_perturb_taped": (
            lambda b: A.abcmb_perturb_taped(b["bg"], k, o, f64(16), S=b["S"], status=b["status"]),
            dict(bg=f64(B, n), S=f64(B, NK, nt, 3), status=i32(B, NK))),
        "abcmb_perturb_adjoint": (
            lambda b: A.abcmb_perturb_adjoint(b["bg"], k, o, b["Sbar"], f64(16), b["recbar"]),
            dict(bg=f64(B, n), Sbar=f64(B, NK, nt, 3), recbar=f64(B, n))),
        "abcmb_cl_adjoint": (
            lambda b: A.abcmb_cl_adjoint(b["bg"], b["Delta"], k, o, b["Clbar"], b["recbar"],
                                         Deltabar=b["Deltabar"]),
            dict(bg=f64(B, n), Delta=f64(*D), Clbar=f64(B, 3, L - 1), recbar=f64(B, n), Deltabar=f64(*D))),
        "abcmb_project_adjoint": (
            lambda b: A.abcmb_project_adjoint(b["bg"], b["S"], k, o, b["Deltabar"], b["recbar"], Sbar=b["Sbar"]),
            dict(bg=f64(B, n), S=f64(B, NK, nt, 3), Deltabar=f64(*D), recbar=f64(B, n),
                 Sbar=f64(B, NK, nt, 3))),
        "abcmb_param_stencil": (
            lambda b: A.abcmb_param_stencil(b["params"], 1e-4, 1e-3),
            dict(params=f64(B, 6))),
        "abcmb_record_vjp": (
            lambda b: A.abcmb_record_vjp(o, b["recbar"], b["rec_plus"], b["rec_minus"], b["h"], grad=b["grad"]),
            dict(recbar=f64(1, n), rec_plus=f64(6, n), rec_minus=f64(6, n), h=f64(1, 6), grad=f64(1, 6))),
    }


NAMES = ["abcmb_background_tables", "abcmb_perturb", "abcmb_matter_pk", "abcmb_project", "abcmb_project_interp",
         "abcmb_cl", "abcmb_project_mixed", "abcmb_cl_mixed", "abcmb_delta_m_nodes", "abcmb_cl_psi", "abcmb_lens",
         "abcmb_grad_count_steps", "abcmb_perturb_taped", "abcmb_perturb_adjoint", "abcmb_cl_adjoint",
         "abcmb_project_adjoint", "abcmb_param_stencil", "abcmb_record_vjp"]


def pointers(args):
    return {a.value for a in args if isinstance(a, ctypes.c_void_p) and a.value}


@pytest.mark.parametrize("name", NAMES)
def test_buffers_of_the_declared_size_reach_the_entry_point(AR, name):
    A, rec = AR
    call, bufs = cases(A)[name]
    call(bufs)
    assert [c[0] for c in rec.calls] == [name]
    assert {t.data_ptr() for t in bufs.values()} <= pointers(rec.calls[0][1])


@pytest.mark.parametrize("name", NAMES)
def test_a_short_buffer_is_refused_before_the_call(AR, name):
    A, rec = AR
    call, bufs = cases(A)[name]
    for key, t in bufs.items():
        short = dict(bufs)
        short[key] = torch.zeros(t.numel() - 1, dtype=t.dtype)
        with pytest.raises(ValueError):
            call(short)
        assert rec.calls == [], (name, key)


def test_wrong_dtype_and_layout_are_refused(AR):
    A, rec = AR
    call, bufs = cases(A)["abcmb_perturb"]
    for key, dt in (("status", torch.int64), ("S", torch.float32)):
        bad = dict(bufs)
        bad[key] = torch.zeros(bufs[key].shape, dtype=dt)
        with pytest.raises(TypeError):
            call(bad)
    bad = dict(bufs)
    bad["S"] = f64(B, NK, 64, 3).transpose(0, 1)  # not contiguous
    with pytest.raises(TypeError):
        call(bad)
    assert rec.calls == []


def test_workspace_goes_over_in_bytes_whatever_its_dtype(AR):
    A, rec = AR
    o = A.options(lmax_hier=80, lmax_cl=40, n_tau=64)
    bg = f64(1, A.bg_doubles(o))
    ws = torch.zeros(1000, dtype=torch.uint8)
    A.abcmb_perturb(bg, f64(3), o, workspace=ws)
    (name, args), = rec.calls
    assert name == "abcmb_perturb" and args[8].value == ws.data_ptr() and args[9] == 1000
    rec.calls.clear()
    A.abcmb_perturb_taped(bg, f64(3), o, torch.zeros(24, dtype=torch.int32))
    assert rec.calls[0][1][8] == 96


def test_a_plan_of_fewer_modes_is_refused(AR):
    A, rec = AR
    o = A.options(lmax_hier=12, lmax_cl=40, n_tau=64)
    acc = torch.full((B, NK), 100, dtype=torch.int32)
    plan, nbytes = A.grad_plan(o, acc)
    assert plan.size == 2 * B * NK + 2 and nbytes > 0
    bg = f64(B, A.bg_doubles(o))
    ws = torch.zeros(nbytes // 8 + 1, dtype=torch.float64)
    with pytest.raises(ValueError):
        A.abcmb_perturb_taped(bg, f64(NK + 1), o, ws, plan=plan)
    with pytest.raises(ValueError):
        A.abcmb_perturb_adjoint(bg, f64(NK), o, f64(B, NK, 64, 3), ws, f64(*bg.shape), plan=plan[:-1].copy())
    assert rec.calls == []
    A.abcmb_perturb_taped(bg, f64(NK), o, ws, plan=plan)
    assert rec.calls[0][1][9].value == plan.ctypes.data


def test_noalloc_checks_types_only(AR):
    A, rec = AR
    o = A.options(lmax_hier=12, lmax_cl=40, n_tau=64)
    bg = f64(1, A.bg_doubles(o))
    with pytest.raises(TypeError):
        A.abcmb_perturb_noalloc(bg, f64(3), o, f64(1), f64(1))
    assert rec.calls == []
    # sizes are left to the library, which refuses a problem beyond its
    # scratch before touching the outputs
    assert A.abcmb_perturb_noalloc(bg, f64(3), o, f64(1), i32(1)) == A.OK
    assert rec.calls[0][0] == "abcmb_perturb_noalloc"


def test_params_must_be_rows_of_six(AR):
    A, rec = AR
    o = A.options(lmax_hier=12, lmax_cl=40, n_tau=64)
    with pytest.raises(ValueError):
        A.abcmb_background_tables(f64(6), o)
    with pytest.raises(ValueError):
        A.abcmb_background_tables(f64(2, 7), o)
    with pytest.raises(ValueError):
        A.abcmb_param_stencil(f64(12), 1e-4, 1e-3)
    assert rec.calls == []
    assert np.array_equal(A.abcmb_background_tables(f64(3, 6), o).shape, (3, A.bg_doubles(o)))


def test_server_submit_takes_six_parameters(AR):
    A, rec = AR
    srv = A.Server.__new__(A.Server)  # no device arena needed to check the arguments
    srv._h = None
    for bad in (np.zeros(5), np.zeros((2, 6)), 3.0):
        with pytest.raises(ValueError):
            srv.submit(1, bad, 100, 8, 1e-4, 0.1)
    assert rec.calls == []
    assert srv.submit(1, np.zeros(6), 100, 8, 1e-4, 0.1) == A.OK
    (name, args), = rec.calls
    assert name == "abcmb_server_submit" and args[3:] == (100, 8, 1e-4, 0.1)


def _args_by_name(name, args):
    from test_binding_signatures import prototypes
    params = prototypes()[name][1]
    assert len(params) == len(args), name
    return {pname: (a.value if isinstance(a, ctypes.c_void_p) else a) for (_, _, pname), a in zip(params, args)}


@pytest.mark.parametrize("mixed", [False, True])
def test_pipeline_threads_its_buffers_through_the_four_calls(AR, mixed):
    A, rec = AR
    o = A.options(lmax_hier=12, lmax_cl=40, n_tau=64)
    pipe = A.Pipeline(B, np.geomspace(1e-4, 0.1, NK), o, device="cpu", mixed=mixed)
    params = f64(B, 6)
    assert pipe.run(params) is pipe.C
    tail = ["abcmb_project_mixed", "abcmb_cl_mixed"] if mixed else ["abcmb_project", "abcmb_cl"]
    assert [c[0] for c in rec.calls] == ["abcmb_background_tables", "abcmb_perturb", *tail]
    bgt, per, proj, cl = (_args_by_name(n, a) for n, a in rec.calls)
    bg, k = pipe.bg.data_ptr(), pipe.k.data_ptr()
    assert bgt["B"] == B and bgt["params"] == params.data_ptr() and bgt["bg"] == bg
    assert per["bg"] == bg and per["k"] == k and per["Nk"] == NK
    assert (per["S"], per["mode_status"], per["steps"]) == (pipe.S.data_ptr(), pipe.status.data_ptr(),
                                                            pipe.steps.data_ptr())
    D = "Delta32" if mixed else "Delta"
    assert proj["bg"] == bg and proj["S"] == pipe.S.data_ptr() and proj["k"] == k and proj["Nk"] == NK
    assert cl["bg"] == bg and cl["k"] == k and cl[D] == proj[D] == pipe.D.data_ptr()
    assert cl["Cl"] == pipe.C.data_ptr()
    assert pipe.D.dtype == (torch.float32 if mixed else torch.float64)
    rec.calls.clear()
    pipe.run()  # no params given: the pipeline's own parameter buffer
    assert _args_by_name(*rec.calls[0])["params"] == pipe.params.data_ptr()


def test_pipeline_status_words_raise(AR):
    A, _ = AR
    pipe = A.Pipeline(B, np.geomspace(1e-4, 0.1, NK), A.options(lmax_hier=12, lmax_cl=40, n_tau=64), device="cpu")
    pipe.bg.zero_()
    pipe.status.zero_()
    pipe.check_status()
    pipe.status[1, 3] = A.E_MAX_STEPS
    with pytest.raises(RuntimeError, match=r"1 modes failed, first \[1, 3\]: step budget"):
        pipe.check_status()
    pipe.bg[1, A.S_INDEX["STATUS"]] = A.E_BACKGROUND
    with pytest.raises(RuntimeError, match=r"background failed for cosmologies \[1\]"):
        pipe.check_status()


class Filler(Recorder):
    """A Recorder whose stubs also write what ClWithGradient reads back on
    the host: clear status words (the background record's and the modes'),
    and a count of accepted steps for the tape plan."""

    def __getattr__(self, name):
        call = super().__getattr__(name)
        if name in SIZE_QUERIES:
            return call

        def fill(*args):
            a = _args_by_name(name, args)
            if name == "abcmb_background_tables":
                ctypes.memset(a["bg"], 0, a["B"] * self.n_bg * 8)
            if "mode_status" in a:
                ctypes.memset(a["mode_status"], 0, a["B"] * a["Nk"] * 4)
            if "accepted" in a:
                acc = np.ctypeslib.as_array((ctypes.c_int32 * (a["B"] * a["Nk"])).from_address(a["accepted"]))
                acc[:] = np.arange(acc.size) + 40  # ragged tapes
            return call(*args)
        return fill


def test_gradient_function_chains_its_calls(real_lib, monkeypatch):
    from paper_2602_15104_gb300 import abcmb as A
    rec = Filler(real_lib)
    monkeypatch.setattr(A, "lib", lambda: rec)
    monkeypatch.setattr(A, "_stream", lambda: None)
    monkeypatch.setattr(A, "_on_gpu", lambda t: isinstance(t, torch.Tensor) and t.is_contiguous())
    o = A.options(lmax_hier=12, lmax_cl=40, n_tau=64)
    rec.n_bg = A.bg_doubles(o)
    params, k = f64(B, 6).requires_grad_(), torch.tensor(np.geomspace(1e-4, 0.1, NK))
    C = A.cl_with_gradient(params, k, o)
    fwd = ["abcmb_background_tables", "abcmb_grad_count_steps", "abcmb_perturb_taped", "abcmb_project", "abcmb_cl"]
    assert [c[0] for c in rec.calls] == fwd
    bg0, cnt, taped, proj, cl = (_args_by_name(n, a) for n, a in rec.calls)
    assert bg0["params"] == params.data_ptr()
    assert cnt["bg"] == taped["bg"] == proj["bg"] == cl["bg"] == bg0["bg"]
    assert taped["S"] == proj["S"] and proj["Delta"] == cl["Delta"] and cl["Cl"] == C.data_ptr()
    # the tapes are sized from the counted steps: the plan's total is the workspace
    acc = np.arange(B * NK, dtype=np.int32) + 40
    plan = np.empty(2 * B * NK + 2, np.int64)
    nb = real_lib.abcmb_grad_plan(B, NK, ctypes.byref(o), acc.ctypes.data_as(ctypes.c_void_p),
                                  plan.ctypes.data_as(ctypes.c_void_p))
    assert nb > 0 and taped["workspace_bytes"] >= nb
    rec.calls.clear()
    Cbar = torch.randn(C.shape, dtype=torch.float64)
    (g,) = torch.autograd.grad(C, params, Cbar)
    back = ["abcmb_cl_adjoint", "abcmb_project_adjoint", "abcmb_perturb_adjoint", "abcmb_param_stencil",
            "abcmb_background_tables", "abcmb_background_tables", "abcmb_record_vjp"]
    assert [c[0] for c in rec.calls] == back
    cla, pra, pea, st, bp, bm, vjp = (_args_by_name(n, a) for n, a in rec.calls)
    assert cla["Clbar"] == Cbar.data_ptr() and cla["Delta"] == cl["Delta"] and cla["bg"] == bg0["bg"]
    assert pra["Deltabar"] == cla["Deltabar"] and pra["S"] == taped["S"]
    assert pea["Sbar"] == pra["Sbar"] and pea["workspace"] == taped["workspace"]
    assert pea["plan_host"] == taped["plan_host"] and pea["workspace_bytes"] == taped["workspace_bytes"]
    assert cla["recbar"] == pra["recbar"] == pea["recbar"] == vjp["recbar"]
    assert st["params"] == params.data_ptr()
    assert bp["params"] == st["params_plus"] and bm["params"] == st["params_minus"]
    assert (vjp["rec_plus"], vjp["rec_minus"], vjp["h"]) == (bp["bg"], bm["bg"], st["h"])
    assert vjp["grad"] == g.data_ptr() and g.shape == (B, 6)
