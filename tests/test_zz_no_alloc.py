"""sc_residual_noalloc: the residual call for callers that cannot allocate.

Some callers cannot give the library a device workspace because they may not
allocate GPU memory at all (a host application's allocator owns the device,
or allocation is forbidden in a latency-bound loop).  For them the library
has one extra entry point that keeps its scratch in a fixed array compiled
into the library.  These tests call it through the C ABI and check it against
the ordinary sc_residual on the same inputs, on two calls in a row with
different inputs (so stale scratch from the first call would show), in both
precisions; check that a call takes no device memory once the first call on
the device has loaded the library's device code; and check that a problem
too large for the built-in scratch, or of a shape sc_residual refuses, is
refused before anything runs.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1910_13908_gb300 import build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1910_13908_gb300 import sagecal as sc  # noqa: E402


def entry():
    build.build()
    f = sc.lib().sc_residual_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [ctypes.POINTER(sc.Dims), vp, vp, vp, vp, vp, ctypes.c_int32, vp, ctypes.c_char_p,
                  ctypes.c_size_t]
    f.restype = ctypes.c_int32
    return f


def call_noalloc(f, shp, X, C, J, prec, want_R=True, R=None, cost=None):
    if R is None and want_R:
        R = torch.empty_like(X)
    if cost is None:
        cost = torch.zeros((), dtype=torch.float64, device=X.device)
    err = ctypes.create_string_buffer(256)
    d = sc.Dims(shp.N, shp.T, shp.F, 1, 0)
    rc = f(ctypes.byref(d), ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(C.data_ptr()),
           ctypes.c_void_p(J.data_ptr()), None if R is None else ctypes.c_void_p(R.data_ptr()),
           ctypes.c_void_p(cost.data_ptr()), prec,
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), err, 256)
    assert rc == 0, err.value
    return R, cost


@pytest.mark.parametrize("prec", [sc.SC_FP64, sc.SC_MIXED])
@pytest.mark.parametrize("N,T,F", [(37, 3, 2), (300, 4, 2)])
def test_noalloc_matches_residual_on_two_calls_in_a_row(prec, N, T, F):
    f = entry()
    spec = synth.JobSpec(N=N, T=T, F=F, K=1, S=5, f_lo=140e6, f_hi=160e6, seed=17)
    uvw, fr, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_coherencies(uvw, fr, sky.l, sky.m, sky.flux, sky.alpha)
    Jt = synth.jones_true(spec)[0]
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    X = torch.as_tensor(O.model_vis(C, Jt) + synth.noise(spec)).to("cuda", cdt).contiguous()
    Cd = torch.as_tensor(C).to("cuda", cdt).contiguous()
    shp = sc.Shape(N, T, F, 1, 5)
    ws = sc.workspace(shp, prec)
    tol = 1e-11 if prec == sc.SC_FP64 else 1e-5
    for J in (Jt * (1 + 0.01j), Jt + 0.02):          # two calls, different inputs
        Jd = torch.as_tensor(J).to("cuda").contiguous()
        R_ref, c_ref = sc.residual(shp, X, Cd, Jd, prec, ws)
        R, c = call_noalloc(f, shp, X, Cd, Jd, prec)
        torch.cuda.synchronize()
        scale = X.abs().max().item()
        assert (R - R_ref).abs().max().item() <= tol * scale
        assert abs(c.item() - c_ref.item()) <= tol * c_ref.item()


def test_noalloc_refuses_problems_beyond_its_scratch():
    f = entry()
    err = ctypes.create_string_buffer(256)
    d = sc.Dims(1000, 1, 1, 1, 0)                     # 499500 baselines > 233013 in FP64
    dummy = torch.zeros(8, dtype=torch.complex128, device="cuda")
    cost = torch.zeros((), dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = f(ctypes.byref(d), p, p, p, None, ctypes.c_void_p(cost.data_ptr()), sc.SC_FP64, None, err, 256)
    assert rc == -1
    assert b"scratch" in err.value and b"233013" in err.value


@pytest.mark.parametrize("prec", [sc.SC_FP64, sc.SC_MIXED])
def test_noalloc_call_takes_no_device_memory(prec):
    """The property the entry point exists for.  After one call has loaded the
    library's device code on this GPU (and with it the built-in scratch),
    another call with its outputs allocated beforehand leaves the free device
    memory and torch's reserved pool exactly as they were."""
    f = entry()
    N, T, F = 300, 4, 2
    spec = synth.JobSpec(N=N, T=T, F=F, K=1, S=5, f_lo=140e6, f_hi=160e6, seed=3)
    uvw, fr, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    C = O.predict_coherencies(uvw, fr, sky.l, sky.m, sky.flux, sky.alpha)
    Jt = synth.jones_true(spec)[0]
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    X = torch.as_tensor(O.model_vis(C, Jt)).to("cuda", cdt).contiguous()
    Cd = torch.as_tensor(C).to("cuda", cdt).contiguous()
    Jd = torch.as_tensor(Jt).to("cuda").contiguous()
    shp = sc.Shape(N, T, F, 1, 5)
    R = torch.empty_like(X)
    cost = torch.zeros((), dtype=torch.float64, device="cuda")
    call_noalloc(f, shp, X, Cd, Jd, prec, R=R, cost=cost)       # loads the device code
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    call_noalloc(f, shp, X, Cd, Jd, prec, R=R, cost=cost)
    torch.cuda.synchronize()
    free1, reserved1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    assert (free1, reserved1) == (free0, reserved0)
    assert cost.item() < 1e-9 * float((X.abs() ** 2).sum())      # noiseless data, true Jones


def test_noalloc_refuses_the_shapes_sc_residual_refuses():
    f = entry()
    err = ctypes.create_string_buffer(256)
    dummy = torch.zeros(8, dtype=torch.complex128, device="cuda")
    cost = torch.zeros((), dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    for dims in ((16, 300, 300), (1, 4, 2), (16, 0, 2)):        # T*F > 65535, N < 2, T < 1
        d = sc.Dims(dims[0], dims[1], dims[2], 1, 0)
        rc = f(ctypes.byref(d), p, p, p, None, ctypes.c_void_p(cost.data_ptr()), sc.SC_FP64, None, err, 256)
        assert rc == -1, dims
        shp = sc.Shape(dims[0], dims[1], dims[2], 1, 0)
        with pytest.raises(Exception):
            sc.workspace_size(shp, sc.SC_FP64)
