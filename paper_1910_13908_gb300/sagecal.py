"""Python binding of the C ABI in include/sagecal_gb.h (ctypes).

Argument marshalling only: every step of the calibration runs in the CUDA
library libsagecal_gb.so.  Tensors are torch CUDA tensors (PyTorch provides
device memory and streams); complex data are torch.complex64 (SC_MIXED) or
torch.complex128 (SC_FP64) with the layouts of the header:

    uvw    float64 [T][N][3]        freqs  float64 [F]
    V, X, R  complex [T][B][F][2][2]
    C      complex [K][T][B][F] (one cluster: [T][B][F])
    jones  complex128 [K][N][2][2] (one cluster: [N][2][2])

There is no fallback: if the library is missing or the device is not a
CUDA device, calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

from . import build as _build

SC_FP64 = 0
SC_MIXED = 1

# device status bits (sc_device_status)
SC_CHOL_SIMT = 0
SC_CHOL_TENSOR = 1
SC_STATUS_NOTPD = 1
SC_STATUS_TIMEOUT = 2
SC_STATUS_SINGULAR = 4
SC_STATUS_BASIS = 8

_c = ctypes
_LIB = None


class Dims(_c.Structure):
    _fields_ = [("N", _c.c_int32), ("T", _c.c_int32), ("F", _c.c_int32),
                ("K", _c.c_int32), ("S_max", _c.c_int32)]


class SkyC(_c.Structure):
    _fields_ = [("offsets", _c.POINTER(_c.c_int32)), ("l", _c.c_void_p), ("m", _c.c_void_p),
                ("flux", _c.c_void_p), ("alpha", _c.c_void_p), ("f0", _c.c_double)]


class SkyFullC(_c.Structure):
    _fields_ = [("offsets", _c.POINTER(_c.c_int32))] + \
        [(n, _c.c_void_p) for n in ("l", "m", "I", "Q", "U", "V", "alpha", "maj", "mnr", "pa")] + \
        [("f0", _c.c_double)]


class LMOpts(_c.Structure):
    _fields_ = [("n_lm", _c.c_int32), ("refine_sweeps", _c.c_int32),
                ("tau", _c.c_double), ("eps_grad", _c.c_double),
                ("max_ctas", _c.c_int32), ("chol_kernel", _c.c_int32)]


class SageOpts(_c.Structure):
    _fields_ = [("n_em", _c.c_int32), ("lm", LMOpts)]


class ConsensusOpts(_c.Structure):
    _fields_ = [("sage", SageOpts), ("n_admm", _c.c_int32), ("n_poly", _c.c_int32), ("rho", _c.c_double)]


class JobC(_c.Structure):
    _fields_ = [("dims", Dims), ("uvw", _c.c_void_p), ("freqs", _c.c_void_p), ("sky", SkyC),
                ("V", _c.c_void_p), ("jones", _c.c_void_p), ("costs", _c.c_void_p),
                ("ws", _c.c_void_p), ("ws_bytes", _c.c_size_t), ("stream", _c.c_void_p)]


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libsagecal_gb.so is not built (run __graft_entry__.build())")
        L = _c.CDLL(path)
        vp, i32, sz = _c.c_void_p, _c.c_int32, _c.c_size_t
        D = _c.POINTER(Dims)
        L.sc_version.restype = i32
        L.sc_last_error.argtypes = [_c.c_char_p, sz]
        L.sc_last_error.restype = i32
        L.sc_workspace_size.argtypes = [D, i32, _c.POINTER(sz)]
        L.sc_device_status.argtypes = [vp, sz, _c.POINTER(_c.c_uint32)]
        L.sc_chol_schedule.argtypes = [i32, i32, _c.POINTER(i32), i32]
        L.sc_predict_coherencies.argtypes = [D, vp, vp, _c.POINTER(SkyC), vp, i32, vp, sz, vp]
        L.sc_predict_coherencies_full.argtypes = [D, vp, vp, _c.POINTER(SkyFullC), vp, i32, vp, sz, vp]
        L.sc_predict_coherencies_full.restype = i32
        L.sc_residual.argtypes = [D, vp, vp, vp, vp, vp, i32, vp, sz, vp]
        L.sc_residual_all.argtypes = [D, vp, vp, vp, i32, vp, vp, i32, vp, sz, vp]
        L.sc_lm_normal_eqs.argtypes = [D, vp, vp, vp, vp, vp, i32, vp, sz, vp]
        L.sc_solve_cluster.argtypes = [D, vp, vp, vp, _c.POINTER(LMOpts), vp, vp, i32, vp, sz, vp]
        L.sc_calibrate_sage.argtypes = [D, vp, vp, _c.POINTER(SkyC), vp, vp, _c.POINTER(SageOpts),
                                        vp, i32, vp, sz, vp]
        L.sc_calibrate_chunks.argtypes = [D, i32, vp, vp, _c.POINTER(SkyC), vp, vp, vp,
                                          _c.POINTER(SageOpts), vp, i32, vp, sz, vp]
        L.sc_calibrate_chunks.restype = i32
        L.sc_calibrate_batch.argtypes = [_c.POINTER(JobC), i32, _c.POINTER(SageOpts), i32]
        L.sc_calibrate_consensus.argtypes = [D, i32, vp, vp, _c.POINTER(SkyC), vp, vp, vp, vp, vp, vp,
                                             _c.POINTER(ConsensusOpts), i32, vp, sz, vp]
        L.sc_calibrate_consensus.restype = i32
        L.sc_graph_capture_sage.argtypes = [D, vp, vp, _c.POINTER(SkyC), vp, vp, _c.POINTER(SageOpts),
                                            vp, i32, vp, sz, vp, _c.POINTER(vp)]
        L.sc_graph_launch.argtypes = [vp, vp]
        L.sc_graph_destroy.argtypes = [vp]
        for f in ("sc_graph_capture_sage", "sc_graph_launch", "sc_graph_destroy"):
            getattr(L, f).restype = i32
        L.sc_calibrate_batch.restype = i32
        L.sc_batched_workspace_size.argtypes = [D, i32, i32, _c.POINTER(sz)]
        L.sc_calibrate_batched.argtypes = [_c.POINTER(JobC), i32, _c.POINTER(SageOpts), i32, i32, vp, sz, vp]
        L.sc_tune_batched.argtypes = [D, i32, i32, _c.POINTER(i32), i32, i32, _c.POINTER(_c.c_double),
                                      _c.POINTER(i32), vp, sz, vp]
        L.sc_batch_order.argtypes = [i32, i32, i32, _c.POINTER(i32), _c.c_int64]
        for f in ("sc_batched_workspace_size", "sc_calibrate_batched", "sc_tune_batched", "sc_batch_order"):
            getattr(L, f).restype = i32
        L.sc_cholesky_workspace_size.argtypes = [i32, i32, _c.POINTER(sz)]
        L.sc_cholesky_solve.argtypes = [i32, vp, i32, vp, vp, i32, i32, vp, sz, vp]
        for f in ("sc_cholesky_workspace_size", "sc_cholesky_solve"):
            getattr(L, f).restype = i32
        L.sc_launch_count.restype = _c.c_uint64
        L.sc_profile_read.argtypes = [i32, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_double)]
        for f in ("sc_profile_begin", "sc_profile_end", "sc_profile_read"):
            getattr(L, f).restype = i32
        for f in ("sc_workspace_size", "sc_device_status", "sc_chol_schedule",
                  "sc_predict_coherencies", "sc_residual", "sc_residual_all", "sc_lm_normal_eqs",
                  "sc_solve_cluster", "sc_calibrate_sage"):
            getattr(L, f).restype = i32
        _LIB = L
    return _LIB


class ScError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("sagecal_gb error %d: %s" % (code, msg))
        self.code = code


def _check(rc):
    if rc < 0:
        buf = _c.create_string_buffer(512)
        lib().sc_last_error(buf, 512)
        raise ScError(rc, buf.value.decode(errors="replace"))
    return rc


def _ptr(t):
    return None if t is None else _c.c_void_p(t.data_ptr())


def _stream():
    import torch
    return _c.c_void_p(torch.cuda.current_stream().cuda_stream)


def _cdt(prec):
    import torch
    return torch.complex64 if prec == SC_MIXED else torch.complex128


def _rdt(prec):
    import torch
    return torch.float32 if prec == SC_MIXED else torch.float64


@dataclasses.dataclass
class Shape:
    N: int
    T: int
    F: int
    K: int = 1
    S_max: int = 0

    @property
    def B(self):
        return self.N * (self.N - 1) // 2

    def c(self):
        return Dims(self.N, self.T, self.F, self.K, self.S_max)


@dataclasses.dataclass
class DeviceSky:
    """Sky model on the device: SoA float64 tensors + host cluster offsets."""
    l: object
    m: object
    flux: object
    alpha: object
    offsets: list
    f0: float = 150e6

    def c(self):
        offs = (_c.c_int32 * len(self.offsets))(*[int(x) for x in self.offsets])
        s = SkyC(offs, _ptr(self.l), _ptr(self.m), _ptr(self.flux), _ptr(self.alpha), float(self.f0))
        s._keep = offs
        return s

    @property
    def K(self):
        return len(self.offsets) - 1

    @property
    def S_max(self):
        return max([b - a for a, b in zip(self.offsets[:-1], self.offsets[1:])] + [0])

    @staticmethod
    def from_synth(sky, device="cuda"):
        import torch
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
        return DeviceSky(t(sky.l), t(sky.m), t(sky.flux), t(sky.alpha),
                         [int(x) for x in sky.offsets], float(sky.f0))


FULL_FIELDS = ("l", "m", "I", "Q", "U", "V", "alpha", "maj", "mnr", "pa")


@dataclasses.dataclass
class DeviceSkyFull:
    """Polarised, possibly extended sky on the device: SoA float64 tensors
    (FULL_FIELDS) + host cluster offsets."""
    arrays: dict
    offsets: list
    f0: float = 150e6

    def c(self):
        offs = (_c.c_int32 * len(self.offsets))(*[int(x) for x in self.offsets])
        s = SkyFullC(offs, *[_ptr(self.arrays[n]) for n in FULL_FIELDS], float(self.f0))
        s._keep = offs
        return s

    @property
    def K(self):
        return len(self.offsets) - 1

    @property
    def S_max(self):
        return max([b - a for a, b in zip(self.offsets[:-1], self.offsets[1:])] + [0])

    @staticmethod
    def from_synth(sky, device="cuda"):
        import torch
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
        return DeviceSkyFull({n: t(getattr(sky, n)) for n in FULL_FIELDS},
                             [int(x) for x in sky.offsets], float(sky.f0))


def workspace_size(shape: Shape, prec: int) -> int:
    n = _c.c_size_t(0)
    d = shape.c()
    _check(lib().sc_workspace_size(_c.byref(d), prec, _c.byref(n)))
    return n.value


def workspace(shape: Shape, prec: int, device="cuda"):
    import torch
    ws = torch.empty(workspace_size(shape, prec), dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


def device_status(ws) -> int:
    import torch
    torch.cuda.synchronize(ws.device)
    st = _c.c_uint32(0)
    _check(lib().sc_device_status(_ptr(ws), ws.numel(), _c.byref(st)))
    return st.value


def chol_schedule(nT: int, which: int = 0):
    n = _check(lib().sc_chol_schedule(nT, which, None, 0))
    buf = (_c.c_int32 * (4 * n))()
    _check(lib().sc_chol_schedule(nT, which, buf, n))
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(n)]


PROFILE_KINDS = ["station_phasors", "coherency", "vis_pass", "station_reduce", "jhj_assemble",
                 "cholesky", "tri_solve", "refine_residual", "lm_control", "other", "lm_stats"]


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(lib().sc_launch_count())


def profile_begin():
    _check(lib().sc_profile_begin())


def profile_end() -> dict:
    """Stops per-kernel timing; returns {kind: (launches, total_ms)}."""
    _check(lib().sc_profile_end())
    out = {}
    for k, name in enumerate(PROFILE_KINDS):
        n, ms = _c.c_int64(0), _c.c_double(0)
        _check(lib().sc_profile_read(k, _c.byref(n), _c.byref(ms)))
        out[name] = (n.value, ms.value)
    return out


def _need(t, dtype, shape, name):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() or not t.is_cuda:
        raise ValueError("%s: expected contiguous CUDA %s %s, got %s %s" %
                         (name, dtype, tuple(shape), t.dtype, tuple(t.shape)))


def predict_coherencies(shape: Shape, uvw, freqs, sky: DeviceSky, prec: int, ws, out=None):
    """C [K][T][B][F] of every cluster."""
    import torch
    K = sky.K
    d = Shape(shape.N, shape.T, shape.F, K, max(shape.S_max, sky.S_max))
    if out is None:
        out = torch.empty((K, d.T, d.B, d.F), dtype=_cdt(prec), device=uvw.device)
    _need(uvw, torch.float64, (d.T, d.N, 3), "uvw")
    _need(freqs, torch.float64, (d.F,), "freqs")
    _need(out, _cdt(prec), (K, d.T, d.B, d.F), "C")
    dc, skc = d.c(), sky.c()
    _check(lib().sc_predict_coherencies(_c.byref(dc), _ptr(uvw), _ptr(freqs), _c.byref(skc),
                                        _ptr(out), prec, _ptr(ws), ws.numel(), _stream()))
    return out


def predict_coherencies_full(shape: Shape, uvw, freqs, sky: DeviceSkyFull, prec: int, ws, out=None):
    """Full 2x2 coherencies C [K][T][B][F][2][2] of a polarised, possibly
    extended sky (sc_predict_coherencies_full)."""
    import torch
    K = sky.K
    d = Shape(shape.N, shape.T, shape.F, K, max(shape.S_max, sky.S_max))
    if out is None:
        out = torch.empty((K, d.T, d.B, d.F, 2, 2), dtype=_cdt(prec), device=uvw.device)
    _need(uvw, torch.float64, (d.T, d.N, 3), "uvw")
    _need(freqs, torch.float64, (d.F,), "freqs")
    _need(out, _cdt(prec), (K, d.T, d.B, d.F, 2, 2), "C")
    dc, skc = d.c(), sky.c()
    _check(lib().sc_predict_coherencies_full(_c.byref(dc), _ptr(uvw), _ptr(freqs), _c.byref(skc),
                                             _ptr(out), prec, _ptr(ws), ws.numel(), _stream()))
    return out


def residual(shape: Shape, X, C, jones, prec: int, ws, out=None, want_cost=True):
    """R = X - J_p C J_q^H for one cluster, and cost = sum |R|^2 (device scalar)."""
    import torch
    d = Shape(shape.N, shape.T, shape.F, 1, shape.S_max)
    _need(X, _cdt(prec), (d.T, d.B, d.F, 2, 2), "X")
    _need(C, _cdt(prec), (d.T, d.B, d.F), "C")
    _need(jones, torch.complex128, (d.N, 2, 2), "jones")
    if out is None:
        out = torch.empty_like(X)
    cost = torch.zeros((), dtype=torch.float64, device=X.device) if want_cost else None
    dc = d.c()
    _check(lib().sc_residual(_c.byref(dc), _ptr(X), _ptr(C), _ptr(jones), _ptr(out), _ptr(cost),
                             prec, _ptr(ws), ws.numel(), _stream()))
    return out, cost


def residual_all(shape: Shape, V, C, jones, prec: int, ws, corr=-1, out=None, want_cost=True):
    """R = V - sum_k J_kp C_kpq J_kq^H over all K clusters, then, if corr >= 0,
    R <- J_cp^{-1} R J_cq^{-H}; cost = sum |R|^2 before the correction
    (device scalar).  out may be V (in place)."""
    import torch
    K = C.shape[0]
    d = Shape(shape.N, shape.T, shape.F, K, shape.S_max)
    _need(V, _cdt(prec), (d.T, d.B, d.F, 2, 2), "V")
    _need(C, _cdt(prec), (K, d.T, d.B, d.F), "C")
    _need(jones, torch.complex128, (K, d.N, 2, 2), "jones")
    if out is None:
        out = torch.empty_like(V)
    _need(out, _cdt(prec), (d.T, d.B, d.F, 2, 2), "out")
    cost = torch.zeros((), dtype=torch.float64, device=V.device) if want_cost else None
    dc = d.c()
    _check(lib().sc_residual_all(_c.byref(dc), _ptr(V), _ptr(C), _ptr(jones), int(corr), _ptr(out),
                                 _ptr(cost), prec, _ptr(ws), ws.numel(), _stream()))
    return out, cost


def lm_normal_eqs(shape: Shape, R, C, jones, prec: int, ws):
    """(J^T J [8N][8N], J^T r [8N]) of one cluster at residual R."""
    import torch
    d = Shape(shape.N, shape.T, shape.F, 1, shape.S_max)
    _need(R, _cdt(prec), (d.T, d.B, d.F, 2, 2), "R")
    _need(C, _cdt(prec), (d.T, d.B, d.F), "C")
    _need(jones, torch.complex128, (d.N, 2, 2), "jones")
    P = 8 * d.N
    JhJ = torch.empty((P, P), dtype=_rdt(prec), device=R.device)
    Jhr = torch.empty((P,), dtype=torch.float64, device=R.device)
    dc = d.c()
    _check(lib().sc_lm_normal_eqs(_c.byref(dc), _ptr(R), _ptr(C), _ptr(jones), _ptr(JhJ), _ptr(Jhr),
                                  prec, _ptr(ws), ws.numel(), _stream()))
    return JhJ, Jhr


def lm_opts(n_lm=10, refine_sweeps=1, tau=1e-3, eps_grad=1e-12, max_ctas=0, chol_kernel=0):
    return LMOpts(int(n_lm), int(refine_sweeps), float(tau), float(eps_grad), int(max_ctas), int(chol_kernel))


def solve_cluster(shape: Shape, X, C, jones, prec: int, ws, n_lm=10, refine_sweeps=1, tau=1e-3,
                  eps_grad=1e-12, chol_kernel=0):
    """LM solve of one cluster; `jones` [N][2][2] complex128 is updated in place.
    Returns (jones, cost, iters) with cost/iters device scalars."""
    import torch
    d = Shape(shape.N, shape.T, shape.F, 1, shape.S_max)
    _need(X, _cdt(prec), (d.T, d.B, d.F, 2, 2), "X")
    _need(C, _cdt(prec), (d.T, d.B, d.F), "C")
    _need(jones, torch.complex128, (d.N, 2, 2), "jones")
    cost = torch.zeros((), dtype=torch.float64, device=X.device)
    iters = torch.zeros((), dtype=torch.int32, device=X.device)
    o = lm_opts(n_lm, refine_sweeps, tau, eps_grad, chol_kernel=chol_kernel)
    dc = d.c()
    _check(lib().sc_solve_cluster(_c.byref(dc), _ptr(X), _ptr(C), _ptr(jones), _c.byref(o),
                                  _ptr(cost), _ptr(iters), prec, _ptr(ws), ws.numel(), _stream()))
    return jones, cost, iters


def cholesky_workspace(n: int, prec: int, device="cuda"):
    import torch
    nb = _c.c_size_t(0)
    _check(lib().sc_cholesky_workspace_size(n, prec, _c.byref(nb)))
    return torch.empty(nb.value, dtype=torch.uint8, device=device)


def cholesky_solve(A, b, prec: int, ws=None, chol_kernel=0):
    """Factorises the SPD matrix A (n x n, float32 for SC_MIXED / float64 for
    SC_FP64, lower triangle read) in place into L and solves A x = b (b float64
    [n] or None); chol_kernel SC_CHOL_SIMT / SC_CHOL_TENSOR.  Returns (A
    holding L in its lower triangle, x)."""
    import torch
    n = A.shape[0]
    rdt = torch.float32 if prec == SC_MIXED else torch.float64
    _need(A, rdt, (n, A.shape[1]), "A")
    if A.shape[1] < n or A.stride(1) != 1:
        raise ValueError("A: expected n x lda row-major with lda >= n")
    if ws is None:
        ws = cholesky_workspace(n, prec, A.device)
    x = None
    if b is not None:
        _need(b, torch.float64, (n,), "b")
        x = torch.empty_like(b)
    _check(lib().sc_cholesky_solve(n, _ptr(A), A.stride(0), None if b is None else _ptr(b),
                                   None if x is None else _ptr(x), prec, chol_kernel, _ptr(ws), ws.numel(),
                                   _stream()))
    return A, x


def calibrate_sage(shape: Shape, uvw, freqs, sky: DeviceSky, V, jones, prec: int, ws, n_em=1,
                   n_lm=10, refine_sweeps=1, tau=1e-3, eps_grad=1e-12, costs=None, max_ctas=0, chol_kernel=0):
    """The whole path for one job; `jones` [K][N][2][2] complex128 is updated in
    place.  Returns (jones, costs [K] device float64)."""
    import torch
    K = sky.K
    d = Shape(shape.N, shape.T, shape.F, K, max(shape.S_max, sky.S_max))
    _need(uvw, torch.float64, (d.T, d.N, 3), "uvw")
    _need(freqs, torch.float64, (d.F,), "freqs")
    _need(V, _cdt(prec), (d.T, d.B, d.F, 2, 2), "V")
    _need(jones, torch.complex128, (K, d.N, 2, 2), "jones")
    if costs is None:
        costs = torch.zeros((K,), dtype=torch.float64, device=V.device)
    o = SageOpts(int(n_em), lm_opts(n_lm, refine_sweeps, tau, eps_grad, max_ctas, chol_kernel))
    dc, skc = d.c(), sky.c()
    _check(lib().sc_calibrate_sage(_c.byref(dc), _ptr(uvw), _ptr(freqs), _c.byref(skc), _ptr(V),
                                   _ptr(jones), _c.byref(o), _ptr(costs), prec, _ptr(ws), ws.numel(),
                                   _stream()))
    return jones, costs


def calibrate_chunks(shape: Shape, uvw, freqs, sky: DeviceSky, V, jones, prec: int, ws, n_em=1,
                     n_lm=10, refine_sweeps=1, tau=1e-3, eps_grad=1e-12, max_ctas=0,
                     want_history=True):
    """Consecutive time chunks, each warm-started from the previous chunk's
    solution.  shape.T is the timeslots of ONE chunk; V is
    [n_chunks][T][B][F][2][2], uvw [n_chunks * T][N][3].  `jones` [K][N][2][2]
    is the initial guess and is left holding the last chunk's solution.
    Returns (jones, history [n_chunks][K][N][2][2] or None, costs [n_chunks][K])."""
    import torch
    K = sky.K
    n = V.shape[0]
    d = Shape(shape.N, shape.T, shape.F, K, max(shape.S_max, sky.S_max))
    _need(uvw, torch.float64, (n * d.T, d.N, 3), "uvw")
    _need(freqs, torch.float64, (d.F,), "freqs")
    _need(V, _cdt(prec), (n, d.T, d.B, d.F, 2, 2), "V")
    _need(jones, torch.complex128, (K, d.N, 2, 2), "jones")
    hist = torch.empty((n, K, d.N, 2, 2), dtype=torch.complex128, device=V.device) if want_history else None
    costs = torch.zeros((n, K), dtype=torch.float64, device=V.device)
    o = SageOpts(int(n_em), lm_opts(n_lm, refine_sweeps, tau, eps_grad, max_ctas))
    dc, skc = d.c(), sky.c()
    _check(lib().sc_calibrate_chunks(_c.byref(dc), int(n), _ptr(uvw), _ptr(freqs), _c.byref(skc),
                                     _ptr(V), _ptr(jones), _ptr(hist), _c.byref(o), _ptr(costs), prec,
                                     _ptr(ws), ws.numel(), _stream()))
    return jones, hist, costs


class Graph:
    """A sc_calibrate_sage call captured once as a CUDA graph (see
    capture_sage).  launch() replays it on the current stream; the tensors
    given at capture are kept alive here, since the graph reads and writes
    them at every replay."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self):
        if self._h is None:
            raise RuntimeError("graph has been closed")
        _check(lib().sc_graph_launch(self._h, _stream()))

    def close(self):
        if self._h is not None:
            lib().sc_graph_destroy(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def capture_sage(shape: Shape, uvw, freqs, sky: DeviceSky, V, jones, prec: int, ws, costs, n_em=1,
                 n_lm=10, refine_sweeps=1, tau=1e-3, eps_grad=1e-12, max_ctas=0):
    """Records calibrate_sage on these tensors as a CUDA graph (nothing runs
    yet).  Each Graph.launch() then calibrates whatever V, jones (initial
    guess in, solution out), uvw and the sky arrays hold at that point;
    costs [K] float64 receives the final cluster costs.  Captured on a side
    stream, since the legacy default stream cannot be captured."""
    import torch
    K = sky.K
    d = Shape(shape.N, shape.T, shape.F, K, max(shape.S_max, sky.S_max))
    _need(uvw, torch.float64, (d.T, d.N, 3), "uvw")
    _need(freqs, torch.float64, (d.F,), "freqs")
    _need(V, _cdt(prec), (d.T, d.B, d.F, 2, 2), "V")
    _need(jones, torch.complex128, (K, d.N, 2, 2), "jones")
    _need(costs, torch.float64, (K,), "costs")
    o = SageOpts(int(n_em), lm_opts(n_lm, refine_sweeps, tau, eps_grad, max_ctas))
    dc, skc = d.c(), sky.c()
    h = _c.c_void_p()
    side = torch.cuda.Stream(device=V.device)
    side.wait_stream(torch.cuda.current_stream(V.device))
    with torch.cuda.stream(side):
        _check(lib().sc_graph_capture_sage(_c.byref(dc), _ptr(uvw), _ptr(freqs), _c.byref(skc), _ptr(V),
                                           _ptr(jones), _c.byref(o), _ptr(costs), prec, _ptr(ws),
                                           ws.numel(), _c.c_void_p(side.cuda_stream), _c.byref(h)))
    return Graph(h, (uvw, freqs, sky, V, jones, costs, ws))


def consensus_workspace(shape: Shape, prec: int, concurrent: int = 1, device="cuda"):
    """Workspace of sc_calibrate_consensus for `concurrent` bands at once:
    that many whole band workspaces (each sc_workspace_size rounded up to
    256 bytes)."""
    import torch
    per = (workspace_size(shape, prec) + 255) // 256 * 256
    return torch.empty(per * max(1, int(concurrent)), dtype=torch.uint8, device=device)


def calibrate_consensus(shape: Shape, uvw, freqs, sky: DeviceSky, V, basis, jones, prec: int, ws, rho,
                        n_admm=3, n_em=1, n_lm=10, refine_sweeps=1, tau=1e-3, eps_grad=1e-12, max_ctas=0,
                        dual=None):
    """Sub-band calibrations coupled by a smooth frequency model
    (sc_calibrate_consensus).  shape is ONE band's (F channels per band);
    freqs [n_bands][F], V [n_bands][T][B][F][2][2], basis [n_bands][n_poly]
    float64, jones [n_bands][K][N][2][2] (updated in place), dual the scaled
    duals (zeros if None; updated in place).
    Returns (jones, dual, Z [K][n_poly][N][2][2], costs [n_bands][K])."""
    import torch
    K = sky.K
    n_bands, n_poly = basis.shape
    d = Shape(shape.N, shape.T, shape.F, K, max(shape.S_max, sky.S_max))
    _need(uvw, torch.float64, (d.T, d.N, 3), "uvw")
    _need(freqs, torch.float64, (n_bands, d.F), "freqs")
    _need(V, _cdt(prec), (n_bands, d.T, d.B, d.F, 2, 2), "V")
    _need(basis, torch.float64, (n_bands, n_poly), "basis")
    _need(jones, torch.complex128, (n_bands, K, d.N, 2, 2), "jones")
    if dual is None:
        dual = torch.zeros_like(jones)
    _need(dual, torch.complex128, (n_bands, K, d.N, 2, 2), "dual")
    Z = torch.empty((K, n_poly, d.N, 2, 2), dtype=torch.complex128, device=V.device)
    costs = torch.zeros((n_bands, K), dtype=torch.float64, device=V.device)
    o = ConsensusOpts(SageOpts(int(n_em), lm_opts(n_lm, refine_sweeps, tau, eps_grad, max_ctas)), int(n_admm),
                      int(n_poly), float(rho))
    dc, skc = d.c(), sky.c()
    _check(lib().sc_calibrate_consensus(_c.byref(dc), int(n_bands), _ptr(uvw), _ptr(freqs), _c.byref(skc),
                                        _ptr(V), _ptr(basis), _ptr(jones), _ptr(dual), _ptr(Z), _ptr(costs),
                                        _c.byref(o), prec, _ptr(ws), ws.numel(), _stream()))
    return jones, dual, Z, costs


@dataclasses.dataclass
class Job:
    """One calibration job of a batch: device inputs, in/out Jones, cost
    output, its own workspace and its own stream."""
    shape: Shape
    uvw: object
    freqs: object
    sky: DeviceSky
    V: object
    jones: object
    costs: object
    ws: object
    stream: object


def calibrate_batch(jobs, prec: int, n_em=1, n_lm=10, refine_sweeps=1, tau=1e-3, eps_grad=1e-12,
                    max_ctas=0):
    """Enqueue every job (sc_calibrate_batch); each runs on job.stream.
    Synchronise the streams (or the device) before reading the results."""
    arr, keep = _job_array(jobs, prec)
    o = SageOpts(int(n_em), lm_opts(n_lm, refine_sweeps, tau, eps_grad, max_ctas))
    _check(lib().sc_calibrate_batch(arr, len(jobs), _c.byref(o), prec))
    del keep
    return jobs


def _job_array(jobs, prec):
    """The jobs as sc_job structs (and the sky structs they point to)."""
    n = len(jobs)
    arr = (JobC * n)()
    keep = []
    for i, j in enumerate(jobs):
        K = j.sky.K
        d = Shape(j.shape.N, j.shape.T, j.shape.F, K, max(j.shape.S_max, j.sky.S_max))
        _need(j.V, _cdt(prec), (d.T, d.B, d.F, 2, 2), "V")
        _need(j.jones, torch_complex128(), (K, d.N, 2, 2), "jones")
        skc = j.sky.c()
        keep.append(skc)
        arr[i] = JobC(d.c(), _ptr(j.uvw), _ptr(j.freqs), skc, _ptr(j.V), _ptr(j.jones), _ptr(j.costs),
                      _ptr(j.ws), j.ws.numel(), _c.c_void_p(j.stream.cuda_stream))
    return arr, keep


def _job_dims(jobs):
    dims = (Dims * len(jobs))()
    for i, j in enumerate(jobs):
        dims[i] = Shape(j.shape.N, j.shape.T, j.shape.F, j.sky.K, max(j.shape.S_max, j.sky.S_max)).c()
    return dims


def batched_workspace(jobs, prec: int, device="cuda"):
    """Workspace of calibrate_batched for these jobs (sc_batched_workspace_size)."""
    import torch
    n = len(jobs)
    dims = _job_dims(jobs)
    nb = _c.c_size_t(0)
    _check(lib().sc_batched_workspace_size(dims, n, prec, _c.byref(nb)))
    ws = torch.empty(nb.value, dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


def calibrate_batched(jobs, prec: int, ws, n_em=1, n_lm=10, refine_sweeps=1, tau=1e-3, eps_grad=1e-12,
                      max_ctas=0, window=0):
    """Lock-step batch (sc_calibrate_batched) of jobs of equal N and K on the
    current stream, the factorisations staggered over `window` jobs (0: as
    many as fit in L2); each job's stream waits for it."""
    arr, keep = _job_array(jobs, prec)
    o = SageOpts(int(n_em), lm_opts(n_lm, refine_sweeps, tau, eps_grad, max_ctas))
    _check(lib().sc_calibrate_batched(arr, len(jobs), _c.byref(o), prec, int(window), _ptr(ws), ws.numel(),
                                      _stream()))
    del keep
    return jobs


def tune_batched(jobs, prec: int, ws, windows=(1, 4, 16, 64, 1 << 20), reps=3):
    """sc_tune_batched: ms per batched factorisation for each window; returns
    (best window, {window: ms}).  Synchronises; overwrites ws."""
    n = len(windows)
    w = (_c.c_int32 * n)(*[int(x) for x in windows])
    ms = (_c.c_double * n)()
    best = _c.c_int32(0)
    _check(lib().sc_tune_batched(_job_dims(jobs), len(jobs), prec, w, n, int(reps), ms, _c.byref(best),
                                 _ptr(ws), ws.numel(), _stream()))
    return best.value, {int(windows[i]): ms[i] for i in range(n)}


def batch_order(nT: int, n_jobs: int, window: int):
    """Host only: positions [n_jobs][tasks per job] of each job's tasks in the
    merged factorisation list (sc_batch_order)."""
    import numpy as np
    n = _check(lib().sc_chol_schedule(nT, 0, None, 0))
    out = (_c.c_int32 * (n * n_jobs))()
    _check(lib().sc_batch_order(nT, n_jobs, window, out, n * n_jobs))
    return np.frombuffer(out, dtype=np.int32).reshape(n_jobs, n).copy()


def torch_complex128():
    import torch
    return torch.complex128
