"""Extrinsic-marginalised likelihood (ILE) of RIFT on one NVIDIA B300.

Thin binding of the C ABI in include/rift_ile.h: every function here only
marshals arguments (PyTorch CUDA tensors or numpy arrays) into the shared
library _rift_ile.so and returns its results.  All computation runs in the
library's CUDA kernels; there is no CPU fallback, and importing this package
fails if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_rift_ile.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python paper_2609_37393_b300/build.py` "
        "(there is no CPU implementation of this package)")

_lib = ctypes.CDLL(LIB_PATH)

FP64 = 0
FP32_MIXED = 1
PARAMS = ("ra", "dec", "psi", "incl", "phase", "lnD", "t")
MAX_DET, MAX_MODES, MAX_ELL = 8, 16, 8

ERRORS = {-1: "INVALID_ARG", -2: "SHAPE", -3: "UNSUPPORTED", -4: "CUDA", -5: "TIMEOUT",
          -6: "ALLOC"}


class RiftError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _PointDesc(ctypes.Structure):
    _fields_ = [
        ("n_det", ctypes.c_int32), ("n_modes", ctypes.c_int32),
        ("ell", ctypes.c_void_p), ("em", ctypes.c_void_p),
        ("Q", ctypes.c_void_p), ("q_dtype", ctypes.c_int32), ("q_len", ctypes.c_int32),
        ("q_t0", ctypes.c_void_p), ("q_dt", ctypes.c_double),
        ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
        ("det_pos", ctypes.c_void_p), ("det_resp", ctypes.c_void_p),
        ("gmst", ctypes.c_double), ("d_ref", ctypes.c_double),
    ]


class _Draws(ctypes.Structure):
    _fields_ = [(p, ctypes.c_void_p) for p in PARAMS] + [
        ("logw", ctypes.c_void_p), ("n", ctypes.c_int64), ("dtype", ctypes.c_int32)]


class _Lse(ctypes.Structure):
    _fields_ = [("m", ctypes.c_double), ("s", ctypes.c_double), ("s2", ctypes.c_double),
                ("n", ctypes.c_double)]


class _Dist(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("lnw", ctypes.c_void_p), ("n", ctypes.c_int32)]


_P = ctypes.c_void_p
_lib.rift_ile_last_error.restype = ctypes.c_char_p
_lib.rift_ile_point_create.argtypes = [_P, _P, _P]
_lib.rift_ile_point_destroy.argtypes = [_P]
_lib.rift_ile_point_info.argtypes = [_P, _P]
_lib.rift_ile_lnL.argtypes = [_P, _P, ctypes.c_int, _P, _P]
_lib.rift_ile_lnL_grad.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P]
_lib.rift_ile_lnZ.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P]
_lib.rift_ile_lnZ_state.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P]
_lib.rift_ile_lnZ_merge.argtypes = [_P, ctypes.c_int32, _P, _P]
_lib.rift_ile_lnZ_state_async.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P]
_lib.rift_ile_lnZ_state_host.argtypes = [_P, _P, ctypes.c_int, _P, ctypes.c_int64, _P, _P]
_lib.rift_ile_lnZ_batch.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int, _P, _P]
_lib.rift_ile_batch_create.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int, _P]
_lib.rift_ile_batch_launch.argtypes = [_P, _P, _P]
_lib.rift_ile_batch_destroy.argtypes = [_P]
_lib.rift_ile_batch_tune.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P]
_lib.rift_ile_lnL_dist.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P, _P]
_lib.rift_ile_dist_nodes.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int32, _P, _P, _P]
_lib.rift_ile_last_oob.restype = ctypes.c_int64
_lib.rift_ile_probe_alu.argtypes = [ctypes.c_int, ctypes.c_double, _P, _P]
_lib.rift_ile_set_small_batch.argtypes = [ctypes.c_int64]
_lib.rift_ile_set_small_batch.restype = ctypes.c_int64


def _check(rc: int):
    if rc != 0:
        raise RiftError(rc, _lib.rift_ile_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _stream(stream=None) -> int:
    """The raw CUDA stream handle of `stream`, or of torch's current stream
    (looked up without building a Stream object, which costs a few
    microseconds per call, where this torch exposes the raw lookup)."""
    torch = _torch()
    if stream is not None:
        return int(stream.cuda_stream)
    raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
    dev = getattr(torch._C, "_cuda_getDevice", None)
    if raw is not None and dev is not None:
        return int(raw(dev()))
    return int(torch.cuda.current_stream().cuda_stream)


def _dev_tensor(x, dtype, device):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=dtype)
    else:
        t = torch.as_tensor(np.asarray(x), device=device, dtype=dtype)
    return t.contiguous()


class Point:
    """An intrinsic point prepared for evaluation (rift_ile_point_create).

    point: dict with K, M, ell[M], em[M], Q[K, n, M] (complex64 or complex128,
    numpy or CUDA tensor), q_t0[K], q_dt, U[K, M, M], V[K, M, M] (complex),
    det_pos[K, 3] (light-seconds), det_resp[K, 6], gmst, d_ref.
    """

    def __init__(self, point: dict, device=None, stream=None):
        torch = _torch()
        device = torch.device(device or "cuda")
        Q = point["Q"]
        if isinstance(Q, torch.Tensor):
            qdt = Q.dtype
        else:
            qdt = {np.dtype(np.complex64): torch.complex64,
                   np.dtype(np.complex128): torch.complex128}[np.asarray(Q).dtype]
        self._Q = _dev_tensor(Q, qdt, device)
        K, n, M = self._Q.shape
        self._host = {
            "ell": np.ascontiguousarray(point["ell"], dtype=np.int32),
            "em": np.ascontiguousarray(point["em"], dtype=np.int32),
            "t0": np.ascontiguousarray(point["q_t0"], dtype=np.float64),
            "U": np.ascontiguousarray(np.asarray(point["U"], dtype=np.complex128)).view(np.float64),
            "V": np.ascontiguousarray(np.asarray(point["V"], dtype=np.complex128)).view(np.float64),
            "pos": np.ascontiguousarray(point["det_pos"], dtype=np.float64),
            "resp": np.ascontiguousarray(point["det_resp"], dtype=np.float64),
        }
        d = _PointDesc()
        d.n_det, d.n_modes = K, M
        d.ell, d.em = self._host["ell"].ctypes.data, self._host["em"].ctypes.data
        d.Q = self._Q.data_ptr()
        d.q_dtype = 1 if qdt == torch.complex128 else 0
        d.q_len = n
        d.q_t0 = self._host["t0"].ctypes.data
        d.q_dt = float(point["q_dt"])
        d.U, d.V = self._host["U"].ctypes.data, self._host["V"].ctypes.data
        d.det_pos, d.det_resp = self._host["pos"].ctypes.data, self._host["resp"].ctypes.data
        d.gmst, d.d_ref = float(point["gmst"]), float(point["d_ref"])
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            _check(_lib.rift_ile_point_create(ctypes.byref(d), ctypes.byref(h), _stream(stream)))
        self._h = h
        self.K, self.M, self.n = K, M, n
        self.device = device
        del self._Q  # the library holds its own copy

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        """K, M, n, whitened dimension R, detector classes, kept null directions."""
        out = (ctypes.c_int32 * 6)()
        _check(_lib.rift_ile_point_info(self._h, out))
        return dict(zip(("K", "M", "n", "R", "ncls", "has_null"), list(out)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.rift_ile_point_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Draws:
    """Device-resident extrinsic draws (rift_ile_draws): seven arrays of equal
    length in float32 or float64, plus optional ln p - ln p_s."""

    def __init__(self, draws: dict, logw=None, dtype=None, device=None):
        torch = _torch()
        device = torch.device(device or "cuda")
        first = draws[PARAMS[0]]
        if dtype is None:
            if isinstance(first, torch.Tensor):
                dtype = first.dtype
            else:
                dtype = torch.float64 if np.asarray(first).dtype == np.float64 else torch.float32
        self.t = {p: _dev_tensor(draws[p], dtype, device) for p in PARAMS}
        self.logw = None if logw is None else _dev_tensor(logw, dtype, device)
        n = self.t[PARAMS[0]].numel()
        for p in PARAMS:
            if self.t[p].numel() != n:
                raise ValueError(f"draw array {p} has {self.t[p].numel()} entries, expected {n}")
        if self.logw is not None and self.logw.numel() != n:
            raise ValueError("logw length differs from the draws")
        self.n = n
        self.dtype = dtype
        s = _Draws()
        for p in PARAMS:
            setattr(s, p, self.t[p].data_ptr() if n else None)
        s.logw = self.logw.data_ptr() if (self.logw is not None and n) else None
        s.n = n
        s.dtype = 1 if dtype == torch.float64 else 0
        self.struct = s

    @property
    def ref(self):
        return ctypes.byref(self.struct)


class HostDraws:
    """Draws in HOST memory for rift_ile_lnZ_state_host: seven arrays (and an
    optional ln p - ln p_s) as numpy arrays or CPU tensors, float32 or float64
    (page-locked CPU tensors let the library overlap copies and kernels)."""

    def __init__(self, draws: dict, logw=None):
        torch = _torch()

        def host(x, dtype=None):
            t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
            if t.is_cuda:
                raise ValueError("HostDraws takes host arrays")
            if dtype is not None and t.dtype != dtype:
                t = t.to(dtype)
            return t.contiguous()

        self.t = {p: host(draws[p]) for p in PARAMS}
        dtype = self.t[PARAMS[0]].dtype
        if dtype not in (torch.float32, torch.float64):
            raise ValueError("draws must be float32 or float64")
        self.t = {p: host(v, dtype) for p, v in self.t.items()}
        self.logw = None if logw is None else host(logw, dtype)
        n = self.t[PARAMS[0]].numel()
        if any(v.numel() != n for v in self.t.values()) or (self.logw is not None and self.logw.numel() != n):
            raise ValueError("host draw arrays differ in length")
        self.n = n
        s = _Draws()
        for p in PARAMS:
            setattr(s, p, self.t[p].data_ptr() if n else None)
        s.logw = self.logw.data_ptr() if (self.logw is not None and n) else None
        s.n = n
        s.dtype = 1 if dtype == torch.float64 else 0
        self.struct = s

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def rift_ile_lnZ_state_host(point: Point, host_draws, precision: int = FP32_MIXED, dist=None,
                            chunk: int = 0, stream=None):
    """LSE state of draws held in host memory, copied in double-buffered chunks
    overlapping the fused kernel (end-to-end path)."""
    d = host_draws if isinstance(host_draws, HostDraws) else HostDraws(host_draws)
    st = _Lse()
    ds, keep = _dist_struct(dist)
    _check(_lib.rift_ile_lnZ_state_host(point.handle, d.ref, precision,
                                        ctypes.byref(ds) if ds is not None else None,
                                        chunk, ctypes.byref(st), _stream(stream)))
    del keep
    return (st.m, st.s, st.s2, st.n)


def _as_draws(draws, logw=None):
    return draws if isinstance(draws, Draws) else Draws(draws, logw)


def rift_ile_lnL(point: Point, draws, precision: int = FP32_MIXED, out=None, stream=None):
    """lnL per draw (float64 CUDA tensor), eq. def:lnL:Decomposed."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(d.n, dtype=torch.float64, device=point.device)
    _check(_lib.rift_ile_lnL(point.handle, d.ref, precision, out.data_ptr() if d.n else None,
                             _stream(stream)))
    return out


def rift_ile_lnL_grad(point: Point, draws, precision: int = FP32_MIXED, lnl_out=None,
                      grad_out=None, stream=None):
    """(lnL[n], grad[7, n]) as float64 CUDA tensors (Sec. II.B)."""
    torch = _torch()
    d = _as_draws(draws)
    if lnl_out is None:
        lnl_out = torch.empty(d.n, dtype=torch.float64, device=point.device)
    if grad_out is None:
        grad_out = torch.empty((7, d.n), dtype=torch.float64, device=point.device)
    _check(_lib.rift_ile_lnL_grad(point.handle, d.ref, precision,
                                  lnl_out.data_ptr() if d.n else None,
                                  grad_out.data_ptr() if d.n else None, _stream(stream)))
    return lnl_out, grad_out


class PreparedCall:
    """One lnL (+ gradient) launch with its C-ABI arguments marshalled once,
    for a caller that evaluates the same point on the same device buffers
    again and again (a sampler updating its draws in place): calling the
    object launches rift_ile_lnL_grad (or rift_ile_lnL) on the stream given
    at preparation and returns the output tensors, with no host
    synchronisation and no per-call argument conversion.  The draws' buffers
    and the outputs must stay alive and keep their size."""

    def __init__(self, point: Point, draws, precision: int, grad: bool, lnl_out=None,
                 grad_out=None, stream=None):
        torch = _torch()
        self.draws = _as_draws(draws)
        n = self.draws.n
        if n == 0:
            raise ValueError("PreparedCall needs at least one draw")
        self.lnl = lnl_out if lnl_out is not None else torch.empty(
            n, dtype=torch.float64, device=point.device)
        self.grad = None
        if grad:
            self.grad = grad_out if grad_out is not None else torch.empty(
                (7, n), dtype=torch.float64, device=point.device)
        self.point = point
        P = ctypes.c_void_p
        s = P(_stream(stream))
        if grad:
            fn = _lib.rift_ile_lnL_grad
            args = (point.handle, self.draws.ref, ctypes.c_int(precision),
                    P(self.lnl.data_ptr()), P(self.grad.data_ptr()), s)
        else:
            fn = _lib.rift_ile_lnL
            args = (point.handle, self.draws.ref, ctypes.c_int(precision),
                    P(self.lnl.data_ptr()), s)
        self._fn, self._args = fn, args

    def __call__(self):
        rc = self._fn(*self._args)
        if rc != 0:
            _check(rc)
        return (self.lnl, self.grad) if self.grad is not None else self.lnl


def prepare_lnL_grad(point: Point, draws, precision: int = FP32_MIXED, lnl_out=None,
                     grad_out=None, stream=None) -> PreparedCall:
    """A PreparedCall of rift_ile_lnL_grad: each call launches lnL and its
    gradient into the same outputs."""
    return PreparedCall(point, draws, precision, True, lnl_out, grad_out, stream)


def prepare_lnL(point: Point, draws, precision: int = FP32_MIXED, lnl_out=None,
                stream=None) -> PreparedCall:
    """A PreparedCall of rift_ile_lnL."""
    return PreparedCall(point, draws, precision, False, lnl_out, None, stream)


def _dist_struct(dist):
    if dist is None:
        return None, None
    x = np.ascontiguousarray(dist[0], dtype=np.float64)
    w = np.ascontiguousarray(dist[1], dtype=np.float64)
    s = _Dist()
    s.x, s.lnw, s.n = x.ctypes.data, w.ctypes.data, x.shape[0]
    return s, (x, w)


def rift_ile_lnL_dist(point: Point, draws, dist, precision: int = FP32_MIXED, out=None,
                      grad=False, grad_out=None, stream=None):
    """Distance-marginalised lnL per draw (eq. ap:dexp on the node table
    dist = (x, lnw)); with grad=True returns (lnL, grad[7, n])."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(d.n, dtype=torch.float64, device=point.device)
    if grad and grad_out is None:
        grad_out = torch.empty((7, d.n), dtype=torch.float64, device=point.device)
    ds, keep = _dist_struct(dist)
    _check(_lib.rift_ile_lnL_dist(point.handle, d.ref, precision, ctypes.byref(ds),
                                  out.data_ptr() if d.n else None,
                                  grad_out.data_ptr() if (grad and d.n) else None, _stream(stream)))
    del keep
    return (out, grad_out) if grad else out


def rift_ile_lnZ_state(point: Point, draws, precision: int = FP32_MIXED, dist=None, stream=None):
    """LSE state (m, s, s2, n) of the draws; dist = (x_nodes, lnw_nodes) or None."""
    d = _as_draws(draws)
    st = _Lse()
    ds, keep = _dist_struct(dist)
    _check(_lib.rift_ile_lnZ_state(point.handle, d.ref, precision,
                                   ctypes.byref(ds) if ds is not None else None,
                                   ctypes.byref(st), _stream(stream)))
    del keep
    return (st.m, st.s, st.s2, st.n)


def rift_ile_lnZ_state_async(point: Point, draws, precision: int = FP32_MIXED, dist=None,
                             out=None, stream=None):
    """LSE state (m, s, s2, n) written to a float64 CUDA tensor of 4 without a
    host synchronisation (chain many on a stream, read once)."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=point.device)
    ds, keep = _dist_struct(dist)
    _check(_lib.rift_ile_lnZ_state_async(point.handle, d.ref, precision,
                                         ctypes.byref(ds) if ds is not None else None,
                                         out.data_ptr(), _stream(stream)))
    del keep
    return out


def rift_ile_lnZ(point: Point, draws, precision: int = FP32_MIXED, dist=None, stream=None):
    """(lnZ, sigma_lnZ, n_eff) of eq. lnL:MonteCarlo / eq. neff."""
    d = _as_draws(draws)
    out = (ctypes.c_double * 3)()
    ds, keep = _dist_struct(dist)
    _check(_lib.rift_ile_lnZ(point.handle, d.ref, precision,
                             ctypes.byref(ds) if ds is not None else None, out, _stream(stream)))
    del keep
    return float(out[0]), float(out[1]), float(out[2])


def rift_ile_lnZ_merge(states):
    """Merge LSE states [(m, s, s2, n), ...] -> ((lnZ, sigma, n_eff), merged state)."""
    arr = (_Lse * max(1, len(states)))()
    for i, s in enumerate(states):
        arr[i] = _Lse(*s)
    out = (ctypes.c_double * 3)()
    merged = _Lse()
    _check(_lib.rift_ile_lnZ_merge(arr, len(states), out, ctypes.byref(merged)))
    return (float(out[0]), float(out[1]), float(out[2])), (merged.m, merged.s, merged.s2, merged.n)


def rift_ile_lnZ_batch(points, draws_list, precision: int = FP32_MIXED, out=None, stream=None):
    """lnZ, sigma, n_eff of many points in one persistent launch ([P, 3] CUDA tensor)."""
    torch = _torch()
    P = len(points)
    ds = [_as_draws(d) for d in draws_list]
    handles = (ctypes.c_void_p * P)(*[p.handle.value for p in points])
    structs = (_Draws * P)(*[d.struct for d in ds])
    if out is None:
        out = torch.empty((P, 3), dtype=torch.float64, device=points[0].device)
    _check(_lib.rift_ile_lnZ_batch(handles, structs, P, precision, out.data_ptr(),
                                   _stream(stream)))
    out._keep_draws = ds  # the launch reads the draws asynchronously
    return out


class Batch:
    """A prepared multi-point lnZ (rift_ile_batch_create); launch() enqueues
    the persistent kernel and the per-point combine (capturable in a CUDA
    graph).  Keeps the points and draws alive while it exists."""

    def __init__(self, points, draws_list, precision: int = FP32_MIXED):
        self.points = list(points)
        self.draws = [_as_draws(d) for d in draws_list]
        P = len(self.points)
        handles = (ctypes.c_void_p * P)(*[p.handle.value for p in self.points])
        structs = (_Draws * P)(*[d.struct for d in self.draws])
        h = ctypes.c_void_p()
        _check(_lib.rift_ile_batch_create(handles, structs, P, precision, ctypes.byref(h)))
        self._h = h
        self.P = P
        self.device = self.points[0].device

    def launch(self, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.P, 3), dtype=torch.float64, device=self.device)
        _check(_lib.rift_ile_batch_launch(self._h, out.data_ptr(), _stream(stream)))
        return out

    def tune(self, reps: int = 3, stream=None):
        """Autotune the draw-tile size and grid of the persistent launch
        (rift_ile_batch_tune); returns (tile, blocks, ms per launch)."""
        tile, blocks, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(_lib.rift_ile_batch_tune(self._h, reps, _stream(stream), ctypes.byref(tile),
                                        ctypes.byref(blocks), ctypes.byref(ms)))
        return tile.value, blocks.value, ms.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.rift_ile_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _comp_mixed(cp, precision) -> bool:
    """Whether a composite point evaluates in its FP32-mixed form: asked for
    and built (rift_ile_comp_mixed_build)."""
    return precision == FP32_MIXED and rift_ile_comp_mixed_info(cp)[0] > 0


def _make_autograd():
    torch = _torch()

    class LnLFunction(torch.autograd.Function):
        """lnL per draw as a differentiable function of the seven extrinsic
        parameter tensors (Sec. II.B: gradient-based extrinsic sampling).

        When any parameter needs a gradient the forward launches the fused
        lnL + adjoint kernel once and keeps the [7, n] gradient; with
        recompute=True it launches the forward-only kernel and the backward
        launches the adjoint kernel again on the saved parameters (less memory,
        one more pass).  Backward returns grad_output * d lnL / d theta in the
        parameters' dtype.  With a distance table the lnD component is zero."""

        @staticmethod
        def forward(ctx, point, precision, dist, recompute, *theta):
            draws = Draws({p: x.detach() for p, x in zip(PARAMS, theta)})
            need = any(ctx.needs_input_grad[4:])
            ctx.point, ctx.precision, ctx.dist = point, precision, dist
            ctx.dtypes = [x.dtype for x in theta]
            ctx.grad = None
            if need and recompute:
                ctx.save_for_backward(*[x.detach() for x in theta])
            if isinstance(point, CompPoint):
                if dist is not None:
                    raise ValueError("distance marginalisation is not built for CompPoint")
                mixed = _comp_mixed(point, precision)
                if need and not recompute:
                    lnl, ctx.grad = (rift_ile_comp_lnL_grad_mixed if mixed
                                     else rift_ile_comp_lnL_grad)(point, draws)
                else:
                    lnl = (rift_ile_comp_lnL_mixed if mixed else rift_ile_comp_lnL)(point, draws)
            elif dist is not None:
                if need and not recompute:
                    lnl, ctx.grad = rift_ile_lnL_dist(point, draws, dist, precision, grad=True)
                else:
                    lnl = rift_ile_lnL_dist(point, draws, dist, precision)
            elif need and not recompute:
                lnl, ctx.grad = rift_ile_lnL_grad(point, draws, precision)
            else:
                lnl = rift_ile_lnL(point, draws, precision)
            return lnl

        @staticmethod
        def backward(ctx, grad_out):
            g = ctx.grad
            if g is None:
                theta = ctx.saved_tensors
                draws = Draws(dict(zip(PARAMS, theta)))
                if isinstance(ctx.point, CompPoint):
                    _, g = (rift_ile_comp_lnL_grad_mixed if _comp_mixed(ctx.point, ctx.precision)
                            else rift_ile_comp_lnL_grad)(ctx.point, draws)
                elif ctx.dist is not None:
                    _, g = rift_ile_lnL_dist(ctx.point, draws, ctx.dist, ctx.precision, grad=True)
                else:
                    _, g = rift_ile_lnL_grad(ctx.point, draws, ctx.precision)
            grads = [None] * 4
            for j in range(7):
                grads.append((g[j] * grad_out).to(ctx.dtypes[j])
                             if ctx.needs_input_grad[4 + j] else None)
            return tuple(grads)

    return LnLFunction


_LnLFunction = None


def lnL(point: Point, ra, dec, psi, incl, phase, lnD, t, precision: int = FP32_MIXED,
        dist=None, recompute: bool = False):
    """Differentiable lnL[n] (float64) of CUDA tensors of draws (torch autograd);
    dist = (x_nodes, lnw_nodes) marginalises the distance (eq. ap:dexp).  A
    CompPoint (composite-index response, Sec. III) evaluates in its FP32-mixed
    form when `precision` is FP32_MIXED and that form is built
    (rift_ile_comp_mixed_build), else in FP64."""
    global _LnLFunction
    if _LnLFunction is None:
        _LnLFunction = _make_autograd()
    return _LnLFunction.apply(point, precision, dist, recompute, ra, dec, psi, incl, phase, lnD, t)


def rift_ile_dist_nodes(d_min, d_max, d_ref, tol, rho_max, max_nodes=1 << 16):
    """Log-uniform lnD node table of eq. ap:dlog: (x_j, ln w_j)."""
    x = np.empty(max_nodes)
    w = np.empty(max_nodes)
    n = ctypes.c_int32()
    _check(_lib.rift_ile_dist_nodes(d_min, d_max, d_ref, tol, rho_max, max_nodes,
                                    x.ctypes.data, w.ctypes.data, ctypes.byref(n)))
    return x[:n.value].copy(), w[:n.value].copy()


def rift_ile_last_oob() -> int:
    return int(_lib.rift_ile_last_oob())


def rift_ile_set_small_batch(max_draws: int) -> int:
    """Draw count up to which FP32-mixed lnL and lnL + gradient calls use the
    warp-per-draw kernel (0 disables it); returns the previous value."""
    return int(_lib.rift_ile_set_small_batch(int(max_draws)))


PROBE_FP32_FMA, PROBE_FP64_FMA, PROBE_MUFU_EX2, PROBE_MUFU_SIN, PROBE_FP32X2_FMA = range(5)


def rift_ile_probe_alu(which: int, target_seconds: float = 0.2):
    """(ops per second, SM MHz seen by the probe) of FP32 FMA (0), FP64 FMA (1),
    MUFU ex2 (2), MUFU sin (3) or packed FP32 pair FMA (4, two ops each)."""
    ops = ctypes.c_double()
    mhz = ctypes.c_double()
    _check(_lib.rift_ile_probe_alu(which, target_seconds, ctypes.byref(ops), ctypes.byref(mhz)))
    return ops.value, mhz.value


def rift_ile_release():
    _check(_lib.rift_ile_release())


def shard_bounds(n: int, rank: int, world: int):
    """Contiguous slice [a, b) of n draws (or points) owned by `rank` of
    `world`: the draws of one point and the points of a batch are
    independent, so ranks share nothing but the final LSE states."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request n={n} rank={rank} world={world}")
    q, r = divmod(n, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def lnZ_merge_ranks(state, group=None):
    """The one exchange step of a draw-sharded lnZ: every rank contributes its
    LSE state (m, s, s2, n) and all ranks get ((lnZ, sigma, n_eff), merged
    state) from rift_ile_lnZ_merge over the states in rank order (an
    all-gather of 32 bytes per rank through torch.distributed)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    states = [None] * world
    dist.all_gather_object(states, tuple(float(v) for v in state), group=group)
    return rift_ile_lnZ_merge(states)


# ------------------------------------------------ composite-index response

RESP_ROTATION = 1
RESP_FINITE_ARM = 2


class _CompDesc(ctypes.Structure):
    _fields_ = [
        ("n_det", ctypes.c_int32), ("n_modes", ctypes.c_int32),
        ("ell", ctypes.c_void_p), ("em", ctypes.c_void_p),
        ("kind", ctypes.c_int32), ("p_max", ctypes.c_int32), ("omega", ctypes.c_double),
        ("arm_x", ctypes.c_void_p), ("arm_y", ctypes.c_void_p),
        ("Q", ctypes.c_void_p), ("q_len", ctypes.c_int32),
        ("q_t0", ctypes.c_void_p), ("q_dt", ctypes.c_double),
        ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
        ("det_pos", ctypes.c_void_p), ("det_resp", ctypes.c_void_p),
        ("gmst", ctypes.c_double), ("d_ref", ctypes.c_double),
    ]


_lib.rift_ile_comp_n_index.argtypes = [ctypes.c_int32, ctypes.c_int32]
_lib.rift_ile_comp_create.argtypes = [_P, _P, _P]
_lib.rift_ile_comp_destroy.argtypes = [_P]
_lib.rift_ile_comp_coeffs.argtypes = [_P, _P, _P, _P]
_lib.rift_ile_comp_lnL.argtypes = [_P, _P, _P, _P]
_lib.rift_ile_comp_lnZ_state.argtypes = [_P, _P, _P, _P]
_lib.rift_ile_comp_lnZ_state_async.argtypes = [_P, _P, _P, _P]
_lib.rift_ile_comp_mixed_build.argtypes = [_P, ctypes.c_double, _P]
_lib.rift_ile_comp_mixed_info.argtypes = [_P, _P]
_lib.rift_ile_comp_lnL_mixed.argtypes = [_P, _P, _P, _P]
_lib.rift_ile_comp_lnL_grad_mixed.argtypes = [_P, _P, _P, _P, _P]
_lib.rift_ile_comp_lnZ_state_mixed.argtypes = [_P, _P, _P, _P]
_lib.rift_ile_comp_lnZ_state_mixed_async.argtypes = [_P, _P, _P, _P]


def rift_ile_comp_n_index(kind: int, p_max: int) -> int:
    """Number of response indices a of the composite response (kind, p_max)."""
    na = _lib.rift_ile_comp_n_index(kind, p_max)
    if na < 0:
        _check(na)
    return na


class CompPoint:
    """An intrinsic point with a composite response (rift_ile_comp_create).

    point: dict with K, M, ell, em, kind (RESP_ROTATION or RESP_FINITE_ARM),
    p_max, omega (rad/s), arm_x[K, 3], arm_y[K, 3] (finite arms), Q[K, n, A]
    complex128 with A = n_index * M (composite index a * M + i), q_t0[K], q_dt,
    U[K, A, A], V[K, A, A], det_pos[K, 3], det_resp[K, 6], gmst, d_ref.
    """

    def __init__(self, point: dict, device=None, stream=None):
        torch = _torch()
        device = torch.device(device or "cuda")
        Q = _dev_tensor(point["Q"], torch.complex128, device)
        K, n, A = Q.shape
        kind, p_max = int(point["kind"]), int(point["p_max"])
        self.na = rift_ile_comp_n_index(kind, p_max)
        M = int(point["M"])
        if A != self.na * M:
            raise ValueError(f"Q has {A} composite columns, expected {self.na} x {M}")
        arms = kind == RESP_FINITE_ARM
        self._host = {
            "ell": np.ascontiguousarray(point["ell"], dtype=np.int32),
            "em": np.ascontiguousarray(point["em"], dtype=np.int32),
            "t0": np.ascontiguousarray(point["q_t0"], dtype=np.float64),
            "U": np.ascontiguousarray(np.asarray(point["U"], dtype=np.complex128)).view(np.float64),
            "V": np.ascontiguousarray(np.asarray(point["V"], dtype=np.complex128)).view(np.float64),
            "pos": np.ascontiguousarray(point["det_pos"], dtype=np.float64),
            "resp": np.ascontiguousarray(point["det_resp"], dtype=np.float64),
            "ax": np.ascontiguousarray(point["arm_x"], dtype=np.float64) if arms else None,
            "ay": np.ascontiguousarray(point["arm_y"], dtype=np.float64) if arms else None,
        }
        h = self._host
        d = _CompDesc()
        d.n_det, d.n_modes = K, M
        d.ell, d.em = h["ell"].ctypes.data, h["em"].ctypes.data
        d.kind, d.p_max, d.omega = kind, p_max, float(point.get("omega", 0.0))
        d.arm_x = h["ax"].ctypes.data if arms else None
        d.arm_y = h["ay"].ctypes.data if arms else None
        d.Q, d.q_len = Q.data_ptr(), n
        d.q_t0, d.q_dt = h["t0"].ctypes.data, float(point["q_dt"])
        d.U, d.V = h["U"].ctypes.data, h["V"].ctypes.data
        d.det_pos, d.det_resp = h["pos"].ctypes.data, h["resp"].ctypes.data
        d.gmst, d.d_ref = float(point["gmst"]), float(point["d_ref"])
        hd = ctypes.c_void_p()
        with torch.cuda.device(device):
            _check(_lib.rift_ile_comp_create(ctypes.byref(d), ctypes.byref(hd), _stream(stream)))
        self._h = hd
        self.K, self.M, self.n, self.A = K, M, n, A
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.rift_ile_comp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rift_ile_comp_coeffs(cp: CompPoint, draws, out=None, stream=None):
    """C~^k_a of every draw: complex128 CUDA tensor [n, K, n_index]."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty((d.n, cp.K, cp.na), dtype=torch.complex128, device=cp.device)
    _check(_lib.rift_ile_comp_coeffs(cp.handle, d.ref, out.data_ptr() if d.n else None,
                                     _stream(stream)))
    return out


def rift_ile_comp_lnL(cp: CompPoint, draws, out=None, stream=None):
    """lnL per draw of the composite response (float64 CUDA tensor), FP64."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(d.n, dtype=torch.float64, device=cp.device)
    _check(_lib.rift_ile_comp_lnL(cp.handle, d.ref, out.data_ptr() if d.n else None,
                                  _stream(stream)))
    return out


def rift_ile_comp_lnZ_state(cp: CompPoint, draws, stream=None):
    """LSE state (m, s, s2, n) of the draws under the composite response."""
    d = _as_draws(draws)
    st = _Lse()
    _check(_lib.rift_ile_comp_lnZ_state(cp.handle, d.ref, ctypes.byref(st), _stream(stream)))
    return (st.m, st.s, st.s2, st.n)


def rift_ile_comp_lnZ_state_async(cp: CompPoint, draws, out=None, stream=None):
    """The LSE state into a float64 CUDA tensor of 4, no host synchronisation."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=cp.device)
    _check(_lib.rift_ile_comp_lnZ_state_async(cp.handle, d.ref, out.data_ptr(), _stream(stream)))
    return out


def rift_ile_comp_lnZ(cp: CompPoint, draws, stream=None):
    """(lnZ, sigma_lnZ, n_eff) under the composite response."""
    return rift_ile_lnZ_merge([rift_ile_comp_lnZ_state(cp, draws, stream)])[0]


def rift_ile_comp_mixed_build(cp: CompPoint, tol: float = 1e-14, stream=None):
    """Builds the FP32-mixed (whitened) form of a composite point, keeping the
    eigen-directions of each class's quadratic form above tol x the largest
    eigenvalue; returns rift_ile_comp_mixed_info."""
    torch = _torch()
    with torch.cuda.device(cp.device):
        _check(_lib.rift_ile_comp_mixed_build(cp.handle, float(tol), _stream(stream)))
    return rift_ile_comp_mixed_info(cp)


def rift_ile_comp_mixed_info(cp: CompPoint):
    """(R, largest kept count of a class, classes, threads per block) of the
    mixed form; zeros before it is built."""
    out = np.zeros(4, dtype=np.int32)
    _check(_lib.rift_ile_comp_mixed_info(cp.handle, out.ctypes.data))
    return tuple(int(v) for v in out)


def rift_ile_comp_lnL_mixed(cp: CompPoint, draws, out=None, stream=None):
    """lnL per draw of the composite response (float64 CUDA tensor), FP32-mixed."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(d.n, dtype=torch.float64, device=cp.device)
    _check(_lib.rift_ile_comp_lnL_mixed(cp.handle, d.ref, out.data_ptr() if d.n else None,
                                        _stream(stream)))
    return out


def rift_ile_comp_lnL_grad_mixed(cp: CompPoint, draws, lnl_out=None, grad_out=None, stream=None):
    """(lnL[n], grad[7, n]) of the composite response as float64 CUDA tensors,
    FP32-mixed (rift_ile_comp_mixed_build first)."""
    torch = _torch()
    d = _as_draws(draws)
    if lnl_out is None:
        lnl_out = torch.empty(d.n, dtype=torch.float64, device=cp.device)
    if grad_out is None:
        grad_out = torch.empty((7, d.n), dtype=torch.float64, device=cp.device)
    _check(_lib.rift_ile_comp_lnL_grad_mixed(cp.handle, d.ref, lnl_out.data_ptr() if d.n else None,
                                             grad_out.data_ptr() if d.n else None,
                                             _stream(stream)))
    return lnl_out, grad_out


def rift_ile_comp_lnZ_state_mixed(cp: CompPoint, draws, stream=None):
    """LSE state (m, s, s2, n) of the draws, FP32-mixed composite likelihood."""
    d = _as_draws(draws)
    st = _Lse()
    _check(_lib.rift_ile_comp_lnZ_state_mixed(cp.handle, d.ref, ctypes.byref(st),
                                              _stream(stream)))
    return (st.m, st.s, st.s2, st.n)


def rift_ile_comp_lnZ_state_mixed_async(cp: CompPoint, draws, out=None, stream=None):
    """The mixed LSE state into a float64 CUDA tensor of 4, no host synchronisation."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=cp.device)
    _check(_lib.rift_ile_comp_lnZ_state_mixed_async(cp.handle, d.ref, out.data_ptr(),
                                                    _stream(stream)))
    return out


def rift_ile_comp_lnZ_mixed(cp: CompPoint, draws, stream=None):
    """(lnZ, sigma_lnZ, n_eff) under the composite response, FP32-mixed."""
    return rift_ile_lnZ_merge([rift_ile_comp_lnZ_state_mixed(cp, draws, stream)])[0]


# ------------------------------------------------------- Q, U, V precompute

class _PrecompDesc(ctypes.Structure):
    _fields_ = [
        ("n_det", ctypes.c_int32), ("n_modes", ctypes.c_int32), ("nf", ctypes.c_int32),
        ("df", ctypes.c_double), ("hlm", ctypes.c_void_p), ("dk", ctypes.c_void_p),
        ("wgt", ctypes.c_void_p), ("q_t0", ctypes.c_void_p), ("q_dt", ctypes.c_double),
        ("q_len", ctypes.c_int32), ("q_dtype", ctypes.c_int32),
    ]


_lib.rift_ile_precompute.argtypes = [_P, _P, _P, _P, _P]


def rift_ile_precompute(hlm, dk, wgt, df, q_t0, q_dt, q_len, q_dtype="complex64", device=None,
                        stream=None):
    """Q[K, q_len, M] (complex64 or complex128), U[K, M, M], V[K, M, M]
    (complex128) of eq. QUV on the GPU from the mode spectra hlm[M, nf], the
    data dk[K, nf] and the weights wgt[K, nf] on the two-sided grid of
    spacing df (nf odd); all CUDA tensors are returned."""
    torch = _torch()
    device = torch.device(device or "cuda")
    h = _dev_tensor(hlm, torch.complex128, device)
    d = _dev_tensor(dk, torch.complex128, device)
    w = _dev_tensor(wgt, torch.float64, device)
    M, nf = h.shape
    K = d.shape[0]
    t0 = np.ascontiguousarray(q_t0, dtype=np.float64)
    qt = {"complex64": torch.complex64, "complex128": torch.complex128}[q_dtype]
    Q = torch.empty((K, int(q_len), M), dtype=qt, device=device)
    U = torch.empty((K, M, M), dtype=torch.complex128, device=device)
    V = torch.empty_like(U)
    s = _PrecompDesc()
    s.n_det, s.n_modes, s.nf, s.df = K, M, nf, float(df)
    s.hlm, s.dk, s.wgt = h.data_ptr(), d.data_ptr(), w.data_ptr()
    s.q_t0, s.q_dt, s.q_len = t0.ctypes.data, float(q_dt), int(q_len)
    s.q_dtype = 1 if qt == torch.complex128 else 0
    with torch.cuda.device(device):
        _check(_lib.rift_ile_precompute(ctypes.byref(s), Q.data_ptr(), U.data_ptr(), V.data_ptr(),
                                        _stream(stream)))
    return Q, U, V


_lib.rift_ile_pregrid.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _P]


def rift_ile_pregrid(q_native, r: int, q_dtype="complex64", out=None, stream=None):
    """The fine table Q_fine[K, r (n - 1) + 1, M] of eq. q-time-pregrid from a
    native-rate table q_native[K, n, M] (complex64 or complex128 CUDA tensor,
    or array-like copied to the current device): reflected series, DFT,
    zero-padding x r, inverse DFT, on the GPU (cuFFT).  The fine spacing is
    the native spacing / r, from the same t0."""
    torch = _torch()
    q = q_native
    if not (torch.is_tensor(q) and q.is_cuda):
        q = torch.as_tensor(np.asarray(q)).to("cuda")
    if q.dtype not in (torch.complex64, torch.complex128):
        q = q.to(torch.complex128)
    q = q.contiguous()
    K, n, M = q.shape
    qt = {"complex64": torch.complex64, "complex128": torch.complex128}[q_dtype]
    if out is None:
        out = torch.empty((K, int(r) * (n - 1) + 1, M), dtype=qt, device=q.device)
    with torch.cuda.device(q.device):
        _check(_lib.rift_ile_pregrid(q.data_ptr(), K, M, n, 1 if q.dtype == torch.complex128 else 0,
                                     int(r), out.data_ptr(), 1 if out.dtype == torch.complex128 else 0,
                                     _stream(stream)))
    return out


_lib.rift_ile_comp_lnL_grad.argtypes = [_P, _P, _P, _P, _P]


def rift_ile_comp_lnL_grad(cp: CompPoint, draws, lnl_out=None, grad_out=None, stream=None):
    """(lnL[n], grad[7, n]) of the composite response as float64 CUDA tensors, FP64."""
    torch = _torch()
    d = _as_draws(draws)
    if lnl_out is None:
        lnl_out = torch.empty(d.n, dtype=torch.float64, device=cp.device)
    if grad_out is None:
        grad_out = torch.empty((7, d.n), dtype=torch.float64, device=cp.device)
    _check(_lib.rift_ile_comp_lnL_grad(cp.handle, d.ref, lnl_out.data_ptr() if d.n else None,
                                       grad_out.data_ptr() if d.n else None, _stream(stream)))
    return lnl_out, grad_out


# ------------------------------------------------- direct marginalisation

class _DirectRule(ctypes.Structure):
    _fields_ = [("n_phi", ctypes.c_int32), ("n_psi", ctypes.c_int32), ("n_gh", ctypes.c_int32),
                ("d_min", ctypes.c_double), ("d_max", ctypes.c_double), ("n_t", ctypes.c_int32),
                ("t_lo", ctypes.c_double), ("t_hi", ctypes.c_double), ("t_up", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("t_local", ctypes.c_int32),
                ("t_c", ctypes.c_double), ("t_tol", ctypes.c_double),
                ("t_mirror", ctypes.c_int32)]


_lib.rift_ile_lnL_direct.argtypes = [_P, _P, _P, _P, _P]
_lib.rift_ile_gauss_hermite.argtypes = [ctypes.c_int32, _P, _P]


def rift_ile_gauss_hermite(n: int):
    """The Gauss-Hermite rule (weight e^{-x^2}) the direct kernel uses: (x, w)."""
    x = np.empty(n)
    w = np.empty(n)
    _check(_lib.rift_ile_gauss_hermite(n, x.ctypes.data, w.ctypes.data))
    return x, w


def rift_ile_lnL_direct(point: Point, draws, n_phi: int, n_psi: int, n_gh: int, d_min: float,
                        d_max: float, n_t: int = 0, t_lo: float = 0.0, t_hi: float = 0.0,
                        t_up: int = 0, precision: int = FP64, out=None, stream=None,
                        t_local: bool = False, t_c: float = 16.0, t_tol: float = 1e-10,
                        t_mirror: bool = False):
    """ln L_dir per draw (float64 CUDA tensor): phase, polarisation and
    distance integrated inside the likelihood (ERAI on an n_phi x n_psi grid,
    adaptive Gauss-Hermite in x); uses each draw's ra, dec, incl and t, or
    with n_t > 0 integrates t over [t_lo, t_hi] on n_t midpoints, or with
    t_up > 1 on t_up sinc-reconstructed fine nodes per interval (eq. ap:tband),
    with t_local on those nodes by the peak-local rule (eq. ap:tlocal: the
    neighbourhoods of t_c sigma_t about the envelope's maxima, the rest
    bounded, the full rule when the bound exceeds t_tol); t_mirror takes the
    fine coefficients from the window's mirrored series instead of the
    truncated sinc sum.
    precision=FP32_MIXED takes the prior-weighted distance sum in float."""
    torch = _torch()
    d = _as_draws(draws)
    if out is None:
        out = torch.empty(d.n, dtype=torch.float64, device=point.device)
    r = _DirectRule(int(n_phi), int(n_psi), int(n_gh), float(d_min), float(d_max), int(n_t),
                    float(t_lo), float(t_hi), int(t_up), int(precision), int(bool(t_local)),
                    float(t_c), float(t_tol), int(bool(t_mirror)))
    _check(_lib.rift_ile_lnL_direct(point.handle, d.ref, ctypes.byref(r),
                                    out.data_ptr() if d.n else None, _stream(stream)))
    return out


_lib.rift_ile_rotation_bank.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int32, _P, _P]


def rift_ile_rotation_bank(hlm, df: float, omega: float, p_max: int, device=None, stream=None):
    """The widened Earth-rotation bank chi^(p,n)_lm [n_index * M, nf]
    (complex128 CUDA tensor) from mode spectra hlm[M, nf] on the two-sided
    grid of spacing df, by the DFT round trip of Appendix B."""
    torch = _torch()
    device = torch.device(device or "cuda")
    h = _dev_tensor(hlm, torch.complex128, device)
    M, nf = h.shape
    na = rift_ile_comp_n_index(RESP_ROTATION, p_max)
    out = torch.empty((na * M, nf), dtype=torch.complex128, device=device)
    with torch.cuda.device(device):
        _check(_lib.rift_ile_rotation_bank(h.data_ptr(), M, nf, float(df), float(omega), int(p_max),
                                           out.data_ptr(), _stream(stream)))
    return out


_lib.rift_ile_arm_bank.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int32, _P, _P]


def rift_ile_arm_bank(hlm, df: float, T: float, p_max: int, device=None, stream=None):
    """The finite-arm bank chi^(p)_lm = e^{-2 pi i f T} W_p(pi f T) h_lm
    [(p_max + 1) M, nf] (complex128 CUDA tensor), T the one-way light time."""
    torch = _torch()
    device = torch.device(device or "cuda")
    h = _dev_tensor(hlm, torch.complex128, device)
    M, nf = h.shape
    out = torch.empty(((p_max + 1) * M, nf), dtype=torch.complex128, device=device)
    with torch.cuda.device(device):
        _check(_lib.rift_ile_arm_bank(h.data_ptr(), M, nf, float(df), float(T), int(p_max),
                                      out.data_ptr(), _stream(stream)))
    return out


_lib.rift_ile_lnZ_direct_state.argtypes = [_P, _P, _P, _P, _P, _P]


def rift_ile_lnZ_direct(point: Point, draws, n_phi: int, n_psi: int, n_gh: int, d_min: float,
                        d_max: float, n_t: int = 0, t_lo: float = 0.0, t_hi: float = 0.0,
                        t_up: int = 0, precision: int = FP64, stream=None,
                        t_local: bool = False, t_c: float = 16.0, t_tol: float = 1e-10,
                        t_mirror: bool = False):
    """(lnZ, sigma_lnZ, n_eff) of the draws with the direct marginal as the
    integrand (the LSE state formed on the device, merged on the host)."""
    torch = _torch()
    d = _as_draws(draws)
    scratch = torch.empty(max(d.n, 1), dtype=torch.float64, device=point.device)
    state = torch.empty(4, dtype=torch.float64, device=point.device)
    r = _DirectRule(int(n_phi), int(n_psi), int(n_gh), float(d_min), float(d_max), int(n_t),
                    float(t_lo), float(t_hi), int(t_up), int(precision), int(bool(t_local)),
                    float(t_c), float(t_tol), int(bool(t_mirror)))
    _check(_lib.rift_ile_lnZ_direct_state(point.handle, d.ref, ctypes.byref(r), scratch.data_ptr(),
                                          state.data_ptr(), _stream(stream)))
    return rift_ile_lnZ_merge([tuple(state.cpu().tolist())])[0]
