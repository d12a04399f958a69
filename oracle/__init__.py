"""Plain FP64 CPU oracle of the extrinsic-marginalised likelihood.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product (the
CUDA library and its binding) never does.  The C source ``rift_oracle.c`` is
written from the paper's equations and shares nothing with the CUDA path;
this module only marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rift_oracle.c")


def _host_key() -> str:
    """Short key of this host's CPU (model and instruction-set flags): the
    oracle is compiled for the host it runs on (-march=native), so each kind
    of host gets its own build."""
    import hashlib
    import platform
    info = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith(("model name", "flags", "Features", "CPU part")):
                    info += line
                if line.strip() == "":
                    break
    except OSError:
        pass
    return hashlib.sha1(info.encode()).hexdigest()[:10]


_LIB = os.path.join(_HERE, f"librift_oracle-{_host_key()}.so")
_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_HERE, "libopcount.so")

NPAR = 7
PARAMS = ("ra", "dec", "psi", "incl", "phase", "lnD", "t")


def _stale(lib: str, *srcs: str) -> bool:
    return not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O3 -march=native for the host it runs
    on, no fast-math), and the op counter (opcount.cpp) beside it."""
    hdr = os.path.join(_HERE, "rift_oracle.h")
    if force or _stale(_LIB, _SRC, hdr):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O3", "-march=native", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm", "-lpthread"]
        )
        os.replace(tmp, _LIB)
    if force or _stale(_OPC_LIB, _OPC_SRC, hdr):
        tmp = _OPC_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp,
                               _OPC_SRC])
        os.replace(tmp, _OPC_LIB)
    return _LIB


class _Point(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int), ("M", ctypes.c_int), ("n", ctypes.c_int),
        ("ell", ctypes.c_void_p), ("em", ctypes.c_void_p),
        ("Q", ctypes.c_void_p), ("t0", ctypes.c_void_p), ("dt", ctypes.c_double),
        ("U", ctypes.c_void_p), ("V", ctypes.c_void_p),
        ("pos", ctypes.c_void_p), ("resp", ctypes.c_void_p),
        ("gmst", ctypes.c_double), ("d_ref", ctypes.c_double),
        ("nf", ctypes.c_int), ("freq", ctypes.c_void_p), ("wgt", ctypes.c_void_p),
        ("hlm", ctypes.c_void_p), ("dk", ctypes.c_void_p),
    ]


_lib = None


def load(path: str):
    """Load an oracle shared library and declare its C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.ora_lnL_batch.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P, P]
    L.ora_grad_batch.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P]
    L.ora_lnZ.argtypes = [P, P, ctypes.c_int64, P]
    L.ora_lnL_distmarg_batch.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int,
                                         ctypes.c_int, P]
    L.ora_grad_distmarg_batch.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int,
                                          ctypes.c_int, P, P]
    L.ora_dist_nodes.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, P, P]
    L.ora_dist_nodes.restype = ctypes.c_int
    L.ora_sylm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                           ctypes.c_double, P, P]
    L.ora_sylm_dtheta.argtypes = L.ora_sylm.argtypes
    L.ora_antenna.argtypes = [P] + [ctypes.c_double] * 4 + [P, P]
    L.ora_delay.argtypes = [P] + [ctypes.c_double] * 4
    L.ora_delay.restype = ctypes.c_double
    L.ora_qinterp.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, P, P]
    L.ora_qinterp.restype = ctypes.c_int
    L.ora_sky_basis.argtypes = [ctypes.c_double] * 3 + [P, P, P]
    L.ora_nthreads_default.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


class use_library:
    """Context manager that routes this module's calls to another build of the
    oracle (the mutation tests compile deliberately broken copies)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = lib()
        _lib = load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def default_threads() -> int:
    return int(lib().ora_nthreads_default())


class OraclePoint:
    """Holds FP64 copies of one point's inputs (promoted exactly from the
    single-precision tables the GPU path reads) and the ctypes struct."""

    def __init__(self, point: dict, exact: dict | None = None):
        K, M = int(point["K"]), int(point["M"])
        Q = np.asarray(point["Q"])
        n = Q.shape[1]
        assert Q.shape == (K, n, M)
        self._keep = {
            "ell": np.ascontiguousarray(point["ell"], dtype=np.int32),
            "em": np.ascontiguousarray(point["em"], dtype=np.int32),
            "Q": np.ascontiguousarray(Q.astype(np.complex128)).view(np.float64),
            "t0": np.ascontiguousarray(point["q_t0"], dtype=np.float64),
            "U": np.ascontiguousarray(np.asarray(point["U"], dtype=np.complex128)).view(np.float64),
            "V": np.ascontiguousarray(np.asarray(point["V"], dtype=np.complex128)).view(np.float64),
            "pos": np.ascontiguousarray(point["det_pos"], dtype=np.float64),
            "resp": np.ascontiguousarray(point["det_resp"], dtype=np.float64),
        }
        s = _Point()
        s.K, s.M, s.n = K, M, n
        for name in ("ell", "em", "Q", "t0", "U", "V", "pos", "resp"):
            setattr(s, name, _ptr(self._keep[name]))
        s.dt = float(point["q_dt"])
        s.gmst = float(point["gmst"])
        s.d_ref = float(point["d_ref"])
        s.nf = 0
        if exact is not None:
            self._keep["freq"] = np.ascontiguousarray(exact["freq"], dtype=np.float64)
            self._keep["wgt"] = np.ascontiguousarray(exact["wgt"], dtype=np.float64)
            self._keep["hlm"] = np.ascontiguousarray(
                np.asarray(exact["hlm"], dtype=np.complex128)).view(np.float64)
            self._keep["dk"] = np.ascontiguousarray(
                np.asarray(exact["dk"], dtype=np.complex128)).view(np.float64)
            s.nf = int(self._keep["freq"].shape[0])
            for name in ("freq", "wgt", "hlm", "dk"):
                setattr(s, name, _ptr(self._keep[name]))
        self.struct = s
        self.K, self.M, self.n = K, M, n

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def _theta(draws: dict | np.ndarray) -> np.ndarray:
    if isinstance(draws, np.ndarray):
        th = np.ascontiguousarray(draws, dtype=np.float64)
        assert th.ndim == 2 and th.shape[1] == NPAR
        return th
    return np.ascontiguousarray(
        np.stack([np.asarray(draws[p], dtype=np.float64) for p in PARAMS], axis=1))


def lnL(pt: OraclePoint, draws, exact_q: bool = False, threads: int | None = None,
        terms: bool = False):
    """lnL per draw (eq. def:lnL:Decomposed).  With terms=True also returns
    the data term, the quadratic term and the out-of-table tap count."""
    th = _theta(draws)
    N = th.shape[0]
    out = np.empty(N)
    td = np.empty(N)
    tq = np.empty(N)
    oob = ctypes.c_int64(0)
    lib().ora_lnL_batch(pt.ref, _ptr(th), N, int(exact_q), threads or default_threads(),
                        _ptr(out), _ptr(td), _ptr(tq), ctypes.addressof(oob))
    if terms:
        return out, td, tq, int(oob.value)
    return out


def lnL_grad(pt: OraclePoint, draws, exact_q: bool = False, threads: int | None = None):
    """(lnL, grad[N, 7]) with the analytic chain-rule gradient (Sec. II.B)."""
    th = _theta(draws)
    N = th.shape[0]
    out = np.empty(N)
    g = np.empty((N, NPAR))
    lib().ora_grad_batch(pt.ref, _ptr(th), N, int(exact_q), threads or default_threads(),
                         _ptr(out), _ptr(g))
    return out, g


def lnZ(lnl: np.ndarray, logw: np.ndarray | None = None):
    """(lnZ, sigma_lnZ, n_eff) of eq. lnL:MonteCarlo and eq. neff."""
    lnl = np.ascontiguousarray(lnl, dtype=np.float64)
    lw = None if logw is None else np.ascontiguousarray(logw, dtype=np.float64)
    out = np.empty(3)
    lib().ora_lnZ(_ptr(lnl), _ptr(lw), lnl.shape[0], _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def dist_nodes(d_min: float, d_max: float, d_ref: float, tol: float, rho_max: float,
               max_nodes: int = 1 << 16):
    """The log-uniform lnD node table of eq. ap:dlog: (x_j, ln w_j)."""
    x = np.empty(max_nodes)
    w = np.empty(max_nodes)
    n = lib().ora_dist_nodes(d_min, d_max, d_ref, tol, rho_max, max_nodes, _ptr(x), _ptr(w))
    if n < 0:
        raise ValueError("node table larger than max_nodes")
    return x[:n].copy(), w[:n].copy()


def lnL_distmarg(pt: OraclePoint, draws, x_nodes, lnw_nodes, threads: int | None = None,
                 grad: bool = False):
    """Distance-marginalised lnL per draw (eq. ap:dexp summed on the nodes)."""
    th = _theta(draws)
    N = th.shape[0]
    xn = np.ascontiguousarray(x_nodes, dtype=np.float64)
    wn = np.ascontiguousarray(lnw_nodes, dtype=np.float64)
    out = np.empty(N)
    if grad:
        g = np.empty((N, NPAR))
        lib().ora_grad_distmarg_batch(pt.ref, _ptr(th), N, _ptr(xn), _ptr(wn), xn.shape[0],
                                      threads or default_threads(), _ptr(out), _ptr(g))
        return out, g
    lib().ora_lnL_distmarg_batch(pt.ref, _ptr(th), N, _ptr(xn), _ptr(wn), xn.shape[0],
                                 threads or default_threads(), _ptr(out))
    return out


def sylm(s: int, l: int, m: int, theta: float, phi: float, dtheta: bool = False) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    fn = lib().ora_sylm_dtheta if dtheta else lib().ora_sylm
    fn(s, l, m, theta, phi, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def antenna(resp, ra, dec, psi, gmst) -> complex:
    r = np.ascontiguousarray(resp, dtype=np.float64)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().ora_antenna(_ptr(r), ra, dec, psi, gmst, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def delay(pos, ra, dec, gmst, tc) -> float:
    p = np.ascontiguousarray(pos, dtype=np.float64)
    return float(lib().ora_delay(_ptr(p), ra, dec, gmst, tc))


def sky_basis(ra, dec, gmst):
    s, e1, e2 = np.empty(3), np.empty(3), np.empty(3)
    lib().ora_sky_basis(ra, dec, gmst, _ptr(s), _ptr(e1), _ptr(e2))
    return s, e1, e2


def qinterp(q: np.ndarray, t0: float, dt: float, t: float):
    """(Q(t)[M], dQ/dt[M], taps out of range) from one detector's table q[n][M]."""
    qq = np.ascontiguousarray(np.asarray(q, dtype=np.complex128)).view(np.float64)
    n, M = q.shape
    out = np.empty(2 * M)
    dout = np.empty(2 * M)
    oob = lib().ora_qinterp(_ptr(qq), n, M, t0, dt, t, _ptr(out), _ptr(dout))
    return out.view(np.complex128), dout.view(np.complex128), int(oob)


_opc = None


def op_counts(pt: OraclePoint, draws, which: str, logw=None, x_nodes=None, lnw_nodes=None):
    """Counted plain evaluation (opcount.cpp) over the draws, one thread.

    which: "lnZ" (lnL and the online log-sum-exp), "grad" (lnL and its
    gradient), "dist" (distance-marginalised lnL over the node table) or
    "dist_grad".  Returns a dict with the per-draw values, the gradient
    [N, 7] (gradient modes), the online LSE (max, sum e, sum e^2) ("lnZ") and
    the totals add, mul, div, special (sin, cos, exp, log) over the N draws;
    flops = add + mul + div."""
    global _opc
    if _opc is None:
        build()
        _opc = ctypes.CDLL(_OPC_LIB)
        P = ctypes.c_void_p
        _opc.ora_count_ops.argtypes = [P, P, ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_int,
                                       P, P, P, P]
        _opc.ora_count_ops.restype = ctypes.c_int
    code = {"lnZ": 0, "grad": 1, "dist": 2, "dist_grad": 3}[which]
    th = _theta(draws)
    N = th.shape[0]
    vals = np.empty(N)
    g = np.zeros((N, NPAR))
    lse = np.zeros(3)
    cnt = np.zeros(4, dtype=np.int64)
    lw = None if logw is None else np.ascontiguousarray(logw, dtype=np.float64)
    xn = None if x_nodes is None else np.ascontiguousarray(x_nodes, dtype=np.float64)
    wn = None if lnw_nodes is None else np.ascontiguousarray(lnw_nodes, dtype=np.float64)
    rc = _opc.ora_count_ops(pt.ref, _ptr(th), N, _ptr(lw), _ptr(xn), _ptr(wn),
                            0 if xn is None else xn.shape[0], code, _ptr(vals), _ptr(g),
                            _ptr(lse), _ptr(cnt))
    if rc != 0:
        raise ValueError(which)
    add, mul, div, special = (int(v) for v in cnt)
    return {"values": vals, "grad": g, "lse": lse, "add": add, "mul": mul, "div": div,
            "special": special, "flops": add + mul + div, "n": N}
