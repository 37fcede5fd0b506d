"""FP64 CPU oracle for the QMC-slicing kernel sum (arXiv 2410.01316).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import it; the
library itself never does, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
slices); this module compiles it with gcc into ``liboracle.so`` next to the
source and wraps it with ctypes.  Each wrapper names the passage of the paper
that the C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KERNEL_IDS = {"gauss": 0, "laplace": 1, "negdist": 2, "matern": 3, "riesz": 4, "tps": 5}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2 -fopenmp, IEEE double)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            lib.o_tau.restype = d
            lib.o_tau.argtypes = [i, d, d]
            lib.o_riesz_const.restype = d
            lib.o_riesz_const.argtypes = [i]
            lib.o_riesz_const_r.restype = d
            lib.o_riesz_const_r.argtypes = [i, d]
            lib.o_tps_const.restype = d
            lib.o_tps_const.argtypes = [i]
            lib.o_F2.restype = d
            lib.o_F2.argtypes = [i, d, d, d]
            lib.o_f2.restype = d
            lib.o_f2.argtypes = [i, d, d, i, d]
            lib.o_fhat2.restype = d
            lib.o_fhat2.argtypes = [i, d, d, i, d]
            lib.o_coeffs2.restype = i
            lib.o_coeffs2.argtypes = [i, d, d, i, d, i, p]
            lib.o2_exact2.restype = i
            lib.o2_exact2.argtypes = [i, d, d, i, i64, p, p, i64, p, p, i]
            lib.o3_grad_negdist.restype = i
            lib.o3_grad_negdist.argtypes = [i, i64, p, p, i64, p, p, i, p, p, i]
            lib.o_esym.restype = i
            lib.o_esym.argtypes = [i, i, p, p, p, i]
            lib.o3_sliced2.restype = i
            lib.o3_sliced2.argtypes = [i, d, d, i, i64, p, p, i64, p, i, p, p, i]
            lib.o_F.restype = d
            lib.o_F.argtypes = [i, d, d]
            lib.o_f.restype = d
            lib.o_f.argtypes = [i, d, i, d]
            lib.o_fhat.restype = d
            lib.o_fhat.argtypes = [i, d, i, d]
            lib.o_coeffs.restype = i
            lib.o_coeffs.argtypes = [i, d, i, d, i, p]
            lib.o1_sum.restype = i
            lib.o1_sum.argtypes = [i, i64, p, p, i64, p, i, p, d, i, p, p, i]
            lib.o1_grad.restype = i
            lib.o1_grad.argtypes = [i, i64, p, p, i64, p, p, i, p, d, i, p,
                                    i64, p, p, p, i64, p, p, i]
            lib.o2_exact.restype = i
            lib.o2_exact.argtypes = [i, d, i, i64, p, p, i64, p, p, i]
            lib.o3_sliced.restype = i
            lib.o3_sliced.argtypes = [i, d, i, i64, p, p, i64, p, i, p, p, i]
            _lib = lib
    return _lib


def _kid(kernel: str) -> int:
    return KERNEL_IDS[kernel]


def _f32(a: np.ndarray | None, shape_last: int | None = None) -> np.ndarray | None:
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------------------
# scalar pieces
# ---------------------------------------------------------------------------
def tau(kernel: str, kparam: float, R: float) -> float:
    """Rescaling factor (App. C Step 1; App. G for the negative distance)."""
    return float(_load().o_tau(_kid(kernel), float(kparam), float(R)))


def riesz_const(d: int, r: float = 1.0) -> float:
    """c_{d,r} with f(t) = -c_{d,r} |t|^r for F(x) = -x^r (Table tab:kernels, Riesz row)."""
    if r == 1.0:
        return float(_load().o_riesz_const(int(d)))
    return float(_load().o_riesz_const_r(int(d), float(r)))


def tps_const(d: int) -> float:
    """C_d with f(t) = d t^2 log|t| + C_d t^2 for F(x) = x^2 log x (Table tab:kernels)."""
    return float(_load().o_tps_const(int(d)))


def F(kernel: str, kparam: float, r: float, nu: float = 0.0) -> float:
    """Radial basis function (Table tab:kernels); Matern takes beta = kparam, nu (half-integers)."""
    return float(_load().o_F2(_kid(kernel), float(kparam), float(nu), float(r)))


def f(kernel: str, kparam: float, d: int, t: float, nu: float = 0.0) -> float:
    """Closed-form 1D basis function (d=1, d=3, or the negative distance, Riesz and thin plate
    spline kernels in any d)."""
    return float(_load().o_f2(_kid(kernel), float(kparam), float(nu), int(d), float(t)))


def fhat(kernel: str, kparam: float, d: int, omega: float, nu: float = 0.0) -> float:
    """F_1[f(|.|)](omega) (Table tab:kernels, corrected constants)."""
    return float(_load().o_fhat2(_kid(kernel), float(kparam), float(nu), int(d), float(omega)))


def coeffs(kernel: str, kparam: float, d: int, tau_: float, n_ft: int, nu: float = 0.0) -> np.ndarray:
    """c_k for k = -n_ft/2 .. n_ft/2-1 (App. C Step 2; App. G)."""
    c = np.zeros(n_ft, dtype=np.float64)
    _check(_load().o_coeffs2(_kid(kernel), float(kparam), float(nu), int(d), float(tau_), int(n_ft),
                             _ptr(c)), "coeffs")
    return c


# ---------------------------------------------------------------------------
# sums
# ---------------------------------------------------------------------------
def o1_sum(x, w, y, xi, tau_: float, c: np.ndarray, threads: int = 0) -> np.ndarray:
    """Sliced, Fourier-truncated sum by direct NDFT (eq. kernel_sum_sliced with
    eq. 1d_sum_fourier); the quantity the fast method approximates."""
    x, y, xi = _f32(x), _f32(y), _f32(xi)
    w = _f32(w)
    c = np.ascontiguousarray(c, dtype=np.float64)
    d = xi.shape[1]
    s = np.zeros(y.shape[0], dtype=np.float64)
    _check(_load().o1_sum(d, x.shape[0], _ptr(x), _ptr(w), y.shape[0], _ptr(y), xi.shape[0],
                          _ptr(xi), float(tau_), c.shape[0], _ptr(c), _ptr(s), int(threads)),
           "o1_sum")
    return s


def o1_grad(x, w, y, v, xi, tau_: float, c: np.ndarray, idx_n=None, idx_m=None,
            want=("x", "w", "y"), threads: int = 0) -> dict:
    """Gradients of L = sum_m v_m s_m for the O1 sum, at sampled indices."""
    x, y, xi, v = _f32(x), _f32(y), _f32(xi), _f32(v)
    w = _f32(w)
    c = np.ascontiguousarray(c, dtype=np.float64)
    d = xi.shape[1]
    N, M = x.shape[0], y.shape[0]
    idx_n = np.arange(N, dtype=np.int64) if idx_n is None else np.ascontiguousarray(idx_n, np.int64)
    idx_m = np.arange(M, dtype=np.int64) if idx_m is None else np.ascontiguousarray(idx_m, np.int64)
    gx = np.zeros((idx_n.size, d)) if "x" in want else None
    gw = np.zeros(idx_n.size) if "w" in want else None
    gy = np.zeros((idx_m.size, d)) if "y" in want else None
    _check(_load().o1_grad(d, N, _ptr(x), _ptr(w), M, _ptr(y), _ptr(v), xi.shape[0], _ptr(xi),
                           float(tau_), c.shape[0], _ptr(c), idx_n.size, _ptr(idx_n), _ptr(gx),
                           _ptr(gw), idx_m.size, _ptr(idx_m), _ptr(gy), int(threads)),
           "o1_grad")
    return {"x": gx, "w": gw, "y": gy}


def o2_exact(kernel: str, kparam: float, x, w, y, threads: int = 0, nu: float = 0.0) -> np.ndarray:
    """Exact kernel sum s_m = sum_n w_n F(|x_n - y_m|) (eq. kernel_sum)."""
    x, y, w = _f32(x), _f32(y), _f32(w)
    s = np.zeros(y.shape[0], dtype=np.float64)
    _check(_load().o2_exact2(_kid(kernel), float(kparam), float(nu), x.shape[1], x.shape[0], _ptr(x),
                             _ptr(w), y.shape[0], _ptr(y), _ptr(s), int(threads)), "o2_exact")
    return s


def o3_sliced(kernel: str, kparam: float, x, w, y, xi, threads: int = 0, nu: float = 0.0) -> np.ndarray:
    """Sliced sum with closed-form f, no Fourier step (eq. kernel_sum_sliced)."""
    x, y, w, xi = _f32(x), _f32(y), _f32(w), _f32(xi)
    s = np.zeros(y.shape[0], dtype=np.float64)
    _check(_load().o3_sliced2(_kid(kernel), float(kparam), float(nu), x.shape[1], x.shape[0], _ptr(x),
                              _ptr(w), y.shape[0], _ptr(y), xi.shape[0], _ptr(xi), _ptr(s), int(threads)),
           "o3_sliced")
    return s


def o1_problem(prob, threads: int = 0, y=None) -> np.ndarray:
    """O1 for a workloads.Problem (optionally on a subset of targets y)."""
    nu = getattr(prob, "kparam2", 0.0)
    t = tau(prob.kernel, prob.kparam, prob.R)
    c = coeffs(prob.kernel, prob.kparam, prob.d, t, prob.n_ft, nu=nu)
    return o1_sum(prob.x, prob.w, prob.y if y is None else y, prob.xi, t, c, threads)


def esym(xi, grad: bool = True, threads: int = 0):
    """Symmetric distance energy E_sym = -2 sum_{p,q} (|xi_p - xi_q| + |xi_p + xi_q|) and its
    gradient (eq. distance-sym; Sec. 2.3 eq. distance-mmd)."""
    xi = _f32(xi)
    P, d = xi.shape
    E = ctypes.c_double(0.0)
    g = np.zeros((P, d)) if grad else None
    _check(_load().o_esym(d, P, _ptr(xi), ctypes.byref(E), _ptr(g), int(threads)), "esym")
    return E.value, g


def o3_grad_negdist(x, w, y, v, xi, threads: int = 0) -> np.ndarray:
    """Gradient in y of L = sum_m v_m s_m for the sliced negative-distance sum with
    closed-form f (eq. kernel_sum_sliced), sign(0) = 0."""
    x, y, w, v, xi = _f32(x), _f32(y), _f32(w), _f32(v), _f32(xi)
    M, d = y.shape
    g = np.zeros((M, d))
    _check(_load().o3_grad_negdist(d, x.shape[0], _ptr(x), _ptr(w), M, _ptr(y), _ptr(v), xi.shape[0], _ptr(xi),
                                   _ptr(g), int(threads)), "o3_grad_negdist")
    return g
