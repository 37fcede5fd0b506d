"""GB300-native fast radial kernel summation via QMC slicing (arXiv 2410.01316).

Python binding of the C ABI in ``include/qmcslice.h``.  PyTorch supplies device
memory and streams; all arithmetic runs in the CUDA library
(``libqmcslice.so``), which must have been built (``build.build()``).

    plan = QSPlan(d=3, kernel="gauss", kparam=0.5, P=64, n_ft=256, radius=2.0,
                  dirs=xi, max_n=N, max_m=M)
    s = plan.sum(x, w, y)          # x: (N, d), w: (N,), y: (M, d) float32 CUDA tensors
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib
from ._lib import QSError

__all__ = ["QSPlan", "QSBatch", "QSError", "KernelSumFn", "directions", "sobol_points", "kernel_sum", "version",
           "distance_design", "distance_energy", "tune_cache_save", "tune_cache_load", "tune_cache_clear",
           "tune_cache_size"]


def version() -> str:
    return _lib.load().qs_version().decode()


def directions(kind: str, d: int, P: int, seed: int = 0) -> np.ndarray:
    """Host-side direction design from the library (Fibonacci / orthogonal / iid / Sobol)."""
    out = np.empty((P, d), dtype=np.float32)
    _lib.check(_lib.load().qs_directions(_lib.DIRS[kind], d, P, seed, out.ctypes.data_as(ctypes.c_void_p)),
               "qs_directions")
    return out


def sobol_points(d: int, P: int, seed: int = 0) -> np.ndarray:
    """The library's Sobol' points in (0, 1)^d (P x d, float64) behind the "sobol" directions;
    seed != 0 applies a random digital shift."""
    out = np.empty((P, d), dtype=np.float64)
    _lib.check(_lib.load().qs_sobol_points(d, P, seed, out.ctypes.data_as(ctypes.c_void_p)), "qs_sobol_points")
    return out


def tune_cache_save(path: str) -> None:
    """Write the library's autotune cache (tuned choices per shape class) to a text file."""
    _lib.check(_lib.load().qs_tune_cache_save(path.encode()), "qs_tune_cache_save")


def tune_cache_load(path: str) -> None:
    """Merge a saved autotune cache into the library's cache."""
    _lib.check(_lib.load().qs_tune_cache_load(path.encode()), "qs_tune_cache_load")


def tune_cache_clear() -> None:
    _lib.check(_lib.load().qs_tune_cache_clear(), "qs_tune_cache_clear")


def tune_cache_size() -> int:
    return int(_lib.load().qs_tune_cache_size())


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class QSPlan:
    """A plan for sums s = sum_n w_n F(|x_n - y_m|) with fixed d, kernel, P, N_ft."""

    def __init__(self, d: int, kernel: str, P: int, n_ft: int, radius: float, kparam: float = 0.0,
                 dirs="orthogonal", seed: int = 0, window: int = 8, proj: str = "auto",
                 max_n: int = 0, max_m: int = 0, device=None, kparam2: float = 0.0, window_kind: str = "es"):
        import torch

        lib = _lib.load()
        self._lib = lib
        self._handle = ctypes.c_void_p()
        desc = _lib.PlanDesc()
        desc.d, desc.kernel, desc.kparam, desc.P = d, _lib.KERNELS[kernel], float(kparam), P
        self._dirs_keep = None
        if isinstance(dirs, str):
            desc.dirs = _lib.DIRS[dirs]
            desc.dirs_host = None
        else:
            arr = np.ascontiguousarray(dirs, dtype=np.float32)
            if arr.shape != (P, d):
                raise ValueError(f"dirs must have shape ({P}, {d}), got {arr.shape}")
            self._dirs_keep = arr
            desc.dirs = _lib.DIRS["user"]
            desc.dirs_host = arr.ctypes.data_as(ctypes.c_void_p)
        desc.seed = seed
        desc.n_ft, desc.window, desc.oversampling = n_ft, window, 2.0
        desc.radius = float(radius)
        desc.proj = _lib.PROJ[proj]
        desc.max_n, desc.max_m = int(max_n), int(max_m)
        desc.kparam2 = float(kparam2)
        desc.window_kind = _lib.WINDOWS[window_kind]
        self.window_kind = window_kind
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            _lib.check(lib.qs_plan_create(ctypes.byref(self._handle), ctypes.byref(desc)), "qs_plan_create")
        self.d, self.kernel, self.kparam, self.kparam2, self.P, self.n_ft = d, kernel, kparam, kparam2, P, n_ft
        self.window, self.proj, self.max_n, self.max_m, self.radius = window, proj, max_n, max_m, radius
        tau = ctypes.c_double()
        G = ctypes.c_int()
        _lib.check(lib.qs_plan_info(self._handle, ctypes.byref(tau), ctypes.byref(G), None, None), "qs_plan_info")
        self.tau, self.G = tau.value, G.value

    # -- lifetime ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_handle", None) and self._handle.value:
            self._lib.qs_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- queries ----------------------------------------------------------
    def directions(self) -> np.ndarray:
        out = np.empty((self.P, self.d), dtype=np.float32)
        _lib.check(self._lib.qs_plan_directions(self._handle, out.ctypes.data_as(ctypes.c_void_p)),
                   "qs_plan_directions")
        return out

    # -- tuning -------------------------------------------------------------
    SPREAD_VARIANTS = ("point1", "point2", "point4", "thread32", "moment", "momentwin32")

    def autotune(self, x, w=None, stream=None) -> str:
        """Time the spread variants on these sources and keep the fastest."""
        self._check_points(x, "x")
        v = ctypes.c_int(-1)
        _lib.check(self._lib.qs_plan_autotune(self._handle, x.data_ptr(), x.shape[0],
                                              None if w is None else w.data_ptr(), ctypes.byref(v),
                                              _stream_handle(stream)), "qs_plan_autotune")
        return self.SPREAD_VARIANTS[v.value]

    def autotune_gemm(self, x, stream=None) -> bool:
        """Time the projection GEMM forms on these points and keep the faster; True for SM pairs."""
        self._check_points(x, "x")
        v = ctypes.c_int(-1)
        _lib.check(self._lib.qs_plan_autotune_gemm(self._handle, x.data_ptr(), x.shape[0], ctypes.byref(v),
                                                   _stream_handle(stream)), "qs_plan_autotune_gemm")
        return v.value == 1

    def set_variant(self, name: str) -> None:
        _lib.check(self._lib.qs_plan_set_variant(self._handle, self.SPREAD_VARIANTS.index(name)),
                   "qs_plan_set_variant")

    def set_gemm(self, pair: bool) -> None:
        """Projection GEMM on SM pairs (tcgen05 cta_group::2, 256-point tiles) or one CTA per SM."""
        _lib.check(self._lib.qs_plan_set_gemm(self._handle, 1 if pair else 0), "qs_plan_set_gemm")

    def gemm_pair(self) -> bool:
        """Whether the projection GEMM runs on SM pairs."""
        v = ctypes.c_int(-1)
        _lib.check(self._lib.qs_plan_gemm(self._handle, ctypes.byref(v), None), "qs_plan_gemm")
        return v.value == 1

    def gemm_ctas(self) -> int:
        """CTAs of a full-size launch of the plan's projection GEMM."""
        v, c = ctypes.c_int(-1), ctypes.c_int(-1)
        _lib.check(self._lib.qs_plan_gemm(self._handle, ctypes.byref(v), ctypes.byref(c)), "qs_plan_gemm")
        return c.value

    def spread_variants(self) -> tuple:
        """Names of the spread variants of this plan's family (bitwise identical to each other)."""
        mask = ctypes.c_uint(0)
        _lib.check(self._lib.qs_plan_variants(self._handle, ctypes.byref(mask), None), "qs_plan_variants")
        return tuple(n for i, n in enumerate(self.SPREAD_VARIANTS) if mask.value >> i & 1)

    def variant(self) -> str:
        """The spread variant in use."""
        cur = ctypes.c_int(-1)
        _lib.check(self._lib.qs_plan_variants(self._handle, None, ctypes.byref(cur)), "qs_plan_variants")
        return self.SPREAD_VARIANTS[cur.value]

    # -- stage timing -----------------------------------------------------
    STAGES = ("prep_x", "project_x", "spread_filter", "prep_y", "project_y", "interp", "reduce")

    def set_timing(self, enable: bool) -> None:
        _lib.check(self._lib.qs_set_timing(self._handle, 1 if enable else 0), "qs_set_timing")

    def stage_times(self) -> dict:
        """Stage durations (ms) of the most recent timed sum, from CUDA events."""
        ms = (ctypes.c_float * len(self.STAGES))()
        _lib.check(self._lib.qs_stage_times(self._handle, ms, len(self.STAGES)), "qs_stage_times")
        return dict(zip(self.STAGES, [float(v) for v in ms]))

    # -- sums -------------------------------------------------------------
    def _check_points(self, t, name, rows=None):
        import torch

        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
        if t.device != self.device:
            raise ValueError(f"{name} is on {t.device}, plan on {self.device}")
        if rows is not None and t.shape[0] != rows:
            raise ValueError(f"{name} has {t.shape[0]} rows, expected {rows}")

    def sum(self, x, w, y, out=None, stream=None):
        """s_m = sum_n w_n F(|x_n - y_m|) on the device (asynchronous on the stream)."""
        import torch

        self._check_points(x, "x")
        self._check_points(y, "y")
        if x.dim() != 2 or x.shape[1] != self.d or y.dim() != 2 or y.shape[1] != self.d:
            raise ValueError("x and y must have shape (*, d)")
        N, M = x.shape[0], y.shape[0]
        if w is not None:
            self._check_points(w, "w", rows=N)
        if out is None:
            out = torch.empty(M, dtype=torch.float32, device=self.device)
        else:
            self._check_points(out, "out", rows=M)
        _lib.check(self._lib.qs_sum(self._handle, x.data_ptr(), N, None if w is None else w.data_ptr(),
                                    y.data_ptr(), M, out.data_ptr(), _stream_handle(stream)), "qs_sum")
        return out

    def sum_sorted(self, x, w, y, out=None, stream=None):
        """The sliced negative-distance sum computed exactly by sorting each slice (no Fourier
        truncation); negdist plans with d <= 64.  The first call allocates the sorting workspace."""
        import torch

        self._check_points(x, "x")
        self._check_points(y, "y")
        if x.dim() != 2 or x.shape[1] != self.d or y.dim() != 2 or y.shape[1] != self.d:
            raise ValueError("x and y must have shape (*, d)")
        N, M = x.shape[0], y.shape[0]
        if w is not None:
            self._check_points(w, "w", rows=N)
        if out is None:
            out = torch.empty(M, dtype=torch.float32, device=self.device)
        else:
            self._check_points(out, "out", rows=M)
        _lib.check(self._lib.qs_sum_sorted(self._handle, x.data_ptr(), N, None if w is None else w.data_ptr(),
                                           y.data_ptr(), M, out.data_ptr(), _stream_handle(stream)), "qs_sum_sorted")
        return out

    def grad_sorted(self, x, w, y, v=None, out=None, stream=None):
        """Gradient in y of sum_m v_m s_m for the exact sliced negative-distance sum (M x d tensor)."""
        import torch

        self._check_points(x, "x")
        self._check_points(y, "y")
        N, M = x.shape[0], y.shape[0]
        if w is not None:
            self._check_points(w, "w", rows=N)
        if v is not None:
            self._check_points(v, "v", rows=M)
        if out is None:
            out = torch.empty((M, self.d), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.qs_grad_sorted(self._handle, x.data_ptr(), N, None if w is None else w.data_ptr(),
                                            y.data_ptr(), M, None if v is None else v.data_ptr(), out.data_ptr(),
                                            _stream_handle(stream)), "qs_grad_sorted")
        return out

    def project(self, x, out=None, stream=None):
        """u[p, n] = G tau <x_n, xi_p> in the plan's projection form (P x N tensor)."""
        import torch

        self._check_points(x, "x")
        N = x.shape[0]
        if out is None:
            out = torch.empty((self.P, N), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.qs_project(self._handle, x.data_ptr(), N, out.data_ptr(), out.stride(0),
                                        _stream_handle(stream)), "qs_project")
        return out

    def grad(self, x, w, y, v=None, want=("x", "w", "y"), stream=None):
        """Gradients of L = sum_m v_m s_m (dict with 'x', 'w', 'y'; None where not wanted)."""
        import torch

        self._check_points(x, "x")
        self._check_points(y, "y")
        N, M = x.shape[0], y.shape[0]
        if w is not None:
            self._check_points(w, "w", rows=N)
        if v is not None:
            self._check_points(v, "v", rows=M)
        gx = torch.empty((N, self.d), dtype=torch.float32, device=self.device) if "x" in want else None
        gw = torch.empty(N, dtype=torch.float32, device=self.device) if "w" in want else None
        gy = torch.empty((M, self.d), dtype=torch.float32, device=self.device) if "y" in want else None
        ptr = lambda t: None if t is None else t.data_ptr()
        _lib.check(self._lib.qs_grad(self._handle, x.data_ptr(), N, ptr(w), y.data_ptr(), M, ptr(v), ptr(gx),
                                     ptr(gw), ptr(gy), _stream_handle(stream)), "qs_grad")
        return {"x": gx, "w": gw, "y": gy}

    def sum_host(self, x: np.ndarray, w, y: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Same sum from host arrays (copies in, computes, copies out, synchronises)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        wp = None
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float32)
            wp = w.ctypes.data_as(ctypes.c_void_p)
        if out is None:
            out = np.empty(y.shape[0], dtype=np.float32)
        _lib.check(self._lib.qs_sum_host(self._handle, x.ctypes.data_as(ctypes.c_void_p), x.shape[0], wp,
                                         y.ctypes.data_as(ctypes.c_void_p), y.shape[0],
                                         out.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)),
                   "qs_sum_host")
        return out

    def check(self, stream=None) -> None:
        """Synchronise and raise QSError if the device flagged a data error."""
        _lib.check(self._lib.qs_check(self._handle, _stream_handle(stream)), "qs_check")

    def status(self, stream=None) -> int:
        """Synchronise and return the device error status without raising."""
        return int(self._lib.qs_check(self._handle, _stream_handle(stream)))


class QSBatch:
    """Many independent problems (one QSPlan each) summed in one persistent launch."""

    def __init__(self, plans):
        self._lib = _lib.load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._handle.value for p in self.plans])
        self._handle = ctypes.c_void_p()
        _lib.check(self._lib.qs_batch_create(ctypes.byref(self._handle), arr, len(self.plans)), "qs_batch_create")
        self._probs = (_lib.Problem * len(self.plans))()

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            self._lib.qs_batch_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tiling(self, targets_per_thread: int) -> None:
        _lib.check(self._lib.qs_batch_set_tiling(self._handle, targets_per_thread), "qs_batch_set_tiling")

    def set_mode(self, concurrent: bool) -> None:
        """Persistent kernel (False, default) or every problem's own pipeline on the batch's streams."""
        _lib.check(self._lib.qs_batch_set_mode(self._handle, 1 if concurrent else 0), "qs_batch_set_mode")

    def autotune(self, problems, stream=None) -> int:
        """Time the persistent kernel's interpolation tilings (1, 2, 4 targets per thread) and the
        concurrent mode on these problems and keep the fastest; returns the tiling, or 0 for the
        concurrent mode."""
        self._fill(problems)
        v = ctypes.c_int(-1)
        _lib.check(self._lib.qs_batch_autotune(self._handle, self._probs, ctypes.byref(v), _stream_handle(stream)),
                   "qs_batch_autotune")
        return v.value

    def sum(self, problems, stream=None):
        """problems: list of (x, w, y, out) CUDA tensors (w may be None), one per plan."""
        self._fill(problems)
        _lib.check(self._lib.qs_sum_batched(self._handle, self._probs, _stream_handle(stream)), "qs_sum_batched")

    def _fill(self, problems):
        if len(problems) != len(self.plans):
            raise ValueError("one problem per plan")
        for k, (x, w, y, out) in enumerate(problems):
            pl = self.plans[k]
            pl._check_points(x, "x")
            pl._check_points(y, "y")
            pl._check_points(out, "out", rows=y.shape[0])
            if w is not None:
                pl._check_points(w, "w", rows=x.shape[0])
            self._probs[k] = _lib.Problem(x.data_ptr(), x.shape[0], None if w is None else w.data_ptr(),
                                          y.data_ptr(), y.shape[0], out.data_ptr())

    def check(self, stream=None) -> None:
        _lib.check(self._lib.qs_batch_check(self._handle, _stream_handle(stream)), "qs_batch_check")


def _make_fn():
    import torch

    class KernelSumFn(torch.autograd.Function):
        """s = plan.sum(x, w, y) with gradients from qs_grad (w may be None).

        backward(v) returns dL/dx, dL/dw, dL/dy for L = <v, s>, computed on the
        device by the adjoint pipeline (derivative filter + back-projection)."""

        @staticmethod
        def forward(ctx, x, w, y, plan):
            ctx.plan = plan
            ctx.has_w = w is not None
            ctx.save_for_backward(x, w if w is not None else x.new_empty(0), y)
            return plan.sum(x.contiguous(), None if w is None else w.contiguous(), y.contiguous())

        @staticmethod
        def backward(ctx, v):
            x, w, y = ctx.saved_tensors
            need = ctx.needs_input_grad
            want = tuple(k for k, n in zip(("x", "w", "y"), need[:3]) if n)
            g = ctx.plan.grad(x.contiguous(), w if ctx.has_w else None, y.contiguous(), v.contiguous(), want=want)
            return g["x"], (g["w"] if ctx.has_w else None), g["y"], None

    return KernelSumFn


class _LazyFn:
    _fn = None

    def __getattr__(self, name):
        if _LazyFn._fn is None:
            _LazyFn._fn = _make_fn()
        return getattr(_LazyFn._fn, name)


KernelSumFn = _LazyFn()


def kernel_sum(x, w, y, kernel: str, kparam: float = 0.0, P: int = 256, n_ft: int = 512, dirs="orthogonal",
               seed: int = 0, radius: float | None = None, proj: str = "auto", window: int = 8,
               kparam2: float = 0.0):
    """One-shot convenience wrapper: builds a plan sized for these inputs (kparam2 = nu for "matern")."""
    import torch

    if radius is None:
        radius = float(x.norm(dim=1).max() + y.norm(dim=1).max()) * (1 + 1e-6)
    with QSPlan(x.shape[1], kernel, P, n_ft, radius, kparam, dirs, seed, window, proj, x.shape[0], y.shape[0],
                device=x.device.index, kparam2=kparam2) as plan:
        s = plan.sum(x, w, y)
        torch.cuda.current_stream().synchronize()
        plan.check()
        return s


def _dirs_tensor(xi):
    import torch

    if not (isinstance(xi, torch.Tensor) and xi.is_cuda and xi.dtype == torch.float32 and xi.is_contiguous()
            and xi.dim() == 2):
        raise TypeError("xi must be a contiguous float32 CUDA tensor of shape (P, d)")
    return xi


def distance_design(xi, iters: int = 300, lr: float | None = None, stream=None) -> float:
    """Refine the unit rows of xi (P x d CUDA tensor, in place) towards a distance QMC design:
    `iters` Adam steps on E_sym = -2 sum_{p,q} (|xi_p - xi_q| + |xi_p + xi_q|) (Sec. 2.3,
    eq. distance-sym), rows renormalised after each step.  Returns E_sym of the result."""
    import torch

    xi = _dirs_tensor(xi)
    P, d = xi.shape
    lr = 0.05 / math.sqrt(d) if lr is None else lr
    E = ctypes.c_double(0.0)
    with torch.cuda.device(xi.device):
        _lib.check(_lib.load().qs_distance_design(xi.data_ptr(), d, P, int(iters), float(lr), ctypes.byref(E),
                                                  _stream_handle(stream)), "qs_distance_design")
    return E.value


def distance_energy(xi, grad: bool = False, stream=None):
    """E_sym of the unit rows of xi and, with grad=True, its gradient (a new P x d tensor)."""
    import torch

    xi = _dirs_tensor(xi)
    P, d = xi.shape
    E = ctypes.c_double(0.0)
    g = torch.empty_like(xi) if grad else None
    with torch.cuda.device(xi.device):
        _lib.check(_lib.load().qs_distance_energy(xi.data_ptr(), d, P, ctypes.byref(E),
                                                  None if g is None else g.data_ptr(), _stream_handle(stream)),
                   "qs_distance_energy")
    return (E.value, g) if grad else E.value
