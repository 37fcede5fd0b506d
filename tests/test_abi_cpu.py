"""CPU-only checks of the C ABI: the library loads, exports every symbol the
header declares, and its host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2410_01316_gb300 import _lib, build as qbuild
from paper_2410_01316_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return _lib.load()


def _declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            src = open(os.path.join(ROOT, "include", name)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            syms |= set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", src))
    return syms


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_symbols()
    assert declared, "no declarations found"
    assert declared == set(_lib.EXPORTS)
    for sym in sorted(declared):
        assert hasattr(lib, sym), sym


def test_status_strings_and_version(lib):
    for code in range(8):
        assert lib.qs_status_string(code).decode()
    assert b"sm_103a" in lib.qs_version()


def test_fibonacci_directions_match_workload_generator(lib):
    out = np.empty((64, 3), np.float32)
    assert lib.qs_directions(1, 3, 64, 0, out.ctypes.data_as(ctypes.c_void_p)) == 0
    ref = W.directions_fibonacci(64)
    assert np.max(np.abs(out - ref)) < 2e-7


@pytest.mark.parametrize("kind,d,P", [("orthogonal", 7, 20), ("orthogonal", 64, 128), ("iid", 5, 50)])
def test_generated_directions_are_unit_and_orthogonal(lib, kind, d, P):
    out = np.empty((P, d), np.float32)
    assert lib.qs_directions(_lib.DIRS[kind], d, P, 123, out.ctypes.data_as(ctypes.c_void_p)) == 0
    nrm = np.linalg.norm(out.astype(np.float64), axis=1)
    assert np.max(np.abs(nrm - 1)) < 1e-6
    if kind == "orthogonal":
        for p0 in range(0, P - d + 1, d):
            blk = out[p0:p0 + d].astype(np.float64)
            assert np.max(np.abs(blk @ blk.T - np.eye(d))) < 1e-6
    # deterministic in the seed, different across seeds
    out2 = np.empty_like(out)
    lib.qs_directions(_lib.DIRS[kind], d, P, 123, out2.ctypes.data_as(ctypes.c_void_p))
    assert np.array_equal(out, out2)
    lib.qs_directions(_lib.DIRS[kind], d, P, 124, out2.ctypes.data_as(ctypes.c_void_p))
    assert not np.array_equal(out, out2)


def test_orthogonal_directions_are_haar_in_distribution(lib):
    # E[xi_1^2] = 1/d for the first coordinate of a uniform direction
    d, P = 6, 6 * 400
    out = np.empty((P, d), np.float32)
    lib.qs_directions(2, d, P, 7, out.ctypes.data_as(ctypes.c_void_p))
    m2 = np.mean(out[:, 0].astype(np.float64) ** 2)
    assert abs(m2 - 1.0 / d) < 4 * np.sqrt(2.0 / (d * d) / P) + 0.01


def test_direction_argument_errors(lib):
    out = np.empty((4, 4), np.float32)
    assert lib.qs_directions(1, 4, 4, 0, out.ctypes.data_as(ctypes.c_void_p)) == 1  # Fibonacci needs d=3
    assert lib.qs_directions(2, 0, 4, 0, out.ctypes.data_as(ctypes.c_void_p)) == 1
    assert lib.qs_directions(2, 4, 4, 0, None) == 1
    assert lib.qs_last_error()


def test_plan_create_argument_errors_need_no_gpu(lib):
    desc = _lib.PlanDesc()
    h = ctypes.c_void_p()
    desc.d, desc.kernel, desc.kparam, desc.P, desc.dirs = 3, 0, 0.5, 16, 1
    desc.n_ft, desc.window, desc.radius, desc.max_n, desc.max_m = 100, 8, 2.0, 10, 10
    assert lib.qs_plan_create(ctypes.byref(h), ctypes.byref(desc)) == 6  # n_ft not a power of two
    desc.n_ft = 128
    desc.radius = -1.0
    assert lib.qs_plan_create(ctypes.byref(h), ctypes.byref(desc)) == 1
    desc.radius = 2.0
    desc.window = 7
    assert lib.qs_plan_create(ctypes.byref(h), ctypes.byref(desc)) == 6
    desc.window = 8
    desc.kparam = 0.0
    assert lib.qs_plan_create(ctypes.byref(h), ctypes.byref(desc)) == 1
    assert lib.qs_plan_create(None, ctypes.byref(desc)) == 1
    assert lib.qs_sum(None, None, 0, None, None, 0, None, None) == 1
    assert lib.qs_check(None, None) == 1
    assert lib.qs_plan_destroy(None) == 0


def test_kernel_parameter_errors_need_no_gpu(lib):
    desc = _lib.PlanDesc()
    h = ctypes.c_void_p()
    desc.d, desc.P, desc.dirs = 3, 16, 1
    desc.n_ft, desc.window, desc.radius, desc.max_n, desc.max_m = 128, 8, 2.0, 10, 10
    for kernel, kp, kp2 in (("matern", 0.5, 0.0), ("matern", -1.0, 1.5), ("riesz", 0.0, 0.0),
                            ("riesz", 2.0, 0.0), ("riesz", -0.5, 0.0)):
        desc.kernel, desc.kparam, desc.kparam2 = _lib.KERNELS[kernel], kp, kp2
        assert lib.qs_plan_create(ctypes.byref(h), ctypes.byref(desc)) == 1, (kernel, kp, kp2)
    desc.kernel = 6
    assert lib.qs_plan_create(ctypes.byref(h), ctypes.byref(desc)) == 1
    assert not h.value


def test_plan_create_without_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    desc = _lib.PlanDesc()
    h = ctypes.c_void_p()
    desc.d, desc.kernel, desc.kparam, desc.P, desc.dirs = 3, 0, 0.5, 16, 1
    desc.n_ft, desc.window, desc.radius, desc.max_n, desc.max_m = 128, 8, 2.0, 10, 10
    assert lib.qs_plan_create(ctypes.byref(h), ctypes.byref(desc)) == 5  # QS_ERR_CUDA
    assert not h.value


def test_plan_level_setters_reject_null_plans(lib):
    # QS_ERR_ARG (1) before any device work
    v = ctypes.c_int(-1)
    assert lib.qs_plan_set_gemm(None, 1) == 1
    assert lib.qs_plan_set_gemm(None, 0) == 1
    assert lib.qs_plan_gemm(None, ctypes.byref(v), None) == 1
    assert lib.qs_plan_set_variant(None, 0) == 1
    assert lib.qs_plan_variants(None, None, None) == 1
    assert lib.qs_sum_host(None, None, 0, None, None, 0, None, None) == 1
    assert "NULL" in lib.qs_last_error().decode()
