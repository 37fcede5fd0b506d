"""The Matern, generalised Riesz and thin plate spline kernels on the GPU.

Parity of the whole sum (and of the gradients) with the oracle's O1 for the
same kernel, on the same seeded inputs and directions, within 1e-5 of
sum|w| max|F|, where max|F| is taken over [0, R]: 1 for Matern, R^q for
Riesz, max(R^2 |log R|, 1/(2e)) for the thin plate spline.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2410_01316_gb300 import QSPlan, _lib
from paper_2410_01316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _maxF(prob):
    if prob.kernel == "matern":
        return 1.0
    if prob.kernel == "riesz":
        return prob.R ** prob.kparam
    if prob.kernel == "tps":
        return max(prob.R ** 2 * abs(math.log(prob.R)), 0.5 / math.e)
    return prob.R if prob.kernel == "negdist" else 1.0


def _plan(prob, proj):
    return QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, proj=proj,
                  max_n=prob.N, max_m=prob.M, kparam2=prob.kparam2)


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_sum(prob, proj):
    with _plan(prob, proj) as plan:
        s = plan.sum(_cuda(prob.x), _cuda(prob.w), _cuda(prob.y))
        plan.check()
        return s.cpu().numpy().astype(np.float64), plan.tau


CASES = [
    ("matern", 0.9, 1.5, 3, "fp32_fused", 512),
    ("matern", 2.0, 3.5, 16, "fp32", 512),
    ("matern", 6.0, 2.5, 64, "bf16x3", 512),
    ("riesz", 0.5, 0.0, 3, "fp32_fused", 256),
    ("riesz", 1.5, 0.0, 16, "fp32", 512),
    ("tps", 0.0, 0.0, 3, "fp32_fused", 256),
    ("tps", 0.0, 0.0, 16, "fp32", 512),
]


@pytest.mark.parametrize("kernel,kp,nu,d,proj,n_ft", CASES)
def test_sum_matches_oracle(kernel, kp, nu, d, proj, n_ft):
    prob = W.tiny(d=d, N=2500, M=700, P=48, kernel=kernel, kparam=kp, n_ft=n_ft, seed=60 + d, kparam2=nu)
    s, tau = _gpu_sum(prob, proj)
    t = oracle.tau(kernel, kp, prob.R)
    assert tau == pytest.approx(t, rel=1e-15)
    ref = oracle.o1_problem(prob)
    err = np.max(np.abs(s - ref)) / (np.abs(prob.w.astype(np.float64)).sum() * _maxF(prob))
    assert err < TOL
    # and the answer is not trivially small against its normalisation
    assert np.max(np.abs(ref)) / (np.abs(prob.w.astype(np.float64)).sum() * _maxF(prob)) > 1e-3


def test_riesz_one_equals_negative_distance():
    # q = 1 is the negative distance kernel: quadrature coefficients vs the closed form
    prob = W.tiny(d=8, N=2000, M=500, P=32, kernel="riesz", kparam=1.0, n_ft=512, seed=9)
    a, _ = _gpu_sum(prob, "fp32")
    prob.kernel, prob.kparam = "negdist", 0.0
    b, _ = _gpu_sum(prob, "fp32")
    assert np.max(np.abs(a - b)) / (np.abs(prob.w.astype(np.float64)).sum() * prob.R) < 1e-6


@pytest.mark.parametrize("kernel,kp,nu,d", [("matern", 1.0, 1.5, 3), ("tps", 0.0, 0.0, 8)])
def test_grad_matches_oracle(kernel, kp, nu, d):
    prob = W.tiny(d=d, N=1200, M=500, P=32, kernel=kernel, kparam=kp, n_ft=256, seed=70 + d, kparam2=nu)
    v = np.random.default_rng(5).standard_normal(prob.M).astype(np.float32)
    with _plan(prob, "fp32_fused") as plan:
        g = plan.grad(_cuda(prob.x), _cuda(prob.w), _cuda(prob.y), _cuda(v))
        plan.check()
        g = {k: t.cpu().numpy().astype(np.float64) for k, t in g.items()}
    t = oracle.tau(kernel, kp, prob.R)
    c = oracle.coeffs(kernel, kp, prob.d, t, prob.n_ft, nu=nu)
    ref = oracle.o1_grad(prob.x, prob.w, prob.y, v, prob.xi, t, c)
    k = np.arange(-prob.n_ft // 2, prob.n_ft // 2)
    D1 = float(np.sum(np.abs(2 * np.pi * k * c)))
    sw, mw = float(np.abs(prob.w).sum()), float(np.abs(prob.w).max())
    sv, mv = float(np.abs(v).sum()), float(np.abs(v).max())
    assert np.max(np.abs(g["y"] - ref["y"])) / (t * sw * mv * D1) < TOL
    assert np.max(np.abs(g["x"] - ref["x"])) / (t * mw * sv * D1) < TOL
    assert np.max(np.abs(g["w"] - ref["w"])) / (sv * _maxF(prob)) < TOL


def test_noalloc_refuses_quadrature_kernels_and_runs_matern():
    import torch

    lib = _lib.load()
    prob = W.tiny(d=3, N=900, M=300, P=16, kernel="matern", kparam=0.8, n_ft=256, seed=4, kparam2=1.5)
    desc = _lib.PlanDesc()
    desc.d, desc.kernel, desc.kparam, desc.kparam2, desc.P = 3, _lib.KERNELS["matern"], 0.8, 1.5, prob.P
    desc.dirs, desc.n_ft, desc.window, desc.oversampling, desc.radius = _lib.DIRS["user"], prob.n_ft, 8, 2.0, prob.R
    desc.proj = _lib.PROJ["fp32_fused"]
    x, w, y, xi = _cuda(prob.x), _cuda(prob.w), _cuda(prob.y), _cuda(prob.xi)
    out = torch.empty(prob.M, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.qs_sum_noalloc(ctypes.byref(desc), xi.data_ptr(), x.data_ptr(), prob.N, w.data_ptr(), y.data_ptr(),
                            prob.M, out.data_ptr(), stream)
    assert rc == 0, lib.qs_last_error().decode()
    ref, _ = _gpu_sum(prob, "fp32_fused")
    assert np.max(np.abs(out.cpu().numpy() - ref)) / np.abs(prob.w).sum() < TOL
    for kernel, kp in (("riesz", 0.5), ("tps", 0.0)):
        desc.kernel, desc.kparam = _lib.KERNELS[kernel], kp
        rc = lib.qs_sum_noalloc(ctypes.byref(desc), xi.data_ptr(), x.data_ptr(), prob.N, w.data_ptr(),
                                y.data_ptr(), prob.M, out.data_ptr(), stream)
        assert rc == 6  # QS_ERR_UNSUPPORTED
