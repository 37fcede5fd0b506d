"""qs_sum_noalloc: the kernel sum for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- code under a framework whose caching
allocator owns the GPU's memory, loops that must never stall on an
allocation, plugins that are handed their buffers and nothing else -- so they
cannot create a plan.  qs_sum_noalloc keeps every intermediate in a static
device array reserved by the library instead.  These tests call it through the
C ABI twice in a row and compare each result with the plan-based qs_sum on the
same inputs, within the parity tolerance of the other GPU tests (1e-5 relative
to sum|w| max|F|).  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_01316_gb300 import QSPlan, _lib
from paper_2410_01316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _desc(prob):
    desc = _lib.PlanDesc()
    desc.d, desc.kernel, desc.kparam, desc.P = prob.d, _lib.KERNELS[prob.kernel], float(prob.kparam), prob.P
    desc.dirs, desc.seed, desc.dirs_host = _lib.DIRS["user"], 0, None
    desc.n_ft, desc.window, desc.oversampling, desc.radius = prob.n_ft, prob.window, 2.0, float(prob.R)
    desc.proj, desc.max_n, desc.max_m = _lib.PROJ["fp32_fused"], 0, 0
    return desc


def _norm(prob, use_w):
    sw = float(np.abs(prob.w.astype(np.float64)).sum()) if use_w else float(prob.N)
    return sw * (prob.R if prob.kernel == "negdist" else 1.0)


@pytest.mark.parametrize("case", ["small_gauss", "negdist_d16_unit_weights"])
def test_noalloc_matches_plan_sum_on_two_calls_in_a_row(case):
    import torch

    if case == "small_gauss":
        prob, use_w = W.small_gauss(), True
    else:
        prob, use_w = W.tiny(d=16, N=3000, M=900, P=48, kernel="negdist", kparam=0.0, n_ft=512, seed=17), False
    x = torch.from_numpy(prob.x).cuda()
    y = torch.from_numpy(prob.y).cuda()
    w = torch.from_numpy(prob.w).cuda() if use_w else None
    with QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, window=prob.window,
                proj="fp32_fused", max_n=prob.N, max_m=prob.M) as plan:
        ref = plan.sum(x, w, y)
        plan.check()
        ref = ref.cpu().numpy().astype(np.float64)

    lib = _lib.load()
    desc = _desc(prob)
    dirs_dev = torch.from_numpy(prob.xi).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty(prob.M, dtype=torch.float32, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        rc = lib.qs_sum_noalloc(ctypes.byref(desc), dirs_dev.data_ptr(), x.data_ptr(), prob.N,
                                None if w is None else w.data_ptr(), y.data_ptr(), prob.M, out.data_ptr(), stream)
        assert rc == 0, lib.qs_last_error().decode()
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) / _norm(prob, use_w) < TOL


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch

    prob = W.tiny(d=3, N=10, M=10, P=4096, kernel="gauss", kparam=1.0, n_ft=4096, seed=1)
    desc = _desc(prob)  # 4096 slices x 8192 cells of grid alone need 128 MiB
    lib = _lib.load()
    dirs_dev = torch.from_numpy(prob.xi).cuda()
    x = torch.from_numpy(prob.x).cuda()
    y = torch.from_numpy(prob.y).cuda()
    out = torch.empty(prob.M, dtype=torch.float32, device="cuda")
    rc = lib.qs_sum_noalloc(ctypes.byref(desc), dirs_dev.data_ptr(), x.data_ptr(), prob.N, None, y.data_ptr(),
                            prob.M, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 6  # QS_ERR_UNSUPPORTED
    assert b"scratch" in lib.qs_last_error()
