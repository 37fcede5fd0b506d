"""qs_sum_noalloc: the kernel sum for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- code under a framework whose caching
allocator owns the GPU's memory, loops that must never stall on an
allocation, plugins that are handed their buffers and nothing else -- so they
cannot create a plan.  qs_sum_noalloc keeps every intermediate in a static
device array reserved by the library instead.  These tests call it through the
C ABI twice in a row and compare each result with the plan-based qs_sum on the
same inputs (bit for bit: both use the same host tables, the same slice-group
count and the same kernels) and with the FP64 oracle, within the parity
tolerance of the other GPU tests (1e-5 relative to sum|w| max|F|).  The file
name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
    desc.window_kind = _lib.WINDOWS[getattr(prob, "window_kind", "es")]
    return desc


def _norm(prob, use_w):
    sw = float(np.abs(prob.w.astype(np.float64)).sum()) if use_w else float(prob.N)
    return sw * (prob.R if prob.kernel == "negdist" else 1.0)


def _case(name):
    if name == "small_gauss":
        return W.small_gauss(), True
    if name == "negdist_d16_unit_weights":
        return W.tiny(d=16, N=3000, M=900, P=48, kernel="negdist", kparam=0.0, n_ft=512, seed=17), False
    if name.startswith("laplace_W"):
        prob = W.tiny(d=4, N=1500, M=700, P=24, kernel="laplace", kparam=1.3, n_ft=256, seed=23)
        prob.window = int(name[len("laplace_W"):].split("_")[0])
        if name.endswith("_kb"):
            prob.window_kind = "kb"
        return prob, True
    # d <= 8 with enough targets that the slice-group count falls below its cap
    # (two targets per interpolation thread in the fused form)
    return W.tiny(d=6, N=2000, M=40000, P=48, kernel="gauss", kparam=1.5, n_ft=512, seed=29), True


@pytest.mark.parametrize("case", ["small_gauss", "negdist_d16_unit_weights", "laplace_W6", "laplace_W10",
                                  "laplace_W12", "laplace_W8_kb", "gauss_d6_many_targets"])
def test_noalloc_matches_plan_sum_on_two_calls_in_a_row(case):
    import torch

    prob, use_w = _case(case)
    x = torch.from_numpy(prob.x).cuda()
    y = torch.from_numpy(prob.y).cuda()
    w = torch.from_numpy(prob.w).cuda() if use_w else None
    with QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, window=prob.window,
                proj="fp32_fused", max_n=prob.N, max_m=prob.M,
                window_kind=getattr(prob, "window_kind", "es")) as plan:
        ref = plan.sum(x, w, y)
        plan.check()
        ref = ref.cpu().numpy().astype(np.float64)
    t = oracle.tau(prob.kernel, prob.kparam, prob.R)
    c = oracle.coeffs(prob.kernel, prob.kparam, prob.d, t, prob.n_ft)
    idx = np.random.default_rng(3).choice(prob.M, min(prob.M, 256), replace=False)
    o1 = oracle.o1_sum(prob.x, prob.w if use_w else None, prob.y[idx], prob.xi, t, c)

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
        assert np.array_equal(got, ref)
        assert np.max(np.abs(got[idx] - o1)) / _norm(prob, use_w) < TOL


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


def test_noalloc_flags_non_finite_directions():
    import torch

    prob = W.tiny(d=3, N=200, M=50, P=8, kernel="gauss", kparam=1.0, n_ft=64, seed=4)
    xi = prob.xi.copy()
    xi[3, 1] = np.nan
    desc = _desc(prob)
    lib = _lib.load()
    x = torch.from_numpy(prob.x).cuda()
    y = torch.from_numpy(prob.y).cuda()
    out = torch.empty(prob.M, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.qs_sum_noalloc(ctypes.byref(desc), torch.from_numpy(xi).cuda().data_ptr(), x.data_ptr(), prob.N, None,
                            y.data_ptr(), prob.M, out.data_ptr(), stream)
    assert rc == 3  # QS_ERR_NONFINITE
    # the next call with valid directions starts from a cleared flag
    rc = lib.qs_sum_noalloc(ctypes.byref(desc), torch.from_numpy(prob.xi).cuda().data_ptr(), x.data_ptr(), prob.N,
                            None, y.data_ptr(), prob.M, out.data_ptr(), stream)
    assert rc == 0, lib.qs_last_error().decode()
