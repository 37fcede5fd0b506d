"""Sorting slicing for the negative distance kernel on the GPU (qs_sum_sorted):
the exact sliced sum (Sec. 2.1 eq. kernel_sum_sliced with f(t) = -c_d |t|) against
the oracle's closed-form sliced sum O3 on the plan's own directions, relative to
sum|w| R.

The 1D sums are exact (FP64 prefix sums over a stable sort); what remains is
the FP32 rounding of the projections (sort keys) and of each slice's value,
which averages out over sources and slices: the error falls like
2^-24 c_d / sqrt(N P).  Measured on GB300: ~2e-9 for the small random cases
(N ~ 1e3, P ~ 50), 1.2e-10 for the large one (N = 6e4, P = 96), 4e-8 with unit
weights (no cancellation between sources, so the slice values are N R large);
the tolerances sit a few times above those."""
import numpy as np
import pytest

import oracle
from paper_2410_01316_gb300 import QSError, QSPlan
from paper_2410_01316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-8          # random weights, small N and P
TOL_UNIT = 2e-7     # unit weights
TOL_LARGE = 1e-9    # N = 6e4, P = 96


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sorted_sum(prob, use_w=True, proj="fp32", idx=None):
    with QSPlan(prob.d, "negdist", prob.P, prob.n_ft, prob.R, dirs=prob.xi, proj=proj, max_n=prob.N,
                max_m=prob.M) as plan:
        w = _cuda(prob.w) if use_w else None
        s = plan.sum_sorted(_cuda(prob.x), w, _cuda(prob.y))
        plan.check()
        xi = plan.directions()
    return s.cpu().numpy().astype(np.float64), xi


@pytest.mark.parametrize("d,N,M,P", [(3, 1000, 700, 40), (16, 3001, 517, 70), (64, 2500, 2048, 33)])
def test_sorted_sum_matches_exact_sliced_sum(d, N, M, P):
    prob = W.tiny(d=d, N=N, M=M, P=P, kernel="negdist", kparam=0.0, n_ft=256, seed=90 + d)
    s, xi = _sorted_sum(prob)
    ref = oracle.o3_sliced("negdist", 0.0, prob.x, prob.w, prob.y, xi)
    err = np.max(np.abs(s - ref)) / (np.abs(prob.w).sum() * prob.R)
    print(f"sorted sum d={d} N={N} M={M} P={P}: error vs exact sliced sum {err:.3e}")
    assert err < TOL


def test_sorted_sum_unit_weights_duplicates_and_empty():
    prob = W.tiny(d=5, N=1200, M=300, P=24, kernel="negdist", kparam=0.0, n_ft=128, seed=3)
    prob.x[100:160] = prob.x[7]          # repeated sources: equal keys
    prob.y[:20] = prob.x[7]              # targets on top of them
    s, xi = _sorted_sum(prob, use_w=False)
    ref = oracle.o3_sliced("negdist", 0.0, prob.x, None, prob.y, xi)
    err = np.max(np.abs(s - ref)) / (prob.N * prob.R)
    print(f"sorted sum with duplicates: error {err:.3e}")
    assert err < TOL_UNIT
    import torch

    with QSPlan(prob.d, "negdist", prob.P, prob.n_ft, prob.R, dirs=prob.xi, proj="fp32", max_n=prob.N,
                max_m=prob.M) as plan:
        out = plan.sum_sorted(torch.empty((0, prob.d), device="cuda"), None, _cuda(prob.y))
        plan.check()
        assert np.all(out.cpu().numpy() == 0.0)


def test_sorted_sum_large_sampled_targets():
    prob = W.gauss64_negdist(N=60000, M=50000, P=96)
    s, xi = _sorted_sum(prob, proj="bf16x3")
    idx = np.random.default_rng(1).choice(prob.M, 64, replace=False)
    ref = oracle.o3_sliced("negdist", 0.0, prob.x, prob.w, prob.y[idx], xi)
    err = np.max(np.abs(s[idx] - ref)) / (np.abs(prob.w).sum() * prob.R)
    print(f"sorted sum large: error {err:.3e}")
    assert err < TOL_LARGE


def test_sorted_sum_refuses_other_kernels():
    prob = W.tiny(d=3, N=100, M=50, P=8, kernel="gauss", kparam=1.0, n_ft=64, seed=1)
    with QSPlan(prob.d, "gauss", prob.P, prob.n_ft, prob.R, 1.0, dirs=prob.xi, max_n=prob.N, max_m=prob.M) as plan:
        with pytest.raises(QSError) as ei:
            plan.sum_sorted(_cuda(prob.x), _cuda(prob.w), _cuda(prob.y))
        assert ei.value.status == 6


@pytest.mark.parametrize("d,N,M,P", [(3, 900, 400, 40), (16, 2000, 700, 70)])
def test_sorted_gradient_matches_exact_sliced_gradient(d, N, M, P):
    prob = W.tiny(d=d, N=N, M=M, P=P, kernel="negdist", kparam=0.0, n_ft=256, seed=120 + d)
    v = np.random.default_rng(9).standard_normal(M).astype(np.float32)
    with QSPlan(prob.d, "negdist", prob.P, prob.n_ft, prob.R, dirs=prob.xi, proj="fp32", max_n=N, max_m=M) as plan:
        g = plan.grad_sorted(_cuda(prob.x), _cuda(prob.w), _cuda(prob.y), _cuda(v))
        plan.check()
        xi = plan.directions()
    ref = oracle.o3_grad_negdist(prob.x, prob.w, prob.y, v, xi)
    norm = oracle.riesz_const(d) * np.abs(prob.w).sum() * np.abs(v).max()
    err = np.max(np.abs(g.cpu().numpy() - ref)) / norm
    print(f"sorted gradient d={d}: error {err:.3e}")
    assert err < TOL
    assert np.max(np.abs(ref)) / norm > 1e-3
