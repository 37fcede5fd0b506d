"""Sorting slicing for the negative distance kernel on the GPU (qs_sum_sorted):
the exact sliced sum (Sec. 2.1 eq. kernel_sum_sliced with f(t) = -c_d |t|) against
the oracle's closed-form sliced sum O3 on the plan's own directions, relative to
sum|w| R.

The 1D sums are exact (64-bit fixed-point prefix sums over a stable sort);
what remains is the FP32 rounding of the projections (sort keys), of the
fixed-point terms (2^-51 of the slice's scale) and of each slice's value,
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
TOL_WIDE = 5e-8     # weights over 70 decades: a few sources carry sum|w|, so the FP32 roundings of
                    # their keys and of the slice values average over few terms (measured 8.9e-9)


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


def test_sorted_sum_scales_exactly_with_power_of_two_weights():
    # the fixed-point scales follow max|w|: multiplying every weight by 2^k moves both exponents
    # by -k, so the integer prefix sums are the same integers and every slice value, compensated
    # sum and the result scale by exactly 2^k (no value leaves the normal FP32 range here)
    import dataclasses

    prob = W.tiny(d=16, N=3001, M=517, P=70, kernel="negdist", kparam=0.0, n_ft=256, seed=7)
    s0, _ = _sorted_sum(prob)
    for k in (-60, 40):
        pk = dataclasses.replace(prob, w=(prob.w * np.float32(2.0 ** k)).astype(np.float32))
        sk, _ = _sorted_sum(pk)
        assert np.array_equal(sk, s0 * 2.0 ** k), k


def test_sorted_sum_with_denormal_and_huge_weight_ranges():
    # weights spanning ~70 orders of magnitude, some of them FP32 denormals: the significands
    # are normalised before the fixed-point products, so only the terms below 2^-51 of the
    # slice's scale are lost
    prob = W.tiny(d=3, N=2000, M=300, P=24, kernel="negdist", kparam=0.0, n_ft=128, seed=11)
    rng = np.random.default_rng(5)
    w = (rng.standard_normal(prob.N) * 10.0 ** rng.uniform(-45, 25, prob.N)).astype(np.float32)
    w[:10] = np.float32(3e-42)  # denormal
    import dataclasses

    pw = dataclasses.replace(prob, w=w)
    s, xi = _sorted_sum(pw)
    ref = oracle.o3_sliced("negdist", 0.0, pw.x, pw.w, pw.y, xi)
    err = np.max(np.abs(s - ref)) / (np.abs(pw.w.astype(np.float64)).sum() * pw.R)
    print(f"sorted sum, weights over 70 decades: error {err:.3e}")
    assert err < TOL_WIDE


def test_sorted_sum_flags_non_finite_weights():
    prob = W.tiny(d=3, N=500, M=100, P=8, kernel="negdist", kparam=0.0, n_ft=64, seed=2)
    w = prob.w.copy()
    w[17] = np.nan
    with QSPlan(prob.d, "negdist", prob.P, prob.n_ft, prob.R, dirs=prob.xi, proj="fp32", max_n=prob.N,
                max_m=prob.M) as plan:
        plan.sum_sorted(_cuda(prob.x), _cuda(w), _cuda(prob.y))
        assert plan.status() == 3  # QS_ERR_NONFINITE
        assert plan.status() == 0  # cleared by the check
