"""Library-side tuners and the autotune cache on the GPU.

qs_plan_autotune (spread variant) and qs_plan_autotune_gemm (projection GEMM
form) record their choice under the plan's shape class; plans created later
for the same class start with it.  qs_batch_autotune picks the interpolation
tiling of a batch; every tiling and every spread variant gives the same bits.
"""
import numpy as np
import pytest

from paper_2410_01316_gb300 import QSBatch, QSPlan, tune_cache_clear, tune_cache_load, tune_cache_save, tune_cache_size
from paper_2410_01316_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _plan(prob, proj):
    return QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, proj=proj,
                  max_n=prob.N, max_m=prob.M)


def test_tuned_choices_reach_later_plans_and_leave_results_unchanged(tmp_path):
    tune_cache_clear()
    prob = W.mnist_laplace(N=4000, M=3000, P=256)
    x, w, y = _cuda(prob.x), _cuda(prob.w), _cuda(prob.y)
    with _plan(prob, "bf16x3") as plan:
        untuned = plan.sum(x, w, y).cpu().numpy()
        variant = plan.autotune(x, w)
        pair = plan.autotune_gemm(x)
        assert plan.variant() == variant and plan.gemm_pair() == pair
        plan.set_gemm(not pair)
        plan.set_gemm(pair)
        tuned = plan.sum(x, w, y).cpu().numpy()
        plan.check()
    assert tune_cache_size() == 1
    if pair == (prob.d >= 256):
        assert np.array_equal(untuned, tuned)  # only the spread variant changed: bitwise neutral
    with _plan(prob, "bf16x3") as again:
        assert again.variant() == variant and again.gemm_pair() == pair
    path = str(tmp_path / "tune.txt")
    tune_cache_save(path)
    tune_cache_clear()
    with _plan(prob, "bf16x3") as fresh:
        default_variant = fresh.variant()
    tune_cache_load(path)
    with _plan(prob, "bf16x3") as loaded:
        assert loaded.variant() == variant and loaded.gemm_pair() == pair
    assert default_variant in ("moment", "point1")
    tune_cache_clear()


def test_gemm_tuner_refuses_plans_without_tensor_cores():
    from paper_2410_01316_gb300 import QSError

    prob = W.tiny(d=8, N=300, M=100, P=16, kernel="gauss", kparam=1.0, n_ft=64, seed=3)
    with _plan(prob, "fp32") as plan:
        with pytest.raises(QSError) as ei:
            plan.autotune_gemm(_cuda(prob.x))
        assert ei.value.status == 6


def test_batch_autotune_picks_a_mode_and_tiling_with_the_expected_results():
    # persistent kernel at any tiling: the same bits as at tiling 1; concurrent mode (0): each
    # plan's own qs_sum, bit for bit
    import torch

    specs = [(3, "gauss", 0.8, 64, 128), (16, "laplace", 0.7, 40, 256), (64, "negdist", 0.0, 48, 512)]
    probs = [W.tiny(d=d, N=2500, M=1800, P=P, kernel=k, kparam=kp, n_ft=nft, seed=600 + i)
             for i, (d, k, kp, P, nft) in enumerate(specs)]
    plans = [_plan(p, "auto") for p in probs]
    data = [(_cuda(p.x), _cuda(p.w), _cuda(p.y), torch.empty(p.M, device="cuda")) for p in probs]
    own = [pl.sum(x, w, y).cpu().numpy() for pl, (x, w, y, _) in zip(plans, data)]
    batch = QSBatch(plans)
    batch.set_tiling(1)
    batch.sum(data)
    persistent = [d[3].cpu().numpy().copy() for d in data]
    tpt = batch.autotune(data)
    assert tpt in (0, 1, 2, 4)
    batch.sum(data)
    batch.check()
    want = own if tpt == 0 else persistent
    for b, d in zip(want, data):
        assert np.array_equal(b, d[3].cpu().numpy())
    batch.close()
    for p in plans:
        p.close()
