"""Batched sums (one persistent launch over many problems) through the C ABI.

Every problem of the batch is checked against the FP64 oracle (1e-5 relative
to sum|w| max|F|) and against its own single-problem qs_sum; the tiling of
the interpolation items must not change a single bit; a CUDA graph capture
of the batched call must replay to the same results.
"""
import numpy as np
import pytest

import oracle
from paper_2410_01316_gb300 import QSBatch, QSPlan
from paper_2410_01316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _problems():
    rng = np.random.default_rng(2024)
    probs = []
    specs = [(3, "gauss", 0.8, 64, 128), (16, "laplace", 0.7, 40, 256), (64, "negdist", 0.0, 48, 512),
             (3, "negdist", 0.0, 16, 64), (16, "gauss", 3.0, 64, 256), (64, "gauss", 6.0, 32, 128),
             (5, "laplace", 1.3, 24, 512), (33, "negdist", 0.0, 20, 256)]
    for i, (d, kern, kp, P, nft) in enumerate(specs):
        N = int(rng.integers(1, 3000)) if i != 3 else 0   # one problem without sources
        M = int(rng.integers(1, 2500))
        probs.append(W.tiny(d=d, N=max(N, 1) if i != 3 else 1, M=M, P=P, kernel=kern, kparam=kp, n_ft=nft,
                            seed=300 + i))
        if i == 3:
            probs[-1].x = probs[-1].x[:0]
            probs[-1].w = probs[-1].w[:0]
    return probs


def _norm(prob):
    sw = max(float(np.abs(prob.w.astype(np.float64)).sum()), 1e-30)
    return sw * (prob.R if prob.kernel == "negdist" else 1.0)


def _setup(probs):
    import torch

    plans = [QSPlan(p.d, p.kernel, p.P, p.n_ft, p.R, p.kparam, dirs=p.xi, proj="fp32_fused", max_n=max(p.N, 1),
                    max_m=p.M) for p in probs]
    data = []
    for p in probs:
        x = torch.from_numpy(np.ascontiguousarray(p.x)).cuda().reshape(p.N, p.d)
        w = torch.from_numpy(np.ascontiguousarray(p.w)).cuda()
        y = torch.from_numpy(p.y).cuda()
        data.append((x, w, y, torch.full((p.M,), float("nan"), device="cuda")))
    return plans, data


def test_batch_matches_oracle_and_single_problem_sums():
    probs = _problems()
    plans, data = _setup(probs)
    batch = QSBatch(plans)
    batch.sum(data)
    batch.check()
    for p, plan, (x, w, y, out) in zip(probs, plans, data):
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        if p.N == 0:
            assert np.all(got == 0.0)
            continue
        ref = oracle.o1_problem(p)
        assert np.max(np.abs(got - ref)) / _norm(p) < TOL, (p.d, p.kernel)
        single = plan.sum(x, w, y).cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - single)) / _norm(p) < 1e-6
    batch.close()


def test_batch_tiling_does_not_change_bits():
    probs = _problems()
    plans, data = _setup(probs)
    batch = QSBatch(plans)
    results = []
    for tpt in (1, 2, 4):
        batch.set_tiling(tpt)
        batch.sum(data)
        batch.check()
        results.append([out.cpu().numpy().copy() for (_, _, _, out) in data])
    for r in results[1:]:
        for a, b in zip(results[0], r):
            assert np.array_equal(a, b)
    batch.close()


def test_batch_graph_capture_replays():
    import torch

    probs = _problems()[:4]
    plans, data = _setup(probs)
    batch = QSBatch(plans)
    batch.sum(data)
    batch.check()
    ref = [out.cpu().numpy().copy() for (_, _, _, out) in data]
    for (_, _, _, out) in data:
        out.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.sum(data, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for a, (_, _, _, out) in zip(ref, data):
            assert np.array_equal(a, out.cpu().numpy())
    batch.check()
    batch.close()


def test_batch_rejects_repeated_plan():
    from paper_2410_01316_gb300 import QSError

    p = _problems()[0]
    plan = QSPlan(p.d, p.kernel, p.P, p.n_ft, p.R, p.kparam, dirs=p.xi, proj="fp32_fused", max_n=p.N, max_m=p.M)
    with pytest.raises(QSError):
        QSBatch([plan, plan])


@pytest.mark.parametrize("proj", ["fp32_fused", "auto"])
def test_concurrent_mode_equals_each_plans_sum_and_replays_in_a_graph(proj):
    # the concurrent mode runs each plan's own qs_sum on the batch's streams: bit for bit that
    # sum, also when the forked call is captured into a CUDA graph and replayed
    import torch

    probs = _problems()
    plans = [QSPlan(p.d, p.kernel, p.P, p.n_ft, p.R, p.kparam, dirs=p.xi, proj=proj, max_n=max(p.N, 1), max_m=p.M)
             for p in probs]
    _, data = _setup(probs)
    refs = []
    for plan, (x, w, y, _) in zip(plans, data):
        refs.append(plan.sum(x, w, y).cpu().numpy())
    batch = QSBatch(plans)
    batch.set_mode(True)
    batch.sum(data)
    batch.check()
    for p, r, (_, _, _, out) in zip(probs, refs, data):
        got = out.cpu().numpy()
        assert np.array_equal(got, r)
        if p.N:
            assert np.max(np.abs(got.astype(np.float64) - oracle.o1_problem(p))) / _norm(p) < TOL
    for (_, _, _, out) in data:
        out.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.sum(data, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for r, (_, _, _, out) in zip(refs, data):
            assert np.array_equal(r, out.cpu().numpy())
    batch.check()
    batch.close()
    for pl in plans:
        pl.close()
