"""Distance QMC designs on the GPU (qs_distance_energy, qs_distance_design,
QS_DIR_DISTANCE plans): energy and gradient parity with the FP64 oracle, and
the optimiser's behaviour where the answer is known (orthonormal systems
minimise the symmetric energy when P <= d)."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_01316_gb300 import QSPlan, directions, distance_design, distance_energy
from paper_2410_01316_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _unit(rng, P, d):
    x = rng.standard_normal((P, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.float32)


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("P,d", [(300, 10), (1000, 3), (200, 64), (129, 130)])
def test_energy_and_gradient_match_oracle(P, d):
    x = _unit(np.random.default_rng(P + d), P, d)
    E, g = distance_energy(_cuda(x), grad=True)
    Eo, go = oracle.esym(x)
    assert E == pytest.approx(Eo, rel=2e-6)
    g = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))


def test_energy_and_gradient_with_near_parallel_and_near_antipodal_pairs():
    # |c_pq| > 1/2 takes the squared distance from the rows (c near 1 or -1 would otherwise
    # amplify the Gram matrix's rounding in the weights); pairs at 1e-2 .. 1e-1 radians of each
    # other or of each other's antipode, mixed with unrelated directions
    rng = np.random.default_rng(21)
    d, k = 6, 60
    base = _unit(rng, k, d).astype(np.float64)
    near = base + rng.uniform(1e-2, 1e-1, (k, 1)) * _unit(rng, k, d).astype(np.float64)
    anti = -base + rng.uniform(1e-2, 1e-1, (k, 1)) * _unit(rng, k, d).astype(np.float64)
    x = np.concatenate([base, near, anti, _unit(rng, 90, d).astype(np.float64)])
    x = (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)
    E, g = distance_energy(_cuda(x), grad=True)
    Eo, go = oracle.esym(x)
    assert E == pytest.approx(Eo, rel=2e-6)
    g = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))


@pytest.mark.parametrize("P,d", [(8, 16), (16, 16), (3, 3)])
def test_optimiser_reaches_orthonormal_minimum_when_p_le_d(P, d):
    x = _cuda(_unit(np.random.default_rng(11), P, d))
    E = distance_design(x, iters=800)
    want = -2 * (2 * math.sqrt(2) * P * (P - 1) + 2 * P)
    assert E == pytest.approx(want, rel=2e-4)
    xi = x.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(xi, axis=1) - 1)) < 1e-5
    gram = xi @ xi.T
    assert np.max(np.abs(gram - np.eye(P))) < 3e-2


def test_optimiser_lowers_energy_below_iid_and_orthogonal_starts():
    d, P = 3, 64
    iid = _unit(np.random.default_rng(5), P, d)
    orth = directions("orthogonal", d, P, seed=5)
    e_iid = oracle.esym(iid, grad=False)[0]
    e_orth = oracle.esym(orth, grad=False)[0]
    x = _cuda(iid)
    E = distance_design(x, iters=600)
    assert E < e_orth < 0 and E < e_iid
    # the oracle agrees on the optimised design
    assert oracle.esym(x.cpu().numpy(), grad=False)[0] == pytest.approx(E, rel=2e-6)


def test_distance_plan_directions_and_sum():
    prob = W.tiny(d=5, N=1500, M=400, P=40, kernel="gauss", kparam=1.2, n_ft=256, seed=13)
    with QSPlan(prob.d, "gauss", prob.P, prob.n_ft, prob.R, prob.kparam, dirs="distance", seed=3,
                proj="fp32_fused", max_n=prob.N, max_m=prob.M) as plan:
        xi = plan.directions()
        s = plan.sum(_cuda(prob.x), _cuda(prob.w), _cuda(prob.y))
        plan.check()
        s = s.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(xi.astype(np.float64), axis=1) - 1)) < 1e-5
    e_dist = oracle.esym(xi, grad=False)[0]
    e_orth = oracle.esym(directions("orthogonal", prob.d, prob.P, seed=3), grad=False)[0]
    assert e_dist < e_orth
    t = oracle.tau("gauss", prob.kparam, prob.R)
    ref = oracle.o1_sum(prob.x, prob.w, prob.y, xi, t, oracle.coeffs("gauss", prob.kparam, prob.d, t, prob.n_ft))
    assert np.max(np.abs(s - ref)) / np.abs(prob.w).sum() < 1e-5
