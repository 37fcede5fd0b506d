"""Pins of the oracle's symmetric distance energy (Sec. 2.3 eq. distance-mmd;
eq. distance-sym in the appendix relating distance designs and orthogonal
points) and its gradient.  CPU only; each check uses something other than the
oracle's own loops: numpy on the doubled point set, finite differences, the
closed form for orthonormal systems, and exact symmetries.
"""
import math

import numpy as np
import pytest

import oracle


def _unit(rng, P, d):
    x = rng.standard_normal((P, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.float32)


def _energy_doubled(x):
    # E((xi, -xi)) with E(z) = -sum_{i,j} |z_i - z_j| over the 2P points (eq. distance-mmd, exponent 1)
    z = np.concatenate([x, -x]).astype(np.float64)
    return -np.linalg.norm(z[:, None] - z[None], axis=2).sum()


@pytest.mark.parametrize("P,d", [(5, 3), (12, 4), (30, 7)])
def test_energy_is_the_doubled_point_set_energy(P, d):
    x = _unit(np.random.default_rng(P), P, d)
    E, _ = oracle.esym(x, grad=False)
    assert E == pytest.approx(_energy_doubled(x), rel=1e-13)


@pytest.mark.parametrize("P,d", [(6, 3), (9, 5)])
def test_gradient_matches_central_differences(P, d):
    x = _unit(np.random.default_rng(7 + P), P, d)
    _, g = oracle.esym(x)
    xf = x.astype(np.float64)
    h = 1e-6
    for i in range(P):
        for j in range(d):
            xp, xm = xf.copy(), xf.copy()
            xp[i, j] += h
            xm[i, j] -= h
            fd = (_energy_doubled(xp) - _energy_doubled(xm)) / (2 * h)
            assert g[i, j] == pytest.approx(fd, abs=1e-6 * P)


@pytest.mark.parametrize("P,d", [(1, 1), (3, 3), (5, 8), (16, 16)])
def test_orthonormal_systems_energy_and_stationarity(P, d):
    # |xi_p -+ xi_q| = sqrt 2 for p != q and |2 xi_p| = 2, so
    # E_sym = -2 (2 sqrt2 P (P - 1) + 2 P); the appendix shows these minimise E_sym for P <= d,
    # so the gradient has no component along the sphere
    q, _ = np.linalg.qr(np.random.default_rng(d).standard_normal((d, d)))
    x = q[:, :P].T.astype(np.float32)
    E, g = oracle.esym(x)
    assert E == pytest.approx(-2 * (2 * math.sqrt(2) * P * (P - 1) + 2 * P), rel=1e-6)
    xd = x.astype(np.float64)
    tang = g - np.sum(g * xd, axis=1, keepdims=True) * xd
    assert np.max(np.abs(tang)) < 1e-5 * max(1.0, np.max(np.abs(g)))


def test_energy_symmetries():
    rng = np.random.default_rng(3)
    x = _unit(rng, 20, 5)
    E, _ = oracle.esym(x, grad=False)
    flip = x.copy()
    flip[::3] *= -1  # antipodes are the same design
    assert oracle.esym(flip, grad=False)[0] == pytest.approx(E, rel=1e-6)
    q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    rot = (x.astype(np.float64) @ q).astype(np.float32)
    assert oracle.esym(rot, grad=False)[0] == pytest.approx(E, rel=1e-6)
    perm = x[rng.permutation(20)]
    assert oracle.esym(perm, grad=False)[0] == pytest.approx(E, rel=1e-12)
