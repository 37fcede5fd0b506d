"""Pins of the oracle's Matern, generalised Riesz and thin plate spline kernels.

CPU only.  Each check compares the oracle with something other than its own
method: closed forms evaluated in arbitrary precision (mpmath), adaptive
quadrature of the defining integrals, special cases that reduce to kernels
pinned elsewhere (Matern nu = 1/2 is the Laplace kernel, Riesz r = 1 is the
negative distance kernel), and the slicing relation F(|x|) = E_xi f(<x, xi>)
(Sec. 2, eq. sliced_basis_function) written out for d = 3 and by quadrature
over the distribution of xi_1 for other d.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------------------
# Matern (Table tab:kernels; App. C Steps 1 and 2)
# ---------------------------------------------------------------------------
def test_matern_tau_uses_paper_parameters():
    g = _golden("paper_parameters.json")
    T, gm = g["rescaling_threshold_T"]["matern"], g["g_max_over_lengthscale"]["value"]
    for R in (0.5, 3.0, 20.0):
        for beta in (0.05, 0.7, 4.0):
            want = min(T / R, 1.0 / (2.0 * gm * beta))
            assert oracle.tau("matern", beta, R) == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("beta", [0.4, 1.3])
def test_matern_half_integer_closed_forms(beta):
    # the textbook forms of nu = 1/2, 3/2, 5/2, 7/2 (exponential times a polynomial)
    for r in (0.0, 0.2, 1.0, 3.7):
        a = math.sqrt(1.0) / beta
        assert oracle.F("matern", beta, r, nu=0.5) == pytest.approx(math.exp(-a * r), rel=1e-13)
        a = math.sqrt(3.0) / beta
        assert oracle.F("matern", beta, r, nu=1.5) == pytest.approx((1 + a * r) * math.exp(-a * r), rel=1e-13)
        a = math.sqrt(5.0) / beta
        want = (1 + a * r + (a * r) ** 2 / 3) * math.exp(-a * r)
        assert oracle.F("matern", beta, r, nu=2.5) == pytest.approx(want, rel=1e-13)
        a = math.sqrt(7.0) / beta
        want = (1 + a * r + 2 * (a * r) ** 2 / 5 + (a * r) ** 3 / 15) * math.exp(-a * r)
        assert oracle.F("matern", beta, r, nu=3.5) == pytest.approx(want, rel=1e-13)


def test_matern_bessel_form():
    # F(x) = 2^{1-nu}/Gamma(nu) (sqrt(2 nu) x / beta)^nu K_nu(sqrt(2 nu) x / beta)  (Table tab:kernels)
    mp = pytest.importorskip("mpmath")
    for nu in (1.5, 3.5):
        for beta in (0.6, 2.0):
            for r in (0.1, 0.8, 2.5):
                z = mp.sqrt(2 * nu) * r / beta
                want = 2 ** (1 - nu) / mp.gamma(nu) * z ** nu * mp.besselk(nu, z)
                assert oracle.F("matern", beta, r, nu=nu) == pytest.approx(float(want), rel=1e-12)


@pytest.mark.parametrize("nu", [1.5, 3.5])
def test_matern_f_d3_satisfies_integral_transform(nu):
    # d = 3: F(r) = int_0^1 f(r s) ds (eq. integral_transform)
    beta = 0.9
    for r in (0.05, 0.6, 2.2):
        val, _ = integrate.quad(lambda s: oracle.f("matern", beta, 3, r * s, nu=nu), 0.0, 1.0, epsabs=1e-14)
        assert val == pytest.approx(oracle.F("matern", beta, r, nu=nu), abs=1e-12)


@pytest.mark.parametrize("nu", [1.5, 3.5])
@pytest.mark.parametrize("d", [1, 3])
def test_matern_fhat_is_fourier_transform_of_closed_form_f(nu, d):
    # F_1[f(|.|)](w) = 2 int_0^inf f(t) cos(2 pi w t) dt  (App. A eq. Fourier)
    # f decays like exp(-sqrt(2 nu) t / beta): beyond 60 beta it is below 1e-40
    beta = 0.8
    for om in (0.0, 0.05, 0.3, 1.1):
        g = lambda t: oracle.f("matern", beta, d, t, nu=nu) * math.cos(2 * math.pi * om * t)
        val, _ = integrate.quad(g, 0.0, 60 * beta, epsabs=1e-14, limit=1000)
        assert 2 * val == pytest.approx(oracle.fhat("matern", beta, d, om, nu=nu), abs=1e-10)


@pytest.mark.parametrize("d", [1, 3, 16, 784])
def test_matern_nu_half_is_laplace(d):
    # nu = 1/2 gives F(x) = exp(-x / beta): the Laplace kernel with alpha = 1/beta,
    # whose f-hat is pinned independently
    beta = 0.7
    for om in (0.0, 0.02, 0.4, 3.0):
        lap = oracle.fhat("laplace", 1.0 / beta, d, om)
        mat = oracle.fhat("matern", beta, d, om, nu=0.5)
        assert mat == pytest.approx(lap, rel=1e-11, abs=1e-300)


@pytest.mark.parametrize("nu,d", [(1.5, 3), (1.5, 16), (3.5, 3), (3.5, 64), (2.0, 784)])
def test_matern_coeff_sum_is_g_at_zero(nu, d):
    # sum_k c_k approaches g~(0) = F(0) = 1 up to the tail int_{tau N/2}^inf f-hat and the
    # Poisson aliases f(l / tau), l != 0; beta = 0.4 with tau = 0.2/3 puts the nearest alias at
    # 37 beta, where f is below 1e-25
    beta = 0.4
    t = oracle.tau("matern", beta, 3.0)
    n_ft = 1 << 14
    c = oracle.coeffs("matern", beta, d, t, n_ft, nu=nu)
    tail, _ = integrate.quad(lambda om: oracle.fhat("matern", beta, d, om, nu=nu), t * (n_ft // 2), np.inf,
                             limit=500, epsabs=1e-15)
    assert c.sum() + 2 * tail == pytest.approx(1.0, abs=1e-8)


# ---------------------------------------------------------------------------
# generalised Riesz F(x) = -x^r and thin plate spline F(x) = x^2 log x
# (Table tab:kernels), periodised like the negative distance kernel (App. G)
# ---------------------------------------------------------------------------
def test_periodised_kernels_use_half_period_tau():
    for R in (0.5, 4.0):
        assert oracle.tau("riesz", 0.5, R) == pytest.approx(1.0 / (2 * R), rel=1e-15)
        assert oracle.tau("tps", 0.0, R) == pytest.approx(1.0 / (2 * R), rel=1e-15)


def test_riesz_constant_closed_forms():
    # d = 3: E_xi |<x, xi>|^r = |x|^r / (r + 1), so c_{3,r} = r + 1; d = 1: c_{1,r} = 1
    for r in (0.3, 1.0, 1.5):
        assert oracle.riesz_const(3, r) == pytest.approx(r + 1, rel=1e-13)
        assert oracle.riesz_const(1, r) == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("d", [2, 5, 16, 64])
@pytest.mark.parametrize("kernel,kp", [("riesz", 0.5), ("riesz", 1.5), ("tps", 0.0)])
def test_slicing_relation_by_quadrature(kernel, kp, d):
    # F(r) = E f(r xi_1) with xi_1 ~ (1 - u^2)^{(d-3)/2} / B((d-1)/2, 1/2) on [-1, 1]
    B = math.exp(math.lgamma((d - 1) / 2) + math.lgamma(0.5) - math.lgamma(d / 2))
    for r in (0.4, 1.0, 2.7):
        val, _ = integrate.quad(lambda u: oracle.f(kernel, kp, d, r * u) * (1 - u * u) ** ((d - 3) / 2) / B,
                                -1.0, 1.0, points=[0.0], epsabs=1e-13, limit=400)
        assert val == pytest.approx(oracle.F(kernel, kp, r), rel=1e-9, abs=1e-10)


def test_tps_constant_d3():
    # H_{3/2} = 8/3 - 2 log 2 gives C_3 = 1 and f(t) = 3 t^2 log t + t^2, for which
    # (1/r) int_0^r f = r^2 log r exactly
    assert oracle.tps_const(3) == pytest.approx(1.0, rel=1e-14)
    for r in (0.3, 2.0):
        assert oracle.f("tps", 0.0, 3, r) == pytest.approx(3 * r * r * math.log(r) + r * r, rel=1e-14)


def _riesz_cos_integral(mp, r, k):
    # int_0^{1/2} x^r cos(2 pi k x) dx = (1/2)^{r+1}/(r+1) 1F2((r+1)/2; 1/2, (r+3)/2; -(pi k / 2)^2)
    return mp.mpf(0.5) ** (r + 1) / (r + 1) * mp.hyp1f2((r + 1) / 2, mp.mpf(0.5), (r + 3) / 2, -(mp.pi * k / 2) ** 2)


@pytest.mark.parametrize("r,d", [(0.5, 3), (1.5, 16), (1.0, 5)])
def test_riesz_coefficients_match_hypergeometric_closed_form(r, d):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    R = 2.5
    t = oracle.tau("riesz", r, R)
    n_ft = 64
    c = oracle.coeffs("riesz", r, d, t, n_ft)
    amp = oracle.riesz_const(d, r) * t ** (-r)
    for k in (0, 1, 2, 5, 17, 31):
        want = -amp * 2 * float(_riesz_cos_integral(mp, mp.mpf(r), k))
        assert c[k + n_ft // 2] == pytest.approx(want, abs=1e-12 * amp)
        assert c[-k + n_ft // 2] == c[k + n_ft // 2]


def test_riesz_r1_coefficients_equal_negative_distance_closed_form():
    for d in (3, 64):
        t = oracle.tau("riesz", 1.0, 1.7)
        a = oracle.coeffs("riesz", 1.0, d, t, 128)
        b = oracle.coeffs("negdist", 0.0, d, t, 128)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


@pytest.mark.parametrize("d", [3, 16])
def test_tps_coefficients_match_closed_form_derivative(d):
    # g(x) = tau^-2 [d x^2 log|x| + (C_d - d log tau) x^2] on [-1/2, 1/2), so
    # c_k = tau^-2 [d dI/dr(2, k) + (C_d - d log tau) I(2, k)], I(r, k) = 2 int_0^{1/2} x^r cos(2 pi k x)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    R = 1.3
    t = oracle.tau("tps", 0.0, R)
    n_ft = 64
    c = oracle.coeffs("tps", 0.0, d, t, n_ft)
    Cd = oracle.tps_const(d)
    scale = t ** -2
    for k in (0, 1, 3, 8, 31):
        I2 = 2 * _riesz_cos_integral(mp, mp.mpf(2), k)
        dI = 2 * mp.diff(lambda rr: _riesz_cos_integral(mp, rr, k), mp.mpf(2))
        want = scale * float(d * dI + (Cd - d * mp.log(t)) * I2)
        assert c[k + n_ft // 2] == pytest.approx(want, abs=1e-12 * scale * d)


@pytest.mark.parametrize("kernel,kp", [("riesz", 1.5), ("tps", 0.0)])
def test_o1_approaches_sliced_sum_as_nft_grows(kernel, kp):
    # O1 (truncated series) -> O3 (closed-form f, no Fourier step) as N_ft grows
    from paper_2410_01316_gb300 import workloads as W

    prob = W.tiny(d=4, N=40, M=12, P=6, kernel=kernel, kparam=kp, n_ft=64, seed=3)
    ref = oracle.o3_sliced(kernel, kp, prob.x, prob.w, prob.y, prob.xi)
    t = oracle.tau(kernel, kp, prob.R)
    errs = []
    for n_ft in (64, 256, 1024):
        c = oracle.coeffs(kernel, kp, prob.d, t, n_ft)
        s = oracle.o1_sum(prob.x, prob.w, prob.y, prob.xi, t, c)
        errs.append(np.max(np.abs(s - ref)) / np.abs(prob.w).sum())
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-4
