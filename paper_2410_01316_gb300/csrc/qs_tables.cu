// Host-side tables shared by plan creation (qs_plan.cu) and the
// allocation-free sum (qs_noalloc.cu): the rescaling rule, the window's tap
// polynomials, the window's Fourier transform and the FFT twiddles.  All of
// them write into caller-provided fixed-size storage (no heap), so the
// allocation-free entry point can use them too, and both paths get bitwise
// identical tables.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include "qs_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// The window on |v| < m = W/2 grid cells, normalised to psi(0) = 1:
//  QS_WINDOW_ES  exponential of semicircle, psi(v) = exp(beta (sqrt(1 - (v/m)^2) - 1)), beta = 2.30 W;
//  QS_WINDOW_KB  Kaiser-Bessel in the sinh form used by NFFT (Keiner, Kunis, Potts 2009),
//                psi(v) = [sinh(b r) / r] / [sinh(b m) / m], r = sqrt(m^2 - v^2), b = pi (2 - 1/sigma_os)
//                = 3 pi / 2 for sigma_os = 2 (the limit b / (sinh(b m) / m) at r = 0).
double window_value(int kind, int m, double v)
{
    if (fabs(v) >= m) return 0.0;
    if (kind == QS_WINDOW_KB) {
        const double b = 1.5 * kPi;
        const double r = sqrt((double)m * m - v * v);
        const double num = r > 1e-12 ? sinh(b * r) / r : b;
        return num / (sinh(b * m) / m);
    }
    const double z = v / m;
    return exp(2.30 * (2 * m) * (sqrt(1.0 - z * z) - 1.0));
}

}  // namespace

// Rescaling factor (App. C Step 1: T = 0.3 Gauss, 0.1 Laplace, 0.2 Matern,
// g_max = 5 sigma, 5 / alpha, 5 beta; App. G for the kernels without a
// classical Fourier transform: the half period T = R, tau = 1/(2R)).
double qs_tau_rule(qs_kernel kernel, double kparam, double R)
{
    switch (kernel) {
        case QS_GAUSS: return fmin(0.3 / R, 1.0 / (2.0 * 5.0 * kparam));
        case QS_LAPLACE: return fmin(0.1 / R, 1.0 / (2.0 * 5.0 / kparam));
        case QS_MATERN: return fmin(0.2 / R, 1.0 / (2.0 * 5.0 * kparam));
        case QS_NEGDIST:
        case QS_RIESZ:
        case QS_TPS: return 1.0 / (2.0 * R);
    }
    return -1.0;
}

// Gauss-Legendre nodes and weights on [-1, 1] (n <= QS_GL_MAX) by Newton's method on P_n.
void qs_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double t = cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int j = 1; j < n; ++j) {
                const double p2 = ((2.0 * j + 1.0) * t * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// Tap polynomials of the window `kind`: Chebyshev interpolation of degree
// qs_tap_degree(W) on s in [-1/2, 1/2] for each tap of the first half,
// converted to monomials in s and split into even and odd parts.
void qs_fit_window(int W, int kind, qs_window* win)
{
    const int m = W / 2;
    const int n = qs_tap_degree(W) + 1;
    memset(win, 0, sizeof(*win));
    // T_k(2s) as monomials in s: tm[k][i]
    double tm[QS_MAX_W + 2][QS_MAX_W + 2];
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) tm[k][i] = 0.0;
    tm[0][0] = 1.0;
    if (n > 1) tm[1][1] = 2.0;
    for (int k = 2; k < n; ++k) {
        for (int i = 0; i < n; ++i) {
            double v = -tm[k - 2][i];
            if (i > 0) v += 4.0 * tm[k - 1][i - 1];  // 2 * (2s) * T_{k-1}
            tm[k][i] = v;
        }
    }
    for (int j = 0; j < m; ++j) {
        double cheb[QS_MAX_W + 2], fval[QS_MAX_W + 2], mono[QS_MAX_W + 2];
        for (int i = 0; i < n; ++i) {
            const double th = kPi * (i + 0.5) / n;
            fval[i] = window_value(kind, m, 0.5 * cos(th) + m - 0.5 - j);
        }
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += fval[i] * cos(k * kPi * (i + 0.5) / n);
            cheb[k] = (k == 0 ? 1.0 : 2.0) * acc / n;
        }
        for (int i = 0; i < n; ++i) mono[i] = 0.0;
        for (int k = 0; k < n; ++k)
            for (int i = 0; i < n; ++i) mono[i] += cheb[k] * tm[k][i];
        for (int i = 0; i < n; ++i) {
            if (i % 2 == 0) win->e[j][i / 2] = (float)mono[i];
            else win->o[j][i / 2] = (float)mono[i];
        }
    }
}

// The tap polynomials in monomials of t = 2 s (s the centred offset):
// atab[j K + k] = a_jk 2^-k with tap_j(s) = sum_k a_jk s^k from the even / odd
// parts (the second half mirrored: tap_{W-1-j}(s) = tap_j(-s)), K = qs_moment_count(W).
void qs_fill_atab(const qs_window* win, int W, float* atab)
{
    const int K = qs_moment_count(W), T = qs_tap_terms(W);
    for (int j = 0; j < W; ++j)
        for (int k = 0; k < K; ++k) {
            const int jj = j < W / 2 ? j : W - 1 - j;
            const int i2 = k >> 1;
            float a = 0.0f;
            if (i2 < T) a = (k & 1) ? (j < W / 2 ? win->o[jj][i2] : -win->o[jj][i2]) : win->e[jj][i2];
            atab[j * K + k] = ldexpf(a, -k);
        }
}

// The FP32 tap polynomial of tap j at offset s, evaluated in double.
double qs_window_tap(const qs_window* win, int W, int j, double s)
{
    const int m = W / 2;
    const int T = qs_tap_terms(W);
    const int jj = j < m ? j : W - 1 - j;
    const double ss = j < m ? s : -s;
    double e = 0.0, o = 0.0;
    for (int i = T - 1; i >= 0; --i) {
        e = e * ss * ss + (double)win->e[jj][i];
        o = o * ss * ss + (double)win->o[jj][i];
    }
    return e + ss * o;
}

// Fourier transform (grid units) of the window as the GPU applies it:
// psi_eff(v) = p_j(v - (m - 1/2 - j)) on the j-th unit cell.  Even, so
// psi^(nu) = sum_j int_{-1/2}^{1/2} p_j(s) cos(2 pi nu (s + m - 1/2 - j)) ds,
// by 24-point Gauss-Legendre per cell, for nu = k / G, k = 0 .. K (out[K + 1]).
void qs_window_transform(const qs_window* win, int W, int K, int G, double* out)
{
    constexpr int nq = 24;
    const int m = W / 2;
    double gx[nq], gw[nq], tap[QS_MAX_W][nq];
    qs_gauss_legendre(nq, gx, gw);
    for (int j = 0; j < W; ++j)
        for (int q = 0; q < nq; ++q) tap[j][q] = qs_window_tap(win, W, j, 0.5 * gx[q]);
    for (int k = 0; k <= K; ++k) {
        const double nu = (double)k / G;
        double acc = 0.0;
        for (int j = 0; j < W; ++j) {
            const double c = m - 0.5 - j;
            for (int q = 0; q < nq; ++q) {
                const double s = 0.5 * gx[q];
                acc += 0.5 * gw[q] * tap[j][q] * cos(2.0 * kPi * nu * (s + c));
            }
        }
        out[k] = acc;
    }
}

// FFT twiddles e^{-2 pi i t / G}, t = 0 .. G/2 - 1 (out[G / 2]).
void qs_twiddles(int G, float2* out)
{
    for (int t = 0; t < G / 2; ++t) {
        const double ang = 2.0 * kPi * (double)t / (double)G;
        out[t] = make_float2((float)cos(ang), (float)(-sin(ang)));
    }
}
