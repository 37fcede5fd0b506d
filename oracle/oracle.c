/*
 * FP64 CPU oracle for fast radial kernel summation via QMC slicing
 * (Hertrich, Jahn, Quellmalz, "Fast Summation of Radial Kernels via QMC
 * Slicing", arXiv 2410.01316).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Every computation is in double precision.  Inputs are the exact FP32 arrays
 * the GPU receives, widened to double, so a comparison measures only the
 * GPU's algorithmic and rounding error.
 *
 * Contents (each function names the passage it follows):
 *   o_tau          rescaling factor tau               (App. C "Step 1"; App. G, eq. radius_xy)
 *   o_riesz_const  constant of the sliced Riesz r=1   (Table tab:kernels, Riesz row)
 *   o_f            1D basis function f, closed forms  (Table tab:kernels; Sec. 2, eq. integral_transform)
 *   o_F            radial basis function F            (Table tab:kernels)
 *   o_fhat         1D Fourier transform of f(|.|)     (Table tab:kernels with the corrected constants)
 *   o_coeffs       Fourier coefficients c_k           (App. C "Step 2"; App. G, eq. Fourier-slicing)
 *   o1_sum         sliced, Fourier-truncated sum      (Sec. 2.1 eq. kernel_sum_sliced + App. C eq. 1d_sum_fourier)
 *   o1_grad        gradients of L = sum_m v_m s_m of the same sum
 *   o2_exact       exact kernel sum, O(NM)            (Sec. 1, eq. kernel_sum)
 *   o3_sliced      sliced sum with closed-form f      (Sec. 2.1, eq. kernel_sum_sliced)
 *
 * Readings of the paper taken here (garbled or silent passages):
 *   - f-hat for the Gauss and Laplace kernels is obtained from the relation
 *     F_1[f](w) = pi^{d/2}/Gamma(d/2) |w|^{d-1} F_d[F(|.|)](|w|), which follows
 *     from the slicing relation (Sec. 2, eq. sliced_basis_function) in polar
 *     coordinates with the Fourier convention of App. A, eq. Fourier.  For the
 *     Gauss kernel this agrees with the expression in the proof of Thm. 2
 *     (App. E); the tabulated Gauss and Laplace entries differ from it by
 *     constant factors, and the relation is the one consistent with f(0)=F(0).
 *   - The negative distance kernel uses the 2T-periodic construction of App. G
 *     with T = R, i.e. tau = 1/(2R); the periodised f(|t|) is a triangle wave
 *     whose Fourier coefficients are known in closed form.
 *   - The kept frequencies are k = -N_ft/2 .. N_ft/2-1 (App. C, Step 2), and
 *     the one-dimensional sums take the real part.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define O_GAUSS 0
#define O_LAPLACE 1
#define O_NEGDIST 2

#define O_OK 0
#define O_EARG (-1)
#define O_EUNSUPPORTED (-2)
#define O_ENOMEM (-3)

static const double O_PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------------- */
/* Rescaling (App. C, Step 1): tau = min(T / c, 1 / (2 g_max)), with       */
/* c = max|x| + max|y| (= R here), g_max = 5 m, m = sigma or 1/alpha,      */
/* T = 0.3 (Gauss), 0.1 (Laplace).  Negative distance (App. G): the        */
/* 2T-periodic series with T = R, i.e. tau = 1/(2R).                       */
/* ---------------------------------------------------------------------- */
double o_tau(int kernel, double kparam, double R)
{
    if (!(R > 0.0)) return -1.0;
    if (kernel == O_GAUSS) {
        double gmax = 5.0 * kparam;
        double t1 = 0.3 / R, t2 = 1.0 / (2.0 * gmax);
        return t1 < t2 ? t1 : t2;
    }
    if (kernel == O_LAPLACE) {
        double gmax = 5.0 / kparam;
        double t1 = 0.1 / R, t2 = 1.0 / (2.0 * gmax);
        return t1 < t2 ? t1 : t2;
    }
    if (kernel == O_NEGDIST) return 1.0 / (2.0 * R);
    return -1.0;
}

/* Riesz kernel F(x) = -x^r with r = 1 (Table tab:kernels):                */
/* f(x) = -sqrt(pi) Gamma((d+1)/2) / (Gamma(d/2) Gamma(1)) |x|.            */
double o_riesz_const(int d)
{
    return exp(0.5 * log(O_PI) + lgamma(0.5 * (d + 1)) - lgamma(0.5 * d));
}

/* Radial basis function F (Table tab:kernels). */
double o_F(int kernel, double kparam, double r)
{
    if (kernel == O_GAUSS) return exp(-r * r / (2.0 * kparam * kparam));
    if (kernel == O_LAPLACE) return exp(-kparam * r);
    if (kernel == O_NEGDIST) return -r;
    return NAN;
}

/* One-dimensional basis function f in closed form where one exists:        */
/*  d = 1: f = F;                                                           */
/*  d = 3: f = (t F(t))' since eq. integral_transform reduces to             */
/*         F(t) = int_0^1 f(ts) ds for d = 3;                                */
/*  negative distance, any d: f(t) = -c_d |t| (Riesz row, r = 1).           */
/* Returns NAN where no closed form is implemented.                         */
double o_f(int kernel, double kparam, int d, double t)
{
    t = fabs(t);
    if (kernel == O_NEGDIST) return -o_riesz_const(d) * t;
    if (d == 1) return o_F(kernel, kparam, t);
    if (d == 3) {
        if (kernel == O_GAUSS) {
            double s2 = kparam * kparam;
            return (1.0 - t * t / s2) * exp(-t * t / (2.0 * s2));
        }
        if (kernel == O_LAPLACE) return (1.0 - kparam * t) * exp(-kparam * t);
    }
    return NAN;
}

/* F_1[f(|.|)](omega), evaluated in log space (|omega|^{d-1} and Gamma     */
/* overflow separately for d in the hundreds).                             */
/*  Gauss:   sqrt(2) pi sigma (2 pi^2 sigma^2 w^2)^{(d-1)/2}                */
/*           exp(-2 pi^2 sigma^2 w^2) / Gamma(d/2)                          */
/*  Laplace: Gamma((d+1)/2) 2^d pi^{d-1/2} |w|^{d-1} / (Gamma(d/2) alpha^d) */
/*           (1 + 4 pi^2 w^2 / alpha^2)^{-(d+1)/2}                          */
double o_fhat(int kernel, double kparam, int d, double omega)
{
    double aw = fabs(omega);
    if (kernel == O_GAUSS) {
        double sig = kparam;
        double q = 2.0 * O_PI * O_PI * sig * sig * aw * aw;
        if (aw == 0.0) return d == 1 ? sqrt(2.0 * O_PI) * sig : 0.0;
        double lg = 0.5 * log(2.0) + log(O_PI) + log(sig) + 0.5 * (d - 1) * log(q) - q
                    - lgamma(0.5 * d);
        return exp(lg);
    }
    if (kernel == O_LAPLACE) {
        double al = kparam;
        if (aw == 0.0) return d == 1 ? 2.0 / al : 0.0;
        double lg = lgamma(0.5 * (d + 1)) + d * log(2.0) + (d - 0.5) * log(O_PI)
                    + (d - 1) * log(aw) - lgamma(0.5 * d) - d * log(al)
                    - 0.5 * (d + 1) * log1p(4.0 * O_PI * O_PI * aw * aw / (al * al));
        return exp(lg);
    }
    return NAN;
}

/* Fourier coefficients c_k, k = -nft/2 .. nft/2-1, stored at c[k + nft/2]. */
/*  Gauss / Laplace (App. C, Step 2): c_k = F_1[g~](k) = tau f-hat(tau k),  */
/*  with g~(x) = f(|x| / tau) (Poisson summation, g~ ~ 0 outside [-1/2,1/2]).*/
/*  Negative distance (App. G): g~ is the 1-periodic triangle wave          */
/*  -(c_d / tau)|t| on [-1/2, 1/2); its coefficients are                    */
/*  c_0 = -(c_d/tau)/4,  c_k = (c_d/tau) / (pi^2 k^2) for odd k, 0 else.    */
int o_coeffs(int kernel, double kparam, int d, double tau, int nft, double* c)
{
    if (nft < 2 || (nft & 1) || !(tau > 0.0) || d < 1 || !c) return O_EARG;
    int K = nft / 2;
    for (int k = -K; k < K; ++k) {
        double v;
        if (kernel == O_GAUSS || kernel == O_LAPLACE) {
            v = tau * o_fhat(kernel, kparam, d, tau * (double)k);
        } else if (kernel == O_NEGDIST) {
            double amp = o_riesz_const(d) / tau;
            if (k == 0) v = -amp / 4.0;
            else if (k % 2 != 0) v = amp / (O_PI * O_PI * (double)k * (double)k);
            else v = 0.0;
        } else {
            return O_EUNSUPPORTED;
        }
        c[k + K] = v;
    }
    return O_OK;
}

/* ---------------------------------------------------------------------- */
/* helpers                                                                 */
/* ---------------------------------------------------------------------- */
static double dot_fd(const float* a, const float* b, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += (double)a[j] * (double)b[j];
    return s;
}

/* e^{sign * 2 pi i k a} for k = k0, k0+1, ..., k0+count-1, written to      */
/* (re, im).  The phasor advances by multiplying with e^{sign 2 pi i a} and */
/* is recomputed from cos/sin every 64 steps; the phase is reduced modulo 1 */
/* before the trigonometric call.                                           */
static void phasors(double a, int sign, int k0, int count, double* re, double* im)
{
    double sr = cos(2.0 * O_PI * a), si = sign * sin(2.0 * O_PI * a);
    double er = 0.0, ei = 0.0;
    for (int i = 0; i < count; ++i) {
        if ((i & 63) == 0) {
            double ka = (double)(k0 + i) * a;
            double ph = ka - nearbyint(ka);
            er = cos(2.0 * O_PI * ph);
            ei = sign * sin(2.0 * O_PI * ph);
        } else {
            double nr = er * sr - ei * si;
            double ni = er * si + ei * sr;
            er = nr;
            ei = ni;
        }
        re[i] = er;
        im[i] = ei;
    }
}

static int n_threads(int requested)
{
#ifdef _OPENMP
    if (requested > 0) return requested;
    return omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* O1: the sliced, Fourier-truncated kernel sum                            */
/*                                                                         */
/*   a_{n,p} = tau <x_n, xi_p>,  b_{m,p} = tau <y_m, xi_p>                  */
/*   w^_{k,p} = sum_n w_n e^{-2 pi i k a_{n,p}}          (adjoint NDFT)     */
/*   t_{m,p} = Re sum_k c_k w^_{k,p} e^{2 pi i k b_{m,p}} (NDFT)            */
/*   s_m     = (1/P) sum_p t_{m,p}                                          */
/*                                                                         */
/* Sec. 2.1 eq. kernel_sum_sliced with each 1D sum by App. C eq.           */
/* 1d_sum_fourier (App. G eq. Fourier-slicing for the periodic case).      */
/* Direct NDFT, no window, no FFT.  Slices run in parallel; the slice      */
/* results are stored and averaged in slice order, so the result does not  */
/* depend on the thread count.  w may be NULL (all weights one).           */
/* ---------------------------------------------------------------------- */
int o1_sum(int d, int64_t N, const float* x, const float* w, int64_t M, const float* y,
           int P, const float* xi, double tau, int nft, const double* c, double* s,
           int nthreads)
{
    if (d < 1 || N < 0 || M < 0 || P < 1 || nft < 2 || (nft & 1) || !s || !c || !xi) return O_EARG;
    if ((N > 0 && !x) || (M > 0 && !y)) return O_EARG;
    if (M == 0) return O_OK;
    int K = nft / 2;
    double* t = (double*)calloc((size_t)P * (size_t)M, sizeof(double));
    if (!t) return O_ENOMEM;
    int err = 0;

#pragma omp parallel num_threads(n_threads(nthreads))
    {
        double* wr = (double*)malloc(sizeof(double) * nft);
        double* wi = (double*)malloc(sizeof(double) * nft);
        double* er = (double*)malloc(sizeof(double) * nft);
        double* ei = (double*)malloc(sizeof(double) * nft);
        if (!wr || !wi || !er || !ei) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < P; ++p) {
            if (err) continue;
            const float* xp = xi + (size_t)p * d;
            for (int k = 0; k < nft; ++k) wr[k] = wi[k] = 0.0;
            /* adjoint NDFT: w^_k = sum_n w_n e^{-2 pi i k a_n} */
            for (int64_t n = 0; n < N; ++n) {
                double a = tau * dot_fd(x + (size_t)n * d, xp, d);
                double wn = w ? (double)w[n] : 1.0;
                phasors(a, -1, -K, nft, er, ei);
                for (int k = 0; k < nft; ++k) {
                    wr[k] += wn * er[k];
                    wi[k] += wn * ei[k];
                }
            }
            /* NDFT: t_m = Re sum_k c_k w^_k e^{2 pi i k b_m} */
            for (int64_t m = 0; m < M; ++m) {
                double b = tau * dot_fd(y + (size_t)m * d, xp, d);
                phasors(b, +1, -K, nft, er, ei);
                double acc = 0.0;
                for (int k = 0; k < nft; ++k) acc += c[k] * (wr[k] * er[k] - wi[k] * ei[k]);
                t[(size_t)p * M + m] = acc;
            }
        }
        free(wr);
        free(wi);
        free(er);
        free(ei);
    }
    if (err) {
        free(t);
        return O_ENOMEM;
    }
    for (int64_t m = 0; m < M; ++m) {
        double acc = 0.0;
        for (int p = 0; p < P; ++p) acc += t[(size_t)p * M + m];
        s[m] = acc / (double)P;
    }
    free(t);
    return O_OK;
}

/* ---------------------------------------------------------------------- */
/* O1 gradients of L = sum_m v_m s_m, with s the O1 sum above.             */
/* Write g~_N(t) = Re sum_k c_k e^{2 pi i k t}; then                       */
/*   s_m = (1/P) sum_p sum_n w_n g~_N(b_{m,p} - a_{n,p}),                   */
/*   dL/dy_m = (tau/P) v_m sum_p xi_p Re sum_k 2 pi i k c_k w^_{k,p} e^{2 pi i k b_{m,p}}, */
/*   dL/dx_n = -(tau/P) w_n sum_p xi_p Re sum_k 2 pi i k c_k e^{-2 pi i k a_{n,p}} v^_{k,p}, */
/*   dL/dw_n = (1/P) sum_p Re sum_k c_k e^{-2 pi i k a_{n,p}} v^_{k,p},     */
/* with v^_{k,p} = sum_m v_m e^{2 pi i k b_{m,p}}.  Gradients are returned  */
/* for the listed indices only (idx_n for gx and gw, idx_m for gy), so     */
/* large problems can be checked on a sample.  Any output may be NULL.     */
/* ---------------------------------------------------------------------- */
int o1_grad(int d, int64_t N, const float* x, const float* w, int64_t M, const float* y,
            const float* v, int P, const float* xi, double tau, int nft, const double* c,
            int64_t n_out, const int64_t* idx_n, double* gx, double* gw,
            int64_t m_out, const int64_t* idx_m, double* gy, int nthreads)
{
    if (d < 1 || N < 0 || M < 0 || P < 1 || nft < 2 || (nft & 1) || !c || !xi || !v) return O_EARG;
    if ((n_out > 0 && !idx_n) || (m_out > 0 && !idx_m)) return O_EARG;
    int K = nft / 2;
    int want_x = (gx || gw) && n_out > 0;
    int want_y = gy && m_out > 0;
    /* per-slice scalars: qx[p][i] = Re sum_k 2 pi i k c_k e^{-2 pi i k a} v^_k,
       qw[p][i] = Re sum_k c_k e^{-2 pi i k a} v^_k,
       qy[p][j] = Re sum_k 2 pi i k c_k w^_k e^{2 pi i k b}            */
    double* qx = want_x ? (double*)calloc((size_t)P * n_out, sizeof(double)) : NULL;
    double* qw = want_x ? (double*)calloc((size_t)P * n_out, sizeof(double)) : NULL;
    double* qy = want_y ? (double*)calloc((size_t)P * m_out, sizeof(double)) : NULL;
    if ((want_x && (!qx || !qw)) || (want_y && !qy)) {
        free(qx);
        free(qw);
        free(qy);
        return O_ENOMEM;
    }
    int err = 0;
#pragma omp parallel num_threads(n_threads(nthreads))
    {
        double* hr = (double*)malloc(sizeof(double) * nft);
        double* hi = (double*)malloc(sizeof(double) * nft);
        double* er = (double*)malloc(sizeof(double) * nft);
        double* ei = (double*)malloc(sizeof(double) * nft);
        if (!hr || !hi || !er || !ei) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < P; ++p) {
            if (err) continue;
            const float* xp = xi + (size_t)p * d;
            if (want_y) {
                for (int k = 0; k < nft; ++k) hr[k] = hi[k] = 0.0;
                for (int64_t n = 0; n < N; ++n) {
                    double a = tau * dot_fd(x + (size_t)n * d, xp, d);
                    double wn = w ? (double)w[n] : 1.0;
                    phasors(a, -1, -K, nft, er, ei);
                    for (int k = 0; k < nft; ++k) {
                        hr[k] += wn * er[k];
                        hi[k] += wn * ei[k];
                    }
                }
                for (int64_t j = 0; j < m_out; ++j) {
                    double b = tau * dot_fd(y + (size_t)idx_m[j] * d, xp, d);
                    phasors(b, +1, -K, nft, er, ei);
                    double acc = 0.0;
                    for (int k = 0; k < nft; ++k) {
                        /* Re( 2 pi i k c_k (hr + i hi)(er + i ei) ) = -2 pi k c_k Im(...) */
                        double im = hr[k] * ei[k] + hi[k] * er[k];
                        acc += -2.0 * O_PI * (double)(k - K) * c[k] * im;
                    }
                    qy[(size_t)p * m_out + j] = acc;
                }
            }
            if (want_x) {
                for (int k = 0; k < nft; ++k) hr[k] = hi[k] = 0.0;
                for (int64_t m = 0; m < M; ++m) {
                    double b = tau * dot_fd(y + (size_t)m * d, xp, d);
                    double vm = (double)v[m];
                    phasors(b, +1, -K, nft, er, ei);
                    for (int k = 0; k < nft; ++k) {
                        hr[k] += vm * er[k];
                        hi[k] += vm * ei[k];
                    }
                }
                for (int64_t i = 0; i < n_out; ++i) {
                    double a = tau * dot_fd(x + (size_t)idx_n[i] * d, xp, d);
                    phasors(a, -1, -K, nft, er, ei);
                    double ad = 0.0, ac = 0.0;
                    for (int k = 0; k < nft; ++k) {
                        double re = hr[k] * er[k] - hi[k] * ei[k];
                        double im = hr[k] * ei[k] + hi[k] * er[k];
                        ac += c[k] * re;
                        ad += -2.0 * O_PI * (double)(k - K) * c[k] * im;
                    }
                    qx[(size_t)p * n_out + i] = ad;
                    qw[(size_t)p * n_out + i] = ac;
                }
            }
        }
        free(hr);
        free(hi);
        free(er);
        free(ei);
    }
    if (err) {
        free(qx);
        free(qw);
        free(qy);
        return O_ENOMEM;
    }
    /* reduce over slices in slice order */
    if (want_y) {
        for (int64_t j = 0; j < m_out; ++j) {
            double vm = (double)v[idx_m[j]];
            for (int q = 0; q < d; ++q) {
                double acc = 0.0;
                for (int p = 0; p < P; ++p) acc += qy[(size_t)p * m_out + j] * (double)xi[(size_t)p * d + q];
                gy[j * d + q] = tau / (double)P * vm * acc;
            }
        }
    }
    if (want_x) {
        for (int64_t i = 0; i < n_out; ++i) {
            double wn = w ? (double)w[idx_n[i]] : 1.0;
            if (gx) {
                for (int q = 0; q < d; ++q) {
                    double acc = 0.0;
                    for (int p = 0; p < P; ++p) acc += qx[(size_t)p * n_out + i] * (double)xi[(size_t)p * d + q];
                    gx[i * d + q] = -tau / (double)P * wn * acc;
                }
            }
            if (gw) {
                double acc = 0.0;
                for (int p = 0; p < P; ++p) acc += qw[(size_t)p * n_out + i];
                gw[i] = acc / (double)P;
            }
        }
    }
    free(qx);
    free(qw);
    free(qy);
    return O_OK;
}

/* ---------------------------------------------------------------------- */
/* O2: exact kernel sum s_m = sum_n w_n F(|x_n - y_m|)  (eq. kernel_sum)    */
/* ---------------------------------------------------------------------- */
int o2_exact(int kernel, double kparam, int d, int64_t N, const float* x, const float* w,
             int64_t M, const float* y, double* s, int nthreads)
{
    if (d < 1 || N < 0 || M < 0 || !s) return O_EARG;
    if (kernel != O_GAUSS && kernel != O_LAPLACE && kernel != O_NEGDIST) return O_EUNSUPPORTED;
#pragma omp parallel for schedule(static) num_threads(n_threads(nthreads))
    for (int64_t m = 0; m < M; ++m) {
        double acc = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double r2 = 0.0;
            for (int j = 0; j < d; ++j) {
                double diff = (double)x[(size_t)n * d + j] - (double)y[(size_t)m * d + j];
                r2 += diff * diff;
            }
            acc += (w ? (double)w[n] : 1.0) * o_F(kernel, kparam, sqrt(r2));
        }
        s[m] = acc;
    }
    return O_OK;
}

/* ---------------------------------------------------------------------- */
/* O3: sliced sum with the closed-form basis function f                    */
/*   s_m = (1/P) sum_p sum_n w_n f(|<xi_p, x_n - y_m>|)  (eq. kernel_sum_sliced) */
/* No Fourier step.  Available where o_f has a closed form.                */
/* ---------------------------------------------------------------------- */
int o3_sliced(int kernel, double kparam, int d, int64_t N, const float* x, const float* w,
              int64_t M, const float* y, int P, const float* xi, double* s, int nthreads)
{
    if (d < 1 || N < 0 || M < 0 || P < 1 || !s || !xi) return O_EARG;
    if (isnan(o_f(kernel, kparam, d, 0.5))) return O_EUNSUPPORTED;
#pragma omp parallel for schedule(static) num_threads(n_threads(nthreads))
    for (int64_t m = 0; m < M; ++m) {
        double tot = 0.0;
        for (int p = 0; p < P; ++p) {
            const float* xp = xi + (size_t)p * d;
            double bm = dot_fd(y + (size_t)m * d, xp, d);
            double acc = 0.0;
            for (int64_t n = 0; n < N; ++n) {
                double an = dot_fd(x + (size_t)n * d, xp, d);
                acc += (w ? (double)w[n] : 1.0) * o_f(kernel, kparam, d, an - bm);
            }
            tot += acc;
        }
        s[m] = tot / (double)P;
    }
    return O_OK;
}
