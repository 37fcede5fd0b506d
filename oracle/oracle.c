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
 *   o_riesz_const_r  the same for any r > -1           (Table tab:kernels, Riesz row)
 *   o_tps_const    C_d of the sliced thin plate spline (Table tab:kernels, Thin Plate Spline row)
 *   o_f            1D basis function f, closed forms  (Table tab:kernels; Sec. 2, eq. integral_transform)
 *   o_F            radial basis function F            (Table tab:kernels)
 *   o_fhat         1D Fourier transform of f(|.|)     (Table tab:kernels with the corrected constants)
 *   o_coeffs       Fourier coefficients c_k           (App. C "Step 2"; App. G, eq. Fourier-slicing)
 *   o1_sum         sliced, Fourier-truncated sum      (Sec. 2.1 eq. kernel_sum_sliced + App. C eq. 1d_sum_fourier)
 *   o1_grad        gradients of L = sum_m v_m s_m of the same sum
 *   o2_exact       exact kernel sum, O(NM)            (Sec. 1, eq. kernel_sum)
 *   o3_sliced      sliced sum with closed-form f      (Sec. 2.1, eq. kernel_sum_sliced)
 *   o3_grad_negdist gradient in y of the sliced negative-distance sum (Sec. 2.1, eq. kernel_sum_sliced)
 *   o_esym         symmetric distance energy and its gradient (Sec. 2.3, eq. distance-mmd;
 *                  App. "Relation between Distance QMC Designs and Orthogonal Points", eq. distance-sym)
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
 *   - Matern (nu = kp2, beta = kp): f-hat from the same relation, which is the
 *     last column of Table tab:kernels; tau = min(0.2 / R, 1 / (2 * 5 beta))
 *     (App. C, Step 1: T = 0.2, g_max = 5 beta).
 *   - Generalised Riesz F = -x^r (0 < r < 2, r = kp) and the thin plate spline
 *     F = x^2 log x have no classical Fourier transform (App. A); like the
 *     negative distance kernel they use the 1-periodic continuation of
 *     g(t) = f(|t| / tau) on [-1/2, 1/2) with tau = 1/(2R), whose coefficients
 *     are the integrals c_k = 2 int_0^{1/2} g(t) cos(2 pi k t) dt, computed here
 *     by Gauss-Legendre quadrature on half-period panels.
 *   - H_{d/2} in C_d is the harmonic number at d/2 (digamma(d/2 + 1) + Euler's
 *     constant), so C_3 = 1 and f(t) = 3 t^2 log|t| + t^2 for d = 3.
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
#define O_MATERN 3
#define O_RIESZ 4
#define O_TPS 5

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
    if (kernel == O_MATERN) {
        double gmax = 5.0 * kparam;
        double t1 = 0.2 / R, t2 = 1.0 / (2.0 * gmax);
        return t1 < t2 ? t1 : t2;
    }
    if (kernel == O_RIESZ || kernel == O_TPS) return 1.0 / (2.0 * R);
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

/* Generalised Riesz F(x) = -x^r (Table tab:kernels):                      */
/* f(x) = -sqrt(pi) Gamma((d+r)/2) / (Gamma(d/2) Gamma((r+1)/2)) |x|^r.    */
double o_riesz_const_r(int d, double r)
{
    return exp(0.5 * log(O_PI) + lgamma(0.5 * (d + r)) - lgamma(0.5 * d) - lgamma(0.5 * (r + 1.0)));
}

/* Thin plate spline (Table tab:kernels): C_d = d/2 (H_{d/2} - 2 + log 4), */
/* H_{d/2} by H_0 = 0, H_{1/2} = 2 - 2 log 2 and H_{x+1} = H_x + 1/(x+1).  */
double o_tps_const(int d)
{
    double h = (d % 2 == 0) ? 0.0 : 2.0 - 2.0 * log(2.0);
    double x = (d % 2 == 0) ? 0.0 : 0.5;
    while (x + 0.25 < 0.5 * d) {
        x += 1.0;
        h += 1.0 / x;
    }
    return 0.5 * d * (h - 2.0 + log(4.0));
}

/* Matern with nu = p + 1/2 (p = 0, 1, 2, ...): F(x) = e^{-a x} sum_{i<=p}  */
/* p!/(2p)! (p+i)!/(i!(p-i)!) (2 a x)^{p-i}, a = sqrt(2 nu)/beta.  Writes  */
/* the coefficients q_j of F(x) = e^{-a x} sum_j q_j x^j; returns p, or -1  */
/* if nu is not a half-integer (no closed form here).                       */
static int matern_poly(double beta, double nu, double* a_out, double q[16])
{
    double pd = nu - 0.5;
    int p = (int)llround(pd);
    if (p < 0 || p > 14 || fabs(pd - p) > 1e-12) return -1;
    double a = sqrt(2.0 * nu) / beta;
    for (int j = 0; j < 16; ++j) q[j] = 0.0;
    double lf_p = lgamma(p + 1.0), lf_2p = lgamma(2.0 * p + 1.0);
    for (int i = 0; i <= p; ++i) {
        int j = p - i;
        double lc = lf_p - lf_2p + lgamma(p + i + 1.0) - lgamma(i + 1.0) - lgamma(j + 1.0);
        q[j] = exp(lc) * pow(2.0 * a, (double)j);
    }
    *a_out = a;
    return p;
}

/* Radial basis function F (Table tab:kernels).  Matern: kp = beta, kp2 =  */
/* nu (half-integers only); Riesz: kp = r.                                  */
double o_F2(int kernel, double kparam, double kp2, double r)
{
    if (kernel == O_GAUSS) return exp(-r * r / (2.0 * kparam * kparam));
    if (kernel == O_LAPLACE) return exp(-kparam * r);
    if (kernel == O_NEGDIST) return -r;
    if (kernel == O_RIESZ) return -pow(r, kparam);
    if (kernel == O_TPS) return r > 0.0 ? r * r * log(r) : 0.0;
    if (kernel == O_MATERN) {
        double a, q[16];
        int p = matern_poly(kparam, kp2, &a, q);
        if (p < 0) return NAN;
        double e = exp(-a * r), acc = 0.0;
        if (e == 0.0) return 0.0; /* far tail: the polynomial may overflow */
        for (int j = p; j >= 0; --j) acc = acc * r + q[j];
        return e * acc;
    }
    return NAN;
}

double o_F(int kernel, double kparam, double r) { return o_F2(kernel, kparam, 0.0, r); }

/* One-dimensional basis function f in closed form where one exists:        */
/*  d = 1: f = F;                                                           */
/*  d = 3: f = (t F(t))' since eq. integral_transform reduces to             */
/*         F(t) = int_0^1 f(ts) ds for d = 3;                                */
/*  negative distance, any d: f(t) = -c_d |t| (Riesz row, r = 1).           */
/* Returns NAN where no closed form is implemented.                         */
double o_f2(int kernel, double kparam, double kp2, int d, double t)
{
    t = fabs(t);
    if (kernel == O_NEGDIST) return -o_riesz_const(d) * t;
    if (kernel == O_RIESZ) return -o_riesz_const_r(d, kparam) * pow(t, kparam);
    if (kernel == O_TPS) return t > 0.0 ? d * t * t * log(t) + o_tps_const(d) * t * t : 0.0;
    if (d == 1) return o_F2(kernel, kparam, kp2, t);
    if (d == 3 && kernel == O_MATERN) {
        /* (t F)' = e^{-a t} (P + t P' - a t P) for F = e^{-a t} P */
        double a, q[16];
        int p = matern_poly(kparam, kp2, &a, q);
        if (p < 0) return NAN;
        double P0 = 0.0, P1 = 0.0;
        if (exp(-a * t) == 0.0) return 0.0;
        for (int j = p; j >= 0; --j) P0 = P0 * t + q[j];
        for (int j = p; j >= 1; --j) P1 = P1 * t + j * q[j];
        return exp(-a * t) * (P0 + t * P1 - a * t * P0);
    }
    if (d == 3) {
        if (kernel == O_GAUSS) {
            double s2 = kparam * kparam;
            return (1.0 - t * t / s2) * exp(-t * t / (2.0 * s2));
        }
        if (kernel == O_LAPLACE) return (1.0 - kparam * t) * exp(-kparam * t);
    }
    return NAN;
}

double o_f(int kernel, double kparam, int d, double t) { return o_f2(kernel, kparam, 0.0, d, t); }

/* F_1[f(|.|)](omega), evaluated in log space (|omega|^{d-1} and Gamma     */
/* overflow separately for d in the hundreds).                             */
/*  Gauss:   sqrt(2) pi sigma (2 pi^2 sigma^2 w^2)^{(d-1)/2}                */
/*           exp(-2 pi^2 sigma^2 w^2) / Gamma(d/2)                          */
/*  Laplace: Gamma((d+1)/2) 2^d pi^{d-1/2} |w|^{d-1} / (Gamma(d/2) alpha^d) */
/*           (1 + 4 pi^2 w^2 / alpha^2)^{-(d+1)/2}                          */
/*  Matern:  Gamma(nu + d/2) 2^{d/2} pi^d beta^d |w|^{d-1}                 */
/*           / (Gamma(d/2) Gamma(nu) nu^{d/2}) (1 + 2 pi^2 beta^2 w^2/nu)^{-(nu+d/2)} */
double o_fhat2(int kernel, double kparam, double kp2, int d, double omega)
{
    double aw = fabs(omega);
    if (kernel == O_MATERN) {
        double be = kparam, nu = kp2;
        if (aw == 0.0 && d > 1) return 0.0;
        double lg = lgamma(nu + 0.5 * d) + 0.5 * d * log(2.0) + d * log(O_PI) + d * log(be)
                    + (d > 1 ? (d - 1) * log(aw) : 0.0) - lgamma(0.5 * d) - lgamma(nu) - 0.5 * d * log(nu)
                    - (nu + 0.5 * d) * log1p(2.0 * O_PI * O_PI * be * be * aw * aw / nu);
        return exp(lg);
    }
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

double o_fhat(int kernel, double kparam, int d, double omega) { return o_fhat2(kernel, kparam, 0.0, d, omega); }

/* ---------------------------------------------------------------------- */
/* 2 int_0^{1/2} g(t) cos(2 pi k t) dt for the periodised kernels, by      */
/* 20-point Gauss-Legendre on the half-periods of the cosine, the first    */
/* one graded geometrically towards the |t|^r or t^2 log t point t = 0.    */
/* ---------------------------------------------------------------------- */
#define O_GL 20
static double o_gl_x[O_GL], o_gl_w[O_GL];
static int o_gl_ready = 0;

static void o_gl_init(void)
{
    if (o_gl_ready) return;
    for (int i = 0; i < O_GL; ++i) {
        double z = cos(O_PI * (i + 0.75) / (O_GL + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= O_GL; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = O_GL * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        o_gl_x[i] = z;
        o_gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    o_gl_ready = 1;
}

/* g(t) for t in (0, 1/2], i.e. f(t / tau) */
static double o_gper(int kernel, double kparam, int d, double tau, double t)
{
    return o_f2(kernel, kparam, 0.0, d, t / tau);
}

static double o_panel(int kernel, double kparam, int d, double tau, int k, double a, double b)
{
    double m = 0.5 * (a + b), h = 0.5 * (b - a), acc = 0.0;
    for (int i = 0; i < O_GL; ++i) {
        double t = m + h * o_gl_x[i];
        acc += o_gl_w[i] * o_gper(kernel, kparam, d, tau, t) * cos(2.0 * O_PI * k * t);
    }
    return acc * h;
}

static double o_periodic_coeff(int kernel, double kparam, int d, double tau, int k)
{
    int ak = k < 0 ? -k : k;
    int npan = ak < 1 ? 1 : ak; /* half-periods of cos(2 pi k t) on [0, 1/2] */
    double hw = 0.5 / npan, acc = 0.0;
    for (int j = 1; j < npan; ++j) acc += o_panel(kernel, kparam, d, tau, ak, j * hw, (j + 1) * hw);
    double b = hw; /* first panel, graded: [hw/2^{l+1}, hw/2^l], l = 0..59 */
    for (int l = 0; l < 60; ++l) {
        acc += o_panel(kernel, kparam, d, tau, ak, 0.5 * b, b);
        b *= 0.5;
    }
    return 2.0 * acc;
}

/* Fourier coefficients c_k, k = -nft/2 .. nft/2-1, stored at c[k + nft/2]. */
/*  Gauss / Laplace (App. C, Step 2): c_k = F_1[g~](k) = tau f-hat(tau k),  */
/*  with g~(x) = f(|x| / tau) (Poisson summation, g~ ~ 0 outside [-1/2,1/2]).*/
/*  Negative distance (App. G): g~ is the 1-periodic triangle wave          */
/*  -(c_d / tau)|t| on [-1/2, 1/2); its coefficients are                    */
/*  c_0 = -(c_d/tau)/4,  c_k = (c_d/tau) / (pi^2 k^2) for odd k, 0 else.    */
/*  Matern: tau f-hat(tau k) as for Gauss / Laplace.  Riesz and thin plate */
/*  spline: the integrals of the periodised g~ above (c_{-k} = c_k).        */
int o_coeffs2(int kernel, double kparam, double kp2, int d, double tau, int nft, double* c)
{
    if (nft < 2 || (nft & 1) || !(tau > 0.0) || d < 1 || !c) return O_EARG;
    int K = nft / 2;
    if (kernel == O_RIESZ || kernel == O_TPS) {
        o_gl_init();
        for (int k = 0; k <= K; ++k) {
            double v = o_periodic_coeff(kernel, kparam, d, tau, k);
            if (k < K) c[k + K] = v;
            c[K - k] = v;
        }
        return O_OK;
    }
    for (int k = -K; k < K; ++k) {
        double v;
        if (kernel == O_GAUSS || kernel == O_LAPLACE || kernel == O_MATERN) {
            v = tau * o_fhat2(kernel, kparam, kp2, d, tau * (double)k);
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

int o_coeffs(int kernel, double kparam, int d, double tau, int nft, double* c)
{
    return o_coeffs2(kernel, kparam, 0.0, d, tau, nft, c);
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
int o2_exact2(int kernel, double kparam, double kp2, int d, int64_t N, const float* x, const float* w,
              int64_t M, const float* y, double* s, int nthreads)
{
    if (d < 1 || N < 0 || M < 0 || !s) return O_EARG;
    if (isnan(o_F2(kernel, kparam, kp2, 0.5))) return O_EUNSUPPORTED;
#pragma omp parallel for schedule(static) num_threads(n_threads(nthreads))
    for (int64_t m = 0; m < M; ++m) {
        double acc = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double r2 = 0.0;
            for (int j = 0; j < d; ++j) {
                double diff = (double)x[(size_t)n * d + j] - (double)y[(size_t)m * d + j];
                r2 += diff * diff;
            }
            acc += (w ? (double)w[n] : 1.0) * o_F2(kernel, kparam, kp2, sqrt(r2));
        }
        s[m] = acc;
    }
    return O_OK;
}

int o2_exact(int kernel, double kparam, int d, int64_t N, const float* x, const float* w,
             int64_t M, const float* y, double* s, int nthreads)
{
    return o2_exact2(kernel, kparam, 0.0, d, N, x, w, M, y, s, nthreads);
}

/* ---------------------------------------------------------------------- */
/* O3: sliced sum with the closed-form basis function f                    */
/*   s_m = (1/P) sum_p sum_n w_n f(|<xi_p, x_n - y_m>|)  (eq. kernel_sum_sliced) */
/* No Fourier step.  Available where o_f has a closed form.                */
/* ---------------------------------------------------------------------- */
int o3_sliced2(int kernel, double kparam, double kp2, int d, int64_t N, const float* x, const float* w,
               int64_t M, const float* y, int P, const float* xi, double* s, int nthreads)
{
    if (d < 1 || N < 0 || M < 0 || P < 1 || !s || !xi) return O_EARG;
    if (isnan(o_f2(kernel, kparam, kp2, d, 0.5))) return O_EUNSUPPORTED;
#pragma omp parallel for schedule(static) num_threads(n_threads(nthreads))
    for (int64_t m = 0; m < M; ++m) {
        double tot = 0.0;
        for (int p = 0; p < P; ++p) {
            const float* xp = xi + (size_t)p * d;
            double bm = dot_fd(y + (size_t)m * d, xp, d);
            double acc = 0.0;
            for (int64_t n = 0; n < N; ++n) {
                double an = dot_fd(x + (size_t)n * d, xp, d);
                acc += (w ? (double)w[n] : 1.0) * o_f2(kernel, kparam, kp2, d, an - bm);
            }
            tot += acc;
        }
        s[m] = tot / (double)P;
    }
    return O_OK;
}

int o3_sliced(int kernel, double kparam, int d, int64_t N, const float* x, const float* w,
              int64_t M, const float* y, int P, const float* xi, double* s, int nthreads)
{
    return o3_sliced2(kernel, kparam, 0.0, d, N, x, w, M, y, P, xi, s, nthreads);
}

/* ---------------------------------------------------------------------- */
/* Symmetric distance energy of P points xi_p in R^d (eq. distance-sym):   */
/*   E_sym = E((xi, -xi)) = -2 sum_{p,q} (|xi_p - xi_q| + |xi_p + xi_q|),   */
/* the energy of eq. distance-mmd (s = d/2, exponent 1) of the points and  */
/* their antipodes.  Its gradient in xi_p, from the plain definition (both */
/* orders of each pair; the p = q pair contributes |2 xi_p|):               */
/*   dE/dxi_p = -4 [ sum_{q != p} ((xi_p - xi_q)/|xi_p - xi_q|              */
/*                                 + (xi_p + xi_q)/|xi_p + xi_q|) + xi_p/|xi_p| ]. */
/* grad (P x d) may be NULL.                                               */
/* ---------------------------------------------------------------------- */
int o_esym(int d, int P, const float* xi, double* E, double* grad, int nthreads)
{
    if (d < 1 || P < 1 || !xi || !E) return O_EARG;
    double tot = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : tot) num_threads(n_threads(nthreads))
    for (int p = 0; p < P; ++p) {
        const float* a = xi + (size_t)p * d;
        double acc = 0.0;
        double* g = grad ? grad + (size_t)p * d : NULL;
        if (g)
            for (int j = 0; j < d; ++j) g[j] = 0.0;
        for (int q = 0; q < P; ++q) {
            const float* b = xi + (size_t)q * d;
            double dm = 0.0, dp = 0.0;
            for (int j = 0; j < d; ++j) {
                double u = (double)a[j] - (double)b[j], v = (double)a[j] + (double)b[j];
                dm += u * u;
                dp += v * v;
            }
            dm = sqrt(dm);
            dp = sqrt(dp);
            acc += dm + dp;
            if (!g) continue;
            if (q == p) {
                for (int j = 0; j < d; ++j) g[j] += 4.0 * (double)a[j] / dp; /* d|2 a|/da = 2 a/|a| = 4 a/|2 a| */
                continue;
            }
            for (int j = 0; j < d; ++j) {
                double u = (double)a[j] - (double)b[j], v = (double)a[j] + (double)b[j];
                g[j] += 2.0 * (u / dm + v / dp);
            }
        }
        if (g)
            for (int j = 0; j < d; ++j) g[j] *= -2.0;
        tot += acc;
    }
    *E = -2.0 * tot;
    return O_OK;
}

/* ---------------------------------------------------------------------- */
/* Gradient in y_m of L = sum_m v_m s_m for the sliced negative-distance   */
/* sum s_m = (1/P) sum_p sum_n w_n (-c_d) |<xi_p, y_m - x_n>|              */
/* (eq. kernel_sum_sliced, f(t) = -c_d |t|):                               */
/*   dL/dy_m = v_m (-c_d / P) sum_p (sum_n w_n sign(<xi_p, y_m - x_n>)) xi_p, */
/* with sign(0) = 0.  gy is M x d.                                         */
/* ---------------------------------------------------------------------- */
int o3_grad_negdist(int d, int64_t N, const float* x, const float* w, int64_t M, const float* y, const float* v,
                    int P, const float* xi, double* gy, int nthreads)
{
    if (d < 1 || N < 0 || M < 0 || P < 1 || !xi || !gy) return O_EARG;
    const double cd = o_riesz_const(d);
#pragma omp parallel for schedule(static) num_threads(n_threads(nthreads))
    for (int64_t m = 0; m < M; ++m) {
        double* g = gy + (size_t)m * d;
        for (int j = 0; j < d; ++j) g[j] = 0.0;
        for (int p = 0; p < P; ++p) {
            const float* xp = xi + (size_t)p * d;
            const double bm = dot_fd(y + (size_t)m * d, xp, d);
            double c = 0.0;
            for (int64_t n = 0; n < N; ++n) {
                const double t = bm - dot_fd(x + (size_t)n * d, xp, d);
                const double wn = w ? (double)w[n] : 1.0;
                c += t > 0.0 ? wn : (t < 0.0 ? -wn : 0.0);
            }
            for (int j = 0; j < d; ++j) g[j] += c * (double)xp[j];
        }
        const double vm = v ? (double)v[m] : 1.0;
        for (int j = 0; j < d; ++j) g[j] *= vm * (-cd) / (double)P;
    }
    return O_OK;
}
