// Sobol' directions on the sphere (Sec. 4.1, "QMC Sequences": a Sobol' sequence
// on [0,1]^d mapped through the inverse normal CDF in every coordinate and
// projected onto the sphere, xi = theta / |theta|).  Host code, no GPU.
//
// The sequence (Sobol' 1967, in the Bratley-Fox form with 32-bit direction
// numbers): coordinate 0 is the van der Corput sequence; coordinate j >= 1
// uses the j-th primitive polynomial over GF(2), in order of degree and then
// of coefficient value, p(x) = x^s + a_1 x^{s-1} + ... + a_{s-1} x + 1, and
// direction numbers v_k = m_k 2^{32-k} with
//   v_k = v_{k-s} ^ (v_{k-s} >> s) ^ a_1 v_{k-1} ^ ... ^ a_{s-1} v_{k-s+1}   (k > s);
// the initial m_1..m_s are odd, m_k < 2^k, drawn once from a fixed seeded
// stream (every such choice gives a Sobol' sequence; published tables tune
// them for two-dimensional projections).  Point i is the XOR of v_{b+1} over
// the set bits b of the Gray code i ^ (i >> 1) (Antonov-Saleev order: the
// first 2^m points are the same set as in the natural order).  A seed != 0
// applies a random digital shift (XOR of a seeded 32-bit word per
// coordinate), which keeps every net property.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "qs_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

uint64_t splitmix64(uint64_t& state)
{
    uint64_t z = (state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// a * b mod p over GF(2); a, b of degree < s, p of degree s.
uint64_t gf2_mulmod(uint64_t a, uint64_t b, uint64_t p, int s)
{
    uint64_t r = 0;
    while (b) {
        if (b & 1) r ^= a;
        b >>= 1;
        a <<= 1;
        if ((a >> s) & 1) a ^= p;
    }
    return r;
}

// x^e mod p over GF(2).
uint64_t gf2_pow_x(uint64_t e, uint64_t p, int s)
{
    uint64_t base = s == 1 ? (2 ^ p) : 2;  // x reduced mod p (x = 1 mod x + 1)
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = gf2_mulmod(r, base, p, s);
        base = gf2_mulmod(base, base, p, s);
        e >>= 1;
    }
    return r;
}

// p (degree s, constant term 1) is primitive iff x has multiplicative order
// 2^s - 1 modulo p: x^n = 1 and x^(n/q) != 1 for every prime q dividing n.
bool gf2_primitive(uint64_t p, int s)
{
    const uint64_t n = (1ull << s) - 1;
    if (gf2_pow_x(n, p, s) != 1) return false;
    uint64_t m = n;
    for (uint64_t q = 2; q * q <= m; ++q) {
        if (m % q) continue;
        if (gf2_pow_x(n / q, p, s) == 1) return false;
        while (m % q == 0) m /= q;
    }
    if (m > 1 && m != n && gf2_pow_x(n / m, p, s) == 1) return false;
    return true;
}

// Direction numbers v[j][k-1], k = 1..32, for coordinates j < d.
bool sobol_directions(int d, std::vector<uint32_t>& v)
{
    v.assign((size_t)d * 32, 0u);
    for (int k = 1; k <= 32; ++k) v[k - 1] = 1u << (32 - k);
    uint64_t stream = 0x50b01d1ec7ULL;  // fixed: the same sequence for every seed
    int j = 1;
    for (int s = 1; j < d && s <= 30; ++s) {
        for (uint64_t c = 0; c < (1ull << (s - 1)) && j < d; ++c) {
            const uint64_t p = (1ull << s) | (c << 1) | 1ull;
            if (!gf2_primitive(p, s)) continue;
            uint32_t* vj = &v[(size_t)j * 32];
            for (int k = 1; k <= s && k <= 32; ++k) {
                const uint32_t m = k == 1 ? 1u : (uint32_t)((splitmix64(stream) % (1ull << (k - 1))) * 2 + 1);
                vj[k - 1] = m << (32 - k);
            }
            for (int k = s + 1; k <= 32; ++k) {
                uint32_t x = vj[k - s - 1] ^ (vj[k - s - 1] >> s);
                for (int i = 1; i < s; ++i)
                    if ((p >> (s - i)) & 1) x ^= vj[k - i - 1];
                vj[k - 1] = x;
            }
            ++j;
        }
    }
    return j >= d;
}

// Quantile of the standard normal distribution for 0 < u < 1: the rational
// start of Abramowitz & Stegun 26.2.23 (absolute error < 4.5e-4) for the
// tail probability p = min(u, 1 - u), refined by three Halley steps on
// Phi(z) = p with Phi(z) = erfc(-z / sqrt 2) / 2, which is accurate in the
// lower tail; the sign follows u - 1/2.
double norm_quantile(double u)
{
    const double p = u < 0.5 ? u : 1.0 - u;
    const double t = sqrt(-2.0 * log(p));
    double z = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                         (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 3; ++it) {
        const double e = 0.5 * erfc(-z / sqrt(2.0)) - p;
        const double dens = exp(-0.5 * z * z) / sqrt(2.0 * kPi);
        const double r = e / dens;
        z -= r / (1.0 + 0.5 * z * r);
    }
    return u < 0.5 ? z : -z;
}

}  // namespace

// Points u_{i,j} = (x_{i,j} + 1/2) / 2^32 of the (shifted) sequence, i < P, j < d.
qs_status qs_sobol_cube(int d, int P, uint64_t seed, double* out)
{
    std::vector<uint32_t> v;
    if (!sobol_directions(d, v)) return QS_ERR_UNSUPPORTED;
    std::vector<uint32_t> shift(d, 0u);
    if (seed != 0) {
        uint64_t st = seed ^ 0x243f6a8885a308d3ULL;
        for (int j = 0; j < d; ++j) shift[j] = (uint32_t)(splitmix64(st) >> 32);
    }
    for (int i = 0; i < P; ++i) {
        const uint32_t gray = (uint32_t)i ^ ((uint32_t)i >> 1);
        for (int j = 0; j < d; ++j) {
            uint32_t x = 0;
            for (int b = 0; b < 32; ++b)
                if ((gray >> b) & 1u) x ^= v[(size_t)j * 32 + b];
            out[(size_t)i * d + j] = ((double)(x ^ shift[j]) + 0.5) * (1.0 / 4294967296.0);
        }
    }
    return QS_OK;
}

// Unit rows xi_i = theta_i / |theta_i|, theta_{i,j} = Phi^{-1}(u_{i,j}).
qs_status qs_sobol_sphere(int d, int P, uint64_t seed, float* out)
{
    std::vector<double> u((size_t)P * d);
    const qs_status st = qs_sobol_cube(d, P, seed, u.data());
    if (st != QS_OK) return st;
    std::vector<double> g(d);
    for (int i = 0; i < P; ++i) {
        double nrm = 0.0;
        for (int j = 0; j < d; ++j) {
            g[j] = norm_quantile(u[(size_t)i * d + j]);
            nrm += g[j] * g[j];
        }
        nrm = sqrt(nrm);
        for (int j = 0; j < d; ++j) out[(size_t)i * d + j] = (float)(g[j] / nrm);
    }
    return QS_OK;
}

extern "C" qs_status qs_sobol_points(int d, int P, uint64_t seed, double* out_host)
{
    if (!out_host || d < 1 || P < 1 || d > QS_SOBOL_MAX_D) {
        qs_set_error_message("qs_sobol_points: need out_host != NULL, P >= 1 and 1 <= d <= 4096");
        return QS_ERR_ARG;
    }
    const qs_status st = qs_sobol_cube(d, P, seed, out_host);
    if (st != QS_OK) qs_set_error_message("qs_sobol_points: not enough primitive polynomials");
    return st;
}
