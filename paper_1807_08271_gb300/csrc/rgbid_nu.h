// Host-side Chebyshev expansion of the constant part of the degrees-of-freedom
// equation ("Error distribution and robust optimisation", eq. robustnessValue).
//
// With w_i = (nu + 1)/(nu + x_i^2) the equation is
//   f(nu) = n [psi((nu + 1)/2) - psi(nu/2) + 1 - ln((nu + 1)/nu)] + sum_i (ln w_i - w_i),
// whose sample-independent part, after ln w_i = ln(nu + 1) - ln(nu + x_i^2), is
//   n g(nu),  g(nu) = psi((nu + 1)/2) - psi(nu/2) + 1 + ln nu.
// g is analytic on [nu_lo, nu_hi] (its nearest singularity is nu = 0), so a
// Chebyshev series in tau = (nu - m)/h converges geometrically; 22 terms over
// [2, 10] err by < 1e-9.  The device adds this series to the sample sums'
// series and bisects on the single polynomial that results.
#pragma once
#include <cmath>

namespace rgbid {

constexpr int kNuGTerms = 22;   // coefficients g_0 .. g_21 (plain convention: g = sum_k g_k T_k)

// digamma for x > 0: the recurrence psi(x) = psi(x + 1) - 1/x up to x >= 12,
// then the asymptotic series ln x - 1/(2x) - sum_k B_2k / (2k x^2k) (7 terms).
static inline double digamma_host(double x) {
    double acc = 0.0;
    while (x < 12.0) {
        acc -= 1.0 / x;
        x += 1.0;
    }
    const double i2 = 1.0 / (x * x);
    const double tail =
        i2 * (1.0 / 12 - i2 * (1.0 / 120 - i2 * (1.0 / 252 - i2 * (1.0 / 240 - i2 * (1.0 / 132 - i2 * (691.0 / 32760 - i2 / 12))))));
    return acc + std::log(x) - 0.5 / x - tail;
}

static inline double nu_g_host(double nu) {
    return digamma_host(0.5 * (nu + 1.0)) - digamma_host(0.5 * nu) + 1.0 + std::log(nu);
}

// g_k for k < kNuGTerms by interpolation at N = 64 Chebyshev nodes (FP64):
// c_k = (2/N) sum_j g(nu(tau_j)) T_k(tau_j), g_0 = c_0 / 2, g_k = c_k.
static inline void nu_g_series(double lo, double hi, float out[kNuGTerms]) {
    constexpr int N = 64;
    const double m = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
    const double pi = 3.14159265358979323846;
    double gv[N], th[N];
    for (int j = 0; j < N; ++j) {
        th[j] = pi * (j + 0.5) / N;
        gv[j] = nu_g_host(m + h * std::cos(th[j]));
    }
    for (int k = 0; k < kNuGTerms; ++k) {
        double s = 0.0;
        for (int j = 0; j < N; ++j) s += gv[j] * std::cos(k * th[j]);
        s *= 2.0 / N;
        out[k] = (float)(k == 0 ? 0.5 * s : s);
    }
}

// The series for the last interval asked for on this thread (the alignment
// entry points pass the same [nu_lo, nu_hi] launch after launch).
static inline const float* nu_g_series_cached(double lo, double hi) {
    thread_local double c_lo = -1.0, c_hi = -1.0;
    thread_local float c_g[kNuGTerms];
    if (!(lo == c_lo && hi == c_hi)) {
        nu_g_series(lo, hi, c_g);
        c_lo = lo;
        c_hi = hi;
    }
    return c_g;
}

// The series the kernels take: g's, with ln h (h the interval's half-width as the
// kernels form it in FP32) folded into the constant term, since f carries -n ln h.
static inline void nu_device_series(double lo, double hi, float out[kNuGTerms]) {
    const float* g = nu_g_series_cached(lo, hi);
    const float h = 0.5f * ((float)hi - (float)lo);
    for (int k = 0; k < kNuGTerms; ++k) out[k] = g[k];
    out[0] = (float)((double)g[0] - std::log((double)h));
}

}  // namespace rgbid
