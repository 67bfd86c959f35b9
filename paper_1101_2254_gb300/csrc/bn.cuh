// bn.cuh -- the Sersic index constant b_n (P(2n, b_n) = 1/2, so that r_e
// encloses half the light) solved by a whole warp, shared by the LM kernels
// (lm.cu: the b_n table and the direct solves) and the network's data kernels
// (cnn.cu: training draws and targets).
#pragma once

#include <math.h>

namespace {

// Regularised lower incomplete gamma P(a, x) by its power series
//   P(a, x) = x^a e^{-x} / Gamma(a+1) * sum_{k>=0} x^k / ((a+1)...(a+k)),
// evaluated by the whole warp: lane l forms the ratios x/(a+k) for
// k = 3l+1 .. 3l+3, a warp scan multiplies them into the terms, a butterfly sums
// them.  96 terms: for the b_n root x < a <= 20, term 96 is below 1e-40.
// Every lane returns the same value.  lg1 = ln Gamma(a + 1).
__device__ double gamma_p_warp(double a, double x, double lg1)
{
    if (x <= 0.0) return 0.0;
    const int lane = threadIdx.x & 31;
    const double k0 = 1.0 + 3.0 * lane;
    const double r0 = x / (a + k0), r1 = x / (a + k0 + 1.0), r2 = x / (a + k0 + 2.0);
    const double p0 = r0, p1 = p0 * r1, p2 = p1 * r2;
    double incl = p2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl *= v;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 1.0;
    double s = excl * (p0 + p1 + p2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return exp(a * log(x) - x - lg1) * (1.0 + s);
}

// b_n: root of P(2n, b) = 1/2 by Newton steps safeguarded with a bisection
// bracket (the median of a Gamma(a) variate lies in (0, a)).  The start is
// `guess` when it lies in the bracket, else the asymptotic expansion of
// Ciotti & Bertin (1999).  Called by all lanes of a warp with equal arguments.
__device__ double sersic_bn_warp(double n, double guess)
{
    const double a = 2.0 * n;
    double lo = 0.0, hi = a;
    double b = guess;
    if (!(b > lo && b < hi)) b = a - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n);
    if (!(b > lo && b < hi)) b = 0.5 * a;
    const double lg1 = lgamma(a + 1.0), lga = lg1 - log(a);
    for (int it = 0; it < 100; ++it) {
        const double f = gamma_p_warp(a, b, lg1) - 0.5;
        if (f == 0.0) break;
        if (f < 0.0)
            lo = b;
        else
            hi = b;
        const double dens = exp((a - 1.0) * log(b) - b - lga);
        double nb = b - f / dens;
        const bool newton = nb > lo && nb < hi;
        if (!newton) nb = 0.5 * (lo + hi);
        // Newton converges quadratically: once a Newton correction is below
        // 1e-6 b, the corrected value is good to ~1e-12 b (far below float32)
        const bool done = newton && fabs(nb - b) <= 1e-6 * b;
        b = nb;
        if (done || hi - lo <= 1e-14 * b) break;
    }
    return b;
}

}  // namespace
