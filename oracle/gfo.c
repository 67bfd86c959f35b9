/*
 * gfo.c -- FP64 CPU oracle for "Fitting Galaxies on GPUs" (Barsdell, Barnes &
 * Fluke).  TEST INFRASTRUCTURE ONLY: loaded by the tests, by the smoke check
 * and by the CPU-baseline leg of the benchmark, never by the product path.
 *
 * Each function states the definition it follows.  The paper fixes the five
 * steps of the loop (Sec. 2) and names the algorithms inside steps 1-3
 * (Sec. 3: transform, FFT + transform, transform + reduce); the profile
 * formulas, the oversampling rule, the chi^2 weights and the LM variant are
 * the standard definitions the paper leaves implicit, and each function
 * names the one it takes.
 */
#include "gfo.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ slots */

int gfo_comp_nslots(int kind)
{
    switch (kind) {
    case GFO_SERSIC: return 8;
    case GFO_EXPDISK: return 7;
    case GFO_GAUSSIAN: return 7;
    case GFO_MOFFAT: return 8;
    case GFO_KING: return 9;
    case GFO_NUKER: return 10;
    case GFO_PSF: return 3;
    case GFO_SKYPLANE: return 3;
    case GFO_SERSIC_F: return 14;
    case GFO_SKY: return 1;
    default: return -1;
    }
}

int gfo_nslots(const gfo_desc* d)
{
    int n = 0;
    for (int k = 0; k < d->ncomp; ++k) n += gfo_comp_nslots(d->kinds[k]);
    return n;
}

/* which component owns slot s, and the slot's index inside it */
static void slot_owner(const gfo_desc* d, int s, int* comp, int* local, int* base)
{
    int off = 0;
    for (int k = 0; k < d->ncomp; ++k) {
        int ns = gfo_comp_nslots(d->kinds[k]);
        if (s < off + ns) {
            *comp = k;
            *local = s - off;
            *base = off;
            return;
        }
        off += ns;
    }
    *comp = -1;
    *local = -1;
    *base = -1;
}

/* The amplitude slots (I_e, I_0) and the sky level enter the model linearly. */
int gfo_slot_is_linear(const gfo_desc* d, int s)
{
    int k, l, b;
    slot_owner(d, s, &k, &l, &b);
    if (k < 0) return 0;
    if (d->kinds[k] == GFO_SKY || d->kinds[k] == GFO_SKYPLANE) return 1;
    return l == 2;
}

/* slot semantics: 0 = position, 1 = amplitude, 2 = radius, 3 = Sersic n,
 * 4 = axis ratio, 5 = position angle, 6 = boxiness, 7 = sky, 8 = Moffat beta,
 * 9 = King truncation radius, 10 = King alpha, 11 = Nuker alpha,
 * 12 = Nuker beta, 13 = Nuker gamma, 14 = sky slope in x, 15 = sky slope in y,
 * 16 = Fourier amplitude, 17 = Fourier phase */
static int slot_role(const gfo_desc* d, int s)
{
    int k, l, b;
    slot_owner(d, s, &k, &l, &b);
    if (k < 0) return -1;
    int kind = d->kinds[k];
    if (kind == GFO_SKY) return 7;
    if (kind == GFO_SKYPLANE) return l == 0 ? 7 : 13 + l;
    if (l <= 1) return 0;
    if (l == 2) return 1;
    if (l == 3) return 2;
    if (kind == GFO_SERSIC) {
        static const int r[8] = {0, 0, 1, 2, 3, 4, 5, 6};
        return r[l];
    }
    if (kind == GFO_SERSIC_F) {
        static const int r[14] = {0, 0, 1, 2, 3, 4, 5, 6, 16, 17, 16, 17, 16, 17};
        return r[l];
    }
    if (kind == GFO_MOFFAT) {
        static const int r[8] = {0, 0, 1, 2, 8, 4, 5, 6};
        return r[l];
    }
    if (kind == GFO_KING) {
        static const int r[9] = {0, 0, 1, 2, 9, 10, 4, 5, 6};
        return r[l];
    }
    if (kind == GFO_NUKER) {
        static const int r[10] = {0, 0, 1, 2, 11, 12, 13, 4, 5, 6};
        return r[l];
    }
    if (kind == GFO_PSF) return -1; /* unreachable: l <= 2 handled above */
    {
        static const int r[7] = {0, 0, 1, 2, 4, 5, 6};
        return r[l];
    }
}

/* ------------------------------------------------------------- b_n, flux */

/* P(a, x) = gamma(a, x) / Gamma(a) by the power series
 * gamma(a, x) = x^a e^{-x} sum_{k>=0} x^k / (a (a+1) ... (a+k)). */
double gfo_gammainc_lower(double a, double x)
{
    if (x <= 0.0) return 0.0;
    double term = 1.0 / a, sum = term;
    for (int k = 1; k < 100000; ++k) {
        term *= x / (a + k);
        sum += term;
        if (term < sum * 1e-17) break;
    }
    return exp(a * log(x) - x - lgamma(a)) * sum;
}

/* b_n solves gamma(2n, b_n) = Gamma(2n)/2, i.e. P(2n, b_n) = 1/2, so that the
 * effective radius r_e encloses half of the total light.  The median of a
 * Gamma(a) variate lies in (0, a), so plain bisection on that bracket. */
double gfo_bn(double n)
{
    double a = 2.0 * n, lo = 0.0, hi = a;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (gfo_gammainc_lower(a, mid) < 0.5)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Total flux of I_e exp(-b_n((r/r_e)^{1/n} - 1)) over the ellipse family
 * (boxiness 0): 2 pi q I_e r_e^2 n e^{b_n} Gamma(2n) / b_n^{2n}. */
double gfo_sersic_flux(double Ie, double re, double n, double q)
{
    double b = gfo_bn(n);
    return 2.0 * M_PI * q * Ie * re * re * n * exp(b + lgamma(2.0 * n) - 2.0 * n * log(b));
}

/* ------------------------------------------------------------------ model */

/* sigma of a Gaussian of full width at half maximum 1: 1 / (2 sqrt(2 ln 2)) */
static double gauss_sigma_per_fwhm(void) { return 1.0 / (2.0 * sqrt(2.0 * log(2.0))); }

/* alpha of a Moffat profile (1 + (r/alpha)^2)^(-beta) of full width at half
 * maximum 1: the half maximum sits where (1 + (r/alpha)^2)^beta = 2, so
 * r = alpha sqrt(2^(1/beta) - 1) = 1/2. */
double gfo_moffat_alpha_per_fwhm(double beta)
{
    return 1.0 / (2.0 * sqrt(pow(2.0, 1.0 / beta) - 1.0));
}

/* d(alpha/FWHM)/d(beta) / (alpha/FWHM) = 2^(1/beta) ln 2 / (2 beta^2 (2^(1/beta) - 1)) */
static double moffat_dlnalpha_dbeta(double beta)
{
    double t = pow(2.0, 1.0 / beta);
    return t * log(2.0) / (2.0 * beta * beta * (t - 1.0));
}

/* Surface brightness of one component at (x, y).
 * Rotation: theta = pa_deg * pi / 180, counter-clockwise from +x to the major
 * axis; x' = dx cos + dy sin, y' = -dx sin + dy cos.
 * Generalised radius: r = (|x'|^C + |y'/q|^C)^{1/C}, C = c + 2.
 * Sersic: I_e exp(-b_n ((r/r_e)^{1/n} - 1)); exponential disk: I_0 exp(-r/r_s);
 * Gaussian: I_0 exp(-r^2 / (2 sigma^2)); Moffat: I_0 (1 + (r/alpha)^2)^(-beta).
 * The Sersic n and the Moffat beta share slot 4. */
/* Cubic convolution kernel of Keys (1981), parameter a = -1/2:
 *   w(x) = 3/2 |x|^3 - 5/2 |x|^2 + 1            for |x| <= 1,
 *   w(x) = -1/2 |x|^3 + 5/2 |x|^2 - 4 |x| + 2    for 1 < |x| < 2,  0 beyond.
 * The weights of the four grid points around any offset sum to 1 and
 * reproduce linear (and quadratic) functions exactly. */
double gfo_keys_weight(double x)
{
    double a = fabs(x);
    if (a <= 1.0) return (1.5 * a - 2.5) * a * a + 1.0;
    if (a < 2.0) return ((-0.5 * a + 2.5) * a - 4.0) * a + 2.0;
    return 0.0;
}

/* Generalised radius of (x, y) about (x0, y0): rotation by pa (degrees,
 * counter-clockwise from +x), axis ratio q, boxiness c (C = c + 2). */
static double gen_radius(double x, double y, double x0, double y0, double q, double pa, double c)
{
    double th = pa * M_PI / 180.0;
    double dx = x - x0, dy = y - y0;
    double xp = dx * cos(th) + dy * sin(th);
    double yp = -dx * sin(th) + dy * cos(th);
    double C = c + 2.0;
    return pow(pow(fabs(xp), C) + pow(fabs(yp / q), C), 1.0 / C);
}

double gfo_comp_value(int kind, const double* p, double x, double y, double bn)
{
    if (kind == GFO_SKY) return p[0];
    if (kind == GFO_SKYPLANE) return NAN; /* depends on the stamp: see gfo_model_ext */
    if (kind == GFO_PSF) {
        /* an unresolved source of flux F at (x0, y0): its value at a grid point
         * is F times the cubic-convolution weights of the offsets, so that the
         * convolved image is the PSF interpolated to the sub-pixel position */
        return p[2] * gfo_keys_weight(x - p[0]) * gfo_keys_weight(y - p[1]);
    }
    if (kind == GFO_KING) {
        /* modified King profile: I_0 [(w - w_t) / (1 - w_t)]^alpha for r < r_t,
         * 0 beyond; w = (1 + (r/r_c)^2)^(-1/alpha), w_t = w(r_t).  I(0) = I_0;
         * alpha = 2 is King's (1962) empirical law. */
        double rc = p[3], rt = p[4], al = p[5];
        double r = gen_radius(x, y, p[0], p[1], p[6], p[7], p[8]);
        if (r >= rt) return 0.0;
        double w = pow(1.0 + (r / rc) * (r / rc), -1.0 / al);
        double wt = pow(1.0 + (rt / rc) * (rt / rc), -1.0 / al);
        return p[2] * pow((w - wt) / (1.0 - wt), al);
    }
    if (kind == GFO_NUKER) {
        /* Nuker law (Lauer et al. 1995): inner slope gamma, outer slope beta,
         * break sharpness alpha, I(r_b) = I_b.  The radius is floored at
         * 1e-6 r_b, where the inner power law (gamma > 0) would diverge. */
        double rb = p[3], al = p[4], be = p[5], ga = p[6];
        double r = gen_radius(x, y, p[0], p[1], p[7], p[8], p[9]);
        double t = fmax(r / rb, 1e-6);
        return p[2] * pow(2.0, (be - ga) / al) * pow(t, -ga) * pow(1.0 + pow(t, al), (ga - be) / al);
    }
    if (kind == GFO_SERSIC_F) {
        /* the Sersic on a radius distorted by Fourier modes m = 1, 3, 4:
         * r_F = r (1 + sum_m a_m cos(m (t - phi_m))), t = atan2(y'/q, x') the
         * angle in the component's circularised frame (t = 0 on the major
         * axis), phi_m in degrees; a_m = 0 gives the plain Sersic */
        double th = p[6] * M_PI / 180.0;
        double dx = x - p[0], dy = y - p[1];
        double xp = dx * cos(th) + dy * sin(th);
        double yp = -dx * sin(th) + dy * cos(th);
        double Y = yp / p[5], C = p[7] + 2.0;
        double r = pow(pow(fabs(xp), C) + pow(fabs(Y), C), 1.0 / C);
        double t = atan2(Y, xp);
        static const int ms[3] = {1, 3, 4};
        double g = 1.0;
        for (int k = 0; k < 3; ++k) g += p[8 + 2 * k] * cos(ms[k] * (t - p[9 + 2 * k] * M_PI / 180.0));
        return p[2] * exp(-bn * (pow(r * g / p[3], 1.0 / p[4]) - 1.0));
    }
    double x0 = p[0], y0 = p[1], amp = p[2], rs = p[3];
    double n = 1.0, q, pa, c;
    if (kind == GFO_SERSIC || kind == GFO_MOFFAT) {
        n = p[4];
        q = p[5];
        pa = p[6];
        c = p[7];
    } else {
        q = p[4];
        pa = p[5];
        c = p[6];
    }
    double th = pa * M_PI / 180.0;
    double dx = x - x0, dy = y - y0;
    double xp = dx * cos(th) + dy * sin(th);
    double yp = -dx * sin(th) + dy * cos(th);
    double C = c + 2.0;
    double r = pow(pow(fabs(xp), C) + pow(fabs(yp / q), C), 1.0 / C);
    if (kind == GFO_SERSIC) return amp * exp(-bn * (pow(r / rs, 1.0 / n) - 1.0));
    if (kind == GFO_GAUSSIAN) {
        double sig = rs * gauss_sigma_per_fwhm();
        return amp * exp(-r * r / (2.0 * sig * sig));
    }
    if (kind == GFO_MOFFAT) {
        double al = rs * gfo_moffat_alpha_per_fwhm(n), t = r / al;
        return amp * pow(1.0 + t * t, -n);
    }
    return amp * exp(-r / rs);
}

/* db_n/dn by central differences of the b_n solver (FP64; the solver is
 * accurate to ~1e-14, so the difference quotient carries ~1e-10 relative). */
double gfo_bn_deriv(double n)
{
    double e = 1e-4 * fmax(n, 1.0);
    return (gfo_bn(n + e) - gfo_bn(n - e)) / (2.0 * e);
}

/* The component's value at (x, y) and its partial derivatives with respect to
 * each of its slots, by the chain rule through the definitions above
 * (analytic Jacobian columns, the "next" step after finite differences).
 *   r^C = |x'|^C + |Y|^C with Y = y'/q:
 *     dr/dx' = sgn(x') (|x'|/r)^(C-1),  dr/dY = sgn(Y) (|Y|/r)^(C-1),
 *     dr/dC  = r [ (|x'|^C ln|x'| + |Y|^C ln|Y|) / (C r^C) - ln(r^C) / C^2 ];
 *   x' = dx cos t + dy sin t, y' = -dx sin t + dy cos t, dx = x - x0, dy = y - y0:
 *     dx'/dx0 = -cos t, dx'/dy0 = -sin t, dy'/dx0 = sin t, dy'/dy0 = -cos t,
 *     dx'/dt = y', dy'/dt = -x', dt/dpa = pi/180, dY/dq = -Y/q;
 *   Sersic, u = (r/r_e)^(1/n), I = I_e exp(-b_n (u - 1)):
 *     dI/dr = -b_n I u / (n r),  dI/dr_e = b_n I u / (n r_e),
 *     dI/dn = I [ (1 - u) db_n/dn + b_n u ln(r/r_e) / n^2 ];
 *   disk, I = I_0 exp(-r/r_s): dI/dr = -I/r_s, dI/dr_s = I r / r_s^2;
 *   Gaussian, I = I_0 exp(-r^2 / (2 s^2)), s = FWHM / (2 sqrt(2 ln 2)):
 *     dI/dr = -I r / s^2, dI/dFWHM = I r^2 / s^3 * ds/dFWHM;
 *   Moffat, I = I_0 w^(-beta), w = 1 + t^2, t = r/alpha, alpha = FWHM a(beta):
 *     dI/dr = -2 beta I t / (alpha w),  dI/dalpha = 2 beta I t^2 / (alpha w),
 *     dI/dFWHM = dI/dalpha * alpha / FWHM,
 *     dI/dbeta = -I ln w + dI/dalpha * alpha * d ln a / d beta;
 *   amplitude: dI/dA = I/A (the profile at unit amplitude); sky: 1.
 * At r = 0 (a sample exactly on the centre) the geometric derivatives are
 * set to 0.  grad has one entry per slot of the component. */
double gfo_comp_grad(int kind, const double* p, double x, double y, double bn, double dbdn,
                     double* grad)
{
    if (kind == GFO_SKY) {
        grad[0] = 1.0;
        return p[0];
    }
    double x0 = p[0], y0 = p[1], amp = p[2], rs = p[3];
    double n = 1.0, q, pa, c;
    int iq, ipa, ic, in = -1;
    if (kind == GFO_SERSIC || kind == GFO_MOFFAT) {
        n = p[4];
        q = p[5];
        pa = p[6];
        c = p[7];
        in = 4;
        iq = 5;
        ipa = 6;
        ic = 7;
    } else {
        q = p[4];
        pa = p[5];
        c = p[6];
        iq = 4;
        ipa = 5;
        ic = 6;
    }
    double th = pa * M_PI / 180.0, cs = cos(th), sn = sin(th);
    double dx = x - x0, dy = y - y0;
    double xp = dx * cs + dy * sn;
    double yp = -dx * sn + dy * cs;
    double Y = yp / q;
    double C = c + 2.0;
    double ax = pow(fabs(xp), C), ay = pow(fabs(Y), C);
    double S = ax + ay;
    double r = pow(S, 1.0 / C);
    double unit, dIdr, dIdrs, dIdn = 0.0;
    if (kind == GFO_SERSIC) {
        double t = r / rs, u = pow(t, 1.0 / n);
        unit = exp(-bn * (u - 1.0));
        double I = amp * unit;
        dIdr = r > 0.0 ? -bn * I * u / (n * r) : 0.0;
        dIdrs = bn * I * u / (n * rs);
        dIdn = r > 0.0 ? I * ((1.0 - u) * dbdn + bn * u * log(t) / (n * n)) : I * dbdn;
    } else if (kind == GFO_GAUSSIAN) {
        /* I = A exp(-r^2 / (2 sigma^2)), sigma = k FWHM:
         * dI/dr = -I r / sigma^2, dI/dFWHM = I r^2 / sigma^3 * k */
        double k = gauss_sigma_per_fwhm(), sig = rs * k;
        unit = exp(-r * r / (2.0 * sig * sig));
        double I = amp * unit;
        dIdr = -I * r / (sig * sig);
        dIdrs = I * r * r / (sig * sig * sig) * k;
    } else if (kind == GFO_MOFFAT) {
        double beta = n, al = rs * gfo_moffat_alpha_per_fwhm(beta);
        double t = r / al, w = 1.0 + t * t;
        unit = pow(w, -beta);
        double I = amp * unit;
        double dIdal = 2.0 * beta * I * t * t / (al * w);
        dIdr = -2.0 * beta * I * t / (al * w);
        dIdrs = dIdal * al / rs;
        dIdn = -I * log(w) + dIdal * al * moffat_dlnalpha_dbeta(beta);
    } else {
        unit = exp(-r / rs);
        double I = amp * unit;
        dIdr = -I / rs;
        dIdrs = I * r / (rs * rs);
    }
    double drdxp = 0.0, drdY = 0.0, drdC = 0.0;
    if (r > 0.0) {
        drdxp = (xp > 0.0 ? 1.0 : (xp < 0.0 ? -1.0 : 0.0)) * pow(fabs(xp) / r, C - 1.0);
        drdY = (Y > 0.0 ? 1.0 : (Y < 0.0 ? -1.0 : 0.0)) * pow(fabs(Y) / r, C - 1.0);
        double lx = ax > 0.0 ? ax * log(fabs(xp)) : 0.0;
        double ly = ay > 0.0 ? ay * log(fabs(Y)) : 0.0;
        drdC = r * ((lx + ly) / (C * S) - log(S) / (C * C));
    }
    grad[0] = dIdr * (drdxp * (-cs) + drdY * (sn / q));
    grad[1] = dIdr * (drdxp * (-sn) + drdY * (-cs / q));
    grad[2] = unit;
    grad[3] = dIdrs;
    if (in >= 0) grad[in] = dIdn;
    grad[iq] = dIdr * drdY * (-Y / q);
    grad[ipa] = dIdr * (drdxp * yp + drdY * (-xp / q)) * (M_PI / 180.0);
    grad[ic] = dIdr * drdC;
    return amp * unit;
}

static void os_block(const gfo_desc* d, int* bx0, int* by0)
{
    *bx0 = d->os_x0 >= 0 ? d->os_x0 : (d->W - d->os_box) / 2;
    *by0 = d->os_y0 >= 0 ? d->os_y0 : (d->H - d->os_box) / 2;
}

/* Pixel value: the profile at the pixel centre, except inside the B x B
 * oversampling block, where it is the mean of s x s samples placed at
 * x = j - 1/2 + (b + 1/2)/s, y = i - 1/2 + (a + 1/2)/s. */
static double comp_pixel_bn(const gfo_desc* d, int kind, const double* p, int i, int j,
                            double bn)
{
    int s = d->os_factor, B = d->os_box;
    /* a point source is not sampled: it stands for an unresolved source whose
     * shape is the PSF's, so it keeps its pixel-centre weights everywhere */
    if (kind != GFO_SKY && kind != GFO_PSF && s > 1 && B > 0) {
        int bx0, by0;
        os_block(d, &bx0, &by0);
        if (i >= by0 && i < by0 + B && j >= bx0 && j < bx0 + B) {
            double acc = 0.0;
            for (int a = 0; a < s; ++a)
                for (int b = 0; b < s; ++b) {
                    double y = i - 0.5 + (a + 0.5) / s;
                    double x = j - 0.5 + (b + 0.5) / s;
                    acc += gfo_comp_value(kind, p, x, y, bn);
                }
            return acc / ((double)s * s);
        }
    }
    return gfo_comp_value(kind, p, (double)j, (double)i, bn);
}

/* d(pixel value)/d(slot `local` of the component): the derivative of the
 * pixel-centre value, or the mean of the sub-sample derivatives inside the
 * oversampling block. */
static double comp_pixel_grad(const gfo_desc* d, int kind, const double* p, int i, int j,
                              double bn, double dbdn, int local)
{
    double gr[8];
    int s = d->os_factor, B = d->os_box;
    if (kind != GFO_SKY && s > 1 && B > 0) {
        int bx0, by0;
        os_block(d, &bx0, &by0);
        if (i >= by0 && i < by0 + B && j >= bx0 && j < bx0 + B) {
            double acc = 0.0;
            for (int a = 0; a < s; ++a)
                for (int b = 0; b < s; ++b) {
                    double y = i - 0.5 + (a + 0.5) / s;
                    double x = j - 0.5 + (b + 0.5) / s;
                    gfo_comp_grad(kind, p, x, y, bn, dbdn, gr);
                    acc += gr[local];
                }
            return acc / ((double)s * s);
        }
    }
    gfo_comp_grad(kind, p, (double)j, (double)i, bn, dbdn, gr);
    return gr[local];
}

/* The derivative of the extended-grid model with respect to slot `slot`. */
int gfo_model_ext_grad(const gfo_desc* d, const double* params, int slot, double* out)
{
    int c = (d->P - 1) / 2;
    int He = d->H + 2 * c, We = d->W + 2 * c;
    int k, l, b;
    slot_owner(d, slot, &k, &l, &b);
    if (k < 0) return -1;
    int kind = d->kinds[k];
    if (kind == GFO_KING || kind == GFO_NUKER || kind == GFO_PSF || kind == GFO_SERSIC_F) {
        /* no analytic gradient for these kinds: the column is undefined */
        for (size_t t = 0; t < (size_t)He * We; ++t) out[t] = NAN;
        return -1;
    }
    const double* p = params + b;
    double bn = (kind == GFO_SERSIC || kind == GFO_SERSIC_F) ? gfo_bn(p[4]) : 0.0;
    double dbdn = kind == GFO_SERSIC ? gfo_bn_deriv(p[4]) : 0.0;
    for (int ie = 0; ie < He; ++ie)
        for (int je = 0; je < We; ++je)
            out[(size_t)ie * We + je] = comp_pixel_grad(d, kind, p, ie - c, je - c, bn, dbdn, l);
    return 0;
}

double gfo_comp_pixel(const gfo_desc* d, int kind, const double* p, int i, int j)
{
    double bn = (kind == GFO_SERSIC || kind == GFO_SERSIC_F) ? gfo_bn(p[4]) : 0.0;
    return comp_pixel_bn(d, kind, p, i, j, bn);
}

/* Step 1 (transform): sum of the components on the extended grid. */
/* Single-precision emulation (an experiment, off by default): when on, every
 * component's pixel value and every convolved model pixel is rounded to
 * float32, the storage precision of the GPU path, while all arithmetic stays
 * FP64.  It shows which differences between the GPU's fits and the FP64
 * oracle's come from float32 storage of the model (for example the noise that
 * a forward difference's 1/h amplifies) rather than from the GPU's code. */
static int g_f32_emulation = 0;

void gfo_set_f32_emulation(int on) { g_f32_emulation = on != 0; }

static double f32_store(double v) { return g_f32_emulation ? (double)(float)v : v; }

int gfo_model_ext(const gfo_desc* d, const double* params, int comp, int unit_amp,
                  double* out)
{
    int c = (d->P - 1) / 2;
    int He = d->H + 2 * c, We = d->W + 2 * c;
    memset(out, 0, sizeof(double) * (size_t)He * We);
    int off = 0;
    for (int k = 0; k < d->ncomp; ++k) {
        int kind = d->kinds[k], ns = gfo_comp_nslots(kind);
        if (ns < 0) return -1;
        if (comp < 0 || comp == k) {
            double p[GFO_COMP_MAXSLOTS];
            memcpy(p, params + off, sizeof(double) * ns);
            if (kind == GFO_SKYPLANE) {
                /* the sky plane at the pixel centres (a linear function: its
                 * sub-sample mean is the centre value) about the stamp centre */
                double xc = 0.5 * (d->W - 1), yc = 0.5 * (d->H - 1);
                if (unit_amp) p[0] = 1.0, p[1] = p[2] = 0.0;
                for (int ie = 0; ie < He; ++ie)
                    for (int je = 0; je < We; ++je)
                        out[(size_t)ie * We + je] +=
                            f32_store(p[0] + p[1] * ((je - c) - xc) + p[2] * ((ie - c) - yc));
                off += ns;
                continue;
            }
            if (unit_amp) p[kind == GFO_SKY ? 0 : 2] = 1.0;
            double bn = (kind == GFO_SERSIC || kind == GFO_SERSIC_F) ? gfo_bn(p[4]) : 0.0;
            for (int ie = 0; ie < He; ++ie)
                for (int je = 0; je < We; ++je)
                    out[(size_t)ie * We + je] += f32_store(comp_pixel_bn(d, kind, p, ie - c, je - c, bn));
        }
        off += ns;
    }
    return 0;
}

/* The extended-grid basis function of a linear slot: the model of the slot's
 * component with that slot set to 1 and the component's other linear slots
 * to 0 (a profile at unit amplitude, the constant sky, or one of the sky
 * plane's three terms). */
int gfo_model_ext_basis(const gfo_desc* d, const double* params, int slot, double* out)
{
    int k, l, b;
    slot_owner(d, slot, &k, &l, &b);
    if (k < 0 || !gfo_slot_is_linear(d, slot)) return -1;
    if (d->kinds[k] != GFO_SKYPLANE) return gfo_model_ext(d, params, k, 1, out);
    double q[GFO_MAX_SLOTS];
    memcpy(q, params, sizeof(double) * gfo_nslots(d));
    q[b] = q[b + 1] = q[b + 2] = 0.0;
    q[slot] = 1.0;
    return gfo_model_ext(d, q, k, 0, out);
}

/* ------------------------------------------------------------ convolution */

/* Step 2 by its definition: out(i,j) = sum_{v,u} psf[v][u] E[i+2c-v][j+2c-u]. */
void gfo_convolve_direct(int H, int W, int P, const double* ext, const double* psf,
                         double* out)
{
    int c = (P - 1) / 2, We = W + 2 * c;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int v = 0; v < P; ++v)
                for (int u = 0; u < P; ++u)
                    acc += psf[v * P + u] * ext[(size_t)(i + 2 * c - v) * We + (j + 2 * c - u)];
            out[(size_t)i * W + j] = acc;
        }
}

int gfo_fft_size(int n)
{
    for (int m = n > 1 ? n : 1;; ++m) {
        int r = m;
        while (r % 2 == 0) r /= 2;
        while (r % 3 == 0) r /= 3;
        while (r % 5 == 0) r /= 5;
        if (r == 1) return m;
    }
}

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Decimation-in-time mixed-radix DFT.
 * X[k] = sum_j x[j] w^{jk}, w = exp(sign 2 pi i / n).  With n = p m and the
 * p decimated sequences x[jp + r], Y_r = DFT_m(x[. p + r]) and
 * X[k + q m] = sum_r w_n^{r (k + q m)} Y_r[k].
 * tw holds exp(2 pi i t / N) for the top-level N; w_n^t = tw[t * N / n]. */
static void fft_rec(int n, const double* ire, const double* iim, int stride, double* ore,
                    double* oim, int sign, const double* twr, const double* twi, int N)
{
    if (n == 1) {
        ore[0] = ire[0];
        oim[0] = iim[0];
        return;
    }
    int p = smallest_factor(n), m = n / p;
    for (int r = 0; r < p; ++r)
        fft_rec(m, ire + (size_t)r * stride, iim + (size_t)r * stride, stride * p, ore + r * m,
                oim + r * m, sign, twr, twi, N);
    double* tr = (double*)malloc(sizeof(double) * p);
    double* ti = (double*)malloc(sizeof(double) * p);
    int tstep = N / n;
    for (int k = 0; k < m; ++k) {
        for (int q = 0; q < p; ++q) {
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < p; ++r) {
                long long e = ((long long)r * (k + q * m)) % n;
                double wr = twr[e * tstep], wi = sign * twi[e * tstep];
                double yr = ore[r * m + k], yi = oim[r * m + k];
                sr += yr * wr - yi * wi;
                si += yr * wi + yi * wr;
            }
            tr[q] = sr;
            ti[q] = si;
        }
        for (int q = 0; q < p; ++q) {
            ore[q * m + k] = tr[q];
            oim[q * m + k] = ti[q];
        }
    }
    free(tr);
    free(ti);
}

void gfo_fft(int n, double* re, double* im, int sign)
{
    double* twr = (double*)malloc(sizeof(double) * n);
    double* twi = (double*)malloc(sizeof(double) * n);
    double* cr = (double*)malloc(sizeof(double) * n);
    double* ci = (double*)malloc(sizeof(double) * n);
    for (int t = 0; t < n; ++t) {
        twr[t] = cos(2.0 * M_PI * t / n);
        twi[t] = sin(2.0 * M_PI * t / n);
    }
    memcpy(cr, re, sizeof(double) * n);
    memcpy(ci, im, sizeof(double) * n);
    fft_rec(n, cr, ci, 1, re, im, sign, twr, twi, n);
    free(twr);
    free(twi);
    free(cr);
    free(ci);
}

/* 2-D DFT: 1-D transforms along every row, then along every column. */
static void fft2(int ny, int nx, double* re, double* im, int sign)
{
    for (int y = 0; y < ny; ++y) gfo_fft(nx, re + (size_t)y * nx, im + (size_t)y * nx, sign);
    double* cr = (double*)malloc(sizeof(double) * ny);
    double* ci = (double*)malloc(sizeof(double) * ny);
    for (int x = 0; x < nx; ++x) {
        for (int y = 0; y < ny; ++y) {
            cr[y] = re[(size_t)y * nx + x];
            ci[y] = im[(size_t)y * nx + x];
        }
        gfo_fft(ny, cr, ci, sign);
        for (int y = 0; y < ny; ++y) {
            re[(size_t)y * nx + x] = cr[y];
            im[(size_t)y * nx + x] = ci[y];
        }
    }
    free(cr);
    free(ci);
}

/* Step 2 in Fourier space (Sec. 3, item 2): the circular convolution at a
 * padded size Ny x Nx >= the extended grid, with the PSF wrapped so that its
 * centre sits at (0, 0), equals the direct sum on the valid region. */
void gfo_convolve_fft(int H, int W, int P, const double* ext, const double* psf,
                      double* out)
{
    int c = (P - 1) / 2, He = H + 2 * c, We = W + 2 * c;
    int ny = gfo_fft_size(He), nx = gfo_fft_size(We);
    size_t n = (size_t)ny * nx;
    double* ar = (double*)calloc(n, sizeof(double));
    double* ai = (double*)calloc(n, sizeof(double));
    double* br = (double*)calloc(n, sizeof(double));
    double* bi = (double*)calloc(n, sizeof(double));
    for (int y = 0; y < He; ++y)
        for (int x = 0; x < We; ++x) ar[(size_t)y * nx + x] = ext[(size_t)y * We + x];
    for (int v = 0; v < P; ++v)
        for (int u = 0; u < P; ++u) {
            int y = ((v - c) % ny + ny) % ny, x = ((u - c) % nx + nx) % nx;
            br[(size_t)y * nx + x] += psf[v * P + u];
        }
    fft2(ny, nx, ar, ai, -1);
    fft2(ny, nx, br, bi, -1);
    for (size_t t = 0; t < n; ++t) {
        double r = ar[t] * br[t] - ai[t] * bi[t];
        double i = ar[t] * bi[t] + ai[t] * br[t];
        ar[t] = r;
        ai[t] = i;
    }
    fft2(ny, nx, ar, ai, +1);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j)
            out[(size_t)i * W + j] = ar[(size_t)(i + c) * nx + (j + c)] / (double)n;
    free(ar);
    free(ai);
    free(br);
    free(bi);
}

/* ------------------------------------------------------------------- chi2 */

typedef struct {
    double s, c;
} nsum;

/* Neumaier's compensated summation */
static void nsum_add(nsum* a, double t)
{
    double s = a->s + t;
    if (fabs(a->s) >= fabs(t))
        a->c += (a->s - s) + t;
    else
        a->c += (t - s) + a->s;
    a->s = s;
}

static int pixel_valid(double d, double s) { return isfinite(d) && isfinite(s) && s > 0.0; }

/* Step 3 (transform + reduce): sum of ((d - m)/sigma)^2 over valid pixels. */
double gfo_chi2(int npix, const double* d, const double* sigma, const double* m)
{
    nsum a = {0.0, 0.0};
    for (int t = 0; t < npix; ++t) {
        if (!pixel_valid(d[t], sigma[t])) continue;
        double z = (d[t] - m[t]) / sigma[t];
        nsum_add(&a, z * z);
    }
    return a.s + a.c;
}

static void convolve(int method, int H, int W, int P, const double* ext, const double* psf,
                     double* out)
{
    if (method == 1)
        gfo_convolve_fft(H, W, P, ext, psf, out);
    else
        gfo_convolve_direct(H, W, P, ext, psf, out);
    if (g_f32_emulation)
        for (size_t t = 0; t < (size_t)H * W; ++t) out[t] = (double)(float)out[t];
}

/* Steps 1-3 for one parameter vector. */
double gfo_eval(const gfo_desc* d, const double* params, const double* psf,
                const double* img, const double* sigma, int method, double* model_out)
{
    int c = (d->P - 1) / 2;
    size_t ne = (size_t)(d->H + 2 * c) * (d->W + 2 * c), np = (size_t)d->H * d->W;
    double* ext = (double*)malloc(sizeof(double) * ne);
    double* m = model_out ? model_out : (double*)malloc(sizeof(double) * np);
    gfo_model_ext(d, params, -1, 0, ext);
    convolve(method, d->H, d->W, d->P, ext, psf, m);
    double x2 = (img && sigma) ? gfo_chi2((int)np, img, sigma, m) : 0.0;
    free(ext);
    if (!model_out) free(m);
    return x2;
}

/* ---------------------------------------------------------------- Jacobian */

/* FD step: positions use fd_rel pixels (they are origin-relative); the other
 * nonlinear slots use fd_rel * max(|v|, 1). */
double gfo_fd_step(const gfo_desc* d, int slot, double v, double fd_rel)
{
    int role = slot_role(d, slot);
    if (role == 0) return fd_rel;
    return fd_rel * fmax(fabs(v), 1.0);
}

/* Jacobian of the convolved model with respect to the free slots:
 * linear slots (amplitudes, sky) by the exact column, the convolution of the
 * component with unit amplitude; nonlinear slots by forward (mode 0) or
 * central (mode 1) differences of the full convolved model, or (mode 2) by the
 * convolution of the analytic derivative of the extended-grid model.  A = J^T W J, g = J^T W r with
 * W = diag(1/sigma^2) on valid pixels and r = d - m. */
double gfo_jacobian(const gfo_desc* d, const double* params, const uint8_t* fixed,
                    const double* psf, const double* img, const double* sigma,
                    int method, double fd_rel, int mode, double* J, double* A,
                    double* g, double* model_out)
{
    int c = (d->P - 1) / 2, ns = gfo_nslots(d);
    size_t ne = (size_t)(d->H + 2 * c) * (d->W + 2 * c), np = (size_t)d->H * d->W;
    double* ext = (double*)malloc(sizeof(double) * ne);
    double* m0 = (double*)malloc(sizeof(double) * np);
    double* mp = (double*)malloc(sizeof(double) * np);
    double* mm = (double*)malloc(sizeof(double) * np);
    int nfree = 0;
    int freeslot[GFO_MAX_SLOTS];
    for (int s = 0; s < ns; ++s)
        if (!fixed || !fixed[s]) freeslot[nfree++] = s;
    double* Jl = (double*)malloc(sizeof(double) * np * (nfree > 0 ? nfree : 1));
    double pp[GFO_MAX_SLOTS];

    gfo_model_ext(d, params, -1, 0, ext);
    convolve(method, d->H, d->W, d->P, ext, psf, m0);
    for (int f = 0; f < nfree; ++f) {
        int s = freeslot[f], k, l, b;
        slot_owner(d, s, &k, &l, &b);
        double* col = Jl + (size_t)f * np;
        if (gfo_slot_is_linear(d, s)) {
            gfo_model_ext_basis(d, params, s, ext);
            convolve(method, d->H, d->W, d->P, ext, psf, col);
            continue;
        }
        if (mode == GFO_JAC_ANALYTIC) {
            gfo_model_ext_grad(d, params, s, ext);
            convolve(method, d->H, d->W, d->P, ext, psf, col);
            continue;
        }
        double h = gfo_fd_step(d, s, params[s], fd_rel);
        memcpy(pp, params, sizeof(double) * ns);
        pp[s] = params[s] + h;
        gfo_model_ext(d, pp, -1, 0, ext);
        convolve(method, d->H, d->W, d->P, ext, psf, mp);
        if (mode == GFO_JAC_CENTRAL) {
            pp[s] = params[s] - h;
            gfo_model_ext(d, pp, -1, 0, ext);
            convolve(method, d->H, d->W, d->P, ext, psf, mm);
            for (size_t t = 0; t < np; ++t) col[t] = (mp[t] - mm[t]) / (2.0 * h);
        } else {
            for (size_t t = 0; t < np; ++t) col[t] = (mp[t] - m0[t]) / h;
        }
    }
    double x2 = 0.0;
    if (img && sigma) {
        x2 = gfo_chi2((int)np, img, sigma, m0);
        for (int a = 0; a < nfree; ++a) {
            nsum ga = {0.0, 0.0};
            for (size_t t = 0; t < np; ++t) {
                if (!pixel_valid(img[t], sigma[t])) continue;
                double w = 1.0 / (sigma[t] * sigma[t]);
                nsum_add(&ga, w * Jl[(size_t)a * np + t] * (img[t] - m0[t]));
            }
            if (g) g[a] = ga.s + ga.c;
            for (int bb = 0; bb < nfree; ++bb) {
                nsum aa = {0.0, 0.0};
                for (size_t t = 0; t < np; ++t) {
                    if (!pixel_valid(img[t], sigma[t])) continue;
                    double w = 1.0 / (sigma[t] * sigma[t]);
                    nsum_add(&aa, w * Jl[(size_t)a * np + t] * Jl[(size_t)bb * np + t]);
                }
                if (A) A[a * nfree + bb] = aa.s + aa.c;
            }
        }
    }
    if (J) memcpy(J, Jl, sizeof(double) * np * nfree);
    if (model_out) memcpy(model_out, m0, sizeof(double) * np);
    free(ext);
    free(m0);
    free(mp);
    free(mm);
    free(Jl);
    return x2;
}

/* ------------------------------------------------------------------- LM */

void gfo_default_opts(gfo_lm_opts* o)
{
    o->lambda0 = 1e-3;
    o->lambda_up = 10.0;
    o->lambda_down = 0.1;
    o->lambda_min = 1e-12;
    o->lambda_max = 1e12;
    o->ftol = 1e-8;
    o->xtol = 1e-8;
    o->fd_rel = 1e-3;
    o->max_iter = 200;
    o->jac_mode = GFO_JAC_FORWARD;
}

/* Default box: I >= 0, radii >= 0.1, n in [0.2, 10], q in [0.05, 1],
 * boxiness in [-1.9, 2], Moffat beta in [0.5, 20], King r_t >= 0.1 and alpha
 * in [0.1, 10], Nuker alpha in [0.1, 10], beta in [0, 10], gamma in [0, 2],
 * Fourier amplitudes in [-0.3, 0.3]; positions, sky and phases free;
 * position angles are wrapped into [0, 180) instead of clamped. */
void gfo_default_bounds(const gfo_desc* d, double* lo, double* hi)
{
    int ns = gfo_nslots(d);
    for (int s = 0; s < ns; ++s) {
        lo[s] = -INFINITY;
        hi[s] = INFINITY;
        switch (slot_role(d, s)) {
        case 1: lo[s] = 0.0; break;
        case 2: lo[s] = 0.1; break;
        case 3: lo[s] = 0.2; hi[s] = 10.0; break;
        case 4: lo[s] = 0.05; hi[s] = 1.0; break;
        case 6: lo[s] = -1.9; hi[s] = 2.0; break;
        case 8: lo[s] = 0.5; hi[s] = 20.0; break;
        case 9: lo[s] = 0.1; break;
        case 10: lo[s] = 0.1; hi[s] = 10.0; break;
        case 11: lo[s] = 0.1; hi[s] = 10.0; break;
        case 12: lo[s] = 0.0; hi[s] = 10.0; break;
        case 13: lo[s] = 0.0; hi[s] = 2.0; break;
        case 16: lo[s] = -0.3; hi[s] = 0.3; break;
        default: break;
        }
    }
}

static void project(const gfo_desc* d, double* p, const double* lo, const double* hi)
{
    int ns = gfo_nslots(d);
    for (int s = 0; s < ns; ++s) {
        if (slot_role(d, s) == 5) {
            double a = fmod(p[s], 180.0);
            if (a < 0.0) a += 180.0;
            if (a >= 180.0) a -= 180.0;
            p[s] = a;
            continue;
        }
        if (p[s] < lo[s]) p[s] = lo[s];
        if (p[s] > hi[s]) p[s] = hi[s];
    }
}

/* scale of slot s in the step-size test |delta| / max(|p|, scale) */
static double xtol_scale(const gfo_desc* d, int s)
{
    int role = slot_role(d, s);
    if (role == 1) return 1e-30;
    if (role == 7) return 1e-3;
    if (role == 14 || role == 15) return 1e-5; /* sky slopes, per pixel */
    return 1.0;
}

/* Cholesky solve of the SPD system M x = b (n <= 16); returns 0 on failure. */
static int cholesky_solve(int n, const double* M, const double* b, double* x)
{
    double L[GFO_MAX_FREE * GFO_MAX_FREE];
    memset(L, 0, sizeof(L));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = M[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0) || !isfinite(s)) return 0;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    double y[GFO_MAX_FREE];
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i)
        if (!isfinite(x[i])) return 0;
    return 1;
}

/* Levenberg-Marquardt (Marquardt's diagonal damping), steps 4 and 5 of the
 * loop, over any problem that supplies its normal equations, its chi^2, a
 * projection into its box and the scales of its step test.
 * One trial = solve (A + lambda diag A) delta = g, project p + delta into the
 * box, evaluate chi^2 there; accept if chi^2 falls (lambda shrinks, a new
 * Jacobian is taken), otherwise reject (lambda grows).  Finishing criteria:
 * the scaled step falls below xtol, or an accepted step lowers chi^2 by less
 * than ftol relative while the linearised model also predicts a relative fall
 * below ftol (converged; the predicted fall of the damped step is
 * delta^T (g + lambda diag(A) delta)); lambda exceeds lambda_max (no
 * convergence); max_iter trials (iteration cap). */
int gfo_lm_core(const gfo_lm_problem* P, double* params, const gfo_lm_opts* o, gfo_lm_result* res)
{
    int ns = P->nslots, nfree = P->nfree;
    const int* fs = P->free_slots;
    gfo_lm_result r = {0.0, o->lambda0, 0, 0, GFO_MAXITER};
    if (nfree == 0 || nfree > GFO_MAX_FREE) {
        r.status = GFO_BADINPUT;
        if (res) *res = r;
        return r.status;
    }
    double p[GFO_MAX_SLOTS], pt[GFO_MAX_SLOTS];
    memcpy(p, params, sizeof(double) * ns);
    P->project(P->ctx, p);
    double A[GFO_MAX_FREE * GFO_MAX_FREE], g[GFO_MAX_FREE], M[GFO_MAX_FREE * GFO_MAX_FREE];
    double rhs[GFO_MAX_FREE], delta[GFO_MAX_FREE];
    double lambda = o->lambda0;
    double chi2 = P->normal(P->ctx, p, A, g);
    while (r.iters < o->max_iter) {
        for (int i = 0; i < nfree; ++i) {
            rhs[i] = g[i];
            for (int j = 0; j < nfree; ++j) M[i * nfree + j] = A[i * nfree + j];
        }
        for (int i = 0; i < nfree; ++i) {
            if (A[i * nfree + i] > 0.0) {
                M[i * nfree + i] = A[i * nfree + i] * (1.0 + lambda);
            } else {
                /* a slot with no influence on the model is held this step */
                for (int j = 0; j < nfree; ++j) M[i * nfree + j] = M[j * nfree + i] = 0.0;
                M[i * nfree + i] = 1.0;
                rhs[i] = 0.0;
            }
        }
        r.iters++;
        int ok = cholesky_solve(nfree, M, rhs, delta);
        if (ok) {
            double step = 0.0;
            for (int i = 0; i < nfree; ++i) {
                double den = fmax(fabs(p[fs[i]]), P->xscale(P->ctx, fs[i]));
                step = fmax(step, fabs(delta[i]) / den);
            }
            if (step < o->xtol) {
                r.status = GFO_CONVERGED;
                break;
            }
            double pred = 0.0;
            for (int i = 0; i < nfree; ++i) {
                double d = A[i * nfree + i] > 0.0 ? A[i * nfree + i] : 0.0;
                pred += delta[i] * (rhs[i] + lambda * d * delta[i]);
            }
            memcpy(pt, p, sizeof(double) * ns);
            for (int i = 0; i < nfree; ++i) pt[fs[i]] += delta[i];
            P->project(P->ctx, pt);
            double chi2t = P->eval(P->ctx, pt);
            if (isfinite(chi2t) && chi2t < chi2) {
                double rel = (chi2 - chi2t) / chi2;
                memcpy(p, pt, sizeof(double) * ns);
                r.accepted++;
                lambda = fmax(lambda * o->lambda_down, o->lambda_min);
                if (rel < o->ftol && pred / chi2 < o->ftol) {
                    chi2 = chi2t;
                    r.status = GFO_CONVERGED;
                    break;
                }
                chi2 = P->normal(P->ctx, p, A, g);
                continue;
            }
        }
        lambda *= o->lambda_up;
        if (lambda > o->lambda_max) {
            r.status = GFO_NOCONV;
            break;
        }
    }
    r.chi2 = chi2;
    r.lambda = lambda;
    memcpy(params, p, sizeof(double) * ns);
    if (res) *res = r;
    return r.status;
}

/* the stamp problem of gfo_lm_fit for gfo_lm_core */
typedef struct {
    const gfo_desc* d;
    const uint8_t* fixed;
    const double *lo, *hi, *psf, *img, *sigma;
    int method;
    const gfo_lm_opts* o;
} stamp_problem;

static double stamp_normal(void* ctx, const double* p, double* A, double* g)
{
    const stamp_problem* q = (const stamp_problem*)ctx;
    return gfo_jacobian(q->d, p, q->fixed, q->psf, q->img, q->sigma, q->method, q->o->fd_rel,
                        q->o->jac_mode, NULL, A, g, NULL);
}

static double stamp_eval(void* ctx, const double* p)
{
    const stamp_problem* q = (const stamp_problem*)ctx;
    return gfo_eval(q->d, p, q->psf, q->img, q->sigma, q->method, NULL);
}

static void stamp_project(void* ctx, double* p)
{
    const stamp_problem* q = (const stamp_problem*)ctx;
    project(q->d, p, q->lo, q->hi);
}

static double stamp_xscale(void* ctx, int s)
{
    return xtol_scale(((const stamp_problem*)ctx)->d, s);
}

int gfo_lm_fit(const gfo_desc* d, double* params, const uint8_t* fixed,
               const double* lo_in, const double* hi_in, const double* psf,
               const double* img, const double* sigma, int method,
               const gfo_lm_opts* opts_in, gfo_lm_result* res)
{
    gfo_lm_opts o;
    if (opts_in)
        o = *opts_in;
    else
        gfo_default_opts(&o);
    int ns = gfo_nslots(d);
    double lo[GFO_MAX_SLOTS], hi[GFO_MAX_SLOTS];
    gfo_default_bounds(d, lo, hi);
    if (lo_in) memcpy(lo, lo_in, sizeof(double) * ns);
    if (hi_in) memcpy(hi, hi_in, sizeof(double) * ns);
    int fs[GFO_MAX_SLOTS], nfree = 0;
    for (int s = 0; s < ns; ++s)
        if (!fixed || !fixed[s]) fs[nfree++] = s;
    stamp_problem q = {d, fixed, lo, hi, psf, img, sigma, method, &o};
    gfo_lm_problem P = {ns, nfree, fs, stamp_normal, stamp_eval, stamp_project, stamp_xscale, &q};
    return gfo_lm_core(&P, params, &o, res);
}

int gfo_lm_fit_batch(int nb, const gfo_desc* ds, double* params, const uint8_t* fixed,
                     const double* psf, const int64_t* psf_off, const double* img,
                     const double* sigma, const int64_t* pix_off, int method,
                     const gfo_lm_opts* opts, gfo_lm_result* res)
{
    int ns = gfo_nslots(&ds[0]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nb; ++b)
        gfo_lm_fit(&ds[b], params + (size_t)b * ns, fixed ? fixed + (size_t)b * ns : NULL, NULL,
                   NULL, psf + psf_off[b], img + pix_off[b], sigma + pix_off[b], method, opts,
                   &res[b]);
    return 0;
}

int gfo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops across stamps from here on (n >= 1). */
void gfo_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
