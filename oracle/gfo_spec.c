/*
 * gfo_spec.c -- FP64 CPU oracle for spectral-line fitting: the fitting loop of
 * Sec. 2 (model, convolution, comparison, adjustment, finish) in one
 * dimension, the "flexible dimensionality" extension of Sec. 5 (spectral line
 * or cube fitting; a cube is fitted spectrum by spectrum).
 *
 * TEST INFRASTRUCTURE ONLY, like gfo.c: the plain statement of what the GPU
 * spectral path computes, loaded only by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.  It shares nothing with the CUDA library.
 *
 * A spectrum has N channels; channel i has its centre at x = i.  Its model is
 * evaluated on the extended grid x = -c .. N-1+c (N + L - 1 points) of an odd
 * line-spread function (LSF) of L taps, c = (L-1)/2, and convolved on the
 * channels by the flipped-kernel sum
 *     m_i = sum_u lsf[u] E(i + c - u),
 * the one-dimensional form of the stamp convention.  The model is a continuum
 * polynomial plus Gaussian lines:
 *     E(x) = sum_{j < n_cont} a_j t^j + sum_k A_k exp(-(x - mu_k)^2 / (2 s_k^2)),
 *     t = (x - (N-1)/2) / h,  h = (N-1)/2 (1 when N = 1),
 * with the parameter vector [a_0 .. a_{n_cont-1}, A_0, mu_0, s_0, A_1, ...].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "gfo.h"

int gfo_spec_nparams(const gfo_spec_desc* d) { return d->n_cont + 3 * d->n_lines; }

/* 0 = continuum coefficient, 1 = line amplitude, 2 = line centre, 3 = line width */
static int spec_role(const gfo_spec_desc* d, int s)
{
    if (s < d->n_cont) return 0;
    return 1 + (s - d->n_cont) % 3;
}

int gfo_spec_slot_is_linear(const gfo_spec_desc* d, int s)
{
    int r = spec_role(d, s);
    return r == 0 || r == 1;
}

static double spec_t(const gfo_spec_desc* d, double x)
{
    double h = d->n_chan > 1 ? 0.5 * (d->n_chan - 1) : 1.0;
    return (x - 0.5 * (d->n_chan - 1)) / h;
}

/* E at x */
double gfo_spec_value(const gfo_spec_desc* d, const double* p, double x)
{
    double t = spec_t(d, x), v = 0.0, tj = 1.0;
    for (int j = 0; j < d->n_cont; ++j) {
        v += p[j] * tj;
        tj *= t;
    }
    for (int k = 0; k < d->n_lines; ++k) {
        const double* q = p + d->n_cont + 3 * k;
        double z = (x - q[1]) / q[2];
        v += q[0] * exp(-0.5 * z * z);
    }
    return v;
}

/* dE/dp_s at x, by differentiating the definition:
 *   d/da_j = t^j;  with z = (x - mu)/s and G = exp(-z^2/2):
 *   d/dA = G,  d/dmu = A G z / s,  d/ds = A G z^2 / s. */
double gfo_spec_grad(const gfo_spec_desc* d, const double* p, int s, double x)
{
    if (s < d->n_cont) return pow(spec_t(d, x), (double)s);
    int k = (s - d->n_cont) / 3, r = (s - d->n_cont) % 3;
    const double* q = p + d->n_cont + 3 * k;
    double z = (x - q[1]) / q[2], G = exp(-0.5 * z * z);
    if (r == 0) return G;
    if (r == 1) return q[0] * G * z / q[2];
    return q[0] * G * z * z / q[2];
}

/* the extended model (N + L - 1 values), or the derivative column of slot s */
void gfo_spec_model_ext(const gfo_spec_desc* d, const double* p, int slot, double* E)
{
    int c = (d->lsf_len - 1) / 2, ne = d->n_chan + d->lsf_len - 1;
    for (int e = 0; e < ne; ++e) {
        double x = (double)(e - c);
        E[e] = slot < 0 ? gfo_spec_value(d, p, x) : gfo_spec_grad(d, p, slot, x);
    }
}

/* m_i = sum_u lsf[u] E[i + 2c - u] (E indexed from x = -c) */
void gfo_spec_convolve(const gfo_spec_desc* d, const double* E, const double* lsf, double* m)
{
    int L = d->lsf_len, c = (L - 1) / 2;
    for (int i = 0; i < d->n_chan; ++i) {
        double acc = 0.0;
        for (int u = 0; u < L; ++u) acc += lsf[u] * E[i + 2 * c - u];
        m[i] = acc;
    }
}

/* convolved model, chi^2 against (spec, sig) (gfo_chi2's validity rule) */
double gfo_spec_eval(const gfo_spec_desc* d, const double* p, const double* lsf,
                     const double* spec, const double* sig, double* m_out)
{
    int N = d->n_chan, ne = N + d->lsf_len - 1;
    double* E = (double*)malloc(sizeof(double) * ne);
    double* m = m_out ? m_out : (double*)malloc(sizeof(double) * N);
    gfo_spec_model_ext(d, p, -1, E);
    gfo_spec_convolve(d, E, lsf, m);
    double x2 = spec ? gfo_chi2(N, spec, sig, m) : 0.0;
    free(E);
    if (!m_out) free(m);
    return x2;
}

/* FD step of slot s: centres take fd_rel channels (like positions), widths
 * fd_rel max(|s|, 1); linear slots have exact columns and no step. */
double gfo_spec_fd_step(const gfo_spec_desc* d, int s, double v, double fd_rel)
{
    return spec_role(d, s) == 2 ? fd_rel : fd_rel * fmax(fabs(v), 1.0);
}

/* Jacobian columns of the free slots (nfree x N, optional), the normal
 * equations A = J^T W J, g = J^T W r (r = spec - m) and chi^2.  Linear slots
 * take the convolved basis function; the centres and widths take forward
 * differences (mode GFO_JAC_FORWARD), central differences (GFO_JAC_CENTRAL) or
 * the convolved derivative (GFO_JAC_ANALYTIC). */
double gfo_spec_jacobian(const gfo_spec_desc* d, const double* p, const uint8_t* fixed,
                         const double* lsf, const double* spec, const double* sig, int mode,
                         double fd_rel, double* J, double* A, double* g)
{
    int N = d->n_chan, ne = N + d->lsf_len - 1, np = gfo_spec_nparams(d);
    int fs[GFO_MAX_SLOTS], nf = 0;
    for (int s = 0; s < np; ++s)
        if (!fixed || !fixed[s]) fs[nf++] = s;
    double* E = (double*)malloc(sizeof(double) * ne);
    double* m = (double*)malloc(sizeof(double) * N);
    double* Jc = (double*)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1) * N);
    double* m2 = (double*)malloc(sizeof(double) * N);
    double pp[GFO_MAX_SLOTS];
    double x2 = gfo_spec_eval(d, p, lsf, spec, sig, m);
    for (int f = 0; f < nf; ++f) {
        int s = fs[f];
        double* col = Jc + (size_t)f * N;
        if (gfo_spec_slot_is_linear(d, s) || mode == GFO_JAC_ANALYTIC) {
            gfo_spec_model_ext(d, p, s, E);
            gfo_spec_convolve(d, E, lsf, col);
            continue;
        }
        double h = gfo_spec_fd_step(d, s, p[s], fd_rel);
        memcpy(pp, p, sizeof(double) * np);
        pp[s] += h;
        gfo_spec_eval(d, pp, lsf, NULL, NULL, col);
        if (mode == GFO_JAC_CENTRAL) {
            pp[s] = p[s] - h;
            gfo_spec_eval(d, pp, lsf, NULL, NULL, m2);
            for (int i = 0; i < N; ++i) col[i] = (col[i] - m2[i]) / (2.0 * h);
        } else {
            for (int i = 0; i < N; ++i) col[i] = (col[i] - m[i]) / h;
        }
    }
    for (int a = 0; a < nf; ++a) {
        double ga = 0.0;
        for (int i = 0; i < N; ++i) {
            double w = (isfinite(spec[i]) && isfinite(sig[i]) && sig[i] > 0.0)
                           ? 1.0 / ((double)sig[i] * sig[i]) : 0.0;
            if (w > 0.0) ga += w * Jc[(size_t)a * N + i] * (spec[i] - m[i]);
        }
        if (g) g[a] = ga;
        for (int b = 0; b < nf; ++b) {
            double s = 0.0;
            for (int i = 0; i < N; ++i) {
                double w = (isfinite(spec[i]) && isfinite(sig[i]) && sig[i] > 0.0)
                               ? 1.0 / ((double)sig[i] * sig[i]) : 0.0;
                if (w > 0.0) s += w * Jc[(size_t)a * N + i] * Jc[(size_t)b * N + i];
            }
            if (A) A[a * nf + b] = s;
        }
    }
    if (J) memcpy(J, Jc, sizeof(double) * (size_t)nf * N);
    free(E);
    free(m);
    free(m2);
    free(Jc);
    return x2;
}

/* Default box: widths s >= 0.25 channels (a narrower line is not resolved by
 * its samples); every other slot free. */
void gfo_spec_default_bounds(const gfo_spec_desc* d, double* lo, double* hi)
{
    int np = gfo_spec_nparams(d);
    for (int s = 0; s < np; ++s) {
        lo[s] = spec_role(d, s) == 3 ? 0.25 : -INFINITY;
        hi[s] = INFINITY;
    }
}

typedef struct {
    const gfo_spec_desc* d;
    const uint8_t* fixed;
    const double *lo, *hi, *lsf, *spec, *sig;
    const gfo_lm_opts* o;
} spec_problem;

static double sp_normal(void* ctx, const double* p, double* A, double* g)
{
    const spec_problem* q = (const spec_problem*)ctx;
    return gfo_spec_jacobian(q->d, p, q->fixed, q->lsf, q->spec, q->sig, q->o->jac_mode,
                             q->o->fd_rel, NULL, A, g);
}

static double sp_eval(void* ctx, const double* p)
{
    const spec_problem* q = (const spec_problem*)ctx;
    return gfo_spec_eval(q->d, p, q->lsf, q->spec, q->sig, NULL);
}

static void sp_project(void* ctx, double* p)
{
    const spec_problem* q = (const spec_problem*)ctx;
    int np = gfo_spec_nparams(q->d);
    for (int s = 0; s < np; ++s) {
        if (p[s] < q->lo[s]) p[s] = q->lo[s];
        if (p[s] > q->hi[s]) p[s] = q->hi[s];
    }
}

/* step-test floors: amplitudes relative (1e-30), continuum coefficients 1e-3
 * (like the sky level), centres and widths 1 */
static double sp_xscale(void* ctx, int s)
{
    int r = spec_role(((const spec_problem*)ctx)->d, s);
    if (r == 1) return 1e-30;
    if (r == 0) return 1e-3;
    return 1.0;
}

int gfo_spec_fit(const gfo_spec_desc* d, double* params, const uint8_t* fixed,
                 const double* lo_in, const double* hi_in, const double* lsf,
                 const double* spec, const double* sig, const gfo_lm_opts* opts_in,
                 gfo_lm_result* res)
{
    gfo_lm_opts o;
    if (opts_in)
        o = *opts_in;
    else
        gfo_default_opts(&o);
    int np = gfo_spec_nparams(d);
    double lo[GFO_MAX_SLOTS], hi[GFO_MAX_SLOTS];
    gfo_spec_default_bounds(d, lo, hi);
    if (lo_in) memcpy(lo, lo_in, sizeof(double) * np);
    if (hi_in) memcpy(hi, hi_in, sizeof(double) * np);
    int fs[GFO_MAX_SLOTS], nf = 0;
    for (int s = 0; s < np; ++s)
        if (!fixed || !fixed[s]) fs[nf++] = s;
    spec_problem q = {d, fixed, lo, hi, lsf, spec, sig, &o};
    gfo_lm_problem P = {np, nf, fs, sp_normal, sp_eval, sp_project, sp_xscale, &q};
    return gfo_lm_core(&P, params, &o, res);
}

/* Independent spectra (a cube, spaxel by spaxel), OpenMP across spectra.
 * params: count x nparams; spec, sig: count x N; lsf: L values shared by all
 * spectra, or count x L when lsf_per_spectrum. */
int gfo_spec_fit_batch(int count, const gfo_spec_desc* d, double* params, const uint8_t* fixed,
                       const double* lsf, int lsf_per_spectrum, const double* spec,
                       const double* sig, const gfo_lm_opts* opts, gfo_lm_result* res)
{
    int np = gfo_spec_nparams(d), N = d->n_chan, L = d->lsf_len;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < count; ++b)
        gfo_spec_fit(d, params + (size_t)b * np, fixed, NULL, NULL,
                     lsf + (lsf_per_spectrum ? (size_t)b * L : 0), spec + (size_t)b * N,
                     sig + (size_t)b * N, opts, res ? res + b : NULL);
    return 0;
}
