// lm.cu -- per-stamp constants and the Levenberg-Marquardt steps 4-5 of the
// fitting loop (Sec. 2 items 4-5; LM is the routine the paper names for GALFIT).
//
// FP64 appears on the device only here: in the per-component constants (b_n
// from P(2n, b_n) = 1/2, the rotation terms, finite-difference steps) and in the
// damped normal-equation solve.  The pixel path receives float32 constants.
//
// LM per stamp, driven by a phase word so that one launch sequence serves a
// whole batch of stamps in different states:
//   PH_NEED_JAC  the Jacobian pass (model/convolution/reduction) runs, -> PH_SOLVE
//   PH_SOLVE     solve (A + lambda diag A) delta = g by Cholesky; a tiny scaled
//                step ends the fit; else project p + delta into the box and
//                build the trial model channel, -> PH_TRIAL
//   PH_TRIAL     the trial pass computes chi^2 at the trial point; accept if it
//                fell (lambda shrinks, -> PH_NEED_JAC; a relative fall below ftol
//                ends the fit), else reject (lambda grows, -> PH_SOLVE)
//   PH_DONE      converged, lambda past lambda_max, max_iter trials, or
//                non-finite chi^2 / normal equations
#include <math.h>

#include "gf_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

// Regularised lower incomplete gamma P(a, x) by its power series
// P(a, x) = x^a e^{-x} / Gamma(a+1) * sum_{k>=0} x^k / ((a+1)...(a+k)).
// lg1 = ln Gamma(a + 1).
__device__ double gamma_p(double a, double x, double lg1)
{
    if (x <= 0.0) return 0.0;
    double sum = 1.0, term = 1.0;
    for (int k = 1; k < 1000; ++k) {
        term *= x / (a + k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return exp(a * log(x) - x - lg1) * sum;
}

// b_n: root of P(2n, b) = 1/2, by Newton steps safeguarded with a bisection
// bracket (the median of a Gamma(a) variate lies in (0, a)).  The start is the
// asymptotic expansion of Ciotti & Bertin (1999).
__device__ double sersic_bn(double n)
{
    const double a = 2.0 * n;
    double lo = 0.0, hi = a;
    double b = a - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n);
    if (!(b > lo && b < hi)) b = 0.5 * a;
    const double lg1 = lgamma(a + 1.0), lga = lg1 - log(a);
    for (int it = 0; it < 200; ++it) {
        const double f = gamma_p(a, b, lg1) - 0.5;
        if (f == 0.0) break;
        if (f < 0.0)
            lo = b;
        else
            hi = b;
        const double dens = exp((a - 1.0) * log(b) - b - lga);
        double nb = b - f / dens;
        if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
        const bool done = fabs(nb - b) <= 1e-14 * b;
        b = nb;
        if (done || hi - lo <= 1e-15 * b) break;
    }
    return b;
}

// float32 constants of one component from its float64 slots q; bn is b_n for
// a Sersic component (ignored otherwise)
__device__ CompConst make_cc(int kind, const double* q, bool unit_amp, double bn)
{
    CompConst k;
    k.kind = kind;
    k.x0h = k.x0l = k.y0h = k.y0l = 0.0f;
    k.cs = 1.0f;
    k.sn = 0.0f;
    k.invq = 1.0f;
    k.C = 2.0f;
    k.invC = 0.5f;
    k.amp = 0.0f;
    k.invr = 1.0f;
    k.invn = 1.0f;
    k.b0 = 0.0f;
    k.b = 1.0f;
    k.ellipse = 1;
    if (kind == GF_SKY) return k;
    const double x0 = q[0], y0 = q[1];
    k.x0h = (float)x0;
    k.x0l = (float)(x0 - (double)k.x0h);
    k.y0h = (float)y0;
    k.y0l = (float)(y0 - (double)k.y0h);
    const double amp = unit_amp ? 1.0 : q[2];
    const double r = q[3];
    double ax, pa, c;
    if (kind == GF_SERSIC) {
        ax = q[5];
        pa = q[6];
        c = q[7];
    } else {
        ax = q[4];
        pa = q[5];
        c = q[6];
    }
    const double th = pa * (kPi / 180.0);
    k.cs = (float)cos(th);
    k.sn = (float)sin(th);
    k.invq = (float)(1.0 / ax);
    k.C = (float)(c + 2.0);
    k.invC = (float)(1.0 / (c + 2.0));
    k.ellipse = (c == 0.0);
    k.amp = (float)amp;
    k.invr = (float)(1.0 / r);
    if (kind == GF_SERSIC) {
        const double n = q[4];
        k.invn = (float)(1.0 / n);
        k.b0 = (float)bn;
        k.b = (float)bn;
    }
    return k;
}

__device__ __forceinline__ double amp_of(const Structure& S, const double* p, int k)
{
    return S.kinds[k] == GF_SKY ? p[S.slot0[k]] : p[S.slot0[k] + 2];
}

__device__ double sky_of(const Structure& S, const double* p)
{
    return S.sky_slot >= 0 ? p[S.sky_slot] : 0.0;
}

// the model channel (sky and all components) at p
__device__ void build_sum(const Structure& S, const double* p, Channel& ch)
{
    ch.type = CH_SUM;
    ch.comp = 0;
    ch.jcol = -1;
    ch.mweight = 1.0f;
    ch.scale = 0.0f;
    ch.sky = (float)sky_of(S, p);
    ch.ncomp = S.ncomp;
    ch.msky = 0.0f;
    for (int k = 0; k < S.ncomp; ++k) {
        const double bn = S.kinds[k] == GF_SERSIC ? sersic_bn(p[S.slot0[k] + 4]) : 0.0;
        ch.cc[k] = make_cc(S.kinds[k], p + S.slot0[k], false, bn);
    }
    ch.pert = ch.cc[0];
}

// FD step of slot s at value v: positions fd_rel pixels, others fd_rel*max(|v|,1)
__device__ __forceinline__ double fd_step(int role, double v, double fd_rel)
{
    return role == R_POS ? fd_rel : fd_rel * fmax(fabs(v), 1.0);
}

// Jacobian-pass channels at p: one unit-amplitude shape per profile component
// (its convolution is the exact amplitude column and, weighted by the
// amplitude, its share of the model), then one FD channel per free nonlinear
// slot.  Returns the channel count.
__device__ int build_jac(const Structure& S, const double* p, double fd_rel, float psum,
                         Channel* out)
{
    CompConst unit[GF_MAX_COMP];
    double bnk[GF_MAX_COMP];
    for (int k = 0; k < S.ncomp; ++k) {
        bnk[k] = S.kinds[k] == GF_SERSIC ? sersic_bn(p[S.slot0[k] + 4]) : 0.0;
        unit[k] = make_cc(S.kinds[k], p + S.slot0[k], true, bnk[k]);
    }
    int nc = 0;
    const double sky = sky_of(S, p);
    for (int k = 0; k < S.ncomp; ++k) {
        if (S.kinds[k] == GF_SKY) continue;
        Channel& ch = out[nc++];
        ch.type = CH_SHAPE;
        ch.comp = k;
        ch.jcol = -1;
        for (int f = 0; f < S.nfree; ++f)
            if (S.freeslot[f] == S.slot0[k] + 2) ch.jcol = f;
        ch.mweight = (float)amp_of(S, p, k);
        ch.scale = 0.0f;
        ch.sky = 0.0f;
        ch.ncomp = S.ncomp;
        ch.msky = 0.0f;
        for (int kk = 0; kk < S.ncomp; ++kk) ch.cc[kk] = unit[kk];
        ch.pert = unit[k];
    }
    double pp[GF_MAX_SLOTS];
    for (int s = 0; s < S.nslots; ++s) pp[s] = p[s];
    for (int f = 0; f < S.nfree; ++f) {
        const int s = S.freeslot[f], role = S.role[s], k = S.owner[s];
        if (role == R_AMP || role == R_SKY) continue;
        const double h = fd_step(role, p[s], fd_rel);
        Channel& ch = out[nc++];
        ch.type = CH_FD;
        ch.comp = k;
        ch.jcol = f;
        ch.mweight = 0.0f;
        ch.scale = (float)(amp_of(S, p, k) / h);
        ch.sky = 0.0f;
        ch.ncomp = S.ncomp;
        ch.msky = 0.0f;
        for (int kk = 0; kk < S.ncomp; ++kk) ch.cc[kk] = unit[kk];
        pp[s] = p[s] + h;
        const double bn = role == R_N ? sersic_bn(pp[s]) : bnk[k];
        ch.pert = make_cc(S.kinds[k], pp + S.slot0[k], true, bn);
        pp[s] = p[s];
    }
    out[0].msky = (float)(sky * (double)psum);
    return nc;
}

__device__ void project(const Structure& S, double* p)
{
    for (int s = 0; s < S.nslots; ++s) {
        if (S.role[s] == R_PA) {
            double a = fmod(p[s], 180.0);
            if (a < 0.0) a += 180.0;
            if (a >= 180.0) a -= 180.0;
            p[s] = a;
            continue;
        }
        if (p[s] < S.lo[s]) p[s] = S.lo[s];
        if (p[s] > S.hi[s]) p[s] = S.hi[s];
    }
}

__device__ __forceinline__ double xtol_scale(int role)
{
    if (role == R_AMP) return 1e-30;
    if (role == R_SKY) return 1e-3;
    return 1.0;
}

// ---------------------------------------------------------------- kernels

__global__ void k_prep_sum(PassArgs a, const double* params, int use_trial)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.count) return;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const Structure& S = *a.S;
    const double* p = params ? params + (long long)b * S.nslots
                             : (use_trial ? a.lm[b].pt : a.lm[b].p);
    Channel* ch = const_cast<Channel*>(a.chan) + (long long)b * a.chan_stride;
    build_sum(S, p, ch[0]);
}

// one thread per stamp
__global__ void k_prep_jac(PassArgs a, const double* params)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.count) return;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const Structure& S = *a.S;
    const double* p = params ? params + (long long)b * S.nslots : a.lm[b].p;
    Channel* ch = const_cast<Channel*>(a.chan) + (long long)b * a.chan_stride;
    build_jac(S, p, S.opts.fd_rel, a.psf_sum[b], ch);
}

__global__ void k_lm_init(int count, const Structure* Sp, LMState* lm, const double* p0)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const Structure& S = *Sp;
    LMState& L = lm[b];
    for (int s = 0; s < S.nslots; ++s) L.p[s] = L.pt[s] = p0[(long long)b * S.nslots + s];
    project(S, L.p);
    L.chi2 = INFINITY;
    L.chi2t = INFINITY;
    L.lambda = S.opts.lambda0;
    L.iters = 0;
    L.accepted = 0;
    L.status = GF_EMAXITER;
    L.phase = PH_NEED_JAC;
}

// Cholesky solve of the SPD system M x = r in place (n <= GF_MAX_FREE)
__device__ bool cholesky_solve(int n, double* M, double* r)
{
    for (int j = 0; j < n; ++j) {
        double d = M[j * n + j];
        for (int k = 0; k < j; ++k) d -= M[j * n + k] * M[j * n + k];
        if (!(d > 0.0) || !isfinite(d)) return false;
        d = sqrt(d);
        M[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = M[i * n + j];
            for (int k = 0; k < j; ++k) s -= M[i * n + k] * M[j * n + k];
            M[i * n + j] = s / d;
        }
    }
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= M[i * n + k] * r[k];
        r[i] = s / M[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = r[i];
        for (int k = i + 1; k < n; ++k) s -= M[k * n + i] * r[k];
        r[i] = s / M[i * n + i];
    }
    for (int i = 0; i < n; ++i)
        if (!isfinite(r[i])) return false;
    return true;
}

__device__ void lm_reject(const Structure& S, LMState& L)
{
    L.lambda *= S.opts.lambda_up;
    if (L.lambda > S.opts.lambda_max) {
        L.status = GF_ENOCONV;
        L.phase = PH_DONE;
    } else {
        L.phase = PH_SOLVE;
    }
}

__device__ void lm_check_iters(const Structure& S, LMState& L)
{
    if (L.phase != PH_DONE && L.iters >= S.opts.max_iter) {
        L.status = GF_EMAXITER;
        L.phase = PH_DONE;
    }
}

__global__ void k_lm_solve(PassArgs a, Channel* trial_chan, int trial_stride)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.count) return;
    LMState& L = a.lm[b];
    if (L.phase != PH_SOLVE) return;
    const Structure& S = *a.S;
    const int nf = S.nfree;
    bool finite = isfinite(L.chi2);
    for (int i = 0; i < nf && finite; ++i) finite = isfinite(L.g[i]) && isfinite(L.A[i * nf + i]);
    if (!finite) {
        L.status = GF_ENONFINITE;
        L.phase = PH_DONE;
        return;
    }
    double M[GF_MAX_FREE * GF_MAX_FREE], r[GF_MAX_FREE];
    for (int i = 0; i < nf; ++i) {
        r[i] = L.g[i];
        for (int j = 0; j < nf; ++j) M[i * nf + j] = L.A[i * nf + j];
    }
    for (int i = 0; i < nf; ++i) {
        const double d = L.A[i * nf + i];
        if (d > 0.0) {
            M[i * nf + i] = d * (1.0 + L.lambda);
        } else {
            // a slot with no influence on the model is held this step
            for (int j = 0; j < nf; ++j) M[i * nf + j] = M[j * nf + i] = 0.0;
            M[i * nf + i] = 1.0;
            r[i] = 0.0;
        }
    }
    L.iters++;
    if (!cholesky_solve(nf, M, r)) {
        lm_reject(S, L);
        lm_check_iters(S, L);
        return;
    }
    double step = 0.0;
    for (int i = 0; i < nf; ++i) {
        const int s = S.freeslot[i];
        step = fmax(step, fabs(r[i]) / fmax(fabs(L.p[s]), xtol_scale(S.role[s])));
    }
    if (step < S.opts.xtol) {
        L.status = GF_OK;
        L.phase = PH_DONE;
        return;
    }
    for (int s = 0; s < S.nslots; ++s) L.pt[s] = L.p[s];
    for (int i = 0; i < nf; ++i) L.pt[S.freeslot[i]] += r[i];
    project(S, L.pt);
    build_sum(S, L.pt, trial_chan[(long long)b * trial_stride]);
    L.phase = PH_TRIAL;
}

__global__ void k_lm_update(PassArgs a, int* active)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.count) return;
    LMState& L = a.lm[b];
    const Structure& S = *a.S;
    if (L.phase == PH_TRIAL) {
        const double xt = L.chi2t;
        if (isfinite(xt) && xt < L.chi2) {
            const double rel = (L.chi2 - xt) / L.chi2;
            for (int s = 0; s < S.nslots; ++s) L.p[s] = L.pt[s];
            L.accepted++;
            L.lambda = fmax(L.lambda * S.opts.lambda_down, S.opts.lambda_min);
            L.chi2 = xt;
            if (rel < S.opts.ftol) {
                L.status = GF_OK;
                L.phase = PH_DONE;
            } else {
                L.phase = PH_NEED_JAC;
            }
        } else {
            lm_reject(S, L);
        }
        lm_check_iters(S, L);
    }
    if (active && L.phase != PH_DONE) atomicAdd(active, 1);
}

}  // namespace

cudaError_t launch_prep_sum(const PassArgs& a, const double* params, int use_trial,
                            cudaStream_t s)
{
    k_prep_sum<<<(a.count + 63) / 64, 64, 0, s>>>(a, params, use_trial);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_prep_jac(const PassArgs& a, const double* params, cudaStream_t s)
{
    k_prep_jac<<<(a.count + 63) / 64, 64, 0, s>>>(a, params);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_lm_init(int count, const Structure* S, LMState* lm, const double* p0,
                           cudaStream_t s)
{
    k_lm_init<<<(count + 127) / 128, 128, 0, s>>>(count, S, lm, p0);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_lm_solve(const PassArgs& a, Channel* trial_chan, cudaStream_t s)
{
    k_lm_solve<<<(a.count + 63) / 64, 64, 0, s>>>(a, trial_chan, 1);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_lm_update(const PassArgs& a, int* active_count, cudaStream_t s)
{
    k_lm_update<<<(a.count + 127) / 128, 128, 0, s>>>(a, active_count);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

namespace {
// compact per-stamp results: p[nslots], chi2, lambda, iters, accepted, status
__global__ void k_lm_export(int count, const Structure* Sp, const LMState* lm, double* out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const int ns = Sp->nslots, stride = ns + 5;
    const LMState& L = lm[b];
    double* o = out + (long long)b * stride;
    for (int s = 0; s < ns; ++s) o[s] = L.p[s];
    o[ns] = L.chi2;
    o[ns + 1] = L.lambda;
    o[ns + 2] = L.iters;
    o[ns + 3] = L.accepted;
    o[ns + 4] = L.status;
}
}  // namespace

cudaError_t launch_lm_export(int count, const Structure* S, const LMState* lm, double* out,
                             cudaStream_t s)
{
    k_lm_export<<<(count + 127) / 128, 128, 0, s>>>(count, S, lm, out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}
