// lm.cu -- per-stamp constants and the Levenberg-Marquardt steps 4-5 of the
// fitting loop (Sec. 2 items 4-5; LM is the routine the paper names for GALFIT).
//
// FP64 appears on the device only here: in the per-component constants (b_n
// from P(2n, b_n) = 1/2, the rotation terms, finite-difference steps) and in the
// damped normal-equation solve.  The pixel path receives float32 constants.
//
// Every kernel here runs one warp per stamp.  GB300's FP64 units are few and
// their latency long, so a single thread walking a chain of dependent FP64
// divisions (the incomplete-gamma series, a Cholesky factorisation) costs
// hundreds of microseconds; spread over 32 lanes the same work is short:
//   - the series terms x^k / ((a+1)...(a+k)) come from one division per term,
//     done in parallel, and a warp prefix product;
//   - Newton on P(2n, b) - 1/2 starts from the stamp's previous b_n (db_n/dn is
//     close to 2), so it usually needs two or three series evaluations;
//   - channel constants are built one channel per lane;
//   - the Cholesky factorisation updates each column across the lanes.
//
// LM per stamp, driven by a phase word so that one launch sequence serves a
// whole batch of stamps in different states:
//   PH_NEED_JAC  the Jacobian pass (model/convolution/reduction) runs, -> PH_SOLVE
//   PH_SOLVE     solve (A + lambda diag A) delta = g by Cholesky; a tiny scaled
//                step ends the fit; else project p + delta into the box and
//                build the trial model channel, -> PH_TRIAL
//   PH_TRIAL     the trial pass computes chi^2 at the trial point; accept if it
//                fell (lambda shrinks, -> PH_NEED_JAC; when both the actual and
//                the predicted relative falls are below ftol the fit ends), else
//                reject (lambda grows, -> PH_SOLVE)
//   PH_DONE      converged, lambda past lambda_max, max_iter trials, or
//                non-finite chi^2 / normal equations
#include <math.h>

#include "chol.cuh"
#include "gf_internal.cuh"
#include "bn.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;
// sigma of a Gaussian per unit full width at half maximum, 1 / (2 sqrt(2 ln 2))
constexpr double kGaussSigmaPerFwhm = 0.42466090014400952136;
constexpr double kLn2 = 0.69314718055994530942;

// alpha / fwhm of a Moffat profile of index beta, 1 / (2 sqrt(2^(1/beta) - 1)),
// and d ln(alpha / fwhm) / d beta = 2^(1/beta) ln 2 / (2 beta^2 (2^(1/beta) - 1))
__device__ __forceinline__ double moffat_alpha_per_fwhm(double beta)
{
    return 0.5 / sqrt(exp2(1.0 / beta) - 1.0);
}
__device__ __forceinline__ double moffat_dlnalpha_dbeta(double beta)
{
    const double t = exp2(1.0 / beta);
    return t * kLn2 / (2.0 * beta * beta * (t - 1.0));
}
constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;

// b_n table: g_bn_tab[k] = b_n at n = BN_N0 + k BN_DN, filled once per device
// by k_bn_table with the solver above; read by 4-point Lagrange interpolation
// (relative error below 1e-11 on [0.2, 10] at this spacing, far under float32).
constexpr double BN_N0 = 0.19, BN_DN = 1.0 / 2048.0;
constexpr int BN_TAB = 20160;  // up to n = 10.033 (the FD step above n = 10)
__device__ double g_bn_tab[BN_TAB];
__device__ int g_bn_ready;

__global__ void k_bn_table()
{
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= BN_TAB) return;
    const double b = sersic_bn_warp(BN_N0 + k * BN_DN, -1.0);
    if ((threadIdx.x & 31) == 0) g_bn_tab[k] = b;
}

__global__ void k_bn_ready() { g_bn_ready = 1; }

// b_n from the table, or NaN when the table is not built or n lies outside it
__device__ double bn_lookup(double n)
{
    if (*(volatile int*)&g_bn_ready != 1) return NAN;
    const double u = (n - BN_N0) * (1.0 / BN_DN);
    if (!(u >= 1.0) || !(u < (double)(BN_TAB - 2))) return NAN;
    const int k = (int)floor(u) - 1;  // nodes k .. k + 3, u between nodes k+1 and k+2
    const double t = u - (double)(k + 1);
    const double f0 = g_bn_tab[k], f1 = g_bn_tab[k + 1], f2 = g_bn_tab[k + 2], f3 = g_bn_tab[k + 3];
    const double tm1 = t - 1.0, tm2 = t - 2.0, tp1 = t + 1.0;
    return -t * tm1 * tm2 * (1.0 / 6.0) * f0 + tp1 * tm1 * tm2 * 0.5 * f1 -
           tp1 * t * tm2 * 0.5 * f2 + tp1 * t * tm1 * (1.0 / 6.0) * f3;
}

// db_n/dn from the table: the derivative of the same 4-point Lagrange
// interpolant (NaN where bn_lookup is NaN)
__device__ double bn_deriv_lookup(double n)
{
    if (*(volatile int*)&g_bn_ready != 1) return NAN;
    const double u = (n - BN_N0) * (1.0 / BN_DN);
    if (!(u >= 1.0) || !(u < (double)(BN_TAB - 2))) return NAN;
    const int k = (int)floor(u) - 1;
    const double t = u - (double)(k + 1);
    const double f0 = g_bn_tab[k], f1 = g_bn_tab[k + 1], f2 = g_bn_tab[k + 2], f3 = g_bn_tab[k + 3];
    const double t2 = 3.0 * t * t;
    const double d = -(t2 - 6.0 * t + 2.0) * (1.0 / 6.0) * f0 + (t2 - 4.0 * t - 1.0) * 0.5 * f1 -
                     (t2 - 2.0 * t - 2.0) * 0.5 * f2 + (t2 - 1.0) * (1.0 / 6.0) * f3;
    return d * (1.0 / BN_DN);
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
    k.e0 = k.e1 = k.e2 = k.e3 = 0.0f;
    k.e4 = k.e5 = k.e6 = k.e7 = k.e8 = 0.0f;
    k.pad_c[0] = k.pad_c[1] = k.pad_c[2] = 0;
    if (is_sky_kind(kind)) return k;
    const double x0 = q[0], y0 = q[1];
    k.x0h = (float)x0;
    k.x0l = (float)(x0 - (double)k.x0h);
    k.y0h = (float)y0;
    k.y0l = (float)(y0 - (double)k.y0h);
    const double amp = unit_amp ? 1.0 : q[2];
    if (kind == GF_PSF) {  // a point source: position and flux only
        k.amp = (float)amp;
        return k;
    }
    const double r = q[3];
    // the axis ratio, position angle and boxiness follow the kind's shape slots
    const int g = (kind == GF_SERSIC || kind == GF_MOFFAT || kind == GF_SERSIC_F) ? 5
                  : kind == GF_KING                        ? 6
                  : kind == GF_NUKER                       ? 7
                                                           : 4;
    const double ax = q[g], pa = q[g + 1], c = q[g + 2];
    // The constants are formed in FP64 and rounded once to float32: the
    // finite-difference channels difference two such constant sets, so their
    // rounding is what the 1/h of a forward difference amplifies.
    const double th = pa * (kPi / 180.0);
    double sth, cth;
    sincos(th, &sth, &cth);  // one range reduction for both
    k.cs = (float)cth;
    k.sn = (float)sth;
    k.invq = (float)(1.0 / ax);
    k.C = (float)(c + 2.0);
    k.invC = (float)(1.0 / (c + 2.0));
    k.ellipse = (c == 0.0);
    k.amp = (float)amp;
    k.invr = (float)(1.0 / r);
    if (kind == GF_GAUSSIAN) {
        // exp(-(r/s)^2 / 2): the exp(b0 - b u) form with u = (r/s)^2
        k.invr = (float)(1.0 / (r * kGaussSigmaPerFwhm));
        k.invn = 2.0f;
        k.b0 = 0.0f;
        k.b = 0.5f;
    }
    if (kind == GF_MOFFAT) {
        // (1 + t^2)^(-beta) = exp(-b u) with u = log2(1 + t^2), b = beta ln 2,
        // t = r / alpha, alpha = fwhm / (2 sqrt(2^(1/beta) - 1)); invn carries
        // beta for the gradient
        const double beta = q[4];
        k.invr = (float)(2.0 * sqrt(exp2(1.0 / beta) - 1.0) / r);
        k.invn = (float)beta;
        k.b0 = 0.0f;
        k.b = (float)(beta * kLn2);
    }
    if (is_sersic_kind(kind)) {
        const double n = q[4];
        k.invn = (float)(1.0 / n);
        k.b0 = (float)bn;
        k.b = (float)bn;
    }
    if (kind == GF_SERSIC_F) {
        // Fourier modes m = 1, 3, 4 (slots 8 .. 13): amplitudes, then cos and
        // sin of m phi_m, formed in FP64
        k.e0 = (float)q[8];
        k.e1 = (float)q[10];
        k.e2 = (float)q[12];
        double sp, cp;
        sincos(q[9] * (kPi / 180.0), &sp, &cp);
        k.e3 = (float)cp;
        k.e4 = (float)sp;
        sincos(3.0 * q[11] * (kPi / 180.0), &sp, &cp);
        k.e5 = (float)cp;
        k.e6 = (float)sp;
        sincos(4.0 * q[13] * (kPi / 180.0), &sp, &cp);
        k.e7 = (float)cp;
        k.e8 = (float)sp;
    }
    if (kind == GF_KING) {
        // slots r_c (3), r_t (4), alpha (5): w_t = (1 + (r_t/r_c)^2)^(-1/alpha)
        const double rt = q[4], al = q[5], x = rt / r;
        const double wt = pow(1.0 + x * x, -1.0 / al);
        k.invn = (float)al;
        k.e0 = (float)(1.0 / al);
        k.e1 = (float)wt;
        k.e2 = (float)(1.0 / (1.0 - wt));
    }
    if (kind == GF_NUKER) {
        // slots r_b (3), alpha (4), beta (5), gamma (6)
        const double al = q[4], be = q[5], ga = q[6];
        k.invn = (float)al;
        k.e0 = (float)ga;
        k.e1 = (float)((be - ga) / al);
        k.e2 = (float)((ga - be) / al);
    }
    return k;
}

__device__ __forceinline__ double amp_of(const Structure& S, const double* p, int k)
{
    return is_sky_kind(S.kinds[k]) ? p[S.slot0[k]] : p[S.slot0[k] + 2];
}

__device__ __forceinline__ double sky_of(const Structure& S, const double* p)
{
    return S.sky_slot >= 0 ? p[S.sky_slot] : 0.0;
}

// FD step of slot s at value v: positions fd_rel pixels, others fd_rel*max(|v|,1)
__device__ __forceinline__ double fd_step(int role, double v, double fd_rel)
{
    return role == R_POS ? fd_rel : fd_rel * fmax(fabs(v), 1.0);
}

__device__ __forceinline__ double xtol_scale(int role)
{
    if (role == R_AMP) return 1e-30;
    if (role == R_SKY) return 1e-3;
    if (role == R_TILTX || role == R_TILTY) return 1e-5;  // sky slopes, per pixel
    return 1.0;
}

// the sky plane's slope along x (0) or y (1), 0 without a plane
__device__ __forceinline__ double tilt_of(const Structure& S, const double* p, int a)
{
    return S.tilt_slot[a] >= 0 ? p[S.tilt_slot[a]] : 0.0;
}

__device__ void project_slot(const Structure& S, double* p, int s)
{
    if (S.role[s] == R_PA) {
        // p - 180 k with k = floor(p / 180): exact for the angles a fit meets
        double a = p[s] - 180.0 * floor(p[s] * (1.0 / 180.0));
        if (a < 0.0) a += 180.0;
        if (a >= 180.0) a -= 180.0;
        p[s] = a;
        return;
    }
    if (p[s] < S.lo[s]) p[s] = S.lo[s];
    if (p[s] > S.hi[s]) p[s] = S.hi[s];
}

// per-warp scratch in shared memory
struct WarpScratch {
    double M[GF_MAX_FREE * GF_MAX_FREE];
    double r[GF_MAX_FREE];
    double p[GF_MAX_SLOTS];
    double bn[GF_MAX_COMP];
    double bnp[GF_MAX_COMP];  // b_n at n + h (FD channel of a free n)
    double dbdn[GF_MAX_COMP]; // db_n/dn (analytic channel of a free n)
    CompConst cc[GF_MAX_COMP];
    int ok;
};

// b_n of every Sersic component at W.p (warm start from the stamp's cache when
// one is given), and at n + h when want_pert and the n slot is free
__device__ void warp_bn(const Structure& S, WarpScratch& W, LMState* L, bool want_pert)
{
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < S.ncomp; ++k) {
        if (!is_sersic_kind(S.kinds[k])) continue;
        const int sn = S.slot0[k] + 4;
        const double n = W.p[sn];
        double b = bn_lookup(n);
        if (isnan(b)) {
            double guess = -1.0;
            if (L && L->bn_n[k] > 0.0) guess = L->bn_b[k] + 2.0 * (n - L->bn_n[k]);
            b = sersic_bn_warp(n, guess);
        }
        __syncwarp();
        if (lane == 0) {
            W.bn[k] = b;
            if (L) {
                L->bn_n[k] = n;
                L->bn_b[k] = b;
            }
        }
        if (want_pert) {
            bool free_n = false;
            for (int f = 0; f < S.nfree; ++f) free_n |= (S.freeslot[f] == sn);
            if (S.opts.jac_mode == GF_JAC_ANALYTIC) {
                double db = bn_deriv_lookup(n);
                if (isnan(db)) {  // outside the table: central differences of the solver
                    const double e = 1e-4 * fmax(n, 1.0);
                    db = (sersic_bn_warp(n + e, b + 2.0 * e) - sersic_bn_warp(n - e, b - 2.0 * e)) /
                         (2.0 * e);
                }
                if (lane == 0) W.dbdn[k] = db;
            } else if (free_n) {
                const double h = fd_step(R_N, n, S.opts.fd_rel);
                double bp = bn_lookup(n + h);
                if (isnan(bp)) bp = sersic_bn_warp(n + h, b + 2.0 * h);
                if (lane == 0) W.bnp[k] = bp;
            }
        }
    }
    __syncwarp();
}

// the model channel (sky and all components) at W.p; lanes build components;
// (xc, yc) is the stamp centre, the origin of a sky plane
__device__ void warp_build_sum(const Structure& S, WarpScratch& W, float xc, float yc, Channel* out)
{
    const int lane = threadIdx.x & 31;
    if (lane < S.ncomp) {
        const int k = lane;
        out->cc[k] = make_cc(S.kinds[k], W.p + S.slot0[k], false, W.bn[k]);
        if (k == 0) out->pert = out->cc[0];
    }
    if (lane == 0) {
        out->type = CH_SUM;
        out->comp = 0;
        out->jcol = -1;
        out->mweight = 1.0f;
        out->scale = 0.0f;
        out->sky = (float)sky_of(S, W.p);
        out->ncomp = S.ncomp;
        out->msky = 0.0f;
        out->pxc = xc;
        out->pyc = yc;
        out->tgx = (float)tilt_of(S, W.p, 0);
        out->tgy = (float)tilt_of(S, W.p, 1);
    }
}

// Jacobian-pass channels at W.p: one unit-amplitude shape per profile component
// (its convolution is the exact amplitude column and, weighted by the
// amplitude, its share of the model), the two slope bases of a sky plane
// (exact columns; weighted by the slopes, the plane's share), then one FD
// channel per free nonlinear slot.  Lane c builds channel c.
__device__ void warp_build_jac(const Structure& S, WarpScratch& W, float psum, float xc, float yc,
                               Channel* out)
{
    const int lane = threadIdx.x & 31;
    if (lane < S.ncomp) W.cc[lane] = make_cc(S.kinds[lane], W.p + S.slot0[lane], true, W.bn[lane]);
    __syncwarp();
    for (int c = lane; c < S.nchan; c += 32) {
        // identify channel c
        int type = CH_SHAPE, comp = -1, slot = -1, jcol = -1;
        int idx = 0;
        for (int k = 0; k < S.ncomp && comp < 0; ++k) {
            if (is_sky_kind(S.kinds[k])) continue;
            if (idx == c) comp = k;
            ++idx;
        }
        if (comp >= 0) {
            for (int f = 0; f < S.nfree; ++f)
                if (S.freeslot[f] == S.slot0[comp] + 2) jcol = f;
        } else if (c < S.nprofile + S.nplane) {
            type = CH_PLANE;
            slot = c - S.nprofile;  // 0: slope along x, 1: along y
            jcol = S.tilt_jcol[slot];
        } else {
            type = CH_FD;
            idx += S.nplane;
            for (int f = 0; f < S.nfree && slot < 0; ++f) {
                const int s = S.freeslot[f];
                if (S.role[s] == R_AMP || S.role[s] == R_SKY || S.role[s] == R_TILTX ||
                    S.role[s] == R_TILTY)
                    continue;
                if (idx == c) {
                    slot = s;
                    jcol = f;
                }
                ++idx;
            }
            comp = S.owner[slot];
        }
        Channel& ch = out[c];
        ch.type = type;
        ch.dslot = 0;
        ch.dbdn = 0.0f;
        ch.comp = comp;
        ch.jcol = jcol;
        ch.sky = 0.0f;
        ch.ncomp = S.ncomp;
        ch.msky = c == 0 ? (float)(sky_of(S, W.p) * (double)psum) : 0.0f;
        ch.pxc = xc;
        ch.pyc = yc;
        ch.tgx = ch.tgy = 0.0f;
        for (int k = 0; k < S.ncomp; ++k) ch.cc[k] = W.cc[k];
        if (type == CH_PLANE) {
            ch.dslot = slot;
            ch.comp = -1;
            ch.mweight = (float)tilt_of(S, W.p, slot);
            ch.scale = 0.0f;
            ch.pert = W.cc[0];
        } else if (type == CH_SHAPE) {
            ch.mweight = (float)amp_of(S, W.p, comp);
            ch.scale = 0.0f;
            ch.pert = W.cc[comp];
        } else if (S.opts.jac_mode == GF_JAC_ANALYTIC) {
            ch.type = CH_DERIV;
            ch.mweight = 0.0f;
            ch.scale = (float)amp_of(S, W.p, comp);
            ch.dslot = slot - S.slot0[comp];
            ch.dbdn = S.kinds[comp] == GF_SERSIC ? (float)W.dbdn[comp] : 0.0f;
            if (S.kinds[comp] == GF_MOFFAT) {
                // the gradient's slot 3 is d/d alpha: alpha / fwhm turns it into
                // d/d fwhm; slot 4 takes d ln(alpha / fwhm) / d beta
                const double beta = W.p[S.slot0[comp] + 4];
                if (ch.dslot == 3) ch.scale = (float)(amp_of(S, W.p, comp) * moffat_alpha_per_fwhm(beta));
                ch.dbdn = (float)moffat_dlnalpha_dbeta(beta);
            }
            ch.pert = W.cc[comp];
        } else {
            const int role = S.role[slot];
            const double h = fd_step(role, W.p[slot], S.opts.fd_rel);
            double q[GF_COMP_MAXSLOTS];
            const int ns = comp_nslots(S.kinds[comp]);
            for (int t = 0; t < ns; ++t) q[t] = W.p[S.slot0[comp] + t];
            q[slot - S.slot0[comp]] += h;
            ch.mweight = 0.0f;
            ch.scale = (float)(amp_of(S, W.p, comp) / h);
            ch.pert = make_cc(S.kinds[comp], q, true, role == R_N ? W.bnp[comp] : W.bn[comp]);
        }
    }
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

// ---------------------------------------------------------------- kernels

// the call's Structure, copied into shared memory by the whole block (the
// per-stamp code walks its tables in dependent chains: slot -> role -> value)
// (8-byte words, four loads in flight per thread before the stores: a 32-thread
// block copies it in two rounds of L2 latency instead of eighteen)
__device__ __forceinline__ void load_structure(Structure* dst, const Structure* src)
{
    static_assert(sizeof(Structure) % 8 == 0, "Structure must be a multiple of 8 bytes");
    constexpr int N = (int)(sizeof(Structure) / 8);
    const uint2* s = reinterpret_cast<const uint2*>(src);
    uint2* d = reinterpret_cast<uint2*>(dst);
    for (int i0 = threadIdx.x; i0 < N; i0 += 4 * blockDim.x) {
        uint2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < N) v[u] = __ldcg(s + i);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < N) d[i] = v[u];
        }
    }
}

#define WARP_STAMP()                                                          \
    __shared__ WarpScratch scratch[kWarpsPerBlock];                           \
    __shared__ Structure S_sh;                                                \
    load_structure(&S_sh, a.S);                                               \
    __syncthreads();                                                          \
    const Structure& S = S_sh;                                                \
    const int lane = threadIdx.x & 31;                                        \
    const int b = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);           \
    if (b >= a.count) return;                                                 \
    WarpScratch& W = scratch[threadIdx.x >> 5];

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_prep_sum(PassArgs a, const double* params,
                                                                  int use_trial)
{
    pdl_entry();
    WARP_STAMP();
    if (a.lm && a.lm[b].phase != a.phase) return;
    const double* p = params ? params + (long long)b * S.nslots
                             : (use_trial ? a.lm[b].pt[0] : a.lm[b].p);
    for (int s = lane; s < S.nslots; s += 32) W.p[s] = p[s];
    __syncwarp();
    warp_bn(S, W, a.lm ? &a.lm[b] : nullptr, false);
    warp_build_sum(S, W, 0.5f * (float)(a.st[b].W - 1), 0.5f * (float)(a.st[b].H - 1),
                   const_cast<Channel*>(a.chan) + (long long)b * a.chan_stride);
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_prep_jac(PassArgs a, const double* params)
{
    pdl_entry();
    WARP_STAMP();
    if (a.lm && a.lm[b].phase != a.phase) return;
    const double* p = params ? params + (long long)b * S.nslots : a.lm[b].p;
    for (int s = lane; s < S.nslots; s += 32) W.p[s] = p[s];
    __syncwarp();
    warp_bn(S, W, a.lm ? &a.lm[b] : nullptr, true);
    warp_build_jac(S, W, a.psf_sum[b], 0.5f * (float)(a.st[b].W - 1), 0.5f * (float)(a.st[b].H - 1),
                   const_cast<Channel*>(a.chan) + (long long)b * a.chan_stride);
}

__global__ void k_lm_init(int count, const Structure* Sp, LMState* lm, const double* p0)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const Structure& S = *Sp;
    LMState& L = lm[b];
    for (int s = 0; s < S.nslots; ++s) L.p[s] = L.pt[0][s] = p0[(long long)b * S.nslots + s];
    for (int s = 0; s < S.nslots; ++s) project_slot(S, L.p, s);
    for (int k = 0; k < GF_MAX_COMP; ++k) L.bn_n[k] = L.bn_b[k] = 0.0;
    L.chi2 = INFINITY;
    L.chi2t = INFINITY;
    L.lambda = S.opts.lambda0;
    for (int r = 0; r < GF_MAX_LADDER; ++r) {
        L.pred[r] = 0.0;
        L.rung[r] = RUNG_FAIL;
    }
    L.rung0 = 0;
    L.iters = 0;
    L.accepted = 0;
    L.status = GF_EMAXITER;
    L.phase = PH_NEED_JAC;
}

// The trial ladder.  Marquardt's rule tries one step at a time: solve with
// lambda, evaluate the trial, and after a rejection solve again with
// lambda*up.  With a ladder of R rungs the damped systems for lambda,
// lambda*up, ..., lambda*up^(R-1) (the damping of each repeated by the same
// multiplications the rule makes) are solved side by side, one warp per rung,
// and their trials are evaluated in one pass.  k_final_update then walks the
// rungs in order, applying the rule to each, and stops where the rule stops (an
// accepted trial, a finishing criterion); the rungs it does not reach are
// discarded.  The fit therefore takes exactly the steps of the one-at-a-time
// rule, in fewer passes when trials are rejected.

// One block per stamp, one warp per rung.  Stamps whose Jacobian pass just ran
// (PH_NEED_JAC; its sums already in A, g and chi^2) and stamps retrying after
// rejections (PH_SOLVE) solve the damped systems, apply the scaled-step test,
// and build one trial model channel per rung.  Rungs before the first one that
// needs a trial (failed solves, a finishing step) are settled here.  Block 0
// also resets the active-stamp counter that k_final_update fills.
__global__ void __launch_bounds__(32 * GF_MAX_LADDER) k_final_solve(PassArgs a, Channel* trial_chan,
                                                                    int* active)
{
    pdl_entry();
    __shared__ Structure S_sh;
    __shared__ WarpScratch Ws[GF_MAX_LADDER];
    __shared__ double As[GF_MAX_FREE * GF_MAX_FREE], gs[GF_MAX_FREE];
    __shared__ int rung_state[GF_MAX_LADDER];
    const int b = blockIdx.x;
    const int nr = blockDim.x >> 5;  // rungs
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (b == 0 && threadIdx.x == 0 && active) *active = 0;
    LMState& L = a.lm[b];
    const int phase = L.phase;
    if (phase != PH_NEED_JAC && phase != PH_SOLVE) return;  // the whole block
    load_structure(&S_sh, a.S);
    const Structure& S = S_sh;
    const int nf = a.S->nfree;
    {
        const int nA = nf * nf;
        for (int i = threadIdx.x; i < nA; i += blockDim.x) As[i] = __ldcg(&L.A[i]);
        if (threadIdx.x < nf) gs[threadIdx.x] = __ldcg(&L.g[threadIdx.x]);
    }
    __syncthreads();
    bool fin = true;
    for (int i = lane; i < nf; i += 32) fin = fin && isfinite(gs[i]) && isfinite(As[i * nf + i]);
    const bool finite = __all_sync(kFull, fin) && isfinite(L.chi2);  // the same in every warp
    if (!finite) {
        if (threadIdx.x == 0) {
            L.status = GF_ENONFINITE;
            L.phase = PH_DONE;
        }
        return;
    }
    WarpScratch& W = Ws[w];
    // damping of rung w: lambda times up, w times over (the rule's own sequence)
    double lam = L.lambda;
    for (int r = 0; r < w; ++r) lam *= S.opts.lambda_up;
    // damped system (A + lambda diag A) delta = g; a slot with A_ii = 0 is held
    // bit i: A_ii > 0 (one FP64 comparison per lane instead of one per entry)
    const unsigned pos = __ballot_sync(kFull, lane < nf && As[lane * nf + lane] > 0.0);
    if (lane < nf) {  // lane i builds row i
        const int i = lane;
        const double aii = As[i * nf + i];
        const bool pi = (pos >> i) & 1u;
        for (int j = 0; j < nf; ++j) {
            double v = As[i * nf + j];
            if (!pi || !((pos >> j) & 1u))
                v = (i == j) ? 1.0 : 0.0;
            else if (i == j)
                v = aii * (1.0 + lam);
            W.M[i * nf + j] = v;
        }
        W.r[i] = pi ? gs[i] : 0.0;
    }
    const bool ok = warp_cholesky_solve(nf, W.M, W.r);
    int state = RUNG_FAIL;
    double pred = 0.0;
    if (ok) {
        // scaled step and predicted fall of chi^2 for the damped step,
        // delta^T (g + lambda diag(A) delta), as warp reductions (the test
        // max_i |delta_i| / s_i < xtol is taken as |delta_i| < xtol s_i for
        // every i: no FP64 division per lane)
        bool small = true;
        for (int i = lane; i < nf; i += 32) {
            const int sl = S.freeslot[i];
            small = small && fabs(W.r[i]) < S.opts.xtol * fmax(fabs(L.p[sl]), xtol_scale(S.role[sl]));
            if ((pos >> i) & 1u) pred += W.r[i] * (gs[i] + lam * As[i * nf + i] * W.r[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pred += __shfl_xor_sync(kFull, pred, o);
        state = __all_sync(kFull, small) ? RUNG_SMALL : RUNG_TRIAL;
    }
    // trial parameters p + delta projected into the box (a rung without a
    // trial keeps p, so that its channel is still a valid model)
    for (int sl = lane; sl < S.nslots; sl += 32) W.p[sl] = L.p[sl];
    __syncwarp();
    if (state == RUNG_TRIAL)
        for (int i = lane; i < nf; i += 32) W.p[S.freeslot[i]] += W.r[i];
    __syncwarp();
    for (int sl = lane; sl < S.nslots; sl += 32) {
        project_slot(S, W.p, sl);
        L.pt[w][sl] = W.p[sl];
    }
    __syncwarp();
    warp_bn(S, W, w == 0 ? &L : nullptr, false);
    warp_build_sum(S, W, 0.5f * (float)(a.st[b].W - 1), 0.5f * (float)(a.st[b].H - 1),
                   trial_chan + (long long)b * nr + w);
    if (lane == 0) {
        L.pred[w] = pred;
        L.rung[w] = state;
        rung_state[w] = state;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // settle the rungs before the first trial, as the rule would, one by one
    int r = 0;
    for (; r < nr; ++r) {
        const int st = rung_state[r];
        if (st == RUNG_TRIAL) break;
        L.iters += 1;
        if (st == RUNG_SMALL) {
            L.status = GF_OK;
            L.phase = PH_DONE;
            return;
        }
        lm_reject(S, L);
        lm_check_iters(S, L);
        if (L.phase == PH_DONE) return;
    }
    if (r < nr) {
        L.rung0 = r;
        L.phase = PH_TRIAL;
    } else {
        L.phase = PH_SOLVE;  // every rung's solve failed: solve again at the grown damping
    }
}

// One block per stamp: stamps in PH_TRIAL sum the trial pass's partials into
// the chi^2 of each rung from rung0 on (deterministic tree, the same for every
// rung), then apply the rule rung by rung: a rejected trial grows lambda and
// passes to the next rung, an accepted one (or a finishing criterion) ends the
// walk.  Every stamp not yet done adds one to the active counter.
// The trial ladder's rule for one stamp, given each rung's chi^2 (x2r): a
// rejected trial grows lambda and passes to the next rung, an accepted one (or
// a finishing criterion) ends the walk; a stamp not yet done adds one to the
// active counter.  One thread.
__device__ void lm_apply_trials(const PassArgs& a, LMState& L, int phase, int nr, const double* x2r,
                                int* active)
{
    const Structure& S = *a.S;
    if (phase == PH_TRIAL) {
        for (int r = L.rung0; r < nr; ++r) {
            L.iters += 1;
            const int st = L.rung[r];
            if (st == RUNG_SMALL) {
                L.status = GF_OK;
                L.phase = PH_DONE;
                break;
            }
            if (st == RUNG_TRIAL) {
                const double xt = x2r[r];
                L.chi2t = xt;
                if (isfinite(xt) && xt < L.chi2) {
                    const double rel = (L.chi2 - xt) / L.chi2;
                    const double prel = L.pred[r] / L.chi2;
                    for (int sl = 0; sl < S.nslots; ++sl) L.p[sl] = L.pt[r][sl];
                    L.accepted++;
                    L.lambda = fmax(L.lambda * S.opts.lambda_down, S.opts.lambda_min);
                    L.chi2 = xt;
                    if (rel < S.opts.ftol && prel < S.opts.ftol) {
                        L.status = GF_OK;
                        L.phase = PH_DONE;
                    } else {
                        L.phase = PH_NEED_JAC;
                    }
                    lm_check_iters(S, L);
                    break;
                }
            }
            lm_reject(S, L);
            lm_check_iters(S, L);
            if (L.phase == PH_DONE) break;
        }
    }
    if (active && L.phase != PH_DONE) atomicAdd(active, 1);
}

// the stamp's partial slots of a trial pass: its reduce blocks, or its 16 x 32
// output blocks when the convolution (direct, or the one-CTA FFT) reduced the trial
__device__ __forceinline__ void trial_slots(const PassArgs& a, int b, int& b0, int& b1)
{
    if (a.conv_chi2) {
        const StampInfo& st = a.st[b];
        b0 = st.wb_off;
        b1 = b0 + ((st.H + 15) / 16) * ((st.W + 31) / 32);
    } else {
        const int* pst = a.pre_static + WK_RED * (a.count + 1);
        b0 = pst[b];
        b1 = pst[b + 1];
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_final_update(PassArgs a, int* active)
{
    pdl_entry();
    __shared__ CSum wsum[RED_THREADS / 32];
    __shared__ double x2r[GF_MAX_LADDER];
    const int b = blockIdx.x;
    LMState& L = a.lm[b];
    const int phase = L.phase;
    const int nr = a.nchan;  // rungs of the trial pass
    if (phase == PH_TRIAL) {
        int b0, b1;
        trial_slots(a, b, b0, b1);
        for (int r = L.rung0; r < nr; ++r) {
            CSum acc = {0.0f, 0.0f};
            for (int k = b0 + threadIdx.x; k < b1; k += RED_THREADS)
                csum_add(acc, a.partial[(long long)k * nr + r]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                CSum other;
                other.s = __shfl_down_sync(kFull, acc.s, o);
                other.c = __shfl_down_sync(kFull, acc.c, o);
                acc = csum_merge(acc, other);
            }
            if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                CSum t = wsum[0];
                for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, wsum[w]);
                x2r[r] = (double)t.s + (double)t.c;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x != 0) return;
    lm_apply_trials(a, L, phase, nr, x2r, active);
}

// The same for batches whose stamps have at most 32 partial slots each: a warp
// per stamp, 8 stamps per CTA.  Lane l holds slot l, and the warp's shuffle
// tree is the block-wide kernel's (whose other warps then add zeros), so the
// chi^2 are the same bits.
__global__ void __launch_bounds__(RED_THREADS) k_final_update_w(PassArgs a, int* active)
{
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (RED_THREADS / 32) + (threadIdx.x >> 5);
    if (b >= a.count) return;  // the whole warp
    LMState& L = a.lm[b];
    const int phase = L.phase;
    const int nr = a.nchan;
    double x2r[GF_MAX_LADDER];
    if (phase == PH_TRIAL) {
        int b0, b1;
        trial_slots(a, b, b0, b1);
        for (int r = L.rung0; r < nr; ++r) {
            CSum acc = {0.0f, 0.0f};
            if (b0 + lane < b1) csum_add(acc, a.partial[(long long)(b0 + lane) * nr + r]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                CSum other;
                other.s = __shfl_down_sync(kFull, acc.s, o);
                other.c = __shfl_down_sync(kFull, acc.c, o);
                acc = csum_merge(acc, other);
            }
            x2r[r] = (double)acc.s + (double)acc.c;
        }
    }
    if (lane != 0) return;
    lm_apply_trials(a, L, phase, nr, x2r, active);
}

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

// The work list of one LM phase: the ids of the stamps in that phase, in
// increasing order, and for each work kind the exclusive prefix sums of their
// blocks (pre[k][i] = blocks of kind k of the listed stamps before the i-th).
// Two coalesced passes over the stamps, 1024 per CTA: k_worklist_count sums each
// CTA's listed stamps and blocks, k_worklist_write adds the earlier CTAs' sums
// and scans its own stamps (warp shuffles, then across warps).
constexpr int WL_THREADS = 1024;
constexpr int WLQ = 1 + WK_KINDS;  // listed stamps, then blocks of each kind

// this thread's stamp: 1 and its blocks of each kind if it is in `phase`
__device__ __forceinline__ void wl_item(int count, const LMState* lm, int phase, const int* pst, int b,
                                        int (&v)[WLQ])
{
    for (int q = 0; q < WLQ; ++q) v[q] = 0;
    if (b < count && lm[b].phase == phase) {
        v[0] = 1;
        for (int k = 0; k < WK_KINDS; ++k) v[1 + k] = pst[k * (count + 1) + b + 1] - pst[k * (count + 1) + b];
    }
}

// block-wide exclusive scan of v (excl) and the block's totals (tot)
__device__ __forceinline__ void wl_block_scan(const int (&v)[WLQ], int (&excl)[WLQ], int (&tot)[WLQ],
                                              int (*wsum)[WLQ])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl[WLQ];
    for (int q = 0; q < WLQ; ++q) {
        int x = v[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += u;
        }
        incl[q] = x;
        if (lane == 31) wsum[warp][q] = x;
    }
    __syncthreads();
    if (warp == 0) {
        for (int q = 0; q < WLQ; ++q) {
            const int x0 = wsum[lane][q];
            int x = x0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += u;
            }
            wsum[lane][q] = x - x0;  // exclusive over warps
            if (lane == 31) wsum[32][q] = x;  // the block's total
        }
    }
    __syncthreads();
    for (int q = 0; q < WLQ; ++q) {
        excl[q] = incl[q] - v[q] + wsum[warp][q];
        tot[q] = wsum[32][q];
    }
}

__global__ void __launch_bounds__(WL_THREADS) k_worklist_count(int count, const LMState* lm, int phase,
                                                               const int* pst, int* blk)
{
    pdl_entry();
    __shared__ int wsum[WL_THREADS / 32 + 1][WLQ];
    int v[WLQ], excl[WLQ], tot[WLQ];
    wl_item(count, lm, phase, pst, blockIdx.x * WL_THREADS + threadIdx.x, v);
    wl_block_scan(v, excl, tot, wsum);
    if (threadIdx.x < WLQ) blk[blockIdx.x * WLQ + threadIdx.x] = tot[threadIdx.x];
}

__global__ void __launch_bounds__(WL_THREADS) k_worklist_write(int count, const LMState* lm, int phase,
                                                               const int* pst, const int* blk, int* n_out,
                                                               int* ids, int* pre)
{
    pdl_entry();
    __shared__ int wsum[WL_THREADS / 32 + 1][WLQ];
    __shared__ int base[WLQ];
    // the earlier CTAs' totals (a warp per quantity)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < WLQ) {
        int x = 0;
        for (int j = lane; j < (int)blockIdx.x; j += 32) x += blk[j * WLQ + warp];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0) base[warp] = x;
    }
    const int b = blockIdx.x * WL_THREADS + threadIdx.x;
    int v[WLQ], excl[WLQ], tot[WLQ];
    wl_item(count, lm, phase, pst, b, v);
    wl_block_scan(v, excl, tot, wsum);  // (its barriers also publish base)
    if (v[0]) {
        const int pos = base[0] + excl[0];
        ids[pos] = b;
        for (int k = 0; k < WK_KINDS; ++k) pre[k * (count + 1) + pos] = base[1 + k] + excl[1 + k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const int n = base[0] + tot[0];
        *n_out = n;
        for (int k = 0; k < WK_KINDS; ++k) pre[k * (count + 1) + n] = base[1 + k] + tot[1 + k];
    }
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The loop's control word before the first body: start time, budget, caps.
__global__ void k_loop_start(LoopCtl* c, unsigned long long budget_ns, int max_bodies)
{
    c->t0 = global_ns();
    c->budget_ns = budget_ns;
    c->bodies = 0;
    c->max_bodies = max_bodies;
    c->cont = 1;
    c->timed_out = 0;
}

// The last kernel of an LM body: counts the body and decides whether another
// one runs -- while k_final_update counted stamps still fitting, fewer than
// max_bodies bodies have run and the time budget is not spent.  When the
// budget has run out, every stamp still fitting stops with GF_ETIMEOUT (its
// last accepted parameters and chi^2 stay) and the active count drops to 0.
// In a CUDA graph the decision sets the WHILE node's condition; otherwise the
// host reads the active count.  One block.
constexpr int CTL_THREADS = 1024;

__global__ void __launch_bounds__(CTL_THREADS) k_loop_ctl(int count, LMState* lm, int* active,
                                                          LoopCtl* c,
                                                          cudaGraphConditionalHandle h,
                                                          int use_handle)
{
    pdl_entry();
    __shared__ int decide;  // 0 stop, 1 run another body, 2 out of time
    if (threadIdx.x == 0) {
        const int bodies = c->bodies + 1;
        c->bodies = bodies;
        const int n = *active;
        int d = (n > 0 && bodies < c->max_bodies) ? 1 : 0;
        if (n > 0 && c->budget_ns != 0ull && global_ns() - c->t0 > c->budget_ns) d = 2;
        decide = d;
    }
    __syncthreads();
    const int d = decide;
    if (d == 2) {
        for (int b = threadIdx.x; b < count; b += CTL_THREADS) {
            LMState& L = lm[b];
            if (L.phase != PH_DONE) {
                L.status = GF_ETIMEOUT;
                L.phase = PH_DONE;
            }
        }
    }
    if (threadIdx.x == 0) {
        if (d == 2) {
            c->timed_out = 1;
            *active = 0;
        }
        c->cont = d == 1;
        if (use_handle) cudaGraphSetConditional(h, d == 1 ? 1u : 0u);
    }
}

inline int warp_blocks(int count) { return (count + kWarpsPerBlock - 1) / kWarpsPerBlock; }

}  // namespace

cudaError_t launch_prep_sum(const PassArgs& a, const double* params, int use_trial,
                            cudaStream_t s)
{
    GF_LAUNCH_PDL(k_prep_sum, dim3(warp_blocks(a.count)), dim3(kWarpsPerBlock * 32), 0, s, a, params, use_trial);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_prep_jac(const PassArgs& a, const double* params, cudaStream_t s)
{
    GF_LAUNCH_PDL(k_prep_jac, dim3(warp_blocks(a.count)), dim3(kWarpsPerBlock * 32), 0, s, a, params);
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

cudaError_t launch_final_solve(const PassArgs& a, Channel* trial_chan, int* active, int nr,
                               cudaStream_t s)
{
    if (nr < 1 || nr > GF_MAX_LADDER) return cudaErrorInvalidValue;
    GF_LAUNCH_PDL(k_final_solve, dim3(a.count), dim3(32 * nr), 0, s, a, trial_chan, active);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_final_update(const PassArgs& a, int* active_count, cudaStream_t s)
{
    if (a.max_trial_slots <= 32) {
        const int per = RED_THREADS / 32;
        GF_LAUNCH_PDL(k_final_update_w, dim3((a.count + per - 1) / per), dim3(RED_THREADS), 0, s, a,
                      active_count);
    } else {
        GF_LAUNCH_PDL(k_final_update, dim3(a.count), dim3(RED_THREADS), 0, s, a, active_count);
    }
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_lm_export(int count, const Structure* S, const LMState* lm, double* out,
                             cudaStream_t s)
{
    k_lm_export<<<(count + 127) / 128, 128, 0, s>>>(count, S, lm, out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

int worklist_blocks(int count) { return (count + WL_THREADS - 1) / WL_THREADS; }

cudaError_t launch_worklist(int count, const LMState* lm, int phase, const int* pre_static,
                            int* n, int* ids, int* pre, int* blk, cudaStream_t s)
{
    const int g = worklist_blocks(count);
    GF_LAUNCH_PDL(k_worklist_count, dim3(g), dim3(WL_THREADS), 0, s, count, lm, phase, pre_static, blk);
    GF_COUNT_LAUNCH();
    GF_LAUNCH_PDL(k_worklist_write, dim3(g), dim3(WL_THREADS), 0, s, count, lm, phase, pre_static, blk, n,
                  ids, pre);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_loop_start(LoopCtl* c, unsigned long long budget_ns, int max_bodies,
                              cudaStream_t s)
{
    k_loop_start<<<1, 1, 0, s>>>(c, budget_ns, max_bodies);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_loop_ctl(int count, LMState* lm, int* active, LoopCtl* c,
                            cudaGraphConditionalHandle h, int use_handle, cudaStream_t s)
{
    GF_LAUNCH_PDL(k_loop_ctl, dim3(1), dim3(CTL_THREADS), 0, s, count, lm, active, c, h,
                  use_handle);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_bn_table(cudaStream_t s)
{
    k_bn_table<<<(BN_TAB * 32 + 255) / 256, 256, 0, s>>>();
    GF_COUNT_LAUNCH();
    k_bn_ready<<<1, 1, 0, s>>>();
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}
