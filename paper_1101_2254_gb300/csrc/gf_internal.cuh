// gf_internal.cuh -- device-side data structures and the per-pixel profile
// evaluation shared by the kernels of libgf.so.
//
// Layout of the work: a call processes a batch of stamps (a single-stamp call is
// a batch of one).  Each stamp carries up to GF_MAX_CHAN "channels": an image on
// the halo-extended grid that the convolution turns into one column of the
// Jacobian or into the model.  Channel kinds:
//   CH_SUM    sky + all components at one parameter vector (the model, step 1)
//   CH_SHAPE  component k with unit amplitude (exact amplitude column)
//   CH_FD     amp_k (S_k(p + h e_s) - S_k(p)) / h for a nonlinear slot s
//   CH_DERIV  amp_k dS_k/dp_s, the analytic derivative for a nonlinear slot s
//   CH_PLANE  x - x_c or y - y_c, a sky plane's slope basis (its exact column)
// Convolved channels are combined per pixel into the model
//   m = sum_ch mweight_ch * Y_ch + sky_const
// and the Jacobian columns; chi^2 and J^T W J, J^T W r are reduced from there.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/gf.h"

#define GF_MAX_CHAN 24
#define GF_NACC_MAX (GF_MAX_FREE * (GF_MAX_FREE + 1) / 2 + GF_MAX_FREE + 1)

enum { CH_SUM = 0, CH_SHAPE = 1, CH_FD = 2, CH_DERIV = 3, CH_PLANE = 4 };

// LM phases of a stamp
enum { PH_NEED_JAC = 0, PH_SOLVE = 1, PH_TRIAL = 2, PH_DONE = 3, PH_NONE = 99 };

// slot roles
enum { R_POS = 0, R_AMP = 1, R_RAD = 2, R_N = 3, R_Q = 4, R_PA = 5, R_BOXY = 6, R_SKY = 7, R_BETA = 8,
       R_RT = 9, R_KALPHA = 10, R_NALPHA = 11, R_NBETA = 12, R_NGAMMA = 13, R_TILTX = 14,
       R_TILTY = 15, R_FAMP = 16, R_FPHI = 17 };

// a Sersic profile (plain or with Fourier modes): b_n from slot 4
__host__ __device__ __forceinline__ bool is_sersic_kind(int kind)
{
    return kind == GF_SERSIC || kind == GF_SERSIC_F;
}

// the constant sky and the sky plane enter the model as a term on the grid,
// not as a profile
__host__ __device__ __forceinline__ bool is_sky_kind(int kind)
{
    return kind == GF_SKY || kind == GF_SKY_PLANE;
}

// slots of a component of kind `kind` (-1 for an unknown kind)
__host__ __device__ __forceinline__ int comp_nslots(int kind)
{
    switch (kind) {
    case GF_SERSIC: return 8;
    case GF_EXPDISK: return 7;
    case GF_SKY: return 1;
    case GF_GAUSSIAN: return 7;
    case GF_MOFFAT: return 8;
    case GF_KING: return 9;
    case GF_NUKER: return 10;
    case GF_PSF: return 3;
    case GF_SKY_PLANE: return 3;
    case GF_SERSIC_F: return 14;
    default: return -1;
    }
}
#define GF_COMP_MAXSLOTS 14

// Float32 constants of one component at one parameter vector.
struct __align__(16) CompConst {  // 112 bytes; aligned so that field loads combine
    float x0h, x0l, y0h, y0l;  // centre split hi + lo so that x - x0 keeps ~48 bits
    float cs, sn, invq;        // rotation and axis ratio
    float C, invC;             // generalised-radius exponent C = c + 2
    float amp;                 // amplitude (1 for unit shapes)
    float invr;                // 1 / r_e, 1 / r_s, 1 / s (Gaussian), 1 / alpha (Moffat)
    float invn;                // 1 / n (1 for the disk); beta for a Moffat
    float b0, b;               // I = amp * exp(b0 - b * (r invr)^invn); Moffat:
                               // amp * exp(-b log2(1 + (r invr)^2)), b = beta ln 2
    int kind;                  // GF_SERSIC / GF_EXPDISK / GF_SKY / GF_GAUSSIAN / GF_MOFFAT /
                               // GF_KING / GF_NUKER / GF_PSF
    int ellipse;               // C == 2 exactly: r by sqrt
    float e0, e1, e2, e3;      // King: 1/alpha, w_t, 1/(1 - w_t) (invn = alpha, invr = 1/r_c);
                               // Nuker: gamma, (beta-gamma)/alpha, (gamma-beta)/alpha
                               // (invn = alpha, invr = 1/r_b);
    float e4, e5, e6, e7, e8;  // Sersic + Fourier modes: a_1, a_3, a_4 in e0..e2, then
                               // cos phi_1 (e3), sin phi_1, cos 3 phi_3, sin 3 phi_3,
                               // cos 4 phi_4, sin 4 phi_4 (e4..e8)
    int pad_c[3];
};
static_assert(sizeof(CompConst) == 112, "CompConst layout");

struct Channel {
    int type;       // CH_*
    int comp;       // component index (CH_SHAPE, CH_FD)
    int jcol;       // Jacobian column or -1
    float mweight;  // weight of the convolved channel in the model
    float scale;    // CH_FD: amp / h_eff
    float sky;      // CH_SUM: sky level added on the grid
    int ncomp;
    float msky;     // channel 0 of a pass: constant added to the convolved model
    int dslot;      // CH_DERIV: the slot's index inside its component; CH_PLANE: 0 x, 1 y
    float dbdn;     // CH_DERIV of a Sersic component: db_n/dn at its n
    float pxc, pyc; // the stamp centre, origin of a sky plane (CH_SUM, CH_PLANE)
    float tgx, tgy; // CH_SUM: the sky plane's slopes (0 without a plane)
    int pad_[2];
    CompConst cc[GF_MAX_COMP];  // all components at the channel's parameter vector
    CompConst pert;             // CH_FD: component `comp` at p + h e_s (unit amplitude)
};

// Static description of one stamp inside a call.
struct StampInfo {
    int H, W, P, c;
    int He, We;
    int os_factor, os_box, os_x0, os_y0;  // block origin resolved
    int nchan;                             // channels of the Jacobian pass
    int conv_tw;                           // direct-convolution tile width (64 or 32)
    int wb_off;                            // first slot of the stamp's 16 x 32 output blocks
                                           // (ceil(H/16) x ceil(W/32), row-major) in a call
    long long pix_off;   // into image / sigma / model (H*W elements)
    long long psf_off;   // into the PSF array (P*P)
    long long ext1_off;  // sum of He*We over the earlier stamps
    long long y1_off;    // sum of H*W over the earlier stamps
};

// channel k of stamp b in a pass of nchan channels per stamp
__host__ __device__ __forceinline__ long long ext_index(const StampInfo& st, int nchan, int k)
{
    return (long long)nchan * st.ext1_off + (long long)k * st.He * st.We;
}
__host__ __device__ __forceinline__ long long y_index(const StampInfo& st, int nchan, int k)
{
    return (long long)nchan * st.y1_off + (long long)k * st.H * st.W;
}

// Structure shared by all stamps of a call (kinds, free slots, bounds, options).
struct Structure {
    int ncomp, nslots, nfree, nprofile;
    int kinds[GF_MAX_COMP];
    int slot0[GF_MAX_COMP];         // first slot of each component
    int freeslot[GF_MAX_FREE];      // slot index of each free parameter
    int role[GF_MAX_SLOTS];         // R_* per slot
    int owner[GF_MAX_SLOTS];        // component per slot
    int sky_slot;                   // -1 if no sky component
    int sky_jcol;                   // Jacobian column of the sky, -1 if held
    int tilt_slot[2];               // the sky plane's slope slots (x, y), -1 without a plane
    int tilt_jcol[2];               // their Jacobian columns, -1 if held
    int nplane;                     // 2 with a sky plane (its two slope channels), else 0
    int nchan;                      // Jacobian-pass channels per stamp
    int nacc;                       // accumulators of the Jacobian reduction
    double lo[GF_MAX_SLOTS], hi[GF_MAX_SLOTS];
    gf_lm_opts opts;
};

// Outcome of the damped solve of one rung of the trial ladder (see lm.cu)
enum { RUNG_FAIL = 0, RUNG_SMALL = 1, RUNG_TRIAL = 2 };

// Per-stamp LM state, resident on the device for the whole fit.  Rung r of the
// trial ladder is the step for lambda * up^r: its trial parameters pt[r], the
// chi^2 fall its linearised model predicts, and the outcome of its solve.
struct LMState {
    double p[GF_MAX_SLOTS];
    double pt[GF_MAX_LADDER][GF_MAX_SLOTS];
    double A[GF_MAX_FREE * GF_MAX_FREE];
    double g[GF_MAX_FREE];
    double chi2, chi2t, lambda;
    double pred[GF_MAX_LADDER];
    double bn_n[GF_MAX_COMP], bn_b[GF_MAX_COMP];  // last (n, b_n) per component: Newton start
    int rung[GF_MAX_LADDER];  // RUNG_* per rung
    int rung0;                // first rung the trial pass decides (earlier ones were settled)
    int iters, accepted, status, phase;
};

// Control word of a batched LM loop run on the device (see k_loop_ctl).
struct LoopCtl {
    unsigned long long t0;         // global timer at the start of the loop (ns)
    unsigned long long budget_ns;  // 0 = no time budget
    int bodies;                    // loop bodies run so far
    int max_bodies;
    int cont;                      // the last body's decision: run another body
    int timed_out;                 // the budget ran out (stamps set to GF_ETIMEOUT)
};

// ------------------------------------------------------------ device helpers

// Cubic-convolution weight of Keys (1981), a = -1/2, at offset x
__device__ __forceinline__ float keys_w(float x)
{
    const float a = fabsf(x);
    if (a <= 1.0f) return fmaf(fmaf(1.5f, a, -2.5f), a * a, 1.0f);
    if (a < 2.0f) return fmaf(fmaf(fmaf(-0.5f, a, 2.5f), a, -4.0f), a, 2.0f);
    return 0.0f;
}

// The further families (King, Nuker, point source) at grid point (xi + ox, yi + oy).
static __device__ __noinline__ float comp_eval_ext(const CompConst& k, float xi, float yi, float ox,
                                            float oy)
{
    if (k.kind == GF_SERSIC_F) {
        // the Sersic of the distorted radius r g(t), g = 1 + sum_m a_m cos m(t - phi_m),
        // t the angle of (x', y'/q): cos and sin of t from the coordinates, of
        // 3t and 4t by the multiple-angle identities
        const float dx = (xi - k.x0h) + (ox - k.x0l);
        const float dy = (yi - k.y0h) + (oy - k.y0l);
        const float xp = fmaf(dx, k.cs, dy * k.sn);
        const float yp = fmaf(dy, k.cs, -dx * k.sn) * k.invq;
        float r;
        if (k.ellipse) {
            r = sqrtf(fmaf(xp, xp, yp * yp));
        } else {
            const float ax = exp2f(k.C * log2f(fabsf(xp)));
            const float ay = exp2f(k.C * log2f(fabsf(yp)));
            r = exp2f(k.invC * log2f(ax + ay));
        }
        const float rho2 = fmaf(xp, xp, yp * yp);
        const float ir = rho2 > 0.0f ? rsqrtf(rho2) : 0.0f;
        const float c = rho2 > 0.0f ? xp * ir : 1.0f, s = yp * ir;
        const float c2 = c * c, s2 = s * s;
        const float c3 = c * fmaf(4.0f, c2, -3.0f), s3 = s * fmaf(-4.0f, s2, 3.0f);
        const float c4 = fmaf(8.0f * c2, c2 - 1.0f, 1.0f), s4 = 4.0f * s * c * fmaf(2.0f, c2, -1.0f);
        float g = 1.0f;
        g = fmaf(k.e0, fmaf(c, k.e3, s * k.e4), g);
        g = fmaf(k.e1, fmaf(c3, k.e5, s3 * k.e6), g);
        g = fmaf(k.e2, fmaf(c4, k.e7, s4 * k.e8), g);
        const float t = r * g * k.invr;
        const float u = exp2f(k.invn * log2f(t));
        return k.amp * expf(fmaf(-k.b, u, k.b0));
    }
    if (k.kind == GF_PSF) {
        // a point source keeps its pixel-centre weights (it is not sampled)
        const float dx = (xi - k.x0h) - k.x0l, dy = (yi - k.y0h) - k.y0l;
        return k.amp * keys_w(dx) * keys_w(dy);
    }
    const float dx = (xi - k.x0h) + (ox - k.x0l);
    const float dy = (yi - k.y0h) + (oy - k.y0l);
    const float xp = fmaf(dx, k.cs, dy * k.sn);
    const float yp = fmaf(dy, k.cs, -dx * k.sn) * k.invq;
    float r;
    if (k.ellipse) {
        r = sqrtf(fmaf(xp, xp, yp * yp));
    } else {
        const float ax = exp2f(k.C * log2f(fabsf(xp)));
        const float ay = exp2f(k.C * log2f(fabsf(yp)));
        r = exp2f(k.invC * log2f(ax + ay));
    }
    const float t = r * k.invr;
    if (k.kind == GF_KING) {
        // w = (1 + t^2)^(-1/alpha); I = amp ((w - w_t) / (1 - w_t))^alpha, 0 from r_t out
        const float w = exp2f(-k.e0 * log2f(fmaf(t, t, 1.0f)));
        const float z = (w - k.e1) * k.e2;
        return z > 0.0f ? k.amp * exp2f(k.invn * log2f(z)) : 0.0f;
    }
    // Nuker: log2(I / amp) = (beta-gamma)/alpha - gamma log2 t
    //                        + (gamma-beta)/alpha log2(1 + t^alpha)
    const float lt = log2f(fmaxf(t, 1e-6f));
    const float at = k.invn * lt;
    const float l1p = at > 30.0f ? at : log2f(1.0f + exp2f(at));  // log2(1 + 2^at)
    return k.amp * exp2f(fmaf(k.e2, l1p, fmaf(-k.e0, lt, k.e1)));
}

// EV, the evaluator variant of the call: 0 Sersic, disk and Gaussian only;
// 1 with a Moffat (one more log and selects per sample); 2 with King, Nuker or
// point-source components (those take comp_eval_ext).  The kernels are
// compiled for each, so that calls without the longer forms keep the shorter
// evaluator.
// comp_eval's arithmetic in three steps (the same operations in the same
// order, so the same floats), for a Jacobian pass that reuses the first ones
// for a finite-difference channel whose perturbed slot enters only later:
//   the generalised radius r from the pixel, centre, rotation and axis ratio;
//   log2 t for t = r / r_e (log2(1 + t^2) for a Moffat);
//   the profile from t and that logarithm.
// comp_eval (below) keeps its one-piece form, which compiles to fewer
// registers in the one-channel passes.
template <int EV>
__device__ __forceinline__ float comp_radius(const CompConst& k, float xi, float yi, float ox,
                                             float oy)
{
    // dx = x - x0 with x = xi + ox: the integer part against the hi word is exact
    // near the centre (Sterbenz), the sub-pixel offset absorbs the lo word.
    float dx = (xi - k.x0h) + (ox - k.x0l);
    float dy = (yi - k.y0h) + (oy - k.y0l);
    float xp = fmaf(dx, k.cs, dy * k.sn);
    float yp = fmaf(dy, k.cs, -dx * k.sn) * k.invq;
    float r;
    if (k.ellipse) {
        r = sqrtf(fmaf(xp, xp, yp * yp));
    } else {
        float ax = exp2f(k.C * log2f(fabsf(xp)));
        float ay = exp2f(k.C * log2f(fabsf(yp)));
        r = exp2f(k.invC * log2f(ax + ay));
    }
    return r;
}

template <int EV>
__device__ __forceinline__ float comp_log_t(const CompConst& k, float t)
{
    if (EV >= 1) {
        const bool moffat = k.kind == GF_MOFFAT;
        return log2f(moffat ? fmaf(t, t, 1.0f) : t);
    }
    return log2f(t);
}

template <int EV>
__device__ __forceinline__ float comp_tail(const CompConst& k, float t, float lt)
{
    float u;
    if (EV >= 1) {
        // one logarithm for every kind: log2 t (Sersic, Gaussian) or
        // log2(1 + t^2) (Moffat), chosen by selects so the loop body stays
        // branch-free
        const bool moffat = k.kind == GF_MOFFAT;
        u = (k.invn == 1.0f) ? t : exp2f(k.invn * lt);
        u = moffat ? lt : u;
    } else {
        u = (k.invn == 1.0f) ? t : exp2f(k.invn * lt);
    }
    return k.amp * expf(fmaf(-k.b, u, k.b0));
}

template <int EV>
__device__ __forceinline__ float comp_eval(const CompConst& k, float xi, float yi, float ox,
                                           float oy)
{
    if (EV == 2 && k.kind >= GF_KING) return comp_eval_ext(k, xi, yi, ox, oy);
    // dx = x - x0 with x = xi + ox: the integer part against the hi word is exact
    // near the centre (Sterbenz), the sub-pixel offset absorbs the lo word.
    float dx = (xi - k.x0h) + (ox - k.x0l);
    float dy = (yi - k.y0h) + (oy - k.y0l);
    float xp = fmaf(dx, k.cs, dy * k.sn);
    float yp = fmaf(dy, k.cs, -dx * k.sn) * k.invq;
    float r;
    if (k.ellipse) {
        r = sqrtf(fmaf(xp, xp, yp * yp));
    } else {
        float ax = exp2f(k.C * log2f(fabsf(xp)));
        float ay = exp2f(k.C * log2f(fabsf(yp)));
        r = exp2f(k.invC * log2f(ax + ay));
    }
    float t = r * k.invr;
    float u;
    if (EV >= 1) {
        // one logarithm for every kind: log2 t (Sersic, Gaussian) or
        // log2(1 + t^2) (Moffat), chosen by selects so the loop body stays
        // branch-free
        const bool moffat = k.kind == GF_MOFFAT;
        const float lt = log2f(moffat ? fmaf(t, t, 1.0f) : t);
        u = (k.invn == 1.0f) ? t : exp2f(k.invn * lt);
        u = moffat ? lt : u;
    } else {
        u = (k.invn == 1.0f) ? t : exp2f(k.invn * log2f(t));
    }
    return k.amp * expf(fmaf(-k.b, u, k.b0));
}

// A component evaluated once per pixel in a Jacobian pass, with the radius,
// t and log2 t its finite-difference channels may reuse
struct EvalCursor {
    int comp;        // the component held (-1: none yet)
    float v, r, t, lt;
};

template <int EV>
__device__ __forceinline__ void comp_eval_keep(const CompConst& k, float xi, float yi, float ox,
                                               float oy, EvalCursor& e)
{
    if (EV == 2 && k.kind >= GF_KING) {
        e.v = comp_eval_ext(k, xi, yi, ox, oy);
        return;
    }
    e.r = comp_radius<EV>(k, xi, yi, ox, oy);
    e.t = e.r * k.invr;
    e.lt = comp_log_t<EV>(k, e.t);
    e.v = comp_tail<EV>(k, e.t, e.lt);
}

// What a finite-difference channel's perturbed component shares with the
// component at p (the same floats, so the reused steps give the values a full
// evaluation gives): 2 radius and r_e (only the profile's tail differs: n,
// beta, b_n), 1 the radius (r_e too differs), 0 nothing reused.
__device__ __forceinline__ int fd_reuse_level(const CompConst& k, const CompConst& p)
{
    if (is_sky_kind(k.kind) || k.kind != p.kind || k.kind >= GF_KING) return 0;
    auto same = [](float u, float v) { return __float_as_int(u) == __float_as_int(v); };
    // the radius's inputs
    if (!(same(k.x0h, p.x0h) && same(k.x0l, p.x0l) && same(k.y0h, p.y0h) && same(k.y0l, p.y0l) &&
          same(k.cs, p.cs) && same(k.sn, p.sn) && same(k.invq, p.invq) && same(k.C, p.C) &&
          same(k.invC, p.invC) && k.ellipse == p.ellipse))
        return 0;
    return __float_as_int(k.invr) == __float_as_int(p.invr) ? 2 : 1;
}

// The unit-amplitude profile of component k at grid point (xi + ox, yi + oy)
// and its derivatives with respect to the component's slots, in slot order
// (Sersic: x0, y0, amplitude, r_e, n, q, pa, c; Moffat: the same with alpha
// and beta for r_e and n; disk and Gaussian: x0, y0, amplitude, r_s or fwhm, q,
// pa, c), by the chain rule through the generalised radius:
//   r^C = |x'|^C + |Y|^C, Y = y'/q:  dr/dx' = sgn(x') (|x'|/r)^(C-1), likewise Y,
//     dr/dC = r [ (|x'|^C ln|x'| + |Y|^C ln|Y|) / (C r^C) - ln(r^C) / C^2 ];
//   dx'/dx0 = -cos, dx'/dy0 = -sin, dy'/dx0 = sin, dy'/dy0 = -cos,
//   dx'/dth = y', dy'/dth = -x', dY/dq = -Y/q;
//   S = exp(b0 - b u), u = (r/r_e)^(1/n):  dS/dr = -b S u / (n r),
//     dS/dr_e = b S u / (n r_e), dS/dn = S ((1 - u) db/dn + b u ln(r/r_e) / n^2)
// (the disk is the case b = 1, b0 = 0, n = 1; the Gaussian b = 1/2, b0 = 0, n = 1/2
// with the radius s = fwhm / (2 sqrt(2 ln 2))).  Float32 throughout, like the
// pixel path; the derivative channels carry no finite-difference step noise.
// At r = 0 (a sample exactly on the centre) the geometric derivatives are 0.
__device__ __forceinline__ float comp_grad(const CompConst& k, float xi, float yi, float ox,
                                           float oy, float dbdn, float (&g)[8])
{
    const float dx = (xi - k.x0h) + (ox - k.x0l);
    const float dy = (yi - k.y0h) + (oy - k.y0l);
    const float xp = fmaf(dx, k.cs, dy * k.sn);
    const float yp = fmaf(dy, k.cs, -dx * k.sn);
    const float Y = yp * k.invq;
    float r, drdx, drdY, drdC;
    if (k.ellipse) {
        const float S2 = fmaf(xp, xp, Y * Y);
        r = sqrtf(S2);
        const float ir = r > 0.0f ? 1.0f / r : 0.0f;
        drdx = xp * ir;
        drdY = Y * ir;
        // C = 2: r [ (x'^2 ln|x'| + Y^2 ln|Y|) / (2 r^2) - ln(r^2) / 4 ]
        const float lx = xp != 0.0f ? xp * xp * logf(fabsf(xp)) : 0.0f;
        const float ly = Y != 0.0f ? Y * Y * logf(fabsf(Y)) : 0.0f;
        drdC = r > 0.0f ? r * ((lx + ly) * (0.5f * ir * ir) - 0.5f * logf(r)) : 0.0f;
    } else {
        const float l2x = log2f(fabsf(xp)), l2y = log2f(fabsf(Y));
        const float ax = exp2f(k.C * l2x), ay = exp2f(k.C * l2y);
        const float S = ax + ay;
        const float l2S = log2f(S);
        const float l2r = k.invC * l2S;
        r = exp2f(l2r);
        const float cm1 = k.C - 1.0f;
        drdx = xp != 0.0f ? copysignf(exp2f(cm1 * (l2x - l2r)), xp) : 0.0f;
        drdY = Y != 0.0f ? copysignf(exp2f(cm1 * (l2y - l2r)), Y) : 0.0f;
        const float ln2 = 0.69314718055994531f;
        const float lx = ax > 0.0f ? ax * l2x : 0.0f, ly = ay > 0.0f ? ay * l2y : 0.0f;
        drdC = r > 0.0f ? r * ln2 * ((lx + ly) / (k.C * S) - l2S * k.invC * k.invC) : 0.0f;
    }
    const float t = r * k.invr;
    float Sv, dSdr, g3, g4 = 0.0f;
    if (k.kind == GF_MOFFAT) {
        // S = w^-beta, w = 1 + t^2:  dS/dr = -2 beta S t / (alpha w),
        // dS/dalpha = 2 beta S t^2 / (alpha w) (the channel scale carries
        // alpha / fwhm), dS/dbeta = S (-ln w + 2 beta t^2 / w * dbdn) with dbdn
        // standing for d ln(alpha / fwhm) / d beta
        const float beta = k.invn, w = fmaf(t, t, 1.0f), iw = 1.0f / w, l2w = log2f(w);
        Sv = expf(-k.b * l2w);
        const float s2 = 2.0f * beta * Sv * t * iw * k.invr;
        dSdr = -s2;
        g3 = s2 * t;
        g4 = Sv * fmaf(2.0f * beta * t * t * iw, dbdn, -0.69314718055994531f * l2w);
    } else {
        const float u = (k.invn == 1.0f) ? t : exp2f(k.invn * log2f(t));
        Sv = expf(fmaf(-k.b, u, k.b0));
        dSdr = r > 0.0f ? -k.b * Sv * u * k.invn / r : 0.0f;
        g3 = k.b * Sv * u * k.invn * k.invr;  // with respect to 1/invr (r_e, r_s, or s)
        if (k.kind == GF_GAUSSIAN) g3 *= 0.42466090014400952f;  // s = fwhm / (2 sqrt(2 ln 2))
        if (k.kind == GF_SERSIC) {
            const float lt = r > 0.0f ? logf(t) : 0.0f;
            g4 = Sv * fmaf(1.0f - u, dbdn, k.b * u * lt * k.invn * k.invn);
        }
    }
    g[0] = dSdr * fmaf(drdx, -k.cs, drdY * (k.sn * k.invq));
    g[1] = dSdr * fmaf(drdx, -k.sn, drdY * (-k.cs * k.invq));
    g[2] = Sv;
    g[3] = g3;
    const float dq = dSdr * drdY * (-Y * k.invq);
    const float dpa = dSdr * fmaf(drdx, yp, drdY * (-xp * k.invq)) * 0.017453292519943295f;
    const float dc = dSdr * drdC;
    if (k.kind == GF_SERSIC || k.kind == GF_MOFFAT) {  // slot 4 is n or beta
        g[4] = g4;
        g[5] = dq;
        g[6] = dpa;
        g[7] = dc;
    } else {
        g[4] = dq;
        g[5] = dpa;
        g[6] = dc;
        g[7] = 0.0f;
    }
    return Sv;
}

// g[i] for a runtime i, by selects (the array stays in registers)
__device__ __forceinline__ float grad_pick(const float (&g)[8], int i)
{
    float v = g[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) v = (i == q) ? g[q] : v;
    return v;
}

// value of a channel at grid point (xi + ox, yi + oy)
template <int EV>
__device__ __forceinline__ float channel_value(const Channel& ch, float xi, float yi, float ox,
                                               float oy)
{
    if (ch.type == CH_DERIV) {
        float g[8];
        comp_grad(ch.cc[ch.comp], xi, yi, ox, oy, ch.dbdn, g);
        return grad_pick(g, ch.dslot) * ch.scale;
    }
    if (ch.type == CH_SUM) {
        // the sky (constant and plane, at the pixel centre), then the profiles
        float v = fmaf(ch.tgy, yi - ch.pyc, fmaf(ch.tgx, xi - ch.pxc, ch.sky));
        for (int k = 0; k < ch.ncomp; ++k)
            if (!is_sky_kind(ch.cc[k].kind)) v += comp_eval<EV>(ch.cc[k], xi, yi, ox, oy);
        return v;
    }
    if (ch.type == CH_PLANE) return ch.dslot == 0 ? xi - ch.pxc : yi - ch.pyc;
    if (ch.type == CH_SHAPE) return comp_eval<EV>(ch.cc[ch.comp], xi, yi, ox, oy);
    float a = comp_eval<EV>(ch.pert, xi, yi, ox, oy);
    float b = comp_eval<EV>(ch.cc[ch.comp], xi, yi, ox, oy);
    return (a - b) * ch.scale;
}

// comp_eval at two points, the two evaluations' steps interleaved (two
// independent dependency chains for the scheduler); each value is the float
// comp_eval gives for its point.
template <int EV>
__device__ __forceinline__ void comp_eval2(const CompConst& k, float x0, float y0, float x1,
                                           float y1, float& v0, float& v1)
{
    if (EV == 2 && k.kind >= GF_KING) {
        v0 = comp_eval_ext(k, x0, y0, 0.0f, 0.0f);
        v1 = comp_eval_ext(k, x1, y1, 0.0f, 0.0f);
        return;
    }
    const float dx0 = (x0 - k.x0h) + (0.0f - k.x0l), dy0 = (y0 - k.y0h) + (0.0f - k.y0l);
    const float dx1 = (x1 - k.x0h) + (0.0f - k.x0l), dy1 = (y1 - k.y0h) + (0.0f - k.y0l);
    const float xp0 = fmaf(dx0, k.cs, dy0 * k.sn), xp1 = fmaf(dx1, k.cs, dy1 * k.sn);
    const float yp0 = fmaf(dy0, k.cs, -dx0 * k.sn) * k.invq;
    const float yp1 = fmaf(dy1, k.cs, -dx1 * k.sn) * k.invq;
    float r0, r1;
    if (k.ellipse) {
        r0 = sqrtf(fmaf(xp0, xp0, yp0 * yp0));
        r1 = sqrtf(fmaf(xp1, xp1, yp1 * yp1));
    } else {
        const float ax0 = exp2f(k.C * log2f(fabsf(xp0))), ax1 = exp2f(k.C * log2f(fabsf(xp1)));
        const float ay0 = exp2f(k.C * log2f(fabsf(yp0))), ay1 = exp2f(k.C * log2f(fabsf(yp1)));
        r0 = exp2f(k.invC * log2f(ax0 + ay0));
        r1 = exp2f(k.invC * log2f(ax1 + ay1));
    }
    const float t0 = r0 * k.invr, t1 = r1 * k.invr;
    float u0, u1;
    if (EV >= 1) {
        const bool moffat = k.kind == GF_MOFFAT;
        const float lt0 = log2f(moffat ? fmaf(t0, t0, 1.0f) : t0);
        const float lt1 = log2f(moffat ? fmaf(t1, t1, 1.0f) : t1);
        u0 = (k.invn == 1.0f) ? t0 : exp2f(k.invn * lt0);
        u1 = (k.invn == 1.0f) ? t1 : exp2f(k.invn * lt1);
        u0 = moffat ? lt0 : u0;
        u1 = moffat ? lt1 : u1;
    } else {
        u0 = (k.invn == 1.0f) ? t0 : exp2f(k.invn * log2f(t0));
        u1 = (k.invn == 1.0f) ? t1 : exp2f(k.invn * log2f(t1));
    }
    v0 = k.amp * expf(fmaf(-k.b, u0, k.b0));
    v1 = k.amp * expf(fmaf(-k.b, u1, k.b0));
}

// channel_value at two pixel centres (ox = oy = 0)
template <int EV>
__device__ __forceinline__ void channel_value2(const Channel& ch, float x0, float y0, float x1,
                                               float y1, float& v0, float& v1)
{
    if (ch.type != CH_SUM) {
        v0 = channel_value<EV>(ch, x0, y0, 0.0f, 0.0f);
        v1 = channel_value<EV>(ch, x1, y1, 0.0f, 0.0f);
        return;
    }
    v0 = fmaf(ch.tgy, y0 - ch.pyc, fmaf(ch.tgx, x0 - ch.pxc, ch.sky));
    v1 = fmaf(ch.tgy, y1 - ch.pyc, fmaf(ch.tgx, x1 - ch.pxc, ch.sky));
    for (int k = 0; k < ch.ncomp; ++k)
        if (!is_sky_kind(ch.cc[k].kind)) {
            float a0, a1;
            comp_eval2<EV>(ch.cc[k], x0, y0, x1, y1, a0, a1);
            v0 += a0;
            v1 += a1;
        }
}

// Neumaier compensated accumulation in float32
struct CSum {
    float s, c;
};
__device__ __forceinline__ void csum_add(CSum& a, float t)
{
    float s = a.s + t;
    if (fabsf(a.s) >= fabsf(t))
        a.c += (a.s - s) + t;
    else
        a.c += (t - s) + a.s;
    a.s = s;
}
// merge two compensated sums (error-free TwoSum of the heads)
__device__ __forceinline__ CSum csum_merge(CSum a, CSum b)
{
    float s = a.s + b.s;
    float bb = s - a.s;
    float err = (a.s - (s - bb)) + (b.s - bb);
    CSum r;
    r.s = s;
    r.c = a.c + b.c + err;
    return r;
}

// decode accumulator index t into (kind, i, j): 0 = A_ij (i <= j), 1 = g_i, 2 = chi^2
__host__ __device__ __forceinline__ int decode_acc(int t, int nf, int& i, int& j)
{
    const int npair = nf * (nf + 1) / 2;
    if (t < npair) {
        int row = 0, rem = t;
        while (rem >= nf - row) {
            rem -= nf - row;
            ++row;
        }
        i = row;
        j = row + rem;
        return 0;
    }
    if (t < npair + nf) {
        i = t - npair;
        j = 0;
        return 1;
    }
    i = j = 0;
    return 2;
}

// stamp index of a block from an exclusive prefix table (upper_bound - 1)
__device__ __forceinline__ int find_stamp(const int* prefix, int count, int blk)
{
    int lo = 0, hi = count;  // prefix[lo] <= blk < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= blk)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ work lists
// Kernel kinds with per-stamp block counts.
// work-item kinds; the direct convolution has one kind per tile width
// (WK_CONV: 32 x 64 tiles, WK_CONV32: 32 x 32 tiles; each stamp uses one)
enum { WK_MODEL = 0, WK_OS = 1, WK_CONV = 2, WK_RED = 3, WK_CONV32 = 4, WK_KINDS = 5 };

// The stamps taking part in a pass (all stamps, or those in the pass's LM
// phase), in stamp order, and per kernel kind the exclusive prefix sums of
// their blocks.  Pass kernels are persistent: each CTA walks one contiguous
// range of the work items (the listed stamps' blocks), so stamps that are done
// cost nothing and a CTA's consecutive items mostly share a stamp and channel.
struct WorkList {
    const int* n;    // [1] number of listed stamps
    const int* ids;  // [count] listed stamp ids
    const int* pre;  // [WK_KINDS][count + 1]
};

// listed index of block `blk`: a short forward walk from the CTA's previous
// position (its items increase), else a binary search
__device__ __forceinline__ int wl_locate(const int* pre, int n, int blk, int& hint)
{
    int i = hint;
    if (i >= 0 && i < n && pre[i] <= blk) {
        for (int step = 0; step < 4; ++step) {
            if (i + 1 >= n || pre[i + 1] > blk) {
                hint = i;
                return i;
            }
            ++i;
        }
    }
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= blk)
            lo = mid;
        else
            hi = mid;
    }
    hint = lo;
    return lo;
}

// ---------------------------------------------------------- host-side launch
// Arguments of the kernel passes; each .cu file implements its own launcher.

struct PassArgs {
    int count;                 // stamps
    const StampInfo* st;       // [count]
    const Structure* S;        // one
    LMState* lm;               // [count] or null (no phase filtering)
    int phase;                 // process stamps whose lm->phase == phase (if lm)
    const Channel* chan;       // [count * chan_stride]
    int chan_stride;           // channels reserved per stamp
    int nchan;                 // channels processed per stamp in this pass
    int jac_pass;              // the channels are a Jacobian pass's (shapes, then FD channels
                               // of the same components); else independent models
    int jac_analytic;          // the Jacobian pass's nonlinear columns are CH_DERIV channels
    int eval_variant;          // 0 Sersic/disk/Gaussian, 1 with Moffat, 2 with King/Nuker/point
    int os_ns;                 // sub-samples per oversampled pixel (os_factor^2)
    int conv_ty;               // direct-convolution tile height (32 or 16)
    int max_trial_slots;       // most trial-pass partial slots of one stamp (reduce blocks, or
                               // 16 x 32 output blocks with conv_chi2)
    int conv_chi2;             // an LM trial pass on the direct path or the one-CTA FFT: the
                               // convolution writes the chi^2 partial of each 16 x 32 output
                               // block per rung (channel), slot st.wb_off + block, instead of
                               // the convolved tile
    float* ext;                // channel grids: ext + ext_index(st[b], nchan, k)
    float* y;                  // convolved channels: y + y_index(st[b], nchan, k)
    const float* psf;
    const float* psf_sum;      // [count] sum of each PSF (float)
    const float* img;
    const float* sig;
    float* partial;            // reduction partials
    int nacc;                  // accumulators per reduce block
    float* J_out;              // optional Jacobian output (nfree x H x W per stamp, packed)
    float* m_out;              // optional model output (H x W per stamp, packed at pix_off)
    WorkList wl;               // the stamps taking part in this pass
    const int* pre_static;     // [WK_KINDS][count + 1] block prefixes over all stamps
    int max_red;               // most reduction blocks of one stamp
    int grid[WK_KINDS];        // persistent launch grid per kernel kind
    int maxitems[WK_KINDS];    // upper bound of work items (all stamps, all channels)
    int P;                     // PSF side (uniform across the stamps of a call)
    unsigned long long* work;  // profiling: algorithmic work per kernel class, or null
};

enum { PROF_MODEL = 0, PROF_CONV = 1, PROF_REDUCE = 2, PROF_LM = 3, PROF_CLASSES = 4 };

// per-device one-time opt-in to large dynamic shared memory for a kernel
cudaError_t ensure_smem_optin(const void* func, int bytes, int* cache_per_device);
cudaError_t ensure_smem_optin_conv_direct(int P, int* cache_per_device);

// ------------------------------------------------ programmatic dependent launch
// The kernels of a pass are launched with programmatic stream serialization:
// a kernel's CTAs may be scheduled while the previous kernel of the stream is
// still finishing, which hides the launch latency between the short kernels of
// an LM body.  Every such kernel starts with pdl_entry(): it waits until the
// previous grid has completed and its memory is visible (so nothing is read or
// overwritten early), then lets the next kernel begin its own launch.  Kernels
// launched without the attribute pass through pdl_entry() at once.
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Params>(args)...);
}

// launch through launch_pdl, returning the launch error from the caller
#define GF_LAUNCH_PDL(...)                                   \
    do {                                                     \
        const cudaError_t e_pdl_ = launch_pdl(__VA_ARGS__);  \
        if (e_pdl_ != cudaSuccess) return e_pdl_;            \
    } while (0)

// every kernel launch of the library increments this counter
extern std::atomic<long long> g_launch_count;
#define GF_COUNT_LAUNCH() g_launch_count.fetch_add(1, std::memory_order_relaxed)

// kernel launchers (return cudaGetLastError())
cudaError_t launch_fma_peak(int fp64, int grid, int iters, void* sink, cudaStream_t s,
                            double* flops);
cudaError_t launch_model(const PassArgs& a, cudaStream_t s);
cudaError_t launch_conv_direct(const PassArgs& a, cudaStream_t s);
cudaError_t launch_conv_direct_width(const PassArgs& a, int tile_w, cudaStream_t s);
cudaError_t launch_reduce_jac(const PassArgs& a, cudaStream_t s);
cudaError_t launch_reduce_chi2(const PassArgs& a, cudaStream_t s);
// chi^2 partials of each channel as its own model (the rungs of a trial pass)
cudaError_t launch_reduce_rungs(const PassArgs& a, cudaStream_t s);
cudaError_t launch_final_jac(const PassArgs& a, double* A_out, double* g_out, double* chi2_out,
                             cudaStream_t s);
cudaError_t launch_bn_table(cudaStream_t s);
// the LM loop's control word: reset before the loop, decided after every body
cudaError_t launch_loop_start(LoopCtl* c, unsigned long long budget_ns, int max_bodies,
                              cudaStream_t s);
cudaError_t launch_loop_ctl(int count, LMState* lm, int* active, LoopCtl* c,
                            cudaGraphConditionalHandle h, int use_handle, cudaStream_t s);
cudaError_t launch_final_chi2(const PassArgs& a, double* chi2_out, cudaStream_t s);
cudaError_t launch_psf_sum(int count, const StampInfo* st, const float* psf, float* out,
                           cudaStream_t s);
// the work list of the stamps whose LM phase is `phase`; blk: scratch of
// worklist_blocks(count) x (1 + WK_KINDS) ints
int worklist_blocks(int count);
cudaError_t launch_worklist(int count, const LMState* lm, int phase, const int* pre_static,
                            int* n, int* ids, int* pre, int* blk, cudaStream_t s);

// parameter / channel preparation and the LM steps (lm.cu)
cudaError_t launch_prep_sum(const PassArgs& a, const double* params, int use_trial,
                            cudaStream_t s);
cudaError_t launch_prep_jac(const PassArgs& a, const double* params, cudaStream_t s);
cudaError_t launch_lm_init(int count, const Structure* S, LMState* lm, const double* p0,
                           cudaStream_t s);
// one block per stamp, one warp per rung of the trial ladder (nr rungs)
cudaError_t launch_final_solve(const PassArgs& a, Channel* trial_chan, int* active, int nr,
                               cudaStream_t s);
cudaError_t launch_final_update(const PassArgs& a, int* active_count, cudaStream_t s);
cudaError_t launch_lm_export(int count, const Structure* S, const LMState* lm, double* out,
                             cudaStream_t s);

// conv tile shape of the direct kernel
#define CONV_TY 32  // default direct-convolution tile height
#define CONV_TX 64
// pixels per block of the reductions
#define RED_THREADS 256
#define RED_CHUNKS 4
#define RED_PIX (RED_THREADS * RED_CHUNKS)
#define MODEL_THREADS 256
#define OS_WARPS 8
#define FINAL_THREADS 128
