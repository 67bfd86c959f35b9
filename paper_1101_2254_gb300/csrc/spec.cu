// spec.cu -- batched spectral-line fitting on the GPU: the fitting loop of
// Sec. 2 (model, convolution, comparison, LM adjustment, finishing criteria)
// in one dimension, which Sec. 5 names as the same procedure with a flexible
// dimensionality (spectral line or cube fitting; a cube is fitted spaxel by
// spaxel).
//
// A spectrum is small (thousands of channels), so one CTA owns one spectrum
// for its whole fit and keeps every intermediate on chip: the kernel is
// persistent over spectra, and an LM iteration is a few passes over the
// spectrum in chunks of ST channels with no launch and no host round trip.
// Per chunk:
//   1. the extended grid of the chunk (ST + L - 1 points): the model and, for
//      a Jacobian pass, one column per free slot (exact basis functions for
//      the linear slots; forward differences or analytic derivatives of the
//      Gaussian lines) into shared memory;
//   2. the LSF convolution of every column, one output channel per thread;
//   3. the residual and weight, and the bordered normal matrix
//      sum w (J, r)(J, r)^T by 4 x 4 tiles (16 pixel groups per chunk, each
//      a plain float32 sum added to compensated totals), or for a trial pass
//      the compensated chi^2 of each thread.
// The group totals merge in a fixed order, so every result is deterministic.
// The damped system is solved in FP64 by one warp (chol.cuh); the rest of the
// LM step follows the stamp fit's rules exactly.
#include <math.h>

#include <algorithm>

#include "chol.cuh"
#include "gf_internal.cuh"
#include "spec.cuh"

namespace {

constexpr int ST = 256;                          // threads, and channels per chunk
constexpr int SSPAN = ST + GF_SPEC_MAX_LSF - 1;  // extended points of a chunk
constexpr int SV = GF_MAX_FREE + 1;              // columns: free slots + model/residual
constexpr int SVP = 20;                          // rows of the column sums (tiles of 4 stay inside)
constexpr int SVC = ST + 4;                      // their row stride (a 16-byte multiple)
constexpr int SGRP = 16;                         // pixel groups of a chunk (16 pixels each)
constexpr int STILE = 15;                        // 4 x 4 tiles of the upper triangle, at most
constexpr unsigned kFull = 0xffffffffu;

static_assert(4 * ((SV + 3) / 4) <= SVP && SVP % 4 == 0, "tiles stay inside the column sums");
static_assert((SV * SSPAN * sizeof(float)) % 16 == 0, "the column sums start 16-byte aligned");
static_assert((SVC * sizeof(float)) % 16 == 0, "column-sum rows 16-byte aligned");
static_assert(sizeof(float) * SVP * SVC >= sizeof(float) * SGRP * STILE * 16, "union");
// the blocked sums read D up to 4 * 63 + 4 ceil((L + 3) / 4) - 1 < SSPAN
static_assert(252 + 4 * ((GF_SPEC_MAX_LSF + 6) / 4) <= SSPAN, "blocked window inside D");

// the LSF zero padded for the blocked sums: tap u at index u + 7 + lsf_pad_off(L)
constexpr int SLSFZ = ((GF_SPEC_MAX_LSF + 17 + 3) / 4) * 4;
__host__ __device__ constexpr int lsf_pad_off(int L) { return (4 - (L + 3) % 4) % 4; }

struct SpecShared {
    float D[SV][SSPAN];        // extended-grid columns of the chunk
    union {
        // the bordered matrix's columns (J_0 .. J_{nf-1}, r, zero rows up to
        // a multiple of 4) by column, one entry per channel of the chunk
        float Vc[SVP][SVC];
        float red[SGRP][STILE][16];  // after the chunks: per group and tile, its 4 x 4 sums
    } u;
    float lsfz[SLSFZ];         // zero-padded LSF of the blocked sums
    float Wt[ST];              // weights 1/sigma^2 (0 on invalid channels)
    float lsf[GF_SPEC_MAX_LSF];
    // float32 constants of the current parameter vector
    float ca[3];                             // continuum coefficients
    float xc, ih;                            // t = (x - xc) ih
    float la[GF_SPEC_MAX_LINES];             // amplitudes
    float lmh[GF_SPEC_MAX_LINES], lml[GF_SPEC_MAX_LINES];  // centres, hi + lo
    float lis[GF_SPEC_MAX_LINES];            // 1 / widths
    float fmh[GF_MAX_FREE], fml[GF_MAX_FREE], fis[GF_MAX_FREE], fih[GF_MAX_FREE];  // FD
    int colC[3], colA[GF_SPEC_MAX_LINES], colM[GF_SPEC_MAX_LINES], colS[GF_SPEC_MAX_LINES];
    CSum wsum[ST / 32];
    double p[GF_SPEC_MAX_PARAMS], pt[GF_SPEC_MAX_PARAMS];
    double A[GF_MAX_FREE * GF_MAX_FREE], g[GF_MAX_FREE];
    double M[GF_MAX_FREE * GF_MAX_FREE], r[GF_MAX_FREE];
    double chi2;
    double pred;
    int ok, small;
};

// role of slot s: 0 continuum, 1 amplitude, 2 centre, 3 width
__device__ __forceinline__ int spec_role(const SpecArgs& a, int s)
{
    return s < a.nc ? 0 : 1 + (s - a.nc) % 3;
}

__device__ __forceinline__ double spec_fd_step(const SpecArgs& a, int s, double v)
{
    return spec_role(a, s) == 2 ? a.opts.fd_rel : a.opts.fd_rel * fmax(fabs(v), 1.0);
}

// Float constants of parameter vector q (and the FD perturbations of the free
// centre and width slots) into shared memory.  Called by warp 0.
__device__ void spec_consts(const SpecArgs& a, SpecShared& S, const double* q, bool cols)
{
    const int lane = threadIdx.x & 31;
    if (lane < a.nc) S.ca[lane] = (float)q[lane];
    if (lane == 0) {
        const double h = a.N > 1 ? 0.5 * (a.N - 1) : 1.0;
        S.xc = (float)(0.5 * (a.N - 1));
        S.ih = (float)(1.0 / h);
    }
    if (lane < a.K) {
        const double* l = q + a.nc + 3 * lane;
        S.la[lane] = (float)l[0];
        const float mh = (float)l[1];
        S.lmh[lane] = mh;
        S.lml[lane] = (float)(l[1] - (double)mh);
        S.lis[lane] = (float)(1.0 / l[2]);
    }
    if (cols && a.opts.jac_mode == GF_JAC_FD && lane < a.nf) {
        const int s = a.fs[lane], role = spec_role(a, s);
        if (role >= 2) {
            const int k = (s - a.nc) / 3;
            const double* l = q + a.nc + 3 * k;
            const double h = spec_fd_step(a, s, q[s]);
            const double mu = role == 2 ? l[1] + h : l[1];
            const double sw = role == 3 ? l[2] + h : l[2];
            const float mh = (float)mu;
            S.fmh[lane] = mh;
            S.fml[lane] = (float)(mu - (double)mh);
            S.fis[lane] = (float)(1.0 / sw);
            S.fih[lane] = (float)(1.0 / h);
        }
    }
    __syncwarp();
}

// Model (column ncol - 1 = nf for a Jacobian pass, column 0 otherwise) and the
// Jacobian columns at the extended points of the chunk starting at channel i0.
__device__ void spec_columns(const SpecArgs& a, SpecShared& S, int i0, bool cols)
{
    const int c = (a.L - 1) / 2;
    // a Jacobian pass fills the whole blocked window (up to 3 points past the
    // extended chunk, whose taps are zero)
    const int span = cols ? 252 + 4 * ((a.L + 6) / 4) : ST + a.L - 1;
    const int mcol = cols ? a.nf : 0;
    const bool fd = a.opts.jac_mode == GF_JAC_FD;
    for (int e = threadIdx.x; e < span; e += ST) {
        const float x = (float)(i0 - c + e);
        const float t = (x - S.xc) * S.ih;
        float model = 0.0f, tj = 1.0f;
        for (int j = 0; j < a.nc; ++j) {
            model = fmaf(S.ca[j], tj, model);
            if (cols && S.colC[j] >= 0) S.D[S.colC[j]][e] = tj;
            tj *= t;
        }
        for (int k = 0; k < a.K; ++k) {
            const float dx = (x - S.lmh[k]) - S.lml[k];
            const float z = dx * S.lis[k];
            const float G = expf(-0.5f * z * z);
            const float Ak = S.la[k];
            model = fmaf(Ak, G, model);
            if (!cols) continue;
            if (S.colA[k] >= 0) S.D[S.colA[k]][e] = G;
            const int fm = S.colM[k], fsg = S.colS[k];
            if (fm >= 0) {
                float v;
                if (fd) {
                    const float z2 = ((x - S.fmh[fm]) - S.fml[fm]) * S.fis[fm];
                    v = Ak * (expf(-0.5f * z2 * z2) - G) * S.fih[fm];
                } else {
                    v = Ak * G * z * S.lis[k];
                }
                S.D[fm][e] = v;
            }
            if (fsg >= 0) {
                float v;
                if (fd) {
                    const float z2 = ((x - S.fmh[fsg]) - S.fml[fsg]) * S.fis[fsg];
                    v = Ak * (expf(-0.5f * z2 * z2) - G) * S.fih[fsg];
                } else {
                    v = Ak * G * z * z * S.lis[k];
                }
                S.D[fsg][e] = v;
            }
        }
        S.D[mcol][e] = model;
    }
}

// One pass over the spectrum at the parameter vector whose constants are in
// S.  cols: the normal equations (S.A, S.g, S.chi2); otherwise chi^2 only
// (S.chi2) and, with m_out, the convolved model.  All threads call it.
__device__ void spec_pass(const SpecArgs& a, SpecShared& S, const float* spec, const float* sig,
                          float* m_out, bool cols)
{
    const int tid = threadIdx.x;
    const int ncol = cols ? a.nf + 1 : 1;
    const int nv = a.nf + 1;
    const int nt = (nv + 3) / 4, ntp = nt * (nt + 1) / 2;
    // tile slot and pixel group of this thread in the normal-matrix tiles
    // thread (tile slot, group): 16 pixel groups of 16 pixels; the 16 threads
    // of a group read the same pixel row (broadcasts)
    const int tslot = tid % 16, grp = tid / 16;
    const bool active_tile = cols && tslot < ntp;
    int ti = 0, tj = 0;
    for (int I = 0, k = 0; I < nt; ++I)
        for (int J = I; J < nt; ++J, ++k)
            if (k == tslot) {
                ti = I;
                tj = J;
            }
    CSum acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = {0.0f, 0.0f};
    CSum x2 = {0.0f, 0.0f};
    for (int i0 = 0; i0 < a.N; i0 += ST) {
        spec_columns(a, S, i0, cols);
        __syncthreads();
        // LSF convolution, one channel per thread: m_i = sum_u lsf[u] E(i + c - u)
        const int i = i0 + tid;
        const bool in = i < a.N;
        float d = 0.0f, s = 0.0f, m = 0.0f;
        if (in && spec) {
            d = spec[i];
            s = sig[i];
        }
        const bool valid = in && isfinite(d) && isfinite(s) && s > 0.0f;
        if (cols) {
            // The Jacobian columns by blocks: item (f, q) sums outputs 4q .. 4q+3
            // of column f from aligned 16-byte windows of D, the taps read as
            // two broadcast float4 of the padded LSF per window: 16 FMAs per
            // three shared loads.  Output r takes window value s with tap
            // u = r + L - 1 - 4b - s, at lsfz[k0 + r - s + 3].
            const int nb = (a.L + 6) / 4;
            const int kb = a.L + 3 + lsf_pad_off(a.L);
            for (int it = tid; it < a.nf * (ST / 4); it += ST) {
                const int f = it / (ST / 4), q = it % (ST / 4);
                const float* Dq = &S.D[f][4 * q];
                float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f, o3 = 0.0f;
                for (int bb = 0; bb < nb; ++bb) {
                    const float4 w = *reinterpret_cast<const float4*>(Dq + 4 * bb);
                    const int k0 = kb - 4 * bb;
                    const float4 ca = *reinterpret_cast<const float4*>(&S.lsfz[k0]);
                    const float4 cb = *reinterpret_cast<const float4*>(&S.lsfz[k0 + 4]);
                    o0 = fmaf(ca.w, w.x, o0); o0 = fmaf(ca.z, w.y, o0);
                    o0 = fmaf(ca.y, w.z, o0); o0 = fmaf(ca.x, w.w, o0);
                    o1 = fmaf(cb.x, w.x, o1); o1 = fmaf(ca.w, w.y, o1);
                    o1 = fmaf(ca.z, w.z, o1); o1 = fmaf(ca.y, w.w, o1);
                    o2 = fmaf(cb.y, w.x, o2); o2 = fmaf(cb.x, w.y, o2);
                    o2 = fmaf(ca.w, w.z, o2); o2 = fmaf(ca.z, w.w, o2);
                    o3 = fmaf(cb.z, w.x, o3); o3 = fmaf(cb.y, w.y, o3);
                    o3 = fmaf(cb.x, w.z, o3); o3 = fmaf(ca.w, w.w, o3);
                }
                *reinterpret_cast<float4*>(&S.u.Vc[f][4 * q]) = make_float4(o0, o1, o2, o3);
            }
        }
        {
            // the model, one channel per thread in tap order (the trial pass
            // sums it the same way, so both passes give the same model)
            float v = 0.0f;
            const float* Dm = &S.D[ncol - 1][tid + a.L - 1];
            for (int u = 0; u < a.L; ++u) v = fmaf(S.lsf[u], Dm[-u], v);
            m = v;
        }
        if (in && m_out) m_out[i] = m;
        if (cols) {
            // the residual row and the zero rows up to a multiple of 4; channels
            // past the spectrum keep finite column sums but weight 0
            S.u.Vc[a.nf][tid] = valid ? d - m : 0.0f;
            for (int f = nv; f < 4 * nt; ++f) S.u.Vc[f][tid] = 0.0f;
            S.Wt[tid] = valid ? 1.0f / (s * s) : 0.0f;
        } else if (valid) {
            const float z = (d - m) / s;
            csum_add(x2, z * z);
        }
        __syncthreads();
        if (active_tile) {
            // 4 pixels per step: the tile's 4 rows and 4 columns as float4 along
            // the pixels, the sums taken pixel by pixel in order
            float sum[4][4];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) sum[x][y] = 0.0f;
            const int c0 = 4 * ti, r0 = 4 * tj;
            for (int pp = 0; pp < ST / SGRP; pp += 4) {
                const int p = grp * (ST / SGRP) + pp;
                const float4 w4 = *reinterpret_cast<const float4*>(&S.Wt[p]);
                float4 va[4], vb[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    va[x] = *reinterpret_cast<const float4*>(&S.u.Vc[c0 + x][p]);
                    vb[x] = *reinterpret_cast<const float4*>(&S.u.Vc[r0 + x][p]);
                }
                const float wk[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const float ax = k == 0 ? va[x].x : k == 1 ? va[x].y : k == 2 ? va[x].z : va[x].w;
                        const float vi = wk[k] * ax;
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            const float by = k == 0 ? vb[y].x : k == 1 ? vb[y].y : k == 2 ? vb[y].z : vb[y].w;
                            sum[x][y] = fmaf(vi, by, sum[x][y]);
                        }
                    }
                }
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) csum_add(acc[x][y], sum[x][y]);
        }
        __syncthreads();  // D and the column sums are rewritten by the next chunk
    }
    if (cols) {
        if (active_tile)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) S.u.red[grp][tslot][x * 4 + y] = acc[x][y].s + acc[x][y].c;
        __syncthreads();
        // entry (r_, c_), r_ <= c_ < nv, of the bordered matrix: merge the 16
        // groups in order
        const int nent = nv * (nv + 1) / 2;
        for (int t = tid; t < nent; t += ST) {
            // t < nent, so the walk ends with r_ < nv
            int r_ = 0, rem = t;
            while (r_ < nv - 1 && rem >= nv - r_) {
                rem -= nv - r_;
                ++r_;
            }
            const int c_ = r_ + rem;
            const int I = r_ / 4, J = c_ / 4;
            int slot = 0;
            for (int II = 0; II < I; ++II) slot += nt - II;
            slot += J - I;
            CSum tot = {0.0f, 0.0f};
            for (int gq = 0; gq < SGRP; ++gq) csum_add(tot, S.u.red[gq][slot][(r_ % 4) * 4 + (c_ % 4)]);
            const double v = (double)tot.s + (double)tot.c;
            if (c_ < a.nf) {
                S.A[r_ * a.nf + c_] = v;
                S.A[c_ * a.nf + r_] = v;
            } else if (r_ < a.nf) {
                S.g[r_] = v;
            } else {
                S.chi2 = v;
            }
        }
        __syncthreads();
        if (a.work && tid == 0) {
            // useful FLOPs: the LSF sums of every column and the upper
            // triangle of the bordered normal matrix, per channel
            const unsigned long long n = (unsigned long long)a.N;
            atomicAdd(a.work, n * (2ull * nv * a.L + (unsigned long long)nv * (nv + 1)));
        }
    } else {
        if (a.work && tid == 0) atomicAdd(a.work, (unsigned long long)a.N * (2ull * a.L + 3ull));
        // deterministic shuffle tree, then the warps in order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            CSum other;
            other.s = __shfl_down_sync(kFull, x2.s, o);
            other.c = __shfl_down_sync(kFull, x2.c, o);
            x2 = csum_merge(x2, other);
        }
        if ((tid & 31) == 0) S.wsum[tid >> 5] = x2;
        __syncthreads();
        if (tid == 0) {
            CSum t = S.wsum[0];
            for (int w = 1; w < ST / 32; ++w) t = csum_merge(t, S.wsum[w]);
            S.chi2 = (double)t.s + (double)t.c;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double spec_xscale(const SpecArgs& a, int s)
{
    const int r = spec_role(a, s);
    return r == 1 ? 1e-30 : (r == 0 ? 1e-3 : 1.0);
}

// S.p -> constants, then a pass (all threads)
__device__ void spec_eval_at(const SpecArgs& a, SpecShared& S, const double* q, const float* spec,
                             const float* sig, float* m_out, bool cols)
{
    if (threadIdx.x < 32) spec_consts(a, S, q, cols);
    __syncthreads();
    spec_pass(a, S, spec, sig, m_out, cols);
}

// The LSF into shared memory, plain and zero padded (tap u at lsfz[u + 7 +
// lsf_pad_off(L)]).  The caller synchronises before use.
__device__ void spec_load_lsf(const SpecArgs& a, SpecShared& S, const float* lsf)
{
    const int off = 7 + lsf_pad_off(a.L);
    for (int k = threadIdx.x; k < SLSFZ; k += ST) {
        const int u = k - off;
        const float v = (u >= 0 && u < a.L) ? lsf[u] : 0.0f;
        S.lsfz[k] = v;
        if (u >= 0 && u < a.L) S.lsf[u] = v;
    }
}

// Spectrum b: the call's mode (model, chi^2, normal equations or the LM fit).
// All threads of the block call it.
__device__ void spec_one(const SpecArgs& a, SpecShared& S, int b)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const float* spec = a.spec ? a.spec + (long long)b * a.N : nullptr;
    const float* sig = a.sig ? a.sig + (long long)b * a.N : nullptr;
    if (a.lsf_stride) {
        spec_load_lsf(a, S, a.lsf + (long long)b * a.lsf_stride);
    }
    if (tid < a.np) S.p[tid] = a.p_in[(long long)b * a.np + tid];
    __syncthreads();
    if (a.mode == SPEC_MODEL) {
        spec_eval_at(a, S, S.p, nullptr, nullptr, a.model + (long long)b * a.N, false);
        return;
    }
    if (a.mode == SPEC_EVAL) {
        spec_eval_at(a, S, S.p, spec, sig, a.model ? a.model + (long long)b * a.N : nullptr,
                     false);
        if (tid == 0) a.chi2[b] = S.chi2;
        return;
    }
    if (a.mode == SPEC_NORMAL) {
        spec_eval_at(a, S, S.p, spec, sig, nullptr, true);
        for (int t = tid; t < a.nf * a.nf; t += ST) a.A[(long long)b * a.nf * a.nf + t] = S.A[t];
        if (tid < a.nf) a.g[(long long)b * a.nf + tid] = S.g[tid];
        if (tid == 0) a.chi2[b] = S.chi2;
        __syncthreads();
        return;
    }
    // ---- SPEC_FIT: Levenberg-Marquardt with Marquardt's diagonal damping
    const gf_lm_opts& o = a.opts;
    const int nf = a.nf;
    if (tid < a.np) S.p[tid] = fmin(fmax(S.p[tid], a.lo[tid]), a.hi[tid]);
    __syncthreads();
    spec_eval_at(a, S, S.p, spec, sig, nullptr, true);
    double chi2 = S.chi2, lambda = o.lambda0;
    int iters = 0, accepted = 0, status = GF_EMAXITER;
    while (iters < o.max_iter) {
        ++iters;
        if (tid < 32) {
            // damped system; a slot with no influence is held this step
            for (int t = lane; t < nf * nf; t += 32) {
                const int i = t / nf, j = t % nf;
                const bool hi_ = S.A[i * nf + i] > 0.0, hj = S.A[j * nf + j] > 0.0;
                double v = (hi_ && hj) ? S.A[t] : 0.0;
                if (i == j) v = hi_ ? S.A[t] * (1.0 + lambda) : 1.0;
                S.M[t] = v;
            }
            if (lane < nf) S.r[lane] = S.A[lane * nf + lane] > 0.0 ? S.g[lane] : 0.0;
            __syncwarp();
            const bool ok = warp_cholesky_solve(nf, S.M, S.r);
            bool small = true;
            double pred = 0.0;
            if (ok) {
                for (int i = lane; i < nf; i += 32) {
                    const int sl = a.fs[i];
                    const double den = fmax(fabs(S.p[sl]), spec_xscale(a, sl));
                    small = small && fabs(S.r[i]) / den < o.xtol;
                    const double dA = S.A[i * nf + i] > 0.0 ? S.A[i * nf + i] : 0.0;
                    const double rhs = S.A[i * nf + i] > 0.0 ? S.g[i] : 0.0;
                    pred += S.r[i] * (rhs + lambda * dA * S.r[i]);
                }
                // the predicted fall summed in lane order, as a serial sum would
                double tot = 0.0;
                for (int l = 0; l < 32; ++l) tot += __shfl_sync(kFull, pred, l);
                pred = tot;
                small = __all_sync(kFull, small);
            }
            for (int sl = lane; sl < a.np; sl += 32) S.pt[sl] = S.p[sl];
            __syncwarp();
            if (ok && !small)
                for (int i = lane; i < nf; i += 32) S.pt[a.fs[i]] += S.r[i];
            __syncwarp();
            for (int sl = lane; sl < a.np; sl += 32) S.pt[sl] = fmin(fmax(S.pt[sl], a.lo[sl]), a.hi[sl]);
            if (lane == 0) {
                S.ok = ok;
                S.small = small;
                S.pred = pred;
            }
        }
        __syncthreads();
        const bool ok = S.ok, small = S.small;
        const double pred = S.pred;
        __syncthreads();  // warp 0 rewrites the flags in the next iteration
        if (ok && small) {
            status = GF_OK;
            break;
        }
        if (ok) {
            spec_eval_at(a, S, S.pt, spec, sig, nullptr, false);
            const double chi2t = S.chi2;
            if (isfinite(chi2t) && chi2t < chi2) {
                const double rel = (chi2 - chi2t) / chi2;
                if (tid < a.np) S.p[tid] = S.pt[tid];
                ++accepted;
                lambda = fmax(lambda * o.lambda_down, o.lambda_min);
                __syncthreads();
                if (rel < o.ftol && pred / chi2 < o.ftol) {
                    chi2 = chi2t;
                    status = GF_OK;
                    break;
                }
                spec_eval_at(a, S, S.p, spec, sig, nullptr, true);
                chi2 = S.chi2;
                continue;
            }
        }
        lambda *= o.lambda_up;
        if (lambda > o.lambda_max) {
            status = GF_ENOCONV;
            break;
        }
    }
    if (tid < a.np) a.p_out[(long long)b * a.np + tid] = S.p[tid];
    if (tid == 0) {
        gf_lm_result r;
        r.chi2 = chi2;
        r.lambda = lambda;
        r.iters = iters;
        r.accepted = accepted;
        r.status = status;
        a.res[b] = r;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(ST, 3) k_spec(const __grid_constant__ SpecArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpecShared& S = *reinterpret_cast<SpecShared*>(smem_raw);
    const int tid = threadIdx.x;
    // column of each free slot in the Jacobian pass (-1: held)
    if (tid < 3) S.colC[tid] = -1;
    if (tid < GF_SPEC_MAX_LINES) S.colA[tid] = S.colM[tid] = S.colS[tid] = -1;
    __syncthreads();
    if (tid < a.nf) {
        const int s = a.fs[tid];
        if (s < a.nc) {
            S.colC[s] = tid;
        } else {
            const int k = (s - a.nc) / 3, r = (s - a.nc) % 3;
            (r == 0 ? S.colA : r == 1 ? S.colM : S.colS)[k] = tid;
        }
    }
    if (a.lsf_stride == 0)
        spec_load_lsf(a, S, a.lsf);
    __syncthreads();
    for (int b = blockIdx.x; b < a.count; b += gridDim.x) spec_one(a, S, b);
}

int g_spec_grid[64];

}  // namespace

cudaError_t launch_spec(const SpecArgs& a, cudaStream_t s)
{
    if (a.count <= 0) return cudaSuccess;
    const int bytes = (int)sizeof(SpecShared);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_spec_grid[dev] == 0) {
        e = cudaFuncSetAttribute(k_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spec, ST, bytes);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_spec_grid[dev] = std::max(1, per_sm) * sms;
    }
    const int grid = std::min(a.count, g_spec_grid[dev]);
    k_spec<<<grid, ST, bytes, s>>>(a);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}
