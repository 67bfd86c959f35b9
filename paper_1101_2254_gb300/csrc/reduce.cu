// reduce.cu -- step 3 of the fitting loop (Sec. 2 item 3; Sec. 3 item 3,
// transform + reduce) and the normal equations of step 4.
//
// Per pixel (a transform): the model m = sum_ch mweight_ch Y_ch + msky, the
// residual r = d - m, the weight 1/sigma^2 on valid pixels (finite d and sigma,
// sigma > 0), and the Jacobian columns (convolved channels; sum(psf) for the
// sky).  Then the reduce:
//   chi^2 = sum (r/sigma)^2,  A_ij = sum w J_i J_j,  g_i = sum w J_i r.
// All sums are compensated float32 (Neumaier per thread, error-free TwoSum when
// partial sums merge) in a fixed order, so results are deterministic.
//
// Two stages: each block of 256 threads reduces RED_PIX = 1024 pixels of one
// stamp into `nacc` partials; a final kernel, one block per stamp, sums the
// partials of the stamp in block order.
#include <math.h>

#include "gf_internal.cuh"

namespace {

struct ChanInfo {
    float mw[GF_MAX_CHAN];
    int jc[GF_MAX_CHAN];
};

__device__ __forceinline__ void load_chan_info(ChanInfo& ci, float& msky, const PassArgs& a,
                                               int b)
{
    const Channel* c = a.chan + (long long)b * a.chan_stride;
    if (threadIdx.x < a.nchan) {
        ci.mw[threadIdx.x] = c[threadIdx.x].mweight;
        ci.jc[threadIdx.x] = c[threadIdx.x].jcol;
    }
    if (threadIdx.x == 0) msky = c[0].msky;
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce_jac(PassArgs a)
{
    __shared__ float Jt[GF_MAX_FREE][RED_THREADS];
    __shared__ float wv[RED_THREADS], wr[RED_THREADS], zz[RED_THREADS];
    __shared__ ChanInfo ci;
    __shared__ float msky;
    const int blk = blockIdx.x;
    const int b = find_stamp(a.pre_red, a.count, blk);
    if (a.lm && a.lm[b].phase != a.phase) return;
    const StampInfo st = a.st[b];
    const int nf = a.S->nfree, nacc = a.nacc, skyc = a.S->sky_jcol;
    load_chan_info(ci, msky, a, b);
    __syncthreads();
    const float psum = a.psf_sum[b];
    const long long HW = (long long)st.H * st.W;
    const float* img = a.img + st.pix_off;
    const float* sig = a.sig + st.pix_off;
    const float* Y = a.y + y_index(st, a.nchan, 0);
    const int tid = threadIdx.x;
    int ai = 0, aj = 0;
    const int akind = (tid < nacc) ? decode_acc(tid, nf, ai, aj) : -1;
    CSum acc = {0.0f, 0.0f};
    const long long base = (long long)(blk - a.pre_red[b]) * RED_PIX;
    for (int q = 0; q < RED_CHUNKS; ++q) {
        const long long px = base + (long long)q * RED_THREADS + tid;
        if (px < HW) {
            const float d = img[px], s = sig[px];
            const bool valid = isfinite(d) && isfinite(s) && s > 0.0f;
            float m = msky;
            for (int k = 0; k < a.nchan; ++k) {
                const float yk = Y[(long long)k * HW + px];
                if (ci.mw[k] != 0.0f) m = fmaf(ci.mw[k], yk, m);
                if (ci.jc[k] >= 0) Jt[ci.jc[k]][tid] = yk;
            }
            if (skyc >= 0) Jt[skyc][tid] = psum;
            const float r = valid ? d - m : 0.0f;
            const float z = valid ? r / s : 0.0f;
            wv[tid] = valid ? 1.0f / (s * s) : 0.0f;
            wr[tid] = valid ? z / s : 0.0f;
            zz[tid] = z * z;
            if (a.m_out) a.m_out[st.pix_off + px] = m;
            if (a.J_out)
                for (int f = 0; f < nf; ++f) a.J_out[(long long)f * HW + px] = Jt[f][tid];
        } else {
            for (int f = 0; f < nf; ++f) Jt[f][tid] = 0.0f;
            wv[tid] = wr[tid] = zz[tid] = 0.0f;
        }
        __syncthreads();
        if (akind == 0) {
            for (int p = 0; p < RED_THREADS; ++p)
                csum_add(acc, __fmul_rn(__fmul_rn(wv[p], Jt[ai][p]), Jt[aj][p]));
        } else if (akind == 1) {
            for (int p = 0; p < RED_THREADS; ++p) csum_add(acc, __fmul_rn(Jt[ai][p], wr[p]));
        } else if (akind == 2) {
            for (int p = 0; p < RED_THREADS; ++p) csum_add(acc, zz[p]);
        }
        __syncthreads();
    }
    if (tid < nacc) a.partial[(long long)blk * nacc + tid] = acc.s + acc.c;
    if (a.work && tid == 0) {
        const long long n = min((long long)RED_PIX, HW - base);
        atomicAdd(&a.work[PROF_REDUCE], (unsigned long long)n * (4ull * a.nchan + 8ull));
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce_chi2(PassArgs a)
{
    __shared__ ChanInfo ci;
    __shared__ float msky;
    __shared__ CSum wsum[RED_THREADS / 32];
    const int blk = blockIdx.x;
    const int b = find_stamp(a.pre_red, a.count, blk);
    if (a.lm && a.lm[b].phase != a.phase) return;
    const StampInfo st = a.st[b];
    load_chan_info(ci, msky, a, b);
    __syncthreads();
    const long long HW = (long long)st.H * st.W;
    const float* img = a.img + st.pix_off;
    const float* sig = a.sig + st.pix_off;
    const float* Y = a.y + y_index(st, a.nchan, 0);
    CSum acc = {0.0f, 0.0f};
    const long long base = (long long)(blk - a.pre_red[b]) * RED_PIX;
    for (int q = 0; q < RED_CHUNKS; ++q) {
        const long long px = base + (long long)q * RED_THREADS + threadIdx.x;
        if (px >= HW) break;
        float m = msky;
        for (int k = 0; k < a.nchan; ++k) m = fmaf(ci.mw[k], Y[(long long)k * HW + px], m);
        if (a.m_out) a.m_out[st.pix_off + px] = m;
        const float d = img[px], s = sig[px];
        if (isfinite(d) && isfinite(s) && s > 0.0f) {
            const float z = (d - m) / s;
            csum_add(acc, z * z);
        }
    }
    // deterministic shuffle tree, then across warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CSum other;
        other.s = __shfl_down_sync(0xffffffffu, acc.s, o);
        other.c = __shfl_down_sync(0xffffffffu, acc.c, o);
        acc = csum_merge(acc, other);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        CSum t = wsum[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, wsum[w]);
        a.partial[blk] = t.s + t.c;
        if (a.work) {
            const long long n = min((long long)RED_PIX, HW - base);
            atomicAdd(&a.work[PROF_REDUCE], (unsigned long long)n * (4ull * a.nchan + 8ull));
        }
    }
}

// one block per stamp: sum the stamp's partials in block order
__global__ void __launch_bounds__(RED_THREADS) k_final_jac(PassArgs a, double* A_out,
                                                           double* g_out, double* chi2_out)
{
    const int b = blockIdx.x;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const int nf = a.S->nfree, nacc = a.nacc, tid = threadIdx.x;
    if (tid >= nacc) return;
    const int b0 = a.pre_red[b], b1 = a.pre_red[b + 1];
    CSum acc = {0.0f, 0.0f};
    for (int k = b0; k < b1; ++k) csum_add(acc, a.partial[(long long)k * nacc + tid]);
    const double v = (double)acc.s + (double)acc.c;
    int i, j;
    const int kind = decode_acc(tid, nf, i, j);
    double* A = a.lm ? a.lm[b].A : A_out + (long long)b * nf * nf;
    double* g = a.lm ? a.lm[b].g : g_out + (long long)b * nf;
    if (kind == 0) {
        A[i * nf + j] = v;
        A[j * nf + i] = v;
    } else if (kind == 1) {
        g[i] = v;
    } else {
        if (a.lm)
            a.lm[b].chi2 = v;
        else
            chi2_out[b] = v;
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_final_chi2(PassArgs a, double* chi2_out)
{
    __shared__ CSum wsum[RED_THREADS / 32];
    const int b = blockIdx.x;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const int b0 = a.pre_red[b], b1 = a.pre_red[b + 1];
    CSum acc = {0.0f, 0.0f};
    for (int k = b0 + threadIdx.x; k < b1; k += RED_THREADS) csum_add(acc, a.partial[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CSum other;
        other.s = __shfl_down_sync(0xffffffffu, acc.s, o);
        other.c = __shfl_down_sync(0xffffffffu, acc.c, o);
        acc = csum_merge(acc, other);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        CSum t = wsum[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, wsum[w]);
        const double v = (double)t.s + (double)t.c;
        if (a.lm)
            a.lm[b].chi2t = v;
        else
            chi2_out[b] = v;
    }
}

// sum of each PSF (the sky column and the sky's share of the model)
__global__ void __launch_bounds__(RED_THREADS) k_psf_sum(int count, const StampInfo* st,
                                                         const float* psf, float* out)
{
    __shared__ CSum wsum[RED_THREADS / 32];
    const int b = blockIdx.x;
    if (b >= count) return;
    const int n = st[b].P * st[b].P;
    const float* p = psf + st[b].psf_off;
    CSum acc = {0.0f, 0.0f};
    for (int k = threadIdx.x; k < n; k += RED_THREADS) csum_add(acc, p[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CSum other;
        other.s = __shfl_down_sync(0xffffffffu, acc.s, o);
        other.c = __shfl_down_sync(0xffffffffu, acc.c, o);
        acc = csum_merge(acc, other);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        CSum t = wsum[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, wsum[w]);
        out[b] = t.s + t.c;
    }
}

}  // namespace

cudaError_t launch_reduce_jac(const PassArgs& a, cudaStream_t s)
{
    if (a.tot_red > 0) {
        k_reduce_jac<<<a.tot_red, RED_THREADS, 0, s>>>(a);
        GF_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_chi2(const PassArgs& a, cudaStream_t s)
{
    if (a.tot_red > 0) {
        k_reduce_chi2<<<a.tot_red, RED_THREADS, 0, s>>>(a);
        GF_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

cudaError_t launch_final_jac(const PassArgs& a, double* A_out, double* g_out, double* chi2_out,
                             cudaStream_t s)
{
    k_final_jac<<<a.count, RED_THREADS, 0, s>>>(a, A_out, g_out, chi2_out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_final_chi2(const PassArgs& a, double* chi2_out, cudaStream_t s)
{
    k_final_chi2<<<a.count, RED_THREADS, 0, s>>>(a, chi2_out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_psf_sum(int count, const StampInfo* st, const float* psf, float* out,
                           cudaStream_t s)
{
    k_psf_sum<<<count, RED_THREADS, 0, s>>>(count, st, psf, out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}
