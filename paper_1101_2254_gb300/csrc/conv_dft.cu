// conv_dft.cu -- step 2 of the fitting loop (Sec. 3 item 2, convolution in
// Fourier space) with the Fourier transforms posed as dense contractions on the
// tensor cores.
//
// Four-step plan, per axis of length N = R1 R2 with index x = x1 R2 + x2 and
// frequency k = k1 + R1 k2:
//   forward   T[k1][x2] = W_N^{k1 x2} sum_x1 F_R1[k1][x1] x[x1][x2]
//             X[k1][k2] = sum_x2 F_R2[k2][x2] T[k1][x2]
// which leaves the spectrum in digit-reversed order (k1, k2); the inverse takes
// that order back to natural order:
//             Z[k1][x2] = W_N^{-k1 x2} sum_k2 F*_R2[x2][k2] X[k1][k2]
//             x[x1][x2] = sum_k1 F*_R1[x1][k1] Z[k1][x2].
// The PSF spectrum is made by the same forward stages, so the product with it
// happens in the permuted order and no transpose is ever needed.  Each stage
// is a batched complex GEMM against a small fixed DFT matrix.
//
// Precision: float32 data and DFT matrices are split x = hi + lo into bf16
// pairs; each real product uses hi*hi + hi*lo + lo*hi (the lo*lo term is ~2^-16
// of the result) with float32 accumulation.
//
// Tensor cores (tcgen05, accumulators in tensor memory).  A stage is a batch
// of rows (orientation A: the (l, q) pairs; B: the m rows), each contracted
// with the R x R DFT matrix along r.  A CTA takes 128 rows at a time as the M
// side of one accumulator of 128 lanes x 2 Rp columns: columns k hold Re and
// Rp + k hold Im of output k, because the B operand stacks the DFT matrix as
//   B1 = [Fr; Fi] (against the real part of the rows) and
//   B2 = [-Fi; Fr] (against the imaginary part),
// so that Re = Xr Fr^T - Xi Fi^T and Im = Xr Fi^T + Xi Fr^T fall out of one
// accumulator: 6 MMAs (M 128, N 2Rp, K 16) per 16 values of r.  Operands sit in
// shared memory in the canonical K-major layout without swizzle (8 x 8 bf16
// core matrices, 128 B each; consecutive along K 128 B apart, consecutive
// 8-row groups Kp * 16 B apart).  One thread issues the MMAs and commits them
// to an mbarrier; every wait on it is bounded and a timeout turns the tile's
// outputs into NaN and raises the stage's error word.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "conv_dft.cuh"
#include "tc.cuh"

namespace {

constexpr int NT = 256;    // 8 warps: staging 2 threads per row, epilogue 2 warps per lane quarter
constexpr int TM = 128;    // rows per tile (the MMA's M)

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l)
{
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// e >= 0 and below 64 * 4096 for every stage, so 32-bit arithmetic suffices
__device__ __forceinline__ float2 twiddle(const DftStage& s, int e)
{
    e %= s.tw_N;
    float2 w = s.tw[e];
    if (s.tw_sign > 0.0f) w.y = -w.y;
    return w;
}

__device__ __forceinline__ float2 in_a(const DftStage& s, int p, int l, int r, int q)
{
    if (s.in_mode == 1) {
        const int y = l, x = r * s.in_xdigit + q;
        if (y >= s.in_rows || x >= s.in_cols) return make_float2(0.f, 0.f);
        return make_float2(s.in_real[(long long)p * s.in_real_pstride + (long long)y * s.in_ld + x],
                           0.f);
    }
    const long long idx = ((long long)l * s.R + r) * s.Q + q;
    float2 v = s.in[(long long)p * s.in_pstride + idx];
    if (s.in_mode == 2) v = cmulf(v, s.hhat[(long long)(p / s.nchan) * s.in_pstride + idx]);
    return v;
}

// One contraction stage on the tensor cores (see the top of the file).
// ORIENT_A: rows are g = l * Q + q, input IN[p][l][r][q], output OUT[p][l][k][q];
// otherwise rows are m, input IN[p][m][r], output OUT[p][m][k].  A CTA runs
// `tpc` consecutive 128-row tiles of problem blockIdx.z.
template <bool ORIENT_A>
__global__ void __launch_bounds__(NT) k_dft_tc(DftStage s, int tpc, unsigned long long* work)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int p = blockIdx.z;
    if (s.lm && s.lm[p / s.nchan].phase != s.phase) return;  // whole CTA
    const int R = s.R, Rp = s.Rp, Kp = Rp, NB = 2 * Rp;
    const long long rows = ORIENT_A ? (long long)s.L * s.Q : (long long)s.M;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // operand planes: B1 hi, B1 lo, B2 hi, B2 lo (NB x Kp); Xr hi, Xr lo, Xi hi, Xi lo (TM x Kp)
    __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    __nv_bfloat16* Ap = Bp + 4 * NB * Kp;
    const int ncols = NB <= 32 ? 32 : (NB <= 64 ? 64 : 128);  // TMEM columns (power of two)

    // stacked DFT matrix: B1 rows n < Rp = Fr[n], n >= Rp = Fi[n - Rp];
    //                     B2 rows n < Rp = -Fi[n], n >= Rp = Fr[n - Rp]
    for (int i = tid; i < NB * Kp; i += NT) {
        const int n = i / Kp, r = i - n * Kp;
        const int k = n < Rp ? n : n - Rp;
        const __nv_bfloat16* F = s.F + k * Rp + r;
        const int RR = Rp * Rp;
        const __nv_bfloat16 frh = F[0], frl = F[RR], fih = F[2 * RR], fil = F[3 * RR];
        const int o = cofs(n, r, Kp);
        Bp[0 * NB * Kp + o] = n < Rp ? frh : fih;
        Bp[1 * NB * Kp + o] = n < Rp ? frl : fil;
        Bp[2 * NB * Kp + o] = n < Rp ? __hneg(fih) : frh;
        Bp[3 * NB * Kp + o] = n < Rp ? __hneg(fil) : frl;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t bar_a = smem_addr(&bar);
    const uint32_t idesc = idesc_bf16(TM, NB);
    const uint32_t lbo = 128, sbo = (uint32_t)Kp * 16;
    uint32_t parity = 0;

    for (int ti = 0; ti < tpc; ++ti) {
        const long long g0 = ((long long)blockIdx.x * tpc + ti) * TM;
        if (g0 >= rows) break;
        // ---- stage the rows: thread (row, half) splits its half of the r range
        {
            const int row = tid & (TM - 1), half = tid >> 7;
            const long long g = g0 + row;
            const int rbeg = half * (Kp / 2), rend = rbeg + Kp / 2;
            int l = 0, q = 0;
            if (ORIENT_A && g < rows) {
                l = (int)(g / s.Q);
                q = (int)(g - (long long)l * s.Q);
            }
            for (int r8 = rbeg; r8 < rend; r8 += 8) {
                __align__(16) __nv_bfloat16 h[4][8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int r = r8 + j;
                    float2 v = make_float2(0.f, 0.f);
                    if (g < rows && r < R) {
                        if (ORIENT_A)
                            v = in_a(s, p, l, r, q);
                        else
                            v = s.in[(long long)p * s.in_pstride + g * R + r];
                    }
                    split_bf16(v.x, h[0][j], h[1][j]);
                    split_bf16(v.y, h[2][j], h[3][j]);
                }
                const int o = cofs(row, r8, Kp);
#pragma unroll
                for (int pl = 0; pl < 4; ++pl)
                    *reinterpret_cast<uint4*>(Ap + pl * TM * Kp + o) = *reinterpret_cast<const uint4*>(h[pl]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- one thread issues the MMAs: acc = Xr B1^T + Xi B2^T, split precision
        if (tid == 0) {
            const uint32_t a0 = smem_addr(Ap), b0 = smem_addr(Bp);
            const uint32_t aps = TM * Kp * 2, bps = NB * Kp * 2;  // plane bytes
            int acc = 0;
            for (int ks = 0; ks < Kp / 16; ++ks) {
                const uint32_t ko = ks * 256;
                // (A plane, B plane): Xr_h B1_h, Xr_h B1_l, Xr_l B1_h, Xi_h B2_h, Xi_h B2_l, Xi_l B2_h
                const int ap[6] = {0, 0, 1, 2, 2, 3}, bp[6] = {0, 1, 0, 2, 3, 2};
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    umma(tmem, mdesc(a0 + ap[t] * aps + ko, lbo, sbo), mdesc(b0 + bp[t] * bps + ko, lbo, sbo),
                         idesc, acc);
                    acc = 1;
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a));
        }
        const bool done = mbar_wait(bar_a, parity);
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!__syncthreads_and(done ? 1 : 0)) {
            // give up: raise the error word, wait once more (bounded) for the
            // MMAs in flight, mark this tile's outputs NaN and return.  The
            // tensor memory is freed only once that second wait has seen the
            // MMAs complete: freeing it under an MMA still in flight would let
            // that MMA write into columns another CTA may have allocated since.
            // If they never complete the columns stay allocated (the error
            // word tells the host the context is no longer trustworthy).
            if (tid == 0 && s.err) atomicExch(s.err, 1);
            const bool drained = __syncthreads_and(mbar_wait(bar_a, parity ^ 1u) ? 1 : 0);
            for (int i = tid; i < TM * R; i += NT) {
                const long long g = g0 + i / R;
                const int k = i % R;
                if (g >= rows) continue;
                const float2 nan2 = make_float2(NAN, NAN);
                if (ORIENT_A) {
                    const int l = (int)(g / s.Q), q = (int)(g - (long long)l * s.Q);
                    if (s.out_mode == 0) {
                        s.out[(long long)p * s.out_pstride + ((long long)l * R + k) * s.Q + q] = nan2;
                    } else {
                        const int y = l - s.crop_y0, x = k * s.out_xdigit + q - s.crop_x0;
                        if (y >= 0 && y < s.crop_H && x >= 0 && x < s.crop_W)
                            s.out_real[(long long)p * s.out_real_pstride + (long long)y * s.crop_W + x] = NAN;
                    }
                } else {
                    s.out[(long long)p * s.out_pstride + g * R + k] = nan2;
                }
            }
            __syncthreads();
            if (drained && warp == 0)
                asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
            return;
        }
        // ---- epilogue: warp w reads lane quarter w % 4, output half w / 4
        {
            const int quarter = warp & 3, khalf = warp >> 2;
            const int row = quarter * 32 + lane;
            const long long g = g0 + row;
            int l = 0, q = 0;
            if (ORIENT_A) {
                l = (int)(g / s.Q);
                q = (int)(g - (long long)l * s.Q);
            }
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
            for (int k0 = khalf * (Rp / 2); k0 < (khalf + 1) * (Rp / 2); k0 += 8) {
                float re[8], im[8];
                tmem_ld8(taddr + k0, re);
                tmem_ld8(taddr + Rp + k0, im);
                if (g >= rows) continue;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + j;
                    if (k >= R) continue;
                    float2 v = make_float2(re[j], im[j]);
                    if (ORIENT_A) {
                        if (s.tw_mode == 1)
                            v = cmulf(v, twiddle(s, k * ((q / s.tw_div) % s.tw_mod)));
                        else if (s.tw_mode == 2)
                            v = cmulf(v, twiddle(s, l * k));
                        if (s.out_mode == 0) {
                            s.out[(long long)p * s.out_pstride + ((long long)l * R + k) * s.Q + q] = v;
                        } else {
                            const int y = l - s.crop_y0, x = k * s.out_xdigit + q - s.crop_x0;
                            if (y >= 0 && y < s.crop_H && x >= 0 && x < s.crop_W)
                                s.out_real[(long long)p * s.out_real_pstride + (long long)y * s.crop_W + x] = v.x;
                        }
                    } else {
                        if (s.tw_mode == 3) v = cmulf(v, twiddle(s, (int)(g % s.tw_mod) * k));
                        s.out[(long long)p * s.out_pstride + g * R + k] = v;
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();  // TMEM read and the row planes free for the next tile
        if (work && tid == 0) {
            const long long rv = min((long long)TM, rows - g0);
            atomicAdd(work, (unsigned long long)(8ull * R * R * rv));  // complex MACs x 8 FLOP
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// F[k][r] = exp(sign 2 pi i k r / R), zero-padded to Rp x Rp, as 4 bf16 planes
__global__ void k_dft_matrix(int R, int Rp, float sign, __nv_bfloat16* F)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Rp * Rp; i += gridDim.x * blockDim.x) {
        const int k = i / Rp, r = i - k * Rp;
        double c = 0.0, sn = 0.0;
        if (k < R && r < R) {
            const long long e = ((long long)k * r) % R;
            sincospi(2.0 * (double)e / (double)R, &sn, &c);
            sn *= (double)sign;
        }
        __nv_bfloat16 h, lo;
        const float cf = (float)c, sf = (float)sn;
        h = __float2bfloat16_rn(cf);
        lo = __float2bfloat16_rn((float)(c - (double)__bfloat162float(h)));
        F[0 * Rp * Rp + i] = h;
        F[1 * Rp * Rp + i] = lo;
        h = __float2bfloat16_rn(sf);
        lo = __float2bfloat16_rn((float)(sn - (double)__bfloat162float(h)));
        F[2 * Rp * Rp + i] = h;
        F[3 * Rp * Rp + i] = lo;
    }
}

size_t smem_tc(int Rp)
{
    const size_t Kp = Rp, NB = 2 * (size_t)Rp;
    return sizeof(__nv_bfloat16) * 4 * (NB * Kp + (size_t)TM * Kp);
}

// tiles per CTA: enough CTAs for every SM (the CTA stages its DFT matrix once)
int tiles_per_cta(long long rows, int nprob)
{
    const long long tiles = (rows + TM - 1) / TM;
    long long tpc = tiles * nprob / (2 * 152);
    return (int)std::max(1LL, std::min(tpc, 8LL));
}

template <bool A>
cudaError_t launch_tc(const DftStage& s, int nprob, unsigned long long* work, cudaStream_t st)
{
    static int optin[64];
    const size_t sm = smem_tc(s.Rp);
    cudaError_t e = ensure_smem_optin((const void*)k_dft_tc<A>, (int)sm, optin);
    if (e != cudaSuccess) return e;
    const long long rows = A ? (long long)s.L * s.Q : (long long)s.M;
    const int tpc = tiles_per_cta(rows, nprob);
    const long long ctas = (rows + (long long)TM * tpc - 1) / ((long long)TM * tpc);
    dim3 grid((unsigned)ctas, 1, nprob);
    k_dft_tc<A><<<grid, NT, sm, st>>>(s, tpc, work);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dft_matrix(int R, int Rp, float sign, __nv_bfloat16* F, cudaStream_t st)
{
    k_dft_matrix<<<(Rp * Rp + 255) / 256, 256, 0, st>>>(R, Rp, sign, F);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_dft_stage_a(const DftStage& s, int nprob, unsigned long long* work,
                               cudaStream_t st)
{
    return launch_tc<true>(s, nprob, work, st);
}

cudaError_t launch_dft_stage_b(const DftStage& s, int nprob, unsigned long long* work,
                               cudaStream_t st)
{
    return launch_tc<false>(s, nprob, work, st);
}
