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
// of the result) with float32 accumulation, and a complex product is four real
// ones with the sign of Im(F) folded into the bf16 sign bits: 12
// mma.m16n8k16 per complex 16 x 8 x 16 block.
#include <math.h>
#include <stdint.h>

#include "conv_dft.cuh"

namespace {

constexpr int NT = 128;   // 4 warps
constexpr int QT = 64;    // orientation A: q columns per CTA tile (16 per warp)
constexpr int MTILE = 64; // orientation B: rows per CTA tile (16 per warp)
constexpr int LPB = 8;    // tiles per CTA (the DFT matrix is staged once for them)

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l)
{
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment (16 x 16, element (m, k) at P[m * ld + k]) at origin (m0, k0)
__device__ __forceinline__ void frag_a(uint32_t* a, const __nv_bfloat16* P, int ld, int m0, int k0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    a[0] = *reinterpret_cast<const uint32_t*>(P + (m0 + g) * ld + k0 + 2 * t);
    a[1] = *reinterpret_cast<const uint32_t*>(P + (m0 + g + 8) * ld + k0 + 2 * t);
    a[2] = *reinterpret_cast<const uint32_t*>(P + (m0 + g) * ld + k0 + 2 * t + 8);
    a[3] = *reinterpret_cast<const uint32_t*>(P + (m0 + g + 8) * ld + k0 + 2 * t + 8);
}

// B fragment (16 x 8, element (k, n) at P[n * ld + k]) at origin (n0, k0)
__device__ __forceinline__ void frag_b(uint32_t* b, const __nv_bfloat16* P, int ld, int n0, int k0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    b[0] = *reinterpret_cast<const uint32_t*>(P + (n0 + g) * ld + k0 + 2 * t);
    b[1] = *reinterpret_cast<const uint32_t*>(P + (n0 + g) * ld + k0 + 2 * t + 8);
}

__device__ __forceinline__ void neg2(uint32_t* d, const uint32_t* s, int n)
{
    for (int i = 0; i < n; ++i) d[i] = s[i] ^ 0x80008000u;
}

// (re, im) += F * X for one 16 x 8 x 16 block; F planes f[0..3] = re hi, re lo,
// im hi, im lo (A or B role per `f_is_a`), X planes x[0..3] likewise.
__device__ __forceinline__ void cmma_fa(float* cre, float* cim, const uint32_t (*f)[4],
                                        const uint32_t (*x)[2])
{
    uint32_t nh[4], nl[4];
    neg2(nh, f[2], 4);
    neg2(nl, f[3], 4);
    mma16816(cre, f[0], x[0]);
    mma16816(cre, f[0], x[1]);
    mma16816(cre, f[1], x[0]);
    mma16816(cre, nh, x[2]);
    mma16816(cre, nh, x[3]);
    mma16816(cre, nl, x[2]);
    mma16816(cim, f[0], x[2]);
    mma16816(cim, f[0], x[3]);
    mma16816(cim, f[1], x[2]);
    mma16816(cim, f[2], x[0]);
    mma16816(cim, f[2], x[1]);
    mma16816(cim, f[3], x[0]);
}

// same with the data as the A operand and F as B: (re, im) += X * F^T
__device__ __forceinline__ void cmma_fb(float* cre, float* cim, const uint32_t (*x)[4],
                                        const uint32_t (*f)[2])
{
    uint32_t nh[2], nl[2];
    neg2(nh, f[2], 2);
    neg2(nl, f[3], 2);
    mma16816(cre, x[0], f[0]);
    mma16816(cre, x[1], f[0]);
    mma16816(cre, x[0], f[1]);
    mma16816(cre, x[2], nh);
    mma16816(cre, x[3], nh);
    mma16816(cre, x[2], nl);
    mma16816(cim, x[2], f[0]);
    mma16816(cim, x[3], f[0]);
    mma16816(cim, x[2], f[1]);
    mma16816(cim, x[0], f[2]);
    mma16816(cim, x[1], f[2]);
    mma16816(cim, x[0], f[3]);
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

// stage the 4 F planes (Rp x Rp) into shared memory with row stride LD
__device__ __forceinline__ void stage_f(__nv_bfloat16* Fs, const DftStage& s, int LD)
{
    const int Rp = s.Rp, n = 4 * Rp * Rp;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int pl = i / (Rp * Rp), rem = i - pl * Rp * Rp, k = rem / Rp, r = rem - k * Rp;
        Fs[(pl * Rp + k) * LD + r] = s.F[i];
    }
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

// Orientation A: OUT[p][l][k][q] = tw * sum_r F[k][r] IN[p][l][r][q].  A CTA holds
// the whole k range for QT columns q of LPB consecutive l.
__global__ void __launch_bounds__(NT) k_dft_a(DftStage s, unsigned long long* work)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Rp = s.Rp, R = s.R, LD = Rp + 8;
    __nv_bfloat16* Fs = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // 4 x Rp x LD
    __nv_bfloat16* Xs = Fs + 4 * Rp * LD;                             // 4 x QT x LD, [q][r]
    const int p = blockIdx.z, q0 = blockIdx.x * QT;
    if (s.lm && s.lm[p / s.nchan].phase != s.phase) return;
    stage_f(Fs, s, LD);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nmt = Rp / 16, nkt = Rp / 16;
    for (int li = 0; li < LPB; ++li) {
        const int l = blockIdx.y * LPB + li;
        if (l >= s.L) break;
        if (s.out_mode == 1 && (l < s.crop_y0 || l >= s.crop_y0 + s.crop_H)) continue;
        __syncthreads();  // Fs staged / previous tile's Xs consumed
        for (int i = threadIdx.x; i < Rp * QT; i += NT) {
            const int r = i / QT, qq = i - r * QT, q = q0 + qq;
            const float2 v = (r < R && q < s.Q) ? in_a(s, p, l, r, q) : make_float2(0.f, 0.f);
            __nv_bfloat16 h, lo;
            split_bf16(v.x, h, lo);
            Xs[(0 * QT + qq) * LD + r] = h;
            Xs[(1 * QT + qq) * LD + r] = lo;
            split_bf16(v.y, h, lo);
            Xs[(2 * QT + qq) * LD + r] = h;
            Xs[(3 * QT + qq) * LD + r] = lo;
        }
        __syncthreads();
        float acc[4][2][2][4];  // [mtile][ntile][re/im][c]
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int d = 0; d < 4; ++d) acc[a][b][c][d] = 0.0f;
        for (int kt = 0; kt < nkt; ++kt) {
            uint32_t xb[2][4][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int pl = 0; pl < 4; ++pl)
                    frag_b(xb[nt][pl], Xs + pl * QT * LD, LD, 16 * warp + 8 * nt, 16 * kt);
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                if (mt >= nmt) break;
                uint32_t fa[4][4];
#pragma unroll
                for (int pl = 0; pl < 4; ++pl) frag_a(fa[pl], Fs + pl * Rp * LD, LD, 16 * mt, 16 * kt);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) cmma_fa(acc[mt][nt][0], acc[mt][nt][1], fa, xb[nt]);
            }
        }
        // epilogue: twiddle and store
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            if (mt >= nmt) break;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int hf = 0; hf < 2; ++hf)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int k = 16 * mt + g + 8 * hf;
                        const int q = q0 + 16 * warp + 8 * nt + 2 * t + j;
                        if (k >= R || q >= s.Q) continue;
                        float2 v = make_float2(acc[mt][nt][0][2 * hf + j], acc[mt][nt][1][2 * hf + j]);
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
                    }
        }
        if (work && threadIdx.x == 0) {
            const int qv = min(QT, s.Q - q0);
            atomicAdd(work, (unsigned long long)(8ull * R * R * qv));  // complex MACs x 8 FLOP
        }
    }
}

// Orientation B: OUT[p][m][k] = tw * sum_r IN[p][m][r] F[k][r].  A CTA holds the
// whole k range for MTILE rows of LPB consecutive row tiles.
__global__ void __launch_bounds__(NT) k_dft_b(DftStage s, unsigned long long* work)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Rp = s.Rp, R = s.R, LD = Rp + 8;
    __nv_bfloat16* Fs = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // 4 x Rp x LD, [k][r]
    __nv_bfloat16* Xs = Fs + 4 * Rp * LD;                             // 4 x MTILE x LD, [m][r]
    const int p = blockIdx.z;
    if (s.lm && s.lm[p / s.nchan].phase != s.phase) return;
    stage_f(Fs, s, LD);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nnt = Rp / 8, nkt = Rp / 16;
    for (int ti = 0; ti < LPB; ++ti) {
        const int m0 = (blockIdx.x * LPB + ti) * MTILE;
        if (m0 >= s.M) break;
        __syncthreads();
        for (int i = threadIdx.x; i < MTILE * Rp; i += NT) {
            const int mm = i / Rp, r = i - mm * Rp, m = m0 + mm;
            float2 v = make_float2(0.f, 0.f);
            if (r < R && m < s.M) v = s.in[(long long)p * s.in_pstride + (long long)m * R + r];
            __nv_bfloat16 h, lo;
            split_bf16(v.x, h, lo);
            Xs[(0 * MTILE + mm) * LD + r] = h;
            Xs[(1 * MTILE + mm) * LD + r] = lo;
            split_bf16(v.y, h, lo);
            Xs[(2 * MTILE + mm) * LD + r] = h;
            Xs[(3 * MTILE + mm) * LD + r] = lo;
        }
        __syncthreads();
        float acc[8][2][4];  // [ntile][re/im][c]
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int d = 0; d < 4; ++d) acc[a][c][d] = 0.0f;
        for (int kt = 0; kt < nkt; ++kt) {
            uint32_t xa[4][4];
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) frag_a(xa[pl], Xs + pl * MTILE * LD, LD, 16 * warp, 16 * kt);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                if (nt >= nnt) break;
                uint32_t fb[4][2];
#pragma unroll
                for (int pl = 0; pl < 4; ++pl) frag_b(fb[pl], Fs + pl * Rp * LD, LD, 8 * nt, 16 * kt);
                cmma_fb(acc[nt][0], acc[nt][1], xa, fb);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= nnt) break;
#pragma unroll
            for (int hf = 0; hf < 2; ++hf)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int m = m0 + 16 * warp + g + 8 * hf;
                    const int k = 8 * nt + 2 * t + j;
                    if (m >= s.M || k >= R) continue;
                    float2 v = make_float2(acc[nt][0][2 * hf + j], acc[nt][1][2 * hf + j]);
                    if (s.tw_mode == 3) v = cmulf(v, twiddle(s, (m % s.tw_mod) * k));
                    s.out[(long long)p * s.out_pstride + (long long)m * R + k] = v;
                }
        }
        if (work && threadIdx.x == 0) {
            const int mv = min(MTILE, s.M - m0);
            atomicAdd(work, (unsigned long long)(8ull * R * R * mv));
        }
    }
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

size_t smem_a(int Rp) { return sizeof(__nv_bfloat16) * 4 * (size_t)(Rp + QT) * (Rp + 8); }
size_t smem_b(int Rp) { return sizeof(__nv_bfloat16) * 4 * (size_t)(Rp + MTILE) * (Rp + 8); }

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
    static int optin[64];
    const size_t sm = smem_a(s.Rp);
    cudaError_t e = ensure_smem_optin((const void*)k_dft_a, (int)sm, optin);
    if (e != cudaSuccess) return e;
    dim3 grid((s.Q + QT - 1) / QT, (s.L + LPB - 1) / LPB, nprob);
    k_dft_a<<<grid, NT, sm, st>>>(s, work);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_dft_stage_b(const DftStage& s, int nprob, unsigned long long* work,
                               cudaStream_t st)
{
    static int optin[64];
    const size_t sm = smem_b(s.Rp);
    cudaError_t e = ensure_smem_optin((const void*)k_dft_b, (int)sm, optin);
    if (e != cudaSuccess) return e;
    const int tiles = (s.M + MTILE - 1) / MTILE;
    dim3 grid((tiles + LPB - 1) / LPB, 1, nprob);
    k_dft_b<<<grid, NT, sm, st>>>(s, work);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}
