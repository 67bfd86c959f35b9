// warp_fft.cuh -- one complex FFT of length N = 32 M per warp, in registers.
//
// Lane l holds the M inputs x[l + 32 j] (j < M).  With n = l + 32 j and
// k = k2 + M k1 the transform factors as
//   X[k2 + M k1] = sum_l e^{s 2 pi i l k1 / 32} e^{s 2 pi i l k2 / N}
//                        sum_j x[l + 32 j] e^{s 2 pi i j k2 / M}
// (s = -1 forward, +1 inverse), so each lane
//   1. takes an M-point DFT of its own registers (M = A B, two levels of
//      direct small DFTs with compile-time indices: no shared memory, no
//      barrier),
//   2. multiplies value k2 by the twiddle e^{s 2 pi i l k2 / N},
//   3. joins a 32-point DFT across the lanes for each k2: five radix-2
//      decimation-in-frequency stages of butterflies between lanes l and l ^ d
//      by register shuffles.
// Lane l then holds X[k2 + M bitrev5(l)] in register k2.  Every twiddle comes
// from the table tw[k] = e^{-2 pi i k / N} (made in FP64 by k_twiddles); the
// inverse conjugates it.  The table is kept in shared memory with one pad
// element after every 16 (index t -> t + t / 16) so that the lanes' strided
// reads of step 2 mostly fall in different banks.
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"

// the factorisation M = A B of the in-register DFT, for the supported M
template <int M> struct WarpFFTFactor;
#define WARP_FFT_FACTOR(M_, A_, B_)                 \
    template <> struct WarpFFTFactor<M_> {          \
        static constexpr int A = A_, B = B_;        \
    }
WARP_FFT_FACTOR(3, 1, 3);
WARP_FFT_FACTOR(4, 2, 2);
WARP_FFT_FACTOR(5, 1, 5);
WARP_FFT_FACTOR(6, 2, 3);
WARP_FFT_FACTOR(8, 2, 4);
WARP_FFT_FACTOR(9, 3, 3);
WARP_FFT_FACTOR(10, 2, 5);
WARP_FFT_FACTOR(12, 3, 4);
WARP_FFT_FACTOR(15, 3, 5);
WARP_FFT_FACTOR(16, 4, 4);
WARP_FFT_FACTOR(18, 3, 6);
WARP_FFT_FACTOR(20, 4, 5);
#undef WARP_FFT_FACTOR

__host__ __device__ constexpr int warp_fft_pad(int t) { return t + t / 16; }
__host__ __device__ constexpr int warp_fft_table_len(int n) { return warp_fft_pad(n - 1) + 1; }

// acc + a w (complex)
__device__ __forceinline__ float2 cfma2(float2 a, float2 w, float2 acc)
{
    return make_float2(fmaf(a.x, w.x, fmaf(-a.y, w.y, acc.x)), fmaf(a.x, w.y, fmaf(a.y, w.x, acc.y)));
}

// table entry t of the padded shared table, conjugated for the inverse
template <bool INV>
__device__ __forceinline__ float2 wf_tw(const float2* tws, int t)
{
    const float2 w = tws[warp_fft_pad(t)];
    return INV ? make_float2(w.x, -w.y) : w;
}

// The M-point DFT of v (in place, natural order in and out); rm[k] is
// e^{s 2 pi i k / M}.
template <int M>
__device__ __forceinline__ void wf_reg_dft(float2 (&v)[M], const float2 (&rm)[M])
{
    constexpr int A = WarpFFTFactor<M>::A, B = WarpFFTFactor<M>::B;
    float2 z[M];
    // B-point DFTs over j2 of v[j1 + A j2], twiddled by e^{s 2 pi i j1 k2 / M}
#pragma unroll
    for (int j1 = 0; j1 < A; ++j1) {
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            float2 acc = v[j1];
#pragma unroll
            for (int j2 = 1; j2 < B; ++j2) {
                const int e = ((j2 * k2) % B) * A;
                if (e == 0)
                    acc = cadd(acc, v[j1 + A * j2]);
                else
                    acc = cfma2(v[j1 + A * j2], rm[e], acc);
            }
            const int t = (j1 * k2) % M;
            z[j1 + A * k2] = (t == 0) ? acc : cmul(acc, rm[t]);
        }
    }
    // A-point DFTs over j1 for each k2: output k2 + B k1
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) {
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            float2 acc = z[A * k2];
#pragma unroll
            for (int j1 = 1; j1 < A; ++j1) {
                const int e = ((j1 * k1) % A) * B;
                if (e == 0)
                    acc = cadd(acc, z[j1 + A * k2]);
                else
                    acc = cfma2(z[j1 + A * k2], rm[e], acc);
            }
            v[k2 + B * k1] = acc;
        }
    }
}

// The FFT of the warp's N = 32 M values (lane l holds x[l + 32 j] in v[j]);
// tws is the padded shared table of e^{-2 pi i k / N}.  On return lane l holds
// X[k2 + M bitrev5(l)] in v[k2].
template <int M, bool INV>
__device__ __forceinline__ void warp_fft(float2 (&v)[M], const float2* tws)
{
    constexpr int N = 32 * M;
    const int l = threadIdx.x & 31;
    float2 rm[M];
#pragma unroll
    for (int k = 0; k < M; ++k) rm[k] = wf_tw<INV>(tws, 32 * k);
    wf_reg_dft<M>(v, rm);
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) v[k2] = cmul(v[k2], wf_tw<INV>(tws, l * k2));
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const bool upper = (l & d) != 0;
        const float2 w = wf_tw<INV>(tws, (l & (d - 1)) * (N / (2 * d)));
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) {
            const float px = __shfl_xor_sync(0xffffffffu, v[k2].x, d);
            const float py = __shfl_xor_sync(0xffffffffu, v[k2].y, d);
            const float2 p = make_float2(px, py);
            v[k2] = upper ? cmul(csub(p, v[k2]), w) : cadd(v[k2], p);
        }
    }
}

__device__ __forceinline__ int bitrev5(int l) { return (int)(__brev((unsigned)l) >> 27); }

// The twiddles one lane's warp_fft reads, kept in registers by a kernel that
// runs many transforms of one length.  The butterfly of stage d then becomes
// a = p + sg v (sg = -1 on the upper lane of the pair, +1 on the lower) and
// v = a ws: the lower lane's factor is 1, and the last stage (d = 1, factor 1
// on both lanes) has no product.  Every value is the one warp_fft computes.
template <int M>
struct WarpTw {
    float2 rm[M];  // e^{-2 pi i k / M}
    float2 tl[M];  // e^{-2 pi i l k2 / N}
    float2 ws[4];  // stages d = 16, 8, 4, 2: the upper lane's twiddle, 1 on the lower
    float sg[5];   // stages d = 16 .. 1: -1 on the upper lane, +1 on the lower
};

template <int M>
__device__ __forceinline__ void warp_tw_load(WarpTw<M>& t, const float2* tws)
{
    constexpr int N = 32 * M;
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        t.rm[k] = wf_tw<false>(tws, 32 * k);
        t.tl[k] = wf_tw<false>(tws, l * k);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int d = 16 >> i;
        const bool upper = (l & d) != 0;
        t.sg[i] = upper ? -1.0f : 1.0f;
        if (i < 4) t.ws[i] = upper ? wf_tw<false>(tws, (l & (d - 1)) * (N / (2 * d))) : make_float2(1.0f, 0.0f);
    }
}

template <bool INV>
__device__ __forceinline__ float2 wf_dir(float2 w)
{
    return INV ? make_float2(w.x, -w.y) : w;
}

// warp_fft with the lane's twiddles in registers (same layout in and out,
// same values)
template <int M, bool INV>
__device__ __forceinline__ void warp_fft_r(float2 (&v)[M], const WarpTw<M>& t)
{
    float2 rm[M];
#pragma unroll
    for (int k = 0; k < M; ++k) rm[k] = wf_dir<INV>(t.rm[k]);
    wf_reg_dft<M>(v, rm);
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) v[k2] = cmul(v[k2], wf_dir<INV>(t.tl[k2]));
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int d = 16 >> i;
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) {
            const float px = __shfl_xor_sync(0xffffffffu, v[k2].x, d);
            const float py = __shfl_xor_sync(0xffffffffu, v[k2].y, d);
            const float2 a = make_float2(fmaf(t.sg[i], v[k2].x, px), fmaf(t.sg[i], v[k2].y, py));
            v[k2] = i < 4 ? cmul(a, wf_dir<INV>(t.ws[i])) : a;
        }
    }
}
