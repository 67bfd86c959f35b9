// fft.cuh -- shared-memory complex FFT used by the Fourier-space convolution.
//
// Stockham autosort formulation (Govindaraju et al., SC 2008): a length
// N = r_1 r_2 ... r_s transform runs s stages; stage t with radix R and span
// Ns = r_1 ... r_{t-1} reads the butterfly inputs in[j + m N/R] (m < R),
// multiplies input m by w^{m k}, k = j mod Ns, w = exp(sign 2 pi i / (Ns R)),
// applies an R-point DFT, and writes out[(j / Ns) Ns R + k + m Ns].  The output
// comes out in natural order, so no bit reversal is needed; stages alternate
// between two shared buffers.
//
// B independent sequences (B a power of two) are transformed at once with
// element (y, b) at index y * B + b, so that consecutive threads touch
// consecutive addresses.  No stage divides at run time: the sequence index is a
// shift, and j / Ns is a multiply-high by a precomputed reciprocal (exact for
// j, Ns < 2^16).
#pragma once

#include <cuda_runtime.h>

#define FFT_MAX_STAGES 24

struct FFTPlan {
    int n;                        // length
    int nst;                      // stages
    int radix[FFT_MAX_STAGES];    // radix of each stage (2, 3, 4, 5 or 8)
    int ns[FFT_MAX_STAGES];       // span Ns before the stage (product of earlier radices)
    unsigned mag[FFT_MAX_STAGES]; // ceil(2^32 / Ns) for Ns > 1
    int twstep[FFT_MAX_STAGES];   // n / (Ns R): twiddle w_{Ns R}^e = tw[e * twstep]
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by sign * i
__device__ __forceinline__ float2 cmul_si(float2 a, float s) { return make_float2(-s * a.y, s * a.x); }

// R-point DFTs with exponent sign s (-1 forward, +1 inverse), in place
__device__ __forceinline__ void dft2(float2* v)
{
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

__device__ __forceinline__ void dft4(float2* v, float s)
{
    const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const float2 t2 = cadd(v[1], v[3]), t3 = cmul_si(csub(v[1], v[3]), s);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}

__device__ __forceinline__ void dft3(float2* v, float s)
{
    // w = exp(s 2 pi i / 3) = -1/2 + s i sqrt(3)/2
    const float c = -0.5f, sn = 0.86602540378443864676f;
    const float2 a = v[0], b = v[1], d = v[2];
    const float2 t = cadd(b, d);
    const float2 u = make_float2(fmaf(c, t.x, a.x), fmaf(c, t.y, a.y));
    const float2 w = cmul_si(csub(b, d), s * sn);
    v[0] = cadd(a, t);
    v[1] = cadd(u, w);
    v[2] = csub(u, w);
}

__device__ __forceinline__ void dft5(float2* v, float s)
{
    // cos/sin of 2 pi / 5 and 4 pi / 5
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 a = v[0];
    const float2 p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
    const float2 p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
    const float2 r1 = make_float2(a.x + c1 * p1.x + c2 * p2.x, a.y + c1 * p1.y + c2 * p2.y);
    const float2 r2 = make_float2(a.x + c2 * p1.x + c1 * p2.x, a.y + c2 * p1.y + c1 * p2.y);
    // i s (s1 m1 + s2 m2) and i s (s2 m1 - s1 m2)
    const float2 q1 = cmul_si(make_float2(s1 * m1.x + s2 * m2.x, s1 * m1.y + s2 * m2.y), s);
    const float2 q2 = cmul_si(make_float2(s2 * m1.x - s1 * m2.x, s2 * m1.y - s1 * m2.y), s);
    v[0] = make_float2(a.x + p1.x + p2.x, a.y + p1.y + p2.y);
    v[1] = cadd(r1, q1);
    v[4] = csub(r1, q1);
    v[2] = cadd(r2, q2);
    v[3] = csub(r2, q2);
}

// 8-point DFT as two 4-point DFTs: split m = m1 + 4 m2; even outputs are the
// DFT4 of v[m1] + v[m1+4], odd outputs the DFT4 of w^m1 (v[m1] - v[m1+4]),
// w = exp(s 2 pi i / 8)
__device__ __forceinline__ void dft8(float2* v, float s)
{
    const float h = 0.70710678118654752440f;
    float2 a[4], b[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        a[m] = cadd(v[m], v[m + 4]);
        b[m] = csub(v[m], v[m + 4]);
    }
    b[1] = make_float2(h * (b[1].x - s * b[1].y), h * (b[1].y + s * b[1].x));
    b[2] = cmul_si(b[2], s);
    b[3] = make_float2(h * (-b[3].x - s * b[3].y), h * (-b[3].y + s * b[3].x));
    dft4(a, s);
    dft4(b, s);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        v[2 * m] = a[m];
        v[2 * m + 1] = b[m];
    }
}

template <int R>
__device__ __forceinline__ void dft_r(float2* v, float s)
{
    if (R == 2) dft2(v);
    else if (R == 3) dft3(v, s);
    else if (R == 4) dft4(v, s);
    else if (R == 5) dft5(v, s);
    else dft8(v, s);
}

// one Stockham stage of radix R over B = 2^logB interleaved sequences of length n
template <int R>
__device__ __forceinline__ void fft_stage(int n, int Ns, unsigned mag, int twstep,
                                          const float2* __restrict__ src,
                                          float2* __restrict__ dst, int logB, const float2* tw,
                                          float sign)
{
    const int nb = n / R;  // butterflies per sequence
    const int B = 1 << logB, total = nb << logB;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int j = t >> logB, q = t & (B - 1);
        const int jd = Ns > 1 ? (int)__umulhi((unsigned)j, mag) : j;  // j / Ns
        const int k = j - jd * Ns;                                    // j mod Ns
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = src[((j + m * nb) << logB) + q];
        if (Ns > 1) {
#pragma unroll
            for (int m = 1; m < R; ++m) {
                float2 w = tw[m * k * twstep];
                if (sign > 0.0f) w = cconj(w);
                v[m] = cmul(v[m], w);
            }
        }
        dft_r<R>(v, sign);
        const int base = jd * Ns * R + k;
#pragma unroll
        for (int m = 0; m < R; ++m) dst[((base + m * Ns) << logB) + q] = v[m];
    }
}

// One FFT of each of 2^logB interleaved sequences held in `a` (shared memory),
// using `b` as the second buffer.  tw[k] = exp(-2 pi i k / n) for k < n
// (shared or global).  sign = -1 forward, +1 inverse (unnormalised).  All
// threads of the block call it; it ends with a barrier.  Returns the buffer
// that holds the result.
static __device__ float2* fft_smem(const FFTPlan& pl, float2* a, float2* b, int logB,
                                   const float2* tw, float sign)
{
    const int n = pl.n;
    float2* src = a;
    float2* dst = b;
    for (int st = 0; st < pl.nst; ++st) {
        const int Ns = pl.ns[st];
        const unsigned mag = pl.mag[st];
        const int tws = pl.twstep[st];
        switch (pl.radix[st]) {
        case 2: fft_stage<2>(n, Ns, mag, tws, src, dst, logB, tw, sign); break;
        case 3: fft_stage<3>(n, Ns, mag, tws, src, dst, logB, tw, sign); break;
        case 4: fft_stage<4>(n, Ns, mag, tws, src, dst, logB, tw, sign); break;
        case 5: fft_stage<5>(n, Ns, mag, tws, src, dst, logB, tw, sign); break;
        default: fft_stage<8>(n, Ns, mag, tws, src, dst, logB, tw, sign); break;
        }
        __syncthreads();
        float2* t = src;
        src = dst;
        dst = t;
    }
    return src;
}
