// cnn.cu -- the learned initial guess: a small convolutional network that maps
// a 64x64 stamp to the eight regression targets of a single Sersic component,
// its training data drawn on the device, the moments-based default guess, and
// the choice between the two starts.
//
// Network (NCHW, one 64x64 input channel, zero padding 1, stride 2, ReLU after
// every layer but the last):
//   conv 3x3 1->32 (64->32), 32->64 (32->16), 64->64 (16->8), 64->128 (8->4),
//   fc 2048->32, fc 32->8.
// Weights and activations are bf16, every accumulation float32.  The master
// parameters are float32, packed layer by layer as weights [out][in][ky][kx]
// (fc: [out][in]) then biases [out] -- 195432 in all.  Two bf16 copies of the
// convolution weights are kept: [in][tap][out] for the forward pass (eight
// consecutive output channels per 16-byte load; the first layer's SIMT loop and
// the tensor-core input gradients read it) and [out][tap][in] (the tensor-core
// forward's B operand).  The convolution layers' activations and gradients are
// channels-last except conv4's output, which is stored in the [c][y][x] order
// fc1 flattens.  Convolutions 2-4 run on the tensor cores in both directions
// (cnn_tc.cu, cnn_bwd_tc.cu); this file holds the first convolution, the fully
// connected layers, the loss and Adam.  Every reduction runs in a fixed order,
// so a training run is reproducible bit for bit.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "bn.cuh"
#include "cnn.cuh"
#include "gf_internal.cuh"

namespace {

struct ConvL {
    int cin, cout, hin, hout;
    int woff, boff;  // offsets in the master parameter array
};

#define CONV_TABLE                                                                              \
    {                                                                                           \
        {1, 32, 64, 32, 0, 288}, {32, 64, 32, 16, 320, 18752}, {64, 64, 16, 8, 18816, 55680}, \
            {64, 128, 8, 4, 55744, 129472}                                                      \
    }
constexpr ConvL CONV[4] = CONV_TABLE;
__constant__ ConvL c_conv[4] = CONV_TABLE;

constexpr int FC1_W = 129600, FC1_B = 195136, FC2_W = 195168, FC2_B = 195424;
constexpr int NPARAM = CNN_NPARAM;
constexpr int CONV_W_END = 129600;  // the conv weights and biases occupy [0, CONV_W_END)
constexpr int SIDE = CNN_SIDE, NPIX = SIDE * SIDE, NOUT = CNN_NOUT;

__device__ __forceinline__ void unpack8(const uint4 u, float* f)
{
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

inline int blocks(long long n, int t) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------- forward
// fc1: thread = (b, o); input the flattened conv4 output (bf16), output float32 after ReLU
__global__ void k_fc1_fwd(const __nv_bfloat16* __restrict__ a3, const __nv_bfloat16* __restrict__ w,
                          const float* __restrict__ master, float* __restrict__ h, int B)
{
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B * 32) return;
    const int b = item / 32, o = item - b * 32;
    const __nv_bfloat16* xr = a3 + (long long)b * 2048;
    const __nv_bfloat16* wr = w + FC1_W + o * 2048;
    float acc = master[FC1_B + o];
    for (int i = 0; i < 2048; i += 8) {
        float xv[8], wv[8];
        unpack8(*reinterpret_cast<const uint4*>(xr + i), xv);
        unpack8(*reinterpret_cast<const uint4*>(wr + i), wv);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc = fmaf(xv[j], wv[j], acc);
    }
    h[item] = fmaxf(acc, 0.0f);
}

// fc2: thread = (b, j); linear output
__global__ void k_fc2_fwd(const float* __restrict__ h, const __nv_bfloat16* __restrict__ w,
                          const float* __restrict__ master, float* __restrict__ y, int B)
{
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B * NOUT) return;
    const int b = item / NOUT, j = item - b * NOUT;
    float acc = master[FC2_B + j];
    for (int o = 0; o < 32; ++o)
        acc = fmaf(__bfloat162float(w[FC2_W + j * 32 + o]), h[b * 32 + o], acc);
    y[item] = acc;
}

// ------------------------------------------------------------------ loss
// loss = mean (y - t)^2 over B x 8 (one block, fixed-order tree); gy = dloss/dy
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ gy,
                      float* __restrict__ loss, int B)
{
    __shared__ float part[256];
    const int n = B * NOUT;
    const float scale = 1.0f / (float)n;
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float e = y[i] - t[i];
        gy[i] = 2.0f * e * scale;
        s = fmaf(e, e, s);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] * scale;
}

// -------------------------------------------------------------- backward
// fc2: weight/bias gradients (thread per (j, o) / j, summed over the batch)
__global__ void k_fc2_bwd_w(const float* __restrict__ gy, const float* __restrict__ h,
                            float* __restrict__ grad, int B)
{
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item < NOUT * 32) {
        const int j = item / 32, o = item - j * 32;
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s = fmaf(gy[b * NOUT + j], h[b * 32 + o], s);
        grad[FC2_W + item] = s;
    } else if (item < NOUT * 32 + NOUT) {
        const int j = item - NOUT * 32;
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s += gy[b * NOUT + j];
        grad[FC2_B + j] = s;
    }
}

// gradient at fc1's pre-activation
__global__ void k_fc2_bwd_x(const float* __restrict__ gy, const float* __restrict__ h,
                            const __nv_bfloat16* __restrict__ w, float* __restrict__ gh, int B)
{
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B * 32) return;
    const int b = item / 32, o = item - b * 32;
    float s = 0.0f;
    for (int j = 0; j < NOUT; ++j) s = fmaf(__bfloat162float(w[FC2_W + j * 32 + o]), gy[b * NOUT + j], s);
    gh[item] = h[item] > 0.0f ? s : 0.0f;
}

// fc1 weight (thread per (o, i)) and bias gradients
__global__ void k_fc1_bwd_w(const float* __restrict__ gh, const __nv_bfloat16* __restrict__ a3,
                            float* __restrict__ grad, int B)
{
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item < 32 * 2048) {
        const int o = item / 2048, i = item - o * 2048;
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s = fmaf(gh[b * 32 + o], __bfloat162float(a3[(long long)b * 2048 + i]), s);
        grad[FC1_W + item] = s;
    } else if (item < 32 * 2048 + 32) {
        const int o = item - 32 * 2048;
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s += gh[b * 32 + o];
        grad[FC1_B + o] = s;
    }
}

// gradient at conv4's pre-activation (through its ReLU), written channels-last
// (b, pixel, channel) for the tensor-core backward; the flattened input index i
// of fc1 is channel * 16 + pixel (conv4's NCHW output)
__global__ void k_fc1_bwd_x(const float* __restrict__ gh, const __nv_bfloat16* __restrict__ a3,
                            const __nv_bfloat16* __restrict__ w, float* __restrict__ g3, int B)
{
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (long long)B * 2048) return;
    const int b = (int)(item / 2048), i = (int)(item - (long long)b * 2048);
    float s = 0.0f;
    for (int o = 0; o < 32; ++o) s = fmaf(__bfloat162float(w[FC1_W + o * 2048 + i]), gh[b * 32 + o], s);
    const int c = i >> 4, pix = i & 15;
    g3[(long long)b * 2048 + pix * 128 + c] = __bfloat162float(a3[item]) > 0.0f ? s : 0.0f;
}

// Weight gradients of the first convolution (one input channel, nine taps per
// output channel: too narrow for the tensor cores), first stage: block =
// (output channel co, input channel ci, chunk of the batch); threads stride over
// (b, oy, ox) keeping the nine tap sums (and the bias sum); a fixed tree merges
// the threads.  gout is channels-last (b, oy, ox, co).
constexpr int WG_THREADS = 256;

__global__ void __launch_bounds__(WG_THREADS) k_conv_bwd_w(const float* __restrict__ gout,
                                                            const __nv_bfloat16* __restrict__ xin,
                                                            float* __restrict__ part, int B,
                                                            int cin, int hin, int cout, int hout,
                                                            int nchunk)
{
    __shared__ float red[10][WG_THREADS];
    const int co = blockIdx.x / cin, ci = blockIdx.x - co * cin, chunk = blockIdx.y;
    const int npix = hout * hout;
    const long long total = (long long)B * npix;
    const long long per = (total + nchunk - 1) / nchunk;
    const long long i0 = chunk * per, i1 = min(total, i0 + per);
    float s[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) s[k] = 0.0f;
    for (long long it = i0 + threadIdx.x; it < i1; it += WG_THREADS) {
        const int b = (int)(it / npix), pix = (int)(it - (long long)b * npix);
        const int oy = pix / hout, ox = pix - oy * hout;
        const float g = gout[((long long)b * npix + pix) * cout + co];
        if (g == 0.0f) continue;
        s[9] += g;
        const __nv_bfloat16* xb = xin + ((long long)b * cin + ci) * hin * hin;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int iy = 2 * oy - 1 + ky;
            if (iy < 0 || iy >= hin) continue;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int ix = 2 * ox - 1 + kx;
                if (ix < 0 || ix >= hin) continue;
                s[ky * 3 + kx] = fmaf(g, __bfloat162float(xb[iy * hin + ix]), s[ky * 3 + kx]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = WG_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    // part layout: [chunk][co][ci][10]
    if (threadIdx.x < 10)
        part[(((long long)chunk * cout + co) * cin + ci) * 10 + threadIdx.x] = red[threadIdx.x][0];
}

// second stage: the chunks summed in order into the packed master layout
__global__ void k_conv_bwd_w_sum(const float* __restrict__ part, float* __restrict__ grad, int cin,
                                 int cout, int nchunk, int woff, int boff)
{
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= cout * cin * 10) return;
    float s = 0.0f;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * cout * cin * 10 + item];
    const int k = item % 10, pair = item / 10, ci = pair % cin, co = pair / cin;
    if (k < 9)
        grad[woff + (co * cin + ci) * 9 + k] = s;
    else if (ci == 0)
        grad[boff + co] = s;
}

// ------------------------------------------------------------ optimiser
// Adam (Kingma & Ba 2015) on the float32 masters; c1, c2 = bias corrections
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 copies of the masters: the packed layout, plus the two transposed
// layouts of the convolution weights
__global__ void k_cast(const float* __restrict__ w, __nv_bfloat16* __restrict__ wp,
                       __nv_bfloat16* __restrict__ wf, __nv_bfloat16* __restrict__ wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
    wp[i] = h;
    if (i >= CONV_W_END) return;
    for (int l = 0; l < 4; ++l) {
        const ConvL L = c_conv[l];
        if (i < L.woff || i >= L.boff) continue;
        const int r = i - L.woff, co = r / (L.cin * 9), ci = (r / 9) % L.cin, tap = r % 9;
        wf[L.woff + (ci * 9 + tap) * L.cout + co] = h;  // [in][tap][out]
        wb[L.woff + (co * 9 + tap) * L.cin + ci] = h;   // [out][tap][in]
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011): ten rounds, each
// multiplying words 0 and 2 by the round constants 0xD2511F53 and 0xCD9E8D57,
// swapping in the high halves xored with the other words and the key, and
// bumping the key by the Weyl constants 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox(uint4 ctr, uint2 key)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, ctr.x), lo0 = 0xD2511F53u * ctr.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, ctr.z), lo1 = 0xCD9E8D57u * ctr.z;
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
    }
    return ctr;
}

__device__ __forceinline__ uint2 key_of(unsigned long long seed)
{
    return make_uint2((unsigned)seed, (unsigned)(seed >> 32));
}

// a uniform in (0, 1) from one 32-bit word
__device__ __forceinline__ double unit(unsigned r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

// one standard normal from counter (n, stream) by the Box-Muller transform
__device__ __forceinline__ float normal1(unsigned long long n, unsigned stream, uint2 key)
{
    const uint4 r = philox(make_uint4((unsigned)n, (unsigned)(n >> 32), stream, 0u), key);
    const float u1 = (float)unit(r.x), u2 = (float)unit(r.y);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__global__ void k_philox(const unsigned* __restrict__ in, unsigned* __restrict__ out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned* a = in + 6 * i;
    const uint4 r = philox(make_uint4(a[0], a[1], a[2], a[3]), make_uint2(a[4], a[5]));
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

// sigma^2 = sigma_read^2 + max(m, 0) / gain; d = m + sigma z
__global__ void k_noise(const float* __restrict__ m, long long n, unsigned long long seed, float sread,
                        float gain, float* __restrict__ d, float* __restrict__ sig)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = m[i];
    const float s = sqrtf(sread * sread + fmaxf(mi, 0.0f) / gain);
    d[i] = mi + s * normal1((unsigned long long)i, 0u, key_of(seed));
    sig[i] = s;
}

// He-normal initial weights N(0, 2 / fan_in), biases 0
__global__ void k_init(float* __restrict__ w, unsigned long long seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    int fan = 0;
    for (int l = 0; l < 4; ++l)
        if (i >= c_conv[l].woff && i < c_conv[l].boff) fan = c_conv[l].cin * 9;
    if (i >= FC1_W && i < FC1_B) fan = 2048;
    if (i >= FC2_W && i < FC2_B) fan = 32;
    w[i] = fan ? normal1((unsigned long long)i, 1u, key_of(seed)) * sqrtf(2.0f / (float)fan) : 0.0f;
}

// --------------------------------------------------- b_n and Sersic flux
// Regularised lower incomplete gamma by its power series
//   P(a, x) = x^a e^{-x} / Gamma(a+1) * sum_k x^k / ((a+1)...(a+k)),
// summed until a term no longer changes the sum (x < a here, so the terms fall).
__device__ double gamma_p(double a, double x, double lg1)
{
    if (x <= 0.0) return 0.0;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 400; ++k) {
        term *= x / (a + k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return exp(a * log(x) - x - lg1) * sum;
}

// b_n: root of P(2n, b) = 1/2 by Newton steps inside a bisection bracket
// (0, 2n), started from the asymptotic series of Ciotti & Bertin (1999).
__device__ double bn_of(double n)
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
        double nb = b - f / exp((a - 1.0) * log(b) - b - lga);
        if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
        const double step = fabs(nb - b);
        b = nb;
        if (step <= 1e-15 * b || hi - lo <= 1e-15 * b) break;
    }
    return b;
}

// the n-dependent factor e^{b} Gamma(2n) / b^{2n} of the closed-form flux
__device__ double sersic_flux_factor(double n)
{
    const double b = bn_of(n);
    return exp(b + lgamma(2.0 * n) - 2.0 * n * log(b));
}

// closed-form total flux of an elliptical Sersic component:
// 2 pi q I_e r_e^2 n e^{b} Gamma(2n) / b^{2n}, given its n-dependent factor e
__device__ double sersic_flux_e(double ie, double re, double n, double q, double e)
{
    return 2.0 * M_PI * q * ie * re * re * n * e;
}

__device__ double sersic_flux(double ie, double re, double n, double q)
{
    return sersic_flux_e(ie, re, n, q, sersic_flux_factor(n));
}

// the factor at n = 2 (the default guess's index), formed once per call by one
// thread instead of once per stamp (the b_n solve is a long serial FP64 chain)
__global__ void k_flux_factor_n2(double* __restrict__ e2) { *e2 = sersic_flux_factor(2.0); }

// ------------------------------------------------ network input scaling
template <class T>
__device__ void bitonic_sort(T* v, int n)  // n a power of two
{
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (j - 1));
                const int p = i + j;
                const bool up = (i & k) == 0;
                const T a = v[i], b = v[p];
                if ((a > b) == up) {
                    v[i] = b;
                    v[p] = a;
                }
            }
            __syncthreads();
        }
}

// pixel k of the outer ring: top row, bottom row, then the left and right
// columns without their corners
__device__ __forceinline__ void ring_ij(int k, int H, int W, int* i, int* j)
{
    if (k < W) {
        *i = 0;
        *j = k;
    } else if (k < 2 * W) {
        *i = H - 1;
        *j = k - W;
    } else if (k < 2 * W + (H - 2)) {
        *i = k - 2 * W + 1;
        *j = 0;
    } else {
        *i = k - 2 * W - (H - 2) + 1;
        *j = W - 1;
    }
}

// block per stamp: a = median of sigma over the outer ring (252 pixels, mean
// of the two middle values), x = asinh(img / a)
__global__ void __launch_bounds__(256) k_cnn_input(const float* __restrict__ img,
                                                    const float* __restrict__ sig,
                                                    float* __restrict__ x)
{
    __shared__ float v[256];
    const long long base = (long long)blockIdx.x * NPIX;
    constexpr int NR = 4 * SIDE - 4;
    if (threadIdx.x < NR) {
        int i, j;
        ring_ij(threadIdx.x, SIDE, SIDE, &i, &j);
        v[threadIdx.x] = sig[base + i * SIDE + j];
    } else {
        v[threadIdx.x] = INFINITY;
    }
    __syncthreads();
    bitonic_sort(v, 256);
    float a = 0.5f * (v[NR / 2 - 1] + v[NR / 2]);
    if (!(a > 0.0f)) a = 1.0f;
    for (int k = threadIdx.x; k < NPIX; k += blockDim.x) x[base + k] = asinhf(img[base + k] / a);
}

// ------------------------------------------------------ training stamps
// Stamp b of the training batch keyed by `seed`: the Sersic + sky parameters
// (9 slots) drawn from the training prior, and the Moffat PSF (beta 3, FWHM
// ~ U[2, 5]) on a psf_size^2 grid, normalised in float64.  Prior: centre
// (31.5, 31.5) + U[-1, 1] each; n ~ U[0.5, 6]; r_e log-uniform [2, 40];
// q ~ U[0.2, 1]; pa ~ U[0, 180); flux log-uniform [1e2, 1e5]; sky 0.05.
__global__ void __launch_bounds__(256) k_train_sample(unsigned long long seed, double* __restrict__ params,
                                                       float* __restrict__ psf, int psf_size)
{
    __shared__ double red[256];
    __shared__ double s_alpha;
    const int b = blockIdx.x;
    if (threadIdx.x < 32) {
        // warp 0: every lane draws the same values; the warp solves for b_n
        const uint2 key = key_of(seed);
        const uint4 r0 = philox(make_uint4((unsigned)b, 0u, 2u, 0u), key);
        const uint4 r1 = philox(make_uint4((unsigned)b, 1u, 2u, 0u), key);
        const double c = 0.5 * (SIDE - 1);
        const double n = 0.5 + 5.5 * unit(r0.z);
        const double bn = sersic_bn_warp(n, -1.0);
        const double re = exp(log(2.0) + (log(40.0) - log(2.0)) * unit(r0.w));
        const double q = 0.2 + 0.8 * unit(r1.x);
        const double pa = 180.0 * unit(r1.y);
        const double F = exp(log(1e2) + (log(1e5) - log(1e2)) * unit(r1.z));
        const double fwhm = 2.0 + 3.0 * unit(r1.w);
        double* p = params + 9 * (long long)b;
        if (threadIdx.x == 0) {
            p[0] = c - 1.0 + 2.0 * unit(r0.x);
            p[1] = c - 1.0 + 2.0 * unit(r0.y);
            p[2] = F / sersic_flux_e(1.0, re, n, q, exp(bn + lgamma(2.0 * n) - 2.0 * n * log(bn)));
            p[3] = re;
            p[4] = n;
            p[5] = q;
            p[6] = pa;
            p[7] = 0.0;
            p[8] = 0.05;
            s_alpha = fwhm / (2.0 * sqrt(exp2(1.0 / 3.0) - 1.0));
        }
    }
    __syncthreads();
    const int c = psf_size / 2, np = psf_size * psf_size;
    const double ia2 = 1.0 / (s_alpha * s_alpha);
    double s = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const int y = k / psf_size - c, x = k % psf_size - c;
        const double u = 1.0 + (double)(x * x + y * y) * ia2;
        s += 1.0 / (u * u * u);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double inv = 1.0 / red[0];
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const int y = k / psf_size - c, x = k % psf_size - c;
        const double u = 1.0 + (double)(x * x + y * y) * ia2;
        psf[(long long)b * np + k] = (float)(inv / (u * u * u));
    }
}

// targets of the first Sersic component (slots 0..6 of a stamp's parameters)
// a warp per stamp (the warp solves for b_n), lane 0 writes the targets
__global__ void k_encode(const double* __restrict__ params, int nslots, int count, int H, int W,
                         float* __restrict__ t)
{
    const int b = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= count) return;  // the whole warp
    const double* p = params + (long long)b * nslots;
    const double bn = sersic_bn_warp(p[4], -1.0);
    if ((threadIdx.x & 31) != 0) return;
    const double l10 = log(10.0);
    const double th = 2.0 * p[6] * M_PI / 180.0;
    float* o = t + (long long)b * NOUT;
    o[0] = (float)(p[0] - 0.5 * (W - 1));
    o[1] = (float)(p[1] - 0.5 * (H - 1));
    const double e = exp(bn + lgamma(2.0 * p[4]) - 2.0 * p[4] * log(bn));
    o[2] = (float)((log(sersic_flux_e(p[2], p[3], p[4], p[5], e)) - 3.5 * l10) / (1.5 * l10));
    o[3] = (float)((log(p[3]) - 0.5 * log(80.0)) / (0.5 * log(20.0)));
    o[4] = (float)((p[4] - 3.25) / 2.75);
    o[5] = (float)((p[5] - 0.6) / 0.4);
    o[6] = (float)cos(th);
    o[7] = (float)sin(th);
}

// inverse of k_encode: Sersic slots (c = 0) plus the sky slot copied from the
// default guess (and its centre, with GF_DECODE_MOMENT_CENTRE); I_e is NaN
// outside the closed-form flux domain
__global__ void k_decode(const float* __restrict__ y, const double* __restrict__ dflt, int count,
                         int H, int W, int flags, double* __restrict__ params)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const float* t = y + (long long)b * NOUT;
    double* p = params + (long long)b * 9;
    const double l10 = log(10.0);
    const double F = exp(3.5 * l10 + 1.5 * l10 * t[2]);
    const double re = exp(0.5 * log(80.0) + 0.5 * log(20.0) * t[3]);
    const double n = 3.25 + 2.75 * t[4];
    const double q = 0.6 + 0.4 * t[5];
    double pa = 0.5 * atan2((double)t[7], (double)t[6]) * 180.0 / M_PI;
    if (pa < 0.0) pa += 180.0;
    p[0] = 0.5 * (W - 1) + t[0];
    p[1] = 0.5 * (H - 1) + t[1];
    p[2] = (n >= 0.2 && n <= 10.0 && q > 0.0 && q <= 1.0) ? F / sersic_flux(1.0, re, n, q) : NAN;
    p[3] = re;
    p[4] = n;
    p[5] = q;
    p[6] = pa;
    p[7] = 0.0;
    p[8] = dflt[(long long)b * 9 + 8];
    if (flags & GF_DECODE_MOMENT_CENTRE) {
        p[0] = dflt[(long long)b * 9];
        p[1] = dflt[(long long)b * 9 + 1];
    }
}

// ------------------------------------------------------- default guess
// Block per stamp of a batch.  Sky = median of the outer ring; centre = first
// moments of the sky-subtracted positive pixels; q and pa from the second
// moments; r_e = semi-major axis of the first elliptical aperture, in 0.25 px
// steps, holding half their summed flux (found by bisection over the aperture
// index: the enclosed flux only grows with it); n = 2; I_e from the summed flux
// by the closed form.  All in float64; the aperture test avoids contracted
// multiply-adds so it takes the same decisions as a plain evaluation.
constexpr int DG_THREADS = 512;

__device__ double block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = DG_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(DG_THREADS) k_default_guess(const int* __restrict__ Hs,
                                                               const int* __restrict__ Ws,
                                                               const long long* __restrict__ off,
                                                               const float* __restrict__ img,
                                                               double* __restrict__ out, int nslots,
                                                               int ring_cap, int cache_cap,
                                                               const double* __restrict__ e2)
{
    // dynamic shared memory: the ring (ring_cap doubles, a power of two >= the
    // longest ring) then, for stamps of at most cache_cap pixels, each pixel's
    // sky-subtracted value and squared elliptical radius
    extern __shared__ double ring[];
    __shared__ double red[DG_THREADS];
    const int b = blockIdx.x;
    const int H = Hs[b], W = Ws[b];
    const float* im = img + off[b];
    const int npx = H * W;
    const bool line = H == 1 || W == 1;
    const int nr = line ? npx : 2 * W + 2 * (H - 2);
    int n2 = 1;
    while (n2 < nr) n2 <<= 1;
    for (int k = threadIdx.x; k < n2; k += blockDim.x) {
        double v = INFINITY;
        if (k < nr) {
            int i = 0, j = k;
            if (!line) ring_ij(k, H, W, &i, &j);
            v = im[i * W + j];  // a single row or column is its own ring, in storage order
        }
        ring[k] = v;
    }
    __syncthreads();
    bitonic_sort(ring, n2);
    const double sky = (nr & 1) ? ring[nr / 2] : 0.5 * (ring[nr / 2 - 1] + ring[nr / 2]);
    // first moments
    double s0 = 0.0, sx = 0.0, sy = 0.0;
    for (int k = threadIdx.x; k < npx; k += blockDim.x) {
        const double v = (double)im[k] - sky;
        if (v <= 0.0) continue;
        const int i = k / W, j = k - i * W;
        s0 += v;
        sx += v * j;
        sy += v * i;
    }
    s0 = block_sum(s0, red);
    sx = block_sum(sx, red);
    sy = block_sum(sy, red);
    const double x0 = s0 > 0.0 ? sx / s0 : 0.5 * (W - 1), y0 = s0 > 0.0 ? sy / s0 : 0.5 * (H - 1);
    // second moments
    double mxx = 0.0, myy = 0.0, mxy = 0.0;
    for (int k = threadIdx.x; k < npx; k += blockDim.x) {
        const double v = (double)im[k] - sky;
        if (v <= 0.0) continue;
        const int i = k / W, j = k - i * W;
        const double dx = j - x0, dy = i - y0;
        mxx += v * dx * dx;
        myy += v * dy * dy;
        mxy += v * dx * dy;
    }
    mxx = block_sum(mxx, red);
    myy = block_sum(myy, red);
    mxy = block_sum(mxy, red);
    if (s0 > 0.0) {
        mxx /= s0;
        myy /= s0;
        mxy /= s0;
    }
    const double tr = mxx + myy, det = mxx * myy - mxy * mxy;
    const double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
    const double l1 = 0.5 * tr + disc, l2 = 0.5 * tr - disc;
    double q = (l1 > 0.0 && l2 > 0.0) ? sqrt(l2 / l1) : 1.0;
    q = fmin(fmax(q, 0.05), 1.0);
    double pa = 0.5 * atan2(2.0 * mxy, mxx - myy) * 180.0 / M_PI;
    pa = fmod(pa, 180.0);
    if (pa < 0.0) pa += 180.0;
    // curve of growth: smallest aperture index k in [1, K] with enclosed >= half
    const double th = __ddiv_rn(__dmul_rn(pa, M_PI), 180.0), cs = cos(th), sn = sin(th);
    const double half = 0.5 * s0;
    const int K = 4 * max(H, W);
    // each pixel's value and squared elliptical radius, formed once (FP64 is
    // slow on this GPU, a division most of all) instead of once per bisection
    // step; the same operations in the same order, so the same numbers
    const bool cached = npx <= cache_cap;
    double* cv = ring + ring_cap;
    double* crr = cv + cache_cap;
    if (cached) {
        for (int k = threadIdx.x; k < npx; k += blockDim.x) {
            const double v = (double)im[k] - sky;
            cv[k] = v;
            if (v <= 0.0) continue;
            const int i = k / W, j = k - i * W;
            const double dx = j - x0, dy = i - y0;
            const double xp = __dadd_rn(__dmul_rn(dx, cs), __dmul_rn(dy, sn));
            const double yp = __ddiv_rn(__dadd_rn(-__dmul_rn(dx, sn), __dmul_rn(dy, cs)), q);
            crr[k] = __dadd_rn(__dmul_rn(xp, xp), __dmul_rn(yp, yp));
        }
        __syncthreads();
    }
    int klo = 0, khi = K + 1;  // enclosed(klo) < half <= enclosed(khi); K + 1 = not reached
    while (khi - klo > 1) {
        const int km = (klo + khi) >> 1;
        const double a = 0.25 * km, a2 = __dmul_rn(a, a);
        double enc = 0.0;
        if (cached) {
            for (int k = threadIdx.x; k < npx; k += blockDim.x) {
                const double v = cv[k];
                if (v <= 0.0) continue;
                if (crr[k] <= a2) enc += v;
            }
        } else {
            for (int k = threadIdx.x; k < npx; k += blockDim.x) {
                const double v = (double)im[k] - sky;
                if (v <= 0.0) continue;
                const int i = k / W, j = k - i * W;
                const double dx = j - x0, dy = i - y0;
                const double xp = __dadd_rn(__dmul_rn(dx, cs), __dmul_rn(dy, sn));
                const double yp = __ddiv_rn(__dadd_rn(-__dmul_rn(dx, sn), __dmul_rn(dy, cs)), q);
                if (__dadd_rn(__dmul_rn(xp, xp), __dmul_rn(yp, yp)) <= a2) enc += v;
            }
        }
        enc = block_sum(enc, red);
        if (enc >= half)
            khi = km;
        else
            klo = km;
    }
    if (threadIdx.x == 0) {
        double re = khi <= K ? 0.25 * khi : 1.0;
        re = fmax(re, 0.5);
        const double F = s0 > 0.0 ? s0 : 1.0;
        double* p = out + (long long)b * nslots;
        p[0] = x0;
        p[1] = y0;
        p[2] = F / sersic_flux_e(1.0, re, 2.0, q, *e2);
        p[3] = re;
        p[4] = 2.0;
        p[5] = q;
        p[6] = pa;
        p[7] = 0.0;
        p[8] = sky;
    }
}

// ------------------------------------------------------ start selection
// The network's start is taken where every slot is finite and inside its
// bounds and its chi^2 is finite and no larger than the default start's.
__global__ void k_select(int count, int nslots, const double* __restrict__ cand,
                         const double* __restrict__ x2c, const double* __restrict__ dflt,
                         const double* __restrict__ x2d, const double* __restrict__ lo,
                         const double* __restrict__ hi, double* __restrict__ out,
                         int* __restrict__ choice)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const double* c = cand + (long long)b * nslots;
    bool ok = isfinite(x2c[b]) && (!isfinite(x2d[b]) || x2c[b] <= x2d[b]);
    for (int s = 0; s < nslots; ++s) ok = ok && isfinite(c[s]) && c[s] >= lo[s] && c[s] <= hi[s];
    const double* src = ok ? c : dflt + (long long)b * nslots;
    for (int s = 0; s < nslots; ++s) out[(long long)b * nslots + s] = src[s];
    if (choice) choice[b] = ok ? 1 : 0;
}

}  // namespace

// ================================================================ launchers

size_t cnn_buffers(void* ws, int B, bool training, CnnBuffers* cb)
{
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    // weight-gradient partials: the first layer's SIMT chunks or layers 2-4's
    // tensor-core chunks, whichever need more
    size_t part = cnn_bwd_tc_part_floats(B);
    {
        const ConvL L = CONV[0];
        const long long total = (long long)B * L.hout * L.hout;
        const long long nchunk = std::min<long long>(std::max<long long>(1, 2048 / (L.cout * L.cin)), total);
        part = std::max(part, (size_t)(nchunk * L.cout * L.cin * 10));
    }
    // the gradient buffers exist only when the call trains
    const size_t T = training ? 1 : 0;
    const size_t wp = take(2ull * NPARAM), wf = take(2ull * CONV_W_END), wb = take(2ull * CONV_W_END),
                 x = take(2ull * B * NPIX), a0 = take(2ull * B * 32 * 32 * 32),
                 a1 = take(2ull * B * 64 * 16 * 16), a2 = take(2ull * B * 64 * 8 * 8),
                 a3 = take(2ull * B * 2048), h = take(4ull * B * 32), y = take(4ull * B * NOUT),
                 gy = take(T * 4ull * B * NOUT), gh = take(T * 4ull * B * 32),
                 g3 = take(T * 4ull * B * 2048), g2 = take(T * 4ull * B * 64 * 8 * 8),
                 g1 = take(T * 4ull * B * 64 * 16 * 16), g0 = take(T * 4ull * B * 32 * 32 * 32),
                 pt = take(T * 4ull * part);
    if (cb && ws) {
        char* p = static_cast<char*>(ws);
        cb->wp = (__nv_bfloat16*)(p + wp);
        cb->wf = (__nv_bfloat16*)(p + wf);
        cb->wb = (__nv_bfloat16*)(p + wb);
        cb->x = (__nv_bfloat16*)(p + x);
        cb->a0 = (__nv_bfloat16*)(p + a0);
        cb->a1 = (__nv_bfloat16*)(p + a1);
        cb->a2 = (__nv_bfloat16*)(p + a2);
        cb->a3 = (__nv_bfloat16*)(p + a3);
        cb->h = (float*)(p + h);
        cb->y = (float*)(p + y);
        cb->gy = (float*)(p + gy);
        cb->gh = (float*)(p + gh);
        cb->g3 = (float*)(p + g3);
        cb->g2 = (float*)(p + g2);
        cb->g1 = (float*)(p + g1);
        cb->g0 = (float*)(p + g0);
        cb->part = (float*)(p + pt);
        cb->part_floats = T * part;
    }
    return o;
}

cudaError_t cnn_prepare(const float* w, const float* x, int B, const CnnBuffers& cb, cudaStream_t s)
{
    k_cast<<<blocks(NPARAM, 256), 256, 0, s>>>(w, cb.wp, cb.wf, cb.wb);
    GF_COUNT_LAUNCH();
    k_to_bf16<<<blocks((long long)B * NPIX, 256), 256, 0, s>>>(x, cb.x, (long long)B * NPIX);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t cnn_forward_fc(const float* w, int B, const CnnBuffers& cb, float* y, cudaStream_t s)
{
    k_fc1_fwd<<<blocks((long long)B * 32, 256), 256, 0, s>>>(cb.a3, cb.wp, w, cb.h, B);
    GF_COUNT_LAUNCH();
    k_fc2_fwd<<<blocks((long long)B * NOUT, 256), 256, 0, s>>>(cb.h, cb.wp, w, y ? y : cb.y, B);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t cnn_backward(const float* t, int B, float* loss, float* grad, const CnnBuffers& cb,
                         cudaStream_t s)
{
    k_mse<<<1, 256, 0, s>>>(cb.y, t, cb.gy, loss, B);
    GF_COUNT_LAUNCH();
    k_fc2_bwd_w<<<blocks(NOUT * 32 + NOUT, 256), 256, 0, s>>>(cb.gy, cb.h, grad, B);
    GF_COUNT_LAUNCH();
    k_fc2_bwd_x<<<blocks((long long)B * 32, 256), 256, 0, s>>>(cb.gy, cb.h, cb.wp, cb.gh, B);
    GF_COUNT_LAUNCH();
    k_fc1_bwd_w<<<blocks(32 * 2048 + 32, 256), 256, 0, s>>>(cb.gh, cb.a3, grad, B);
    GF_COUNT_LAUNCH();
    k_fc1_bwd_x<<<blocks((long long)B * 2048, 256), 256, 0, s>>>(cb.gh, cb.a3, cb.wp, cb.g3, B);
    GF_COUNT_LAUNCH();
    // layers 4-2 on the tensor cores (weight gradients and the channels-last
    // gradients at the pre-activations of layers 3-1), then layer 1's weights
    float* gout[4] = {cb.g0, cb.g1, cb.g2, cb.g3};
    const __nv_bfloat16* ins[4] = {cb.x, cb.a0, cb.a1, cb.a2};
    cudaError_t e = cnn_backward_tc(B, grad, gout, ins, cb.wf, cb.part, cb.part_floats, s);
    if (e != cudaSuccess) return e;
    const ConvL L = CONV[0];
    const long long total = (long long)B * L.hout * L.hout;
    const int nchunk = (int)std::min<long long>(std::max<long long>(1, 2048 / (L.cout * L.cin)), total);
    k_conv_bwd_w<<<dim3(L.cout * L.cin, nchunk), WG_THREADS, 0, s>>>(cb.g0, cb.x, cb.part, B, L.cin, L.hin,
                                                                     L.cout, L.hout, nchunk);
    GF_COUNT_LAUNCH();
    k_conv_bwd_w_sum<<<blocks((long long)L.cout * L.cin * 10, 256), 256, 0, s>>>(cb.part, grad, L.cin, L.cout,
                                                                                nchunk, L.woff, L.boff);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t cnn_adam(float* w, float* m, float* v, const float* g, int step, float lr,
                     cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<blocks(NPARAM, 256), 256, 0, s>>>(w, m, v, g, NPARAM, lr, b1, b2, 1e-8f, c1, c2);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t cnn_init(float* w, unsigned long long seed, cudaStream_t s)
{
    k_init<<<blocks(NPARAM, 256), 256, 0, s>>>(w, seed);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t cnn_input(const float* img, const float* sig, int B, float* x, cudaStream_t s)
{
    k_cnn_input<<<B, 256, 0, s>>>(img, sig, x);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t cnn_encode(const double* params, int nslots, int count, int H, int W, float* t,
                       cudaStream_t s)
{
    k_encode<<<blocks((long long)count * 32, 128), 128, 0, s>>>(params, nslots, count, H, W, t);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t cnn_decode(const float* y, const double* dflt, int count, int H, int W, int flags,
                       double* params, cudaStream_t s)
{
    k_decode<<<blocks(count, 128), 128, 0, s>>>(y, dflt, count, H, W, flags, params);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t train_sample(unsigned long long seed, int count, double* params, float* psf,
                         int psf_size, cudaStream_t s)
{
    k_train_sample<<<count, 256, 0, s>>>(seed, params, psf, psf_size);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t noise_fill(const float* m, long long n, unsigned long long seed, float sread,
                       float gain, float* d, float* sig, cudaStream_t s)
{
    k_noise<<<blocks(n, 256), 256, 0, s>>>(m, n, seed, sread, gain, d, sig);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t philox_blocks(const unsigned* in, unsigned* out, int n, cudaStream_t s)
{
    k_philox<<<blocks(n, 128), 128, 0, s>>>(in, out, n);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

size_t default_guess_smem(int H, int W)
{
    const int nr = (H == 1 || W == 1) ? H * W : 2 * W + 2 * (H - 2);
    int n2 = 1;
    while (n2 < nr) n2 <<= 1;
    return sizeof(double) * (size_t)n2;
}

// pixels per stamp the per-pixel cache of k_default_guess holds at most (96 KB)
constexpr int DG_CACHE_MAX = 6144;

cudaError_t default_guess(int count, const int* H, const int* W, const long long* off,
                          const float* img, double* out, int nslots, size_t smem, int max_npx,
                          double* e2, cudaStream_t s)
{
    static int optin[64];
    const int ring_cap = (int)(smem / sizeof(double));
    const int cache_cap = max_npx <= DG_CACHE_MAX ? max_npx : 0;
    const size_t bytes = smem + 2 * sizeof(double) * (size_t)cache_cap;
    cudaError_t e = ensure_smem_optin((const void*)k_default_guess, (int)bytes, optin);
    if (e != cudaSuccess) return e;
    k_flux_factor_n2<<<1, 1, 0, s>>>(e2);
    GF_COUNT_LAUNCH();
    k_default_guess<<<count, DG_THREADS, bytes, s>>>(H, W, off, img, out, nslots, ring_cap,
                                                     cache_cap, e2);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t guess_select(int count, int nslots, const double* cand, const double* x2c,
                         const double* dflt, const double* x2d, const double* lo, const double* hi,
                         double* out, int* choice, cudaStream_t s)
{
    k_select<<<blocks(count, 128), 128, 0, s>>>(count, nslots, cand, x2c, dflt, x2d, lo, hi, out, choice);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}
