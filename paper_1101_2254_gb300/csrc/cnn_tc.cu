// cnn_tc.cu -- the network's forward pass with its 3x3 stride-2
// convolutions 2-4 as implicit GEMMs on the tensor cores (tcgen05).
//
// The forward of both inference and training.  A convolution layer is the
// contraction
//   y[m][n] = relu(bias[n] + sum_k A[m][k] B[n][k]),
// over m = (sample, output pixel) (M = batch x hout^2 rows), n = output channel
// (N = 64 or 128) and k = tap * cin + input channel (K = 9 cin = 288 or 576).
// A is the im2col view of the input, gathered on the fly: activations are kept
// channels-last (NHWC), so the 8 consecutive k of one tap are one 16-byte load.
// B is the bf16 weight copy in [out][tap][in] order, which is already B's
// K-major layout.
//
// A CTA of 256 threads stages B whole in shared memory once, then walks tiles
// of 128 rows (persistent grid): per K chunk of 288 values it gathers the A
// tile into the canonical K-major layout, one thread issues the MMAs
// (M 128, N, K 16) into a tensor-memory accumulator of 128 lanes x N columns and
// commits them to an mbarrier (bounded wait); the epilogue reads the
// accumulator (tcgen05.ld), adds the bias, applies the ReLU, rounds to bf16 and
// stores NHWC (layers 2-3) or NCHW (layer 4, the layout the first fully
// connected layer reads).  Layer 1 (one input channel: K = 9) stays a SIMT loop.
//
// Arithmetic is the network's specified one: bf16 weights and activations,
// float32 accumulation, in the tensor cores' summation order.  The training
// backward (cnn_bwd_tc.cu) reads the channels-last activations this writes.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "cnn.cuh"
#include "gf_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int CT_THREADS = 256;
constexpr int CT_TM = 128;  // rows per tile (the MMA's M)
constexpr int CT_KC = 288;  // K per staged chunk of A

struct ConvTC {
    const __nv_bfloat16* x;  // input, NHWC: B x hin x hin x cin
    const __nv_bfloat16* w;  // weights [out][tap][in] (cout x 9 cin)
    const float* bias;
    __nv_bfloat16* y;        // output, NHWC or NCHW
    int B, cin, hin, hout, out_nchw;
};

template <int N>
__global__ void __launch_bounds__(CT_THREADS) k_conv_tc(ConvTC a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = 9 * a.cin, nchunk = K / CT_KC;
    __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // N x K
    __nv_bfloat16* As = Bs + N * K;                                    // 128 x CT_KC
    // B whole, once: row n of the weights is K contiguous bf16
    for (int i = tid; i < N * (K / 8); i += CT_THREADS) {
        const int n = i / (K / 8), k8 = (i - n * (K / 8)) * 8;
        *reinterpret_cast<uint4*>(Bs + cofs(n, k8, K)) =
            *reinterpret_cast<const uint4*>(a.w + (long long)n * K + k8);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t bar_a = smem_addr(&bar);
    const uint32_t idesc = idesc_bf16(CT_TM, N);
    const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
    const int hw = a.hout * a.hout;
    const long long M = (long long)a.B * hw;
    const long long tiles = (M + CT_TM - 1) / CT_TM;
    uint32_t parity = 0;
    bool failed = false;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long m0 = tile * CT_TM;
        for (int c = 0; c < nchunk && !failed; ++c) {
            const int kc0 = c * CT_KC;
            // gather the A chunk: (row, 8 consecutive k of one tap) per item.  A
            // warp takes 8 rows x 4 consecutive 8-k groups: the 8 lanes of each
            // 16-byte store phase write 8 different rows of one core matrix
            // (distinct banks), and each row's 4 groups are 64 contiguous bytes
            // of the input.
            static_assert(CT_KC % 32 == 0 && CT_THREADS % 32 == 0, "lane mapping");
            for (int i = tid; i < CT_TM * (CT_KC / 8); i += CT_THREADS) {
                const int lane_i = i & 31, rest = i >> 5;
                const int kq = rest % (CT_KC / 32), rg = rest / (CT_KC / 32);
                const int row = rg * 8 + (lane_i & 7), k8 = (kq * 4 + (lane_i >> 3)) * 8;
                const int k = kc0 + k8;
                const long long m = m0 + row;
                const __nv_bfloat16* src = a.x;  // (not read when the copy is a zero fill)
                bool in = false;
                if (m < M) {
                    const int b = (int)(m / hw), pix = (int)(m - (long long)b * hw);
                    const int oy = pix / a.hout, ox = pix - oy * a.hout;
                    const int tap = k / a.cin, ci = k - tap * a.cin;
                    const int iy = 2 * oy - 1 + tap / 3, ix = 2 * ox - 1 + tap % 3;
                    in = iy >= 0 && iy < a.hin && ix >= 0 && ix < a.hin;
                    if (in) src = a.x + (((long long)b * a.hin + iy) * a.hin + ix) * a.cin + ci;
                }
                // 16 bytes by cp.async (zeros outside the input): every item of the
                // chunk is in flight at once
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                                 smem_addr(As + cofs(row, k8, CT_KC))),
                             "l"(src), "r"(in ? 16 : 0)
                             : "memory");
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0) {
                for (int ks = 0; ks < CT_KC / 16; ++ks)
                    umma(tmem, mdesc(a0 + ks * 256, 128, CT_KC * 16),
                         mdesc(b0 + (uint32_t)(kc0 + ks * 16) * 16, 128, (uint32_t)K * 16), idesc,
                         (c > 0 || ks > 0) ? 1 : 0);
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        bar_a));
            }
            const bool done = mbar_wait(bar_a, parity);
            parity ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!__syncthreads_and(done ? 1 : 0)) {
                // the MMAs did not complete in the bounded wait: from here on
                // this CTA issues no MMA and writes its tiles' outputs as NaN
                // (a non-finite network output makes the caller fall back to
                // the default start)
                failed = true;
                break;
            }
        }
        // epilogue: warp w reads lane quarter w % 4, column half w / 4
        const int quarter = warp & 3, nhalf = warp >> 2;
        const int row = quarter * 32 + lane;
        const long long m = m0 + row;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
        int b = 0, pix = 0;
        if (m < M) {
            b = (int)(m / hw);
            pix = (int)(m - (long long)b * hw);
        }
        for (int n0 = nhalf * (N / 2); n0 < (nhalf + 1) * (N / 2); n0 += 8) {
            float v[8];
            if (!failed) {
                tmem_ld8(taddr + n0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = NAN;
            }
            if (m >= M) continue;
            __align__(16) __nv_bfloat16 o[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(fmaxf(v[j] + a.bias[n0 + j], 0.0f));
            if (failed) {
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(NAN);
            }
            if (a.out_nchw) {
#pragma unroll
                for (int j = 0; j < 8; ++j) a.y[((long long)b * N + n0 + j) * hw + pix] = o[j];
            } else {
                *reinterpret_cast<uint4*>(a.y + m * N + n0) = *reinterpret_cast<const uint4*>(o);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();  // the accumulator is read before the next tile's MMAs
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    // free the tensor memory once no MMA can still be writing it: on the normal
    // path every commit was waited for; after a timeout, wait (bounded) once more
    bool drained = true;
    if (failed) drained = __syncthreads_and(mbar_wait(bar_a, parity ^ 1u) ? 1 : 0);
    if (drained && warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N));
}

// layer 1 (one input channel), channels-last output: thread = (sample, 8
// output channels, output pixel), the taps in (ky, kx) order
__global__ void k_conv1_nhwc(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ wt,
                             const float* __restrict__ bias, __nv_bfloat16* __restrict__ y, int B,
                             int hin, int cout, int hout)
{
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ncg = cout / 8, npix = hout * hout;
    if (item >= (long long)B * ncg * npix) return;
    const int cg = (int)(item % ncg);
    const long long r = item / ncg;
    const int pix = (int)(r % npix), b = (int)(r / npix);
    const int oy = pix / hout, ox = pix - oy * hout;
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = bias[cg * 8 + j];
    const __nv_bfloat16* xb = x + (long long)b * hin * hin;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
        const int iy = 2 * oy - 1 + ky;
        if (iy < 0 || iy >= hin) continue;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const int ix = 2 * ox - 1 + kx;
            if (ix < 0 || ix >= hin) continue;
            const float v = __bfloat162float(xb[iy * hin + ix]);
            const uint4 u = *reinterpret_cast<const uint4*>(wt + (ky * 3 + kx) * cout + cg * 8);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 t = __bfloat1622float2(h[q]);
                acc[2 * q] = fmaf(t.x, v, acc[2 * q]);
                acc[2 * q + 1] = fmaf(t.y, v, acc[2 * q + 1]);
            }
        }
    }
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(fmaxf(acc[j], 0.0f));
    *reinterpret_cast<uint4*>(y + ((long long)b * npix + pix) * cout + cg * 8) =
        *reinterpret_cast<const uint4*>(o);
}

template <int N>
cudaError_t launch_tc(const ConvTC& a, cudaStream_t s)
{
    static int optin[64];
    const int K = 9 * a.cin;
    const size_t smem = sizeof(__nv_bfloat16) * ((size_t)N * K + (size_t)CT_TM * CT_KC);
    cudaError_t e = ensure_smem_optin((const void*)k_conv_tc<N>, (int)smem, optin);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // the largest shared-memory carveout, so that the occupancy query (and the
    // launch) can place as many of these shared-memory-heavy CTAs as fit
    if ((e = cudaFuncSetAttribute((const void*)k_conv_tc<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_tc<N>, CT_THREADS, smem)) !=
        cudaSuccess)
        return e;
    const long long tiles = ((long long)a.B * a.hout * a.hout + CT_TM - 1) / CT_TM;
    const int grid = (int)std::min<long long>(tiles, (long long)sms * std::max(per_sm, 1));
    k_conv_tc<N><<<grid, CT_THREADS, smem, s>>>(a);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace

// Layer table of the network (as in cnn.cu): cin, cout, hin, hout, weight and
// bias offsets in the master array.
cudaError_t cnn_forward_tc(const float* w, int B, const CnnBuffers& cb, float* y, cudaStream_t s)
{
    struct L {
        int cin, cout, hin, hout, woff, boff;
    };
    const L layers[4] = {{1, 32, 64, 32, 0, 288},
                         {32, 64, 32, 16, 320, 18752},
                         {64, 64, 16, 8, 18816, 55680},
                         {64, 128, 8, 4, 55744, 129472}};
    {
        const L& l = layers[0];
        const long long n = (long long)B * (l.cout / 8) * l.hout * l.hout;
        k_conv1_nhwc<<<(int)((n + 255) / 256), 256, 0, s>>>(cb.x, cb.wf + l.woff, w + l.boff, cb.a0, B,
                                                            l.hin, l.cout, l.hout);
        GF_COUNT_LAUNCH();
    }
    __nv_bfloat16* outs[4] = {cb.a0, cb.a1, cb.a2, cb.a3};
    for (int i = 1; i < 4; ++i) {
        const L& l = layers[i];
        ConvTC a;
        a.x = outs[i - 1];
        a.w = cb.wb + l.woff;
        a.bias = w + l.boff;
        a.y = outs[i];
        a.B = B;
        a.cin = l.cin;
        a.hin = l.hin;
        a.hout = l.hout;
        a.out_nchw = i == 3;
        const cudaError_t e = l.cout == 64 ? launch_tc<64>(a, s) : launch_tc<128>(a, s);
        if (e != cudaSuccess) return e;
    }
    return cnn_forward_fc(w, B, cb, y, s);
}
