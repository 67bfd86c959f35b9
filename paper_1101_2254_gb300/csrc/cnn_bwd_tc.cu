// cnn_bwd_tc.cu -- the network's training backward with the weight and input
// gradients of convolutions 2-4 as implicit GEMMs on the tensor cores (tcgen05).
//
// With G the gradient at a layer's pre-activation (float32, channels-last: row
// m = (sample, output pixel), cout columns) and X the layer's input (bf16
// activations, channels-last, cin columns):
//   weight gradient  D[n][co] = sum_m Xcol[n][m] G[m][co],   n = tap * cin + ci,
//                    plus a row n = 9 cin of ones, whose sums are the bias gradient;
//   input gradient   E[m'][ci] = sum_{tap, co} Gcol[m'][tap, co] W[ci][tap][co]
//                    over input pixels m' (b, iy, ix), where Gcol holds G at the
//                    output pixel (oy, ox) = ((iy + 1 - ky) / 2, (ix + 1 - kx) / 2)
//                    when both are whole numbers in range (stride 2, padding 1)
//                    and zero otherwise; E is then masked by the ReLU below
//                    (X > 0), giving the next layer's G.
// G enters the MMAs as three bf16 planes hi + mid + lo whose sum is G exactly
// (round to nearest, then the rounded-off rest twice: 8 significant bits each),
// so every product with a bf16 activation or weight is exact and each
// contraction is float32 accumulation of the float32 gradient, as in a SIMT
// loop, in the tensor cores' order.
//
// Both kernels stage operands in shared memory in the canonical K-major layout
// without swizzle (tc.cuh), let one thread issue the MMAs (M 128, K 16) into a
// tensor-memory accumulator, commit them to an mbarrier and wait with a bound;
// a CTA whose wait runs out issues nothing more and writes NaN, which the
// caller sees as a non-finite gradient.
//
// Weight gradient: a CTA owns 128 rows n and a contiguous chunk of m (the
// accumulator holds its 128 x cout partial sums); the chunks' partials are
// added in chunk order by a second kernel, so the result does not depend on
// scheduling.  Input gradient: a persistent CTA walks tiles of 128 input
// pixels, with the weights (cin x 9 cout) resident in shared memory.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "cnn.cuh"
#include "gf_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int BT_THREADS = 256;
constexpr int BT_KB = 64;  // K (rows m, or taps x channels) per staged block

// x = hi + mid + lo exactly, each a bf16 (x normal float32)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&v)[8])
{
    uint4 u;
    uint32_t* w = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        w[i] = (uint32_t)__bfloat16_as_ushort(v[2 * i]) | ((uint32_t)__bfloat16_as_ushort(v[2 * i + 1]) << 16);
    return u;
}

__device__ __forceinline__ void mma_fence_sync()
{
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// NCOL tensor-memory columns for the CTA, their address written to *slot by warp 0
template <int NCOL>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot)
{
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}

struct ConvBwd {
    const float* g;          // gradient at the pre-activation, NHWC: B x hout^2 x cout
    const __nv_bfloat16* x;  // the layer's input, NHWC: B x hin^2 x cin
    const __nv_bfloat16* w;  // weights [in][tap][out] (cin rows of 9 cout)
    float* out;              // dW partials [chunk][nrows][cout], or the input gradient NHWC
    int B, cin, hin, cout, hout;
    int nrows;               // dW: 128 x n-tiles (rows n >= 9 cin + 1 are zero padding)
    int nchunk;              // dW: chunks of the m range
};

// ------------------------------------------------------------ weight gradient
// grid (n-tiles, chunks); NCO = cout
template <int NCO>
__global__ void __launch_bounds__(BT_THREADS) k_conv_dw_tc(ConvBwd a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // 128 x BT_KB (A)
    __nv_bfloat16* Gs = Xs + 128 * BT_KB;                              // 3 planes NCO x BT_KB (B)
    tmem_alloc<NCO>(&tmem_slot);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot, bar_a = smem_addr(&bar);
    const uint32_t idesc = idesc_bf16(128, NCO);
    const uint32_t xa = smem_addr(Xs), ga = smem_addr(Gs);
    constexpr uint32_t PLANE = NCO * BT_KB * 2;  // bytes per G plane
    const int hw = a.hout * a.hout, n0 = blockIdx.x * 128, nw = 9 * a.cin;
    const long long M = (long long)a.B * hw;
    const long long nkb = (M + BT_KB - 1) / BT_KB;
    const long long kb0 = nkb * blockIdx.y / a.nchunk, kb1 = nkb * (blockIdx.y + 1) / a.nchunk;
    uint32_t parity = 0;
    bool failed = false;
    for (long long kb = kb0; kb < kb1 && !failed; ++kb) {
        const long long mb = kb * BT_KB;
        // A: rows n of this tile x 64 m (an 8 x 8 block per item, transposed)
        for (int it = tid; it < 16 * 8 + (NCO / 8) * 8; it += BT_THREADS) {
            if (it < 128) {
                const int ng = it >> 3, mg = it & 7;
                const int n = n0 + 8 * ng;
                __nv_bfloat16 v[8][8];  // [m][n]
                if (n < nw) {
                    const int tap = n / a.cin, ci = n - tap * a.cin;
                    const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const long long m = mb + 8 * mg + i;
                        uint4 u = make_uint4(0u, 0u, 0u, 0u);
                        if (m < M) {
                            const int b = (int)(m / hw), pix = (int)(m - (long long)b * hw);
                            const int oy = pix / a.hout, ox = pix - oy * a.hout;
                            const int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
                            if (iy >= 0 && iy < a.hin && ix >= 0 && ix < a.hin)
                                u = *reinterpret_cast<const uint4*>(
                                    a.x + (((long long)b * a.hin + iy) * a.hin + ix) * a.cin + ci);
                        }
                        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
                        for (int j = 0; j < 8; ++j) v[i][j] = h[j];
                    }
                } else {
                    // the bias row (ones where m is in range) and the padding rows
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const bool in = mb + 8 * mg + i < M;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            v[i][j] = __float2bfloat16_rn((n + j == nw && in) ? 1.0f : 0.0f);
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __nv_bfloat16 r[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) r[i] = v[i][j];
                    *reinterpret_cast<uint4*>(Xs + cofs(8 * ng + j, 8 * mg, BT_KB)) = pack8(r);
                }
            } else {
                // B: G rows m x 8 channels, split into three planes and transposed
                const int q = it - 128, cg = q >> 3, mg = q & 7;
                __nv_bfloat16 hi[8][8], mid[8][8], lo[8][8];  // [co][m]
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const long long m = mb + 8 * mg + i;
                    float f[8];
                    if (m < M) {
                        const float4* src = reinterpret_cast<const float4*>(a.g + m * NCO + 8 * cg);
                        const float4 p0 = src[0], p1 = src[1];
                        f[0] = p0.x; f[1] = p0.y; f[2] = p0.z; f[3] = p0.w;
                        f[4] = p1.x; f[5] = p1.y; f[6] = p1.z; f[7] = p1.w;
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) f[j] = 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) split3(f[j], hi[j][i], mid[j][i], lo[j][i]);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int o = cofs(8 * cg + j, 8 * mg, BT_KB);
                    *reinterpret_cast<uint4*>(Gs + o) = pack8(hi[j]);
                    *reinterpret_cast<uint4*>(Gs + PLANE / 2 + o) = pack8(mid[j]);
                    *reinterpret_cast<uint4*>(Gs + PLANE + o) = pack8(lo[j]);
                }
            }
        }
        mma_fence_sync();
        if (tid == 0) {
            for (int ks = 0; ks < BT_KB / 16; ++ks)
                for (int p = 0; p < 3; ++p)
                    umma(tmem, mdesc(xa + ks * 256, 128, BT_KB * 16),
                         mdesc(ga + p * PLANE + ks * 256, 128, BT_KB * 16), idesc,
                         (kb > kb0 || ks > 0 || p > 0) ? 1 : 0);
            mma_commit(bar_a);
        }
        const bool done = mbar_wait(bar_a, parity);
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!__syncthreads_and(done ? 1 : 0)) failed = true;
    }
    // epilogue: warp w reads lane quarter w % 4 (rows n), column half w / 4
    const int quarter = warp & 3, chalf = warp >> 2;
    const int row = quarter * 32 + lane;
    float* dst = a.out + ((long long)blockIdx.y * a.nrows + n0 + row) * NCO;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int c0 = chalf * (NCO / 2); c0 < (chalf + 1) * (NCO / 2); c0 += 8) {
        float v[8];
        if (kb1 > kb0 && !failed) {
            tmem_ld8(taddr + c0, v);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = failed ? NAN : 0.0f;  // an empty chunk adds zero
        }
        *reinterpret_cast<float4*>(dst + c0) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(dst + c0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    bool drained = true;
    if (failed) drained = __syncthreads_and(mbar_wait(bar_a, parity ^ 1u) ? 1 : 0);
    if (drained && warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCO));
}

// the chunks' partials added in chunk order into the packed master layout
// (weights [out][in][ky][kx], then the biases)
__global__ void k_conv_dw_sum(const float* __restrict__ part, float* __restrict__ grad, int cin,
                              int cout, int nrows, int nchunk, int woff, int boff)
{
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = 9 * cin;
    if (item >= (nw + 1) * cout) return;
    const int n = item / cout, co = item - n * cout;
    float s = 0.0f;
    for (int c = 0; c < nchunk; ++c) s += part[((long long)c * nrows + n) * cout + co];
    if (n < nw) {
        const int tap = n / cin, ci = n - tap * cin;
        grad[woff + (co * cin + ci) * 9 + tap] = s;
    } else {
        grad[boff + co] = s;
    }
}

// ------------------------------------------------------------- input gradient
// persistent grid over tiles of 128 input pixels; NCI = cin
template <int NCI>
__global__ void __launch_bounds__(BT_THREADS) k_conv_dx_tc(ConvBwd a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = 9 * a.cout;
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // NCI x K (B)
    __nv_bfloat16* As = Ws + NCI * K;                                  // 3 planes 128 x BT_KB (A)
    constexpr uint32_t PLANE = 128 * BT_KB * 2;
    for (int i = tid; i < NCI * (K / 8); i += BT_THREADS) {
        const int n = i / (K / 8), k8 = (i - n * (K / 8)) * 8;
        *reinterpret_cast<uint4*>(Ws + cofs(n, k8, K)) =
            *reinterpret_cast<const uint4*>(a.w + (long long)n * K + k8);
    }
    tmem_alloc<NCI>(&tmem_slot);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot, bar_a = smem_addr(&bar);
    const uint32_t idesc = idesc_bf16(128, NCI);
    const uint32_t wa = smem_addr(Ws), aa = smem_addr(As);
    const int hwi = a.hin * a.hin;
    const long long M = (long long)a.B * hwi;
    const long long tiles = (M + 127) / 128;
    const int nkc = K / BT_KB;  // a block never straddles two taps (cout is a multiple of 64)
    uint32_t parity = 0;
    bool failed = false;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long m0 = tile * 128;
        for (int c = 0; c < nkc && !failed; ++c) {
            const int kc0 = c * BT_KB, tap = kc0 / a.cout, co0 = kc0 - tap * a.cout;
            const int ky = tap / 3, kx = tap - 3 * ky;
            // A: (input pixel, 8 channels of G at the pixel the tap maps it to).
            // A warp takes 8 rows x 4 channel groups, so the 8 lanes of each
            // 16-byte store phase write 8 different rows (distinct banks).
            static_assert(BT_KB % 32 == 0 && (128 * (BT_KB / 8)) % BT_THREADS == 0, "lane mapping");
            constexpr int PER = 128 * (BT_KB / 8) / BT_THREADS;  // items per thread
            float f[PER][8];
            int orow[PER], oj[PER];
            // every item's loads first (all in flight), then the splits and stores
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int it = tid + u * BT_THREADS;
                const int lane_i = it & 31, rest = it >> 5;
                const int jq = rest % (BT_KB / 32), rg = rest / (BT_KB / 32);
                const int r = rg * 8 + (lane_i & 7), j = jq * 4 + (lane_i >> 3);
                orow[u] = r;
                oj[u] = j;
                const long long m = m0 + r;
                float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
                if (m < M) {
                    const int b = (int)(m / hwi), pix = (int)(m - (long long)b * hwi);
                    const int iy = pix / a.hin, ix = pix - iy * a.hin;
                    const int ty = iy + 1 - ky, tx = ix + 1 - kx;
                    if (ty >= 0 && tx >= 0 && !(ty & 1) && !(tx & 1) && (ty >> 1) < a.hout &&
                        (tx >> 1) < a.hout) {
                        const float4* src = reinterpret_cast<const float4*>(
                            a.g + (((long long)b * a.hout + (ty >> 1)) * a.hout + (tx >> 1)) * a.cout + co0 +
                            8 * j);
                        p0 = src[0];
                        p1 = src[1];
                    }
                }
                f[u][0] = p0.x; f[u][1] = p0.y; f[u][2] = p0.z; f[u][3] = p0.w;
                f[u][4] = p1.x; f[u][5] = p1.y; f[u][6] = p1.z; f[u][7] = p1.w;
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                __nv_bfloat16 hi[8], mid[8], lo[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) split3(f[u][q], hi[q], mid[q], lo[q]);
                const int o = cofs(orow[u], 8 * oj[u], BT_KB);
                *reinterpret_cast<uint4*>(As + o) = pack8(hi);
                *reinterpret_cast<uint4*>(As + PLANE / 2 + o) = pack8(mid);
                *reinterpret_cast<uint4*>(As + PLANE + o) = pack8(lo);
            }
            mma_fence_sync();
            if (tid == 0) {
                for (int ks = 0; ks < BT_KB / 16; ++ks)
                    for (int p = 0; p < 3; ++p)
                        umma(tmem, mdesc(aa + p * PLANE + ks * 256, 128, BT_KB * 16),
                             mdesc(wa + (uint32_t)(kc0 + ks * 16) * 16, 128, (uint32_t)K * 16), idesc,
                             (c > 0 || ks > 0 || p > 0) ? 1 : 0);
                mma_commit(bar_a);
            }
            const bool done = mbar_wait(bar_a, parity);
            parity ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!__syncthreads_and(done ? 1 : 0)) {
                failed = true;
                break;
            }
        }
        // epilogue: the gradient through the ReLU of the layer below (X > 0)
        const int quarter = warp & 3, chalf = warp >> 2;
        const int row = quarter * 32 + lane;
        const long long m = m0 + row;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int c0 = chalf * (NCI / 2); c0 < (chalf + 1) * (NCI / 2); c0 += 8) {
            float v[8];
            if (!failed) {
                tmem_ld8(taddr + c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = NAN;
            }
            if (m >= M) continue;
            const uint4 u = *reinterpret_cast<const uint4*>(a.x + m * NCI + c0);
            const __nv_bfloat16* xv = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (!(__bfloat162float(xv[j]) > 0.0f) && !failed) v[j] = 0.0f;
            float* dst = a.out + m * NCI + c0;
            *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();  // the accumulator is read before the next tile's MMAs
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    bool drained = true;
    if (failed) drained = __syncthreads_and(mbar_wait(bar_a, parity ^ 1u) ? 1 : 0);
    if (drained && warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCI));
}

inline size_t dw_smem(int nco) { return sizeof(__nv_bfloat16) * (size_t)(128 + 3 * nco) * BT_KB; }
inline size_t dx_smem(int nci, int cout)
{
    return sizeof(__nv_bfloat16) * ((size_t)nci * 9 * cout + 3 * 128 * (size_t)BT_KB);
}

// chunks of the m range for a weight gradient with `ntile` row tiles: about
// two CTAs per SM in all (the kernel's registers allow two), at most one per
// 64-row block
int dw_chunks(long long M, int ntile, int sms)
{
    const long long nkb = (M + BT_KB - 1) / BT_KB;
    return (int)std::max<long long>(1, std::min<long long>(nkb, (2 * sms + ntile - 1) / ntile));
}

template <int NCO>
cudaError_t launch_dw(const ConvBwd& a, int ntile, cudaStream_t s)
{
    static int optin[64];
    const size_t smem = dw_smem(NCO);
    cudaError_t e = ensure_smem_optin((const void*)k_conv_dw_tc<NCO>, (int)smem, optin);
    if (e != cudaSuccess) return e;
    k_conv_dw_tc<NCO><<<dim3(ntile, a.nchunk), BT_THREADS, smem, s>>>(a);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

template <int NCI>
cudaError_t launch_dx(const ConvBwd& a, cudaStream_t s)
{
    static int optin[64];
    const size_t smem = dx_smem(NCI, a.cout);
    cudaError_t e = ensure_smem_optin((const void*)k_conv_dx_tc<NCI>, (int)smem, optin);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // the largest shared-memory carveout, so that the occupancy query (and the
    // launch) can place as many of these shared-memory-heavy CTAs as fit
    if ((e = cudaFuncSetAttribute((const void*)k_conv_dx_tc<NCI>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_dx_tc<NCI>, BT_THREADS, smem)) !=
        cudaSuccess)
        return e;
    const long long tiles = ((long long)a.B * a.hin * a.hin + 127) / 128;
    const int grid = (int)std::min<long long>(tiles, (long long)sms * std::max(per_sm, 1));
    k_conv_dx_tc<NCI><<<grid, BT_THREADS, smem, s>>>(a);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

// the network's layers 2-4: cin, cout, hin, hout, weight and bias offsets
struct BwdL {
    int cin, cout, hin, hout, woff, boff;
};
constexpr BwdL BWD_LAYERS[3] = {{32, 64, 32, 16, 320, 18752},
                                {64, 64, 16, 8, 18816, 55680},
                                {64, 128, 8, 4, 55744, 129472}};

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 148;
    return sms;
}

}  // namespace

size_t cnn_bwd_tc_part_floats(int B)
{
    size_t most = 0;
    for (const BwdL& l : BWD_LAYERS) {
        const int ntile = (9 * l.cin + 1 + 127) / 128;
        // sized for any SM count up to 160 (the grid rule caps chunks by SMs)
        const int nch = dw_chunks((long long)B * l.hout * l.hout, ntile, 160);  // (2 x 160 CTAs)
        most = std::max(most, (size_t)nch * ntile * 128 * l.cout);
    }
    return most;
}

// Weight gradients of layers 2-4 and input gradients of layers 4-2 (the
// latter written NHWC into gin[l - 1]): gout[l] is the NHWC gradient at layer
// l's pre-activation, ins[l] its NHWC input.
cudaError_t cnn_backward_tc(int B, float* grad, float* const* gout, const __nv_bfloat16* const* ins,
                            const __nv_bfloat16* wf, float* part, size_t part_floats, cudaStream_t s)
{
    const int sms = std::min(sm_count(), 160);
    for (int li = 2; li >= 0; --li) {
        const BwdL& l = BWD_LAYERS[li];
        const int L = li + 1;  // the network's layer index
        ConvBwd a;
        a.g = gout[L];
        a.x = ins[L];
        a.w = wf + l.woff;
        a.B = B;
        a.cin = l.cin;
        a.hin = l.hin;
        a.cout = l.cout;
        a.hout = l.hout;
        const int ntile = (9 * l.cin + 1 + 127) / 128;
        a.nrows = ntile * 128;
        a.nchunk = dw_chunks((long long)B * l.hout * l.hout, ntile, sms);
        if ((size_t)a.nchunk * a.nrows * l.cout > part_floats) return cudaErrorInvalidValue;
        a.out = part;
        cudaError_t e = l.cout == 64 ? launch_dw<64>(a, ntile, s) : launch_dw<128>(a, ntile, s);
        if (e != cudaSuccess) return e;
        const int n = (9 * l.cin + 1) * l.cout;
        k_conv_dw_sum<<<(n + 255) / 256, 256, 0, s>>>(part, grad, l.cin, l.cout, a.nrows, a.nchunk, l.woff,
                                                      l.boff);
        GF_COUNT_LAUNCH();
        a.out = gout[L - 1];
        e = l.cin == 32 ? launch_dx<32>(a, s) : launch_dx<64>(a, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}
