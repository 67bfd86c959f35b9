// conv_direct.cu -- step 2 of the fitting loop (Sec. 2 item 2) as a tiled
// direct sum, for PSFs up to GF_DIRECT_MAX_PSF pixels on a side.
//
//   out(i, j) = sum_{v,u} psf[v][u] * E[i+2c-v][j+2c-u]
//             = sum_{v,u} k[v][u]   * E[i+v][j+u],   k[v][u] = psf[P-1-v][P-1-u]
//
// One CTA computes a TY x TX output tile of one channel: TX = 64 or 32,
// chosen per stamp (the two kinds of work item), and TY = 32 or 16, chosen per
// call; TX/32 x TY/16 warps.  Both, and the persistent grid, come from the
// device's tuning table (gf_autotune) or its defaults (TY 32, 8 CTAs per SM).  The
// flipped PSF (rows padded with zeros to P4, a multiple of 4 taps) and the
// (TY+P-1) x SW halo tile of the channel grid are staged in shared memory; for
// PSFs up to 35 pixels the tile is double-buffered and filled by cp.async, so a
// CTA's next tile arrives while its current one is summed.
// A warp covers 16 x 32 outputs: lane 8 cg + rl owns the 8 contiguous columns
// 8 cg .. 8 cg + 7 of rows rl and rl + 8.  For each tap row and group of 4
// taps a thread holds, per row, a sliding window of 12 grid values (one new
// 16-byte load per group) and the 4 taps (one broadcast 16-byte load), and
// issues 2 x 8 x 4 = 64 FMAs: 3 shared loads per 64 FMAs.  (Packing the two
// rows' FMAs into __ffma2_rn pairs was measured slower: forming the register
// pairs cost more ALU instructions than the pairing saved.)  In the kernels
// specialised on the padded tap count, the last group of a tap row issues only
// the FMAs of its real taps (P - P4 + 4 of them): for P = 33 that is 33 FMAs
// per output and tap row instead of 36.
// The eight lanes of a quarter-warp read the same columns of eight
// consecutive rows; with the tile's row stride SW = 4 (mod 8) floats their
// 16-byte reads fall in distinct bank groups, so a load takes the minimum four
// wavefronts per warp and shared-memory traffic stays at half the FMA rate.
// The outputs go back through shared memory (row stride TX + 1, conflict-free)
// so that the global stores are coalesced rows.
//
// Each output accumulates its taps in the order v, then u, as a chain of FMAs.
// The work is bound by the FP32 FMA pipe (2 P^2 flop per output pixel against
// 8 bytes of HBM traffic), not by HBM.
#include "gf_internal.cuh"

namespace {

// row stride of the staged grid tile: >= TX + P4 and 4 (mod 8)
__host__ __device__ __forceinline__ int conv_sw(int TX, int P4)
{
    const int w = TX + P4;  // a multiple of 4
    return (w % 8 == 0) ? w + 4 : w;
}

constexpr int RPT = 2;  // rows per thread (rows rl + 8 i)

// acc[o] += sum_t kk[t] win[o + t] for the 8 outputs of one row
__device__ __forceinline__ void fma_row(float (&acc)[8], const float4 kk, const float (&win)[12])
{
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        float x = acc[o];
        x = fmaf(kk.x, win[o], x);
        x = fmaf(kk.y, win[o + 1], x);
        x = fmaf(kk.z, win[o + 2], x);
        x = fmaf(kk.w, win[o + 3], x);
        acc[o] = x;
    }
}

// fma_row for a last tap group with t = 1, 2 or 3 real taps (uniform across
// the warp: the branch costs no divergence)
__device__ __forceinline__ void fma_row_tail(float (&acc)[8], const float4 kk, const float (&win)[12],
                                             int t)
{
    if (t == 1) {
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = fmaf(kk.x, win[o], acc[o]);
    } else if (t == 2) {
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = fmaf(kk.y, win[o + 1], fmaf(kk.x, win[o], acc[o]));
    } else {
#pragma unroll
        for (int o = 0; o < 8; ++o)
            acc[o] = fmaf(kk.z, win[o + 2], fmaf(kk.y, win[o + 1], fmaf(kk.x, win[o], acc[o])));
    }
}

// One tap row v for the thread's RPT rows: er0 points at the first row's first
// window column.  With the tap count P4K known at compile time (PSFs up to
// 35 pixels) the loop over tap groups unrolls completely and the sliding
// window costs no register moves; otherwise (P4K = 0) it runs over P4.
template <int P4K>
__device__ __forceinline__ void tap_row(float (&acc)[RPT][8], const float* kr, const float* er0,
                                        int SW, int P4, int tail)
{
    float win[RPT][12];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const float* er = er0 + i * 8 * SW;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(er + 4 * q);
            win[i][4 * q] = t.x;
            win[i][4 * q + 1] = t.y;
            win[i][4 * q + 2] = t.z;
            win[i][4 * q + 3] = t.w;
        }
    }
    const int pend = P4K > 0 ? P4K : P4;
#pragma unroll(P4K > 0 ? P4K / 4 : 1)
    for (int m = 0; m < pend; m += 4) {
        const float4 kk = *reinterpret_cast<const float4*>(kr + m);
        if (P4K > 0 && m + 4 == pend && tail < 4) {
            // the last group holds only `tail` real taps (the rest are the zero
            // padding): skip the padded ones.  fmaf(0, x, acc) == acc for finite
            // x, so the sums are unchanged.
#pragma unroll
            for (int i = 0; i < RPT; ++i) fma_row_tail(acc[i], kk, win[i], tail);
        } else {
#pragma unroll
            for (int i = 0; i < RPT; ++i) fma_row(acc[i], kk, win[i]);
        }
        if (m + 4 < pend) {
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const float4 t = *reinterpret_cast<const float4*>(er0 + i * 8 * SW + m + 12);
#pragma unroll
                for (int q = 0; q < 8; ++q) win[i][q] = win[i][q + 4];
                win[i][8] = t.x;
                win[i][9] = t.y;
                win[i][10] = t.z;
                win[i][11] = t.w;
            }
        }
    }
}

// One work item's addresses and extent: the channel grid E (He x We) it reads,
// the convolved channel Y (H x W) it writes, its PSF, and the tile's origin.
struct ConvItem {
    const float* E;
    float* Y;
    const float* psf;
    long long pix_off;  // the stamp's image / sigma offset
    int b, ch, wb_off, He, We, H, W, ty0, tx0;
};

template <int TX, int TY>
__device__ __forceinline__ ConvItem conv_item(const PassArgs& a, const int* pre, int n, int tot,
                                              long long it, int& hint)
{
    const int ch = (int)(it / tot), blk = (int)(it - (long long)ch * tot);
    const int li = wl_locate(pre, n, blk, hint);
    ConvItem q;
    q.b = a.wl.ids[li];
    q.ch = ch;
    const StampInfo& st = a.st[q.b];
    q.pix_off = st.pix_off;
    q.wb_off = st.wb_off;
    q.He = st.He;
    q.We = st.We;
    q.H = st.H;
    q.W = st.W;
    const int tiles_x = (st.W + TX - 1) / TX;
    const int t = blk - pre[li];
    q.ty0 = (t / tiles_x) * TY;
    q.tx0 = (t % tiles_x) * TX;
    q.E = a.ext + ext_index(st, a.nchan, ch);
    q.Y = a.y + y_index(st, a.nchan, ch);
    q.psf = a.psf + st.psf_off;
    return q;
}

// asynchronous global -> shared copies (cp.async); a copy whose `in` is false
// reads nothing and writes zeros
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool in)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(in ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool in)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(in ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The SH x SW halo tile of item q into es by cp.async, a warp per row: 16-byte
// copies where the grid's rows are 16-byte aligned (We a multiple of 4, so a
// chunk lies wholly inside or wholly outside the grid), else 4-byte ones.
// Outside the grid the tile holds zeros, as the synchronous staging writes.
template <int NT>
__device__ __forceinline__ void stage_tile_async(float* es, const ConvItem& q, int SH, int SW)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool vec = (q.We & 3) == 0 && (reinterpret_cast<uintptr_t>(q.E) & 15) == 0;
    for (int r = warp; r < SH; r += NT / 32) {
        const int gy = q.ty0 + r;
        const bool row_in = gy < q.He;
        const float* Er = q.E + (long long)(row_in ? gy : 0) * q.We;
        float* er = es + r * SW;
        if (vec) {
            for (int c4 = lane; c4 < (SW >> 2); c4 += 32) {
                const int gx = q.tx0 + 4 * c4;
                const bool in = row_in && gx < q.We;
                cp_async16(er + 4 * c4, in ? Er + gx : q.E, in);
            }
        } else {
            for (int col = lane; col < SW; col += 32) {
                const int gx = q.tx0 + col;
                const bool in = row_in && gx < q.We;
                cp_async4(er + col, in ? Er + gx : q.E, in);
            }
        }
    }
}

// The same tile by plain loads, four per lane in flight.
template <int NT>
__device__ __forceinline__ void stage_tile_sync(float* es, const ConvItem& q, int SH, int SW)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < SH; r += NT / 32) {
        const int gy = q.ty0 + r;
        const bool row_in = gy < q.He;
        const float* Er = q.E + (long long)gy * q.We;
        float* er = es + r * SW;
        for (int c0_ = lane; c0_ < SW; c0_ += 128) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int col = c0_ + 32 * u, gx = q.tx0 + col;
                v[u] = (row_in && col < SW && gx < q.We) ? __ldg(&Er[gx]) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c0_ + 32 * u < SW) er[c0_ + 32 * u] = v[u];
        }
    }
}

// Work item = (channel, output tile of a listed stamp of this tile width).
// With DB (the kernels specialised on the tap count, P <= 35) the halo tile is
// double-buffered: the cp.async copies of item it + 1 are in flight while item
// it's taps run, so the FMA pipe does not wait on global memory between items.
// The generic kernel (larger PSFs, whose two tiles would not fit in shared
// memory) stages each tile synchronously.  The sums are the same either way.
template <int TX, int TY, int P4K>
__global__ void __launch_bounds__(TX * TY / 16) k_conv_direct(PassArgs a)
{
    pdl_entry();
    constexpr bool DB = P4K > 0;
    constexpr int NT = TX * TY / 16, WX = TX / 32;  // threads, warps across
    extern __shared__ __align__(16) float smem[];
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + (TX == 64 ? WK_CONV : WK_CONV32) * (a.count + 1);
    const int tot = pre[n];
    const long long items = (long long)tot * a.nchan;
    const int P = a.P, P4 = (P + 3) & ~3;
    const int SW = conv_sw(TX, P4), SH = TY + P - 1;
    float* ks = smem;                         // P x P4 flipped taps
    float* const es0 = smem + P * P4;         // SH x SW grid tile(s) (P*P4, SW multiples of 4)
    float* const es1 = es0 + (DB ? SH * SW : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rl = lane & 7, cg = lane >> 3;
    const int wr0 = (warp / WX) * 16, wc0 = (warp % WX) * 32;
    const int r0 = wr0 + rl;       // the thread's first row in the tile
    const int c0 = wc0 + 8 * cg;   // the thread's first column in the tile
    int hint = -1, psf_b = -1;
    const long long chunk = (items + gridDim.x - 1) / gridDim.x;
    const long long it0 = (long long)blockIdx.x * chunk, it1 = min(items, it0 + chunk);
    if (it0 >= it1) return;
    ConvItem q = conv_item<TX, TY>(a, pre, n, tot, it0, hint);
    if (DB) {
        stage_tile_async<NT>(es0, q, SH, SW);
        cp_async_commit();
    }
    int cb = 0;  // the buffer holding item it's tile
    for (long long it = it0; it < it1; ++it) {
        __syncthreads();  // the previous item is done with the taps and both tiles
        // item it + 1 (its tile's copies issued now where the tile is double-buffered)
        ConvItem qn = q;
        if (it + 1 < it1) qn = conv_item<TX, TY>(a, pre, n, tot, it + 1, hint);
        if (DB) {
            if (it + 1 < it1) stage_tile_async<NT>(cb ? es0 : es1, qn, SH, SW);
            cp_async_commit();  // (an empty group on the last item)
        }
        if (q.b != psf_b) {
            for (int idx = threadIdx.x; idx < P * P4; idx += NT) {
                const int v = idx / P4, u = idx - v * P4;
                ks[idx] = (u < P) ? __ldg(&q.psf[(P - 1 - v) * P + (P - 1 - u)]) : 0.0f;
            }
            psf_b = q.b;
        }
        float* es = cb ? es1 : es0;
        if (DB)
            cp_async_wait<1>();  // every group but the newest (item it + 1's) is complete
        else
            stage_tile_sync<NT>(es, q, SH, SW);
        __syncthreads();

        // the warp's block meets the stamp
        const bool active = q.ty0 + wr0 < q.H && q.tx0 + wc0 < q.W;
        // an LM trial pass reduces chi^2 here: the thread's 16 image and sigma
        // values are loaded now, so that their latency hides under the taps
        // (outside the stamp: sigma = 0, a pixel that counts nothing)
        float dv[RPT][8], sv[RPT][8];
        float tmw = 0.0f, tmsky = 0.0f;
        if (a.conv_chi2) {
            const Channel& chn = a.chan[(long long)q.b * a.chan_stride + q.ch];
            tmw = chn.mweight;
            tmsky = chn.msky;
            const float* img = a.img + q.pix_off;
            const float* sig = a.sig + q.pix_off;
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int y = q.ty0 + r0 + 8 * i;
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const int x = q.tx0 + c0 + o;
                    const bool in = active && y < q.H && x < q.W;
                    const long long px = (long long)y * q.W + x;
                    dv[i][o] = in ? __ldg(&img[px]) : 0.0f;
                    sv[i][o] = in ? __ldg(&sig[px]) : 0.0f;
                }
            }
        }
        float acc[RPT][8];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int o = 0; o < 8; ++o) acc[i][o] = 0.0f;
        if (active)
            for (int v = 0; v < P; ++v)
                tap_row<P4K>(acc, ks + v * P4, es + (r0 + v) * SW + c0, SW, P4, P - (P4 - 4));

        if (active && a.work && lane == 0) {
            const unsigned long long rows = (unsigned long long)min(16, q.H - q.ty0 - wr0);
            const unsigned long long cols = (unsigned long long)min(32, q.W - q.tx0 - wc0);
            atomicAdd(&a.work[PROF_CONV], 2ull * (unsigned long long)P * P * rows * cols);
        }
        if (a.conv_chi2) {
            // an LM trial pass: this rung's chi^2 over the warp's 16 x 32 block
            // (each thread its 16 outputs in order, then the warp's shuffle
            // tree), one partial per block, and no convolved tile written.  The
            // blocks are the same under every tile shape, so the sums are too.
            CSum cs = {0.0f, 0.0f};
            if (active)
#pragma unroll
                for (int i = 0; i < RPT; ++i)
#pragma unroll
                    for (int o = 0; o < 8; ++o) {
                        const float d = dv[i][o], sg = sv[i][o];
                        if (isfinite(d) && isfinite(sg) && sg > 0.0f) {
                            const float z = (d - fmaf(tmw, acc[i][o], tmsky)) / sg;
                            csum_add(cs, z * z);
                        }
                    }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                CSum other;
                other.s = __shfl_down_sync(0xffffffffu, cs.s, o);
                other.c = __shfl_down_sync(0xffffffffu, cs.c, o);
                cs = csum_merge(cs, other);
            }
            if (active && lane == 0) {
                const int nbx = (q.W + 31) / 32;
                const long long slot = q.wb_off + (long long)((q.ty0 + wr0) / 16) * nbx + (q.tx0 + wc0) / 32;
                a.partial[slot * a.nchan + q.ch] = cs.s + cs.c;
            }
            q = qn;
            cb ^= 1;
            continue;
        }
        // the tile through shared memory (row stride TX + 1), then coalesced rows
        __syncthreads();
        constexpr int OS = TX + 1;
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int o = 0; o < 8; ++o) es[(r0 + 8 * i) * OS + c0 + o] = acc[i][o];
        __syncthreads();
        const int rows = min(TY, q.H - q.ty0), cols = min(TX, q.W - q.tx0);
        for (int idx = threadIdx.x; idx < TY * TX; idx += NT) {
            const int r = idx / TX, c = idx - r * TX;
            if (r < rows && c < cols) q.Y[(long long)(q.ty0 + r) * q.W + q.tx0 + c] = es[r * OS + c];
        }
        q = qn;
        cb ^= 1;
    }
    if (DB) cp_async_wait<0>();
}

}  // namespace

cudaError_t ensure_smem_optin_conv_direct(int P, int* cache);

// shared memory of k_conv_direct<TX, TY, P4K> for a P x P PSF: the taps and one
// halo tile, or two where the kernel double-buffers (P4K > 0)
template <int TX, int TY, int P4K>
size_t conv_smem(int P)
{
    const int P4 = (P + 3) & ~3;
    return sizeof(float) * ((size_t)P * P4 + (P4K > 0 ? 2 : 1) * (size_t)(TY + P - 1) * conv_sw(TX, P4));
}

// one opt-in record per kernel instance and device
template <int TX, int TY, int P4K>
int* conv_optin_cache()
{
    static int cache[64];
    return cache;
}

template <int TX, int TY, int P4K>
cudaError_t launch_p4(const PassArgs& a, int kind, cudaStream_t s)
{
    GF_LAUNCH_PDL((k_conv_direct<TX, TY, P4K>), dim3(a.grid[kind]), dim3(TX * TY / 16),
                  conv_smem<TX, TY, P4K>(a.P), s, a);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

template <int TX, int TY>
cudaError_t launch_tile_h(const PassArgs& a, int kind, cudaStream_t s)
{
    switch ((a.P + 3) & ~3) {
    case 4: return launch_p4<TX, TY, 4>(a, kind, s);
    case 8: return launch_p4<TX, TY, 8>(a, kind, s);
    case 12: return launch_p4<TX, TY, 12>(a, kind, s);
    case 16: return launch_p4<TX, TY, 16>(a, kind, s);
    case 20: return launch_p4<TX, TY, 20>(a, kind, s);
    case 24: return launch_p4<TX, TY, 24>(a, kind, s);
    case 28: return launch_p4<TX, TY, 28>(a, kind, s);
    case 32: return launch_p4<TX, TY, 32>(a, kind, s);
    case 36: return launch_p4<TX, TY, 36>(a, kind, s);
    default: return launch_p4<TX, TY, 0>(a, kind, s);
    }
}

template <int TX>
cudaError_t launch_tile(const PassArgs& a, int kind, cudaStream_t s)
{
    if (a.maxitems[kind] <= 0) return cudaSuccess;
    return a.conv_ty == 16 ? launch_tile_h<TX, 16>(a, kind, s) : launch_tile_h<TX, 32>(a, kind, s);
}

cudaError_t launch_conv_direct(const PassArgs& a, cudaStream_t s)
{
    cudaError_t e = ensure_smem_optin_conv_direct(a.P, nullptr);
    if (e != cudaSuccess) return e;
    if ((e = launch_tile<64>(a, WK_CONV, s)) != cudaSuccess) return e;
    return launch_tile<32>(a, WK_CONV32, s);
}

// launch one tile width alone (the tuner times the two against each other)
cudaError_t launch_conv_direct_width(const PassArgs& a, int tile_w, cudaStream_t s)
{
    cudaError_t e = ensure_smem_optin_conv_direct(a.P, nullptr);
    if (e != cudaSuccess) return e;
    return tile_w == 64 ? launch_tile<64>(a, WK_CONV, s) : launch_tile<32>(a, WK_CONV32, s);
}

// The shared-memory opt-in of the four tile shapes' kernels for a P x P PSF,
// made before the first launch (and cached per device), so that a call made
// before a stream capture leaves nothing to set inside it.
template <int P4K>
cudaError_t optin_p4(int P)
{
    cudaError_t e = ensure_smem_optin((const void*)k_conv_direct<64, 32, P4K>,
                                      (int)conv_smem<64, 32, P4K>(P), conv_optin_cache<64, 32, P4K>());
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_conv_direct<32, 32, P4K>, (int)conv_smem<32, 32, P4K>(P),
                              conv_optin_cache<32, 32, P4K>());
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_conv_direct<64, 16, P4K>, (int)conv_smem<64, 16, P4K>(P),
                              conv_optin_cache<64, 16, P4K>());
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_conv_direct<32, 16, P4K>, (int)conv_smem<32, 16, P4K>(P),
                              conv_optin_cache<32, 16, P4K>());
    return e;
}

cudaError_t ensure_smem_optin_conv_direct(int P, int*)
{
    switch ((P + 3) & ~3) {
    case 4: return optin_p4<4>(P);
    case 8: return optin_p4<8>(P);
    case 12: return optin_p4<12>(P);
    case 16: return optin_p4<16>(P);
    case 20: return optin_p4<20>(P);
    case 24: return optin_p4<24>(P);
    case 28: return optin_p4<28>(P);
    case 32: return optin_p4<32>(P);
    case 36: return optin_p4<36>(P);
    default: return optin_p4<0>(P);
    }
}
