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
// (32+P-1) x SW halo tile of the channel grid are staged in shared memory.
// A warp covers 16 x 32 outputs: lane 8 cg + rl owns the 8 contiguous columns
// 8 cg .. 8 cg + 7 of rows rl and rl + 8.  For each tap row and group of 4
// taps a thread holds, per row, a sliding window of 12 grid values (one new
// 16-byte load per group) and the 4 taps (one broadcast 16-byte load), and
// issues 2 x 8 x 4 = 64 FMAs: 3 shared loads per 64 FMAs.  In the kernels
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

// Work item = (channel, output tile of a listed stamp of this tile width).
template <int TX, int TY, int P4K>
__global__ void __launch_bounds__(TX * TY / 16) k_conv_direct(PassArgs a)
{
    pdl_entry();
    constexpr int NT = TX * TY / 16, WX = TX / 32;  // threads, warps across
    extern __shared__ __align__(16) float smem[];
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + (TX == 64 ? WK_CONV : WK_CONV32) * (a.count + 1);
    const int tot = pre[n];
    const long long items = (long long)tot * a.nchan;
    const int P = a.P, P4 = (P + 3) & ~3;
    const int SW = conv_sw(TX, P4), SH = TY + P - 1;
    float* ks = smem;               // P x P4 flipped taps
    float* es = smem + P * P4;      // SH x SW grid tile (P*P4 is a multiple of 4)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rl = lane & 7, cg = lane >> 3;
    const int wr0 = (warp / WX) * 16, wc0 = (warp % WX) * 32;
    const int r0 = wr0 + rl;       // the thread's first row in the tile
    const int c0 = wc0 + 8 * cg;   // the thread's first column in the tile
    int hint = -1, psf_b = -1;
    const long long chunk = (items + gridDim.x - 1) / gridDim.x;
    const long long it0 = (long long)blockIdx.x * chunk, it1 = min(items, it0 + chunk);
    for (long long it = it0; it < it1; ++it) {
        const int ch = (int)(it / tot), blk = (int)(it - (long long)ch * tot);
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        const StampInfo st = a.st[b];
        const int tiles_x = (st.W + TX - 1) / TX;
        const int t = blk - pre[li];
        const int ty0 = (t / tiles_x) * TY, tx0 = (t % tiles_x) * TX;
        __syncthreads();  // the previous item is done with the shared tiles
        if (b != psf_b) {
            const float* psf = a.psf + st.psf_off;
            for (int idx = threadIdx.x; idx < P * P4; idx += NT) {
                const int v = idx / P4, u = idx - v * P4;
                ks[idx] = (u < P) ? __ldg(&psf[(P - 1 - v) * P + (P - 1 - u)]) : 0.0f;
            }
            psf_b = b;
        }
        // the halo tile, a warp per row (coalesced, no index division), four
        // loads per lane in flight
        const float* E = a.ext + ext_index(st, a.nchan, ch);
        for (int r = warp; r < SH; r += NT / 32) {
            const int gy = ty0 + r;
            const bool row_in = gy < st.He;
            const float* Er = E + (long long)gy * st.We;
            float* er = es + r * SW;
            for (int c0_ = lane; c0_ < SW; c0_ += 128) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int col = c0_ + 32 * u, gx = tx0 + col;
                    v[u] = (row_in && col < SW && gx < st.We) ? __ldg(&Er[gx]) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (c0_ + 32 * u < SW) er[c0_ + 32 * u] = v[u];
            }
        }
        __syncthreads();

        // the warp's block meets the stamp
        const bool active = ty0 + wr0 < st.H && tx0 + wc0 < st.W;
        float acc[RPT][8];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int o = 0; o < 8; ++o) acc[i][o] = 0.0f;
        if (active)
            for (int v = 0; v < P; ++v)
                tap_row<P4K>(acc, ks + v * P4, es + (r0 + v) * SW + c0, SW, P4, P - (P4 - 4));

        if (active && a.work && lane == 0) {
            const unsigned long long rows = (unsigned long long)min(16, st.H - ty0 - wr0);
            const unsigned long long cols = (unsigned long long)min(32, st.W - tx0 - wc0);
            atomicAdd(&a.work[PROF_CONV], 2ull * (unsigned long long)P * P * rows * cols);
        }
        // the tile through shared memory (row stride TX + 1), then coalesced rows
        __syncthreads();
        constexpr int OS = TX + 1;
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int o = 0; o < 8; ++o) es[(r0 + 8 * i) * OS + c0 + o] = acc[i][o];
        __syncthreads();
        float* Y = a.y + y_index(st, a.nchan, ch);
        const int rows = min(TY, st.H - ty0), cols = min(TX, st.W - tx0);
        for (int idx = threadIdx.x; idx < TY * TX; idx += NT) {
            const int r = idx / TX, c = idx - r * TX;
            if (r < rows && c < cols) Y[(long long)(ty0 + r) * st.W + tx0 + c] = es[r * OS + c];
        }
    }
}

}  // namespace

cudaError_t ensure_smem_optin_conv_direct(int P, int* cache);

template <int TX, int TY>
size_t conv_smem(int P)
{
    const int P4 = (P + 3) & ~3;
    return sizeof(float) * ((size_t)P * P4 + (size_t)(TY + P - 1) * conv_sw(TX, P4));
}

size_t conv_direct_smem(int P) { return conv_smem<64, 32>(P); }

template <int TX, int TY, int P4K>
cudaError_t launch_p4(const PassArgs& a, int kind, cudaStream_t s)
{
    GF_LAUNCH_PDL((k_conv_direct<TX, TY, P4K>), dim3(a.grid[kind]), dim3(TX * TY / 16),
                  conv_smem<TX, TY>(a.P), s, a);
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

// one cache per device and width for every caller, so that a call made before a
// stream capture leaves nothing to set inside it
static int g_conv_optin[4][64];

// (the specialised kernels serve PSFs up to 35 pixels, whose tiles stay below the
// default 48 KB of shared memory; only the generic ones need the opt-in)
cudaError_t ensure_smem_optin_conv_direct(int P, int*)
{
    cudaError_t e = ensure_smem_optin((const void*)k_conv_direct<64, 32, 0>,
                                      (int)conv_smem<64, 32>(P), g_conv_optin[0]);
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_conv_direct<32, 32, 0>, (int)conv_smem<32, 32>(P),
                              g_conv_optin[1]);
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_conv_direct<64, 16, 0>, (int)conv_smem<64, 16>(P),
                              g_conv_optin[2]);
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_conv_direct<32, 16, 0>, (int)conv_smem<32, 16>(P),
                              g_conv_optin[3]);
    return e;
}
