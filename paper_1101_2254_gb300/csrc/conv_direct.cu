// conv_direct.cu -- step 2 of the fitting loop (Sec. 2 item 2) as a tiled
// direct sum, for PSFs up to GF_DIRECT_MAX_PSF pixels on a side.
//
//   out(i, j) = sum_{v,u} psf[v][u] * E[i+2c-v][j+2c-u]
//             = sum_{v,u} k[v][u]   * E[i+v][j+u],   k[v][u] = psf[P-1-v][P-1-u]
//
// One CTA computes a 32 x TX output tile of one channel: TX = 64 (4 warps) or
// TX = 32 (2 warps), chosen per stamp (the two kinds of work item).  The
// flipped PSF (rows padded with zeros to a multiple of 4 taps) and the
// (32+P-1) x (TX+P4) halo tile of the channel grid are staged in shared memory.
// A warp covers 16 x 32 outputs with lanes arranged 4 (rows) x 8 (columns); a
// thread owns a 4 x 4 block.  A warp whose 16 x 32 quadrant lies wholly outside
// the stamp skips the taps (its issue slots go to the SM's other CTAs).  For each tap row v and each group of 4 taps, a thread
// issues one broadcast 16-byte load of the taps and one 16-byte load of the
// next 4 grid values per output row, then 64 FMAs: 5 shared loads per 64 FMAs.
// Eight lanes of a quarter-warp read 128 contiguous bytes, so the grid loads
// are free of bank conflicts; the tap loads are broadcasts.
//
// The work is bound by the FP32 FMA pipe (2 P^2 flop per output pixel against
// 8 bytes of HBM traffic), not by HBM.
#include "gf_internal.cuh"

namespace {

constexpr int TY = CONV_TY;

// One tap row v: acc += sum_u k[v][u] E[r0 + v + r][c0 + o + u].  With the tap
// count P4K known at compile time (PSFs up to 33 pixels) the loop over tap
// groups unrolls completely and the sliding 8-value window costs no register
// moves; otherwise (P4K = 0) it runs over the runtime P4.
template <int P4K>
__device__ __forceinline__ void tap_row(float (&acc)[4][4], const float* kr, const float* er, int SW,
                                        int P4)
{
    float4 w0[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) w0[r] = *reinterpret_cast<const float4*>(er + r * SW);
    constexpr int PU = P4K > 0 ? P4K : 4;
    const int pend = P4K > 0 ? P4K : P4;
#pragma unroll(P4K > 0 ? P4K / 4 : 2)
    for (int m = 0; m < pend; m += 4) {
        const float4 kk = *reinterpret_cast<const float4*>(kr + m);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 w1 = *reinterpret_cast<const float4*>(er + r * SW + m + 4);
            const float win[8] = {w0[r].x, w0[r].y, w0[r].z, w0[r].w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                float x = acc[r][o];
                x = fmaf(kk.x, win[o], x);
                x = fmaf(kk.y, win[o + 1], x);
                x = fmaf(kk.z, win[o + 2], x);
                x = fmaf(kk.w, win[o + 3], x);
                acc[r][o] = x;
            }
            w0[r] = w1;
        }
    }
    (void)PU;
}

// Work item = (channel, output tile of a listed stamp of this tile width).
template <int TX, int P4K>
__global__ void __launch_bounds__(TX * 2) k_conv_direct(PassArgs a)
{
    pdl_entry();
    constexpr int NT = TX * 2, WX = TX / 32;  // threads, warps across
    extern __shared__ __align__(16) float smem[];
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + (TX == 64 ? WK_CONV : WK_CONV32) * (a.count + 1);
    const int tot = pre[n];
    const long long items = (long long)tot * a.nchan;
    const int P = a.P, P4 = (P + 3) & ~3;
    const int SW = TX + P4, SH = TY + P - 1;
    float* ks = smem;               // P x P4 flipped taps
    float* es = smem + P * P4;      // SH x SW grid tile (P*P4 is a multiple of 4)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wr0 = (warp / WX) * 16, wc0 = (warp % WX) * 32;
    const int r0 = wr0 + (lane >> 3) * 4;
    const int c0 = wc0 + (lane & 7) * 4;
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
        const float* E = a.ext + ext_index(st, a.nchan, ch);
        for (int idx = threadIdx.x; idx < SH * SW; idx += NT) {
            const int r = idx / SW, col = idx - r * SW;
            const int gy = ty0 + r, gx = tx0 + col;
            es[idx] = (gy < st.He && gx < st.We) ? __ldg(&E[(long long)gy * st.We + gx]) : 0.0f;
        }
        __syncthreads();

        if (ty0 + wr0 >= st.H || tx0 + wc0 >= st.W) continue;  // quadrant outside the stamp
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[r][o] = 0.0f;

        for (int v = 0; v < P; ++v)
            tap_row<P4K>(acc, ks + v * P4, es + (r0 + v) * SW + c0, SW, P4);

        if (a.work && (lane | (warp / WX)) == 0) {  // lane 0 of the first warp of each column
            const unsigned long long rows = (unsigned long long)min(TY, st.H - ty0);
            const unsigned long long cols = (unsigned long long)min(32, st.W - tx0 - wc0);
            atomicAdd(&a.work[PROF_CONV], 2ull * (unsigned long long)P * P * rows * cols);
        }
        float* Y = a.y + y_index(st, a.nchan, ch);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int oy = ty0 + r0 + r;
            if (oy >= st.H) continue;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int ox = tx0 + c0 + o;
                if (ox < st.W) Y[(long long)oy * st.W + ox] = acc[r][o];
            }
        }
    }
}

}  // namespace

cudaError_t ensure_smem_optin_conv_direct(int P, int* cache);

template <int TX>
size_t conv_smem(int P)
{
    const int P4 = (P + 3) & ~3;
    return sizeof(float) * ((size_t)P * P4 + (size_t)(TY + P - 1) * (TX + P4));
}

size_t conv_direct_smem(int P) { return conv_smem<64>(P); }

template <int TX, int P4K>
cudaError_t launch_p4(const PassArgs& a, int kind, cudaStream_t s)
{
    GF_LAUNCH_PDL(k_conv_direct<TX, P4K>, dim3(a.grid[kind]), dim3(TX * 2), conv_smem<TX>(a.P), s, a);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

template <int TX>
cudaError_t launch_tile(const PassArgs& a, int kind, cudaStream_t s)
{
    if (a.maxitems[kind] <= 0) return cudaSuccess;
    switch ((a.P + 3) & ~3) {
    case 4: return launch_p4<TX, 4>(a, kind, s);
    case 8: return launch_p4<TX, 8>(a, kind, s);
    case 12: return launch_p4<TX, 12>(a, kind, s);
    case 16: return launch_p4<TX, 16>(a, kind, s);
    case 20: return launch_p4<TX, 20>(a, kind, s);
    case 24: return launch_p4<TX, 24>(a, kind, s);
    case 28: return launch_p4<TX, 28>(a, kind, s);
    case 32: return launch_p4<TX, 32>(a, kind, s);
    case 36: return launch_p4<TX, 36>(a, kind, s);
    default: return launch_p4<TX, 0>(a, kind, s);
    }
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
static int g_conv_optin64[64], g_conv_optin32[64];

// (the specialised kernels serve PSFs up to 33 pixels, whose tiles stay below the
// default 48 KB of shared memory; only the generic ones need the opt-in)
cudaError_t ensure_smem_optin_conv_direct(int P, int*)
{
    cudaError_t e = ensure_smem_optin((const void*)k_conv_direct<64, 0>, (int)conv_smem<64>(P),
                                      g_conv_optin64);
    if (e != cudaSuccess) return e;
    return ensure_smem_optin((const void*)k_conv_direct<32, 0>, (int)conv_smem<32>(P),
                             g_conv_optin32);
}
