// conv_fft.cu -- step 2 of the fitting loop in Fourier space (Sec. 3 item 2
// places the PSF convolution there: forward FFTs, a pointwise product, an
// inverse FFT).
//
// The halo-extended grid (He x We) is convolved circularly at a padded size
// Ny x Nx (smallest 2^a 3^b 5^c >= He, and the smallest even one >= We); with
// the PSF wrapped so that its centre sits at (0, 0), the circular result equals
// the direct sum on the valid region, because every output pixel reads only
// grid pixels inside the extended grid.
//
// Extended grids up to 160 x 160 are padded to Nx, Ny in {96, 128, 160} and
// convolved by k_conv_fft_small, one CTA per channel with the half spectrum in
// shared memory (its own comment below).  Larger ones take three passes per
// channel, through shared-memory Stockham or warp register FFTs (fft.cuh,
// warp_fft.cuh), the half spectra held in a global scratch between passes:
//   rows    two real grid rows packed as one complex row, forward FFT, unpacked
//           into the two half spectra (Nx/2 + 1 bins each);
//   columns CPC adjacent spectrum columns per CTA (coalesced), forward FFT along
//           y, product with the PSF spectrum, inverse FFT; only the rows the
//           output needs are written back;
//   rows    inverse of the packing: two half spectra form one complex row, one
//           inverse FFT gives both output rows; only the valid region is kept.
// The PSF spectrum, scaled by 1/(Ny Nx), is computed once per call by the same
// kernels.  Grid rows beyond He are zeros and are never read or written.
#include <math.h>

#include "fft.cuh"
#include "gf_internal.cuh"
#include "conv_fft.cuh"
#include "warp_fft.cuh"

namespace {

constexpr int ROW_THREADS = 128;
constexpr int COL_THREADS = 256;
constexpr int COL_UNROLL = 8;   // column-block loads in flight per thread
constexpr int COL_HPRE = 12;    // PSF-spectrum values a thread may hold in registers

__global__ void k_twiddles(int n, float2* tw)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)n, &s, &c);
        tw[k] = make_float2((float)c, (float)-s);
    }
}

__device__ __forceinline__ void load_tw(float2* dst, const float2* src, int n)
{
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// The wrapped, normalised PSF on the Ny x Nx grid: psf[v][u] / (Ny Nx) at
// ((v - c) mod Ny, (u - c) mod Nx); the grid was zeroed by the caller.
__global__ void k_psf_wrap(FFTArgs f, int count, const StampInfo* st, const float* psf)
{
    const int b = blockIdx.x >> 3, part = blockIdx.x & 7;  // 8 CTAs per stamp
    if (b >= count) return;
    const int P = st[b].P, c = st[b].c;
    const float scale = (float)(1.0 / ((double)f.Ny * (double)f.Nx));
    float* g = f.psfgrid + (long long)b * f.Ny * f.Nx;
    const float* p = psf + st[b].psf_off;
    for (int t = part * blockDim.x + threadIdx.x; t < P * P; t += 8 * blockDim.x) {
        const int v = t / P, u = t - v * P;
        const int y = ((v - c) % f.Ny + f.Ny) % f.Ny, x = ((u - c) % f.Nx + f.Nx) % f.Nx;
        g[(long long)y * f.Nx + x] = p[t] * scale;
    }
}

// Forward row pass.  Problem p = blockIdx.x / io.nblk covers one real grid (rows `rows`
// valid of row stride `ld`, `width` valid columns) and one half-spectrum array
// (Kx = Nx/2 + 1 bins per row).  Block x of the problem handles rows 2x and 2x + 1.
// (Every FFT pass numbers its CTAs problem-major in one grid dimension: a
// problem count of count * channels may exceed the 65,535 of the y dimension.)
__global__ void __launch_bounds__(ROW_THREADS) k_fft_rows_fwd(FFTArgs f, RowIO io, PassArgs a)
{
    pdl_entry();
    extern __shared__ __align__(16) float2 sm[];
    const int p = blockIdx.x / io.nblk, bx = blockIdx.x - p * io.nblk;
    if (a.lm && a.lm[p / io.nchan].phase != a.phase) return;
    const int Nx = f.Nx, Kx = Nx / 2 + 1;
    float2* bufA = sm;
    float2* bufB = sm + Nx;
    float2* tw = sm + 2 * Nx;
    load_tw(tw, f.tw_x, Nx);
    const int y0 = 2 * bx, y1 = y0 + 1;
    const float* in = io.in + (long long)p * io.in_stride;
    for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
        const bool cx = x < io.width;
        const float va = (cx && y0 < io.rows) ? in[(long long)y0 * io.ld + x] : 0.0f;
        const float vb = (cx && y1 < io.rows) ? in[(long long)y1 * io.ld + x] : 0.0f;
        bufA[x] = make_float2(va, vb);
    }
    __syncthreads();
    const float2* Z = fft_smem(f.px, bufA, bufB, 0, tw, -1.0f);
    float2* out = io.spec + (long long)p * io.spec_stride;
    for (int k = threadIdx.x; k < Kx; k += blockDim.x) {
        const float2 zk = Z[k], zm = cconj(Z[(Nx - k) % Nx]);
        const float2 s = cadd(zk, zm), d = csub(zk, zm);
        // A = (Z[k] + conj Z[N-k]) / 2,  B = (Z[k] - conj Z[N-k]) / (2i)
        if (y0 < io.out_rows) out[(long long)y0 * Kx + k] = make_float2(0.5f * s.x, 0.5f * s.y);
        if (y1 < io.out_rows) out[(long long)y1 * Kx + k] = make_float2(0.5f * d.y, -0.5f * d.x);
    }
    if (a.work && threadIdx.x == 0) atomicAdd(&a.work[PROF_CONV], (unsigned long long)f.flops_row);
}

// Column pass.  mode 0: forward only, all Ny rows written (the PSF spectrum);
// mode 1: forward, product with the PSF spectrum, inverse, rows [c, c + H)
// written back in place.
__global__ void __launch_bounds__(COL_THREADS) k_fft_cols(FFTArgs f, ColIO io, PassArgs a, int mode)
{
    pdl_entry();
    extern __shared__ __align__(16) float2 sm[];
    const int p = blockIdx.x / io.nblk, bx = blockIdx.x - p * io.nblk;
    const int b = p / io.nchan;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const int Ny = f.Ny, Kx = f.Nx / 2 + 1, B = f.cpc, logB = __ffs(B) - 1;  // B a power of two
    float2* bufA = sm;
    float2* bufB = sm + Ny * B;
    float2* tw = sm + 2 * Ny * B;
    load_tw(tw, f.tw_y, Ny);
    const int kx0 = bx * B;
    float2* spec = io.spec + (long long)p * io.spec_stride;
    const int total = Ny * B;
    // the column block: eight loads per thread in flight before their stores
    for (int t0 = threadIdx.x; t0 < total; t0 += COL_UNROLL * COL_THREADS) {
        float2 v[COL_UNROLL];
#pragma unroll
        for (int u = 0; u < COL_UNROLL; ++u) {
            const int t = t0 + u * COL_THREADS;
            const int y = t >> logB, kx = kx0 + (t & (B - 1));
            v[u] = (t < total && y < io.rows_in && kx < Kx) ? spec[(long long)y * Kx + kx]
                                                            : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < COL_UNROLL; ++u) {
            const int t = t0 + u * COL_THREADS;
            if (t < total) bufA[t] = v[u];
        }
    }
    // the PSF spectrum this thread multiplies, fetched now so that its latency
    // hides behind the forward transform (when it fits the registers)
    const float2* Hs = f.hhat + (long long)b * Ny * Kx;
    float2 hv[COL_HPRE];
    const bool hpre = mode == 1 && total <= COL_HPRE * COL_THREADS;
    if (hpre) {
#pragma unroll
        for (int u = 0; u < COL_HPRE; ++u) {
            const int t = threadIdx.x + u * COL_THREADS;
            const int y = t >> logB, kx = kx0 + (t & (B - 1));
            hv[u] = (t < total && kx < Kx) ? Hs[(long long)y * Kx + kx] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    float2* X = fft_smem(f.py, bufA, bufB, logB, tw, -1.0f);
    if (a.work && threadIdx.x == 0) atomicAdd(&a.work[PROF_CONV], (unsigned long long)f.flops_col);
    if (mode == 0) {
        for (int t = threadIdx.x; t < Ny * B; t += blockDim.x) {
            const int y = t >> logB, kx = kx0 + (t & (B - 1));
            if (kx < Kx) spec[(long long)y * Kx + kx] = X[t];
        }
        return;
    }
    if (hpre) {
#pragma unroll
        for (int u = 0; u < COL_HPRE; ++u) {
            const int t = threadIdx.x + u * COL_THREADS;
            const int kx = kx0 + (t & (B - 1));
            if (t < total && kx < Kx) X[t] = cmul(X[t], hv[u]);
        }
    } else {
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int y = t >> logB, kx = kx0 + (t & (B - 1));
            if (kx < Kx) X[t] = cmul(X[t], Hs[(long long)y * Kx + kx]);
        }
    }
    __syncthreads();
    float2* other = (X == bufA) ? bufB : bufA;
    const float2* Yv = fft_smem(f.py, X, other, logB, tw, 1.0f);
    const int r0 = io.row0, r1 = io.row0 + io.nrows_out;
    for (int t = threadIdx.x; t < Ny * B; t += blockDim.x) {
        const int y = t >> logB, kx = kx0 + (t & (B - 1));
        if (kx < Kx && y >= r0 && y < r1) spec[(long long)y * Kx + kx] = Yv[t];
    }
}

// Inverse row pass: output rows 2x, 2x + 1 of an H x W result from spectrum
// rows row0 + 2x, row0 + 2x + 1; grid columns [col0, col0 + W) are kept.
__global__ void __launch_bounds__(ROW_THREADS) k_fft_rows_inv(FFTArgs f, RowInvIO io, PassArgs a)
{
    pdl_entry();
    extern __shared__ __align__(16) float2 sm[];
    const int p = blockIdx.x / io.nblk, bx = blockIdx.x - p * io.nblk;
    if (a.lm && a.lm[p / io.nchan].phase != a.phase) return;
    const int Nx = f.Nx, Kx = Nx / 2 + 1;
    float2* bufA = sm;
    float2* bufB = sm + Nx;
    float2* tw = sm + 2 * Nx;
    load_tw(tw, f.tw_x, Nx);
    const int i0 = 2 * bx, i1 = i0 + 1;
    const bool has1 = i1 < io.H;
    const float2* spec = io.spec + (long long)p * io.spec_stride;
    const float2* sa = spec + (long long)(io.row0 + i0) * Kx;
    const float2* sb = spec + (long long)(io.row0 + i1) * Kx;
    for (int k = threadIdx.x; k < Nx; k += blockDim.x) {
        float2 A, Bv;
        if (k < Kx) {
            A = sa[k];
            Bv = has1 ? sb[k] : make_float2(0.f, 0.f);
        } else {
            A = cconj(sa[Nx - k]);
            Bv = has1 ? cconj(sb[Nx - k]) : make_float2(0.f, 0.f);
        }
        bufA[k] = make_float2(A.x - Bv.y, A.y + Bv.x);  // A + i B
    }
    __syncthreads();
    const float2* z = fft_smem(f.px, bufA, bufB, 0, tw, 1.0f);
    float* out = io.out + (long long)p * io.out_stride;
    for (int j = threadIdx.x; j < io.W; j += blockDim.x) {
        const float2 v = z[io.col0 + j];
        out[(long long)i0 * io.W + j] = v.x;
        if (has1) out[(long long)i1 * io.W + j] = v.y;
    }
    if (a.work && threadIdx.x == 0) atomicAdd(&a.work[PROF_CONV], (unsigned long long)f.flops_row);
}

// ---------------------------------------------------------- warp row passes
// For Nx = 32 M with M in the WarpFFTFactor list the row passes use one warp
// per pair of rows and the register FFT of warp_fft.cuh: no block barrier
// between stages, every input load of a lane issued before the first
// butterfly.  The CTA's four warps share the padded twiddle table; each warp
// has an Nx-element buffer to bring its result into natural order (and, in the
// forward pass, to pair Z[k] with Z[Nx - k] for the unpacking).
constexpr int WROW_WARPS = 4;

template <int M>
__global__ void __launch_bounds__(WROW_WARPS * 32) k_fft_rows_fwd_w(FFTArgs f, RowIO io, PassArgs a)
{
    pdl_entry();
    constexpr int N = 32 * M, Kx = N / 2 + 1;
    extern __shared__ __align__(16) float2 sm[];
    const int p = blockIdx.x / io.nblk, bx = blockIdx.x - p * io.nblk;
    if (a.lm && a.lm[p / io.nchan].phase != a.phase) return;
    float2* tws = sm;
    for (int t = threadIdx.x; t < N; t += blockDim.x) tws[warp_fft_pad(t)] = f.tw_x[t];
    __syncthreads();
    const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int y0 = 2 * (bx * WROW_WARPS + warp), y1 = y0 + 1;
    if (y0 >= io.out_rows) return;
    const float* in = io.in + (long long)p * io.in_stride;
    float2 v[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int x = l + 32 * j;
        const bool cx = x < io.width;
        const float va = (cx && y0 < io.rows) ? in[(long long)y0 * io.ld + x] : 0.0f;
        const float vb = (cx && y1 < io.rows) ? in[(long long)y1 * io.ld + x] : 0.0f;
        v[j] = make_float2(va, vb);
    }
    warp_fft<M, false>(v, tws);
    float2* z = sm + warp_fft_table_len(N) + warp * N;
    const int br = bitrev5(l);
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) z[k2 + M * br] = v[k2];
    __syncwarp();
    float2* out = io.spec + (long long)p * io.spec_stride;
    for (int k = l; k < Kx; k += 32) {
        const float2 zk = z[k], zm = cconj(z[(N - k) % N]);
        const float2 s = cadd(zk, zm), d = csub(zk, zm);
        // A = (Z[k] + conj Z[N-k]) / 2,  B = (Z[k] - conj Z[N-k]) / (2i)
        out[(long long)y0 * Kx + k] = make_float2(0.5f * s.x, 0.5f * s.y);
        if (y1 < io.out_rows) out[(long long)y1 * Kx + k] = make_float2(0.5f * d.y, -0.5f * d.x);
    }
    if (a.work && l == 0) atomicAdd(&a.work[PROF_CONV], (unsigned long long)f.flops_row);
}

template <int M>
__global__ void __launch_bounds__(WROW_WARPS * 32) k_fft_rows_inv_w(FFTArgs f, RowInvIO io, PassArgs a)
{
    pdl_entry();
    constexpr int N = 32 * M, Kx = N / 2 + 1;
    extern __shared__ __align__(16) float2 sm[];
    const int p = blockIdx.x / io.nblk, bx = blockIdx.x - p * io.nblk;
    if (a.lm && a.lm[p / io.nchan].phase != a.phase) return;
    float2* tws = sm;
    for (int t = threadIdx.x; t < N; t += blockDim.x) tws[warp_fft_pad(t)] = f.tw_x[t];
    __syncthreads();
    const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int i0 = 2 * (bx * WROW_WARPS + warp), i1 = i0 + 1;
    if (i0 >= io.H) return;
    const bool has1 = i1 < io.H;
    const float2* spec = io.spec + (long long)p * io.spec_stride;
    const float2* sa = spec + (long long)(io.row0 + i0) * Kx;
    const float2* sb = spec + (long long)(io.row0 + i1) * Kx;
    float2 v[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int k = l + 32 * j;
        float2 A, Bv;
        if (k < Kx) {
            A = sa[k];
            Bv = has1 ? sb[k] : make_float2(0.f, 0.f);
        } else {
            A = cconj(sa[N - k]);
            Bv = has1 ? cconj(sb[N - k]) : make_float2(0.f, 0.f);
        }
        v[j] = make_float2(A.x - Bv.y, A.y + Bv.x);  // A + i B
    }
    warp_fft<M, true>(v, tws);
    float2* z = sm + warp_fft_table_len(N) + warp * N;
    const int br = bitrev5(l);
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) z[k2 + M * br] = v[k2];
    __syncwarp();
    float* out = io.out + (long long)p * io.out_stride;
    for (int j = l; j < io.W; j += 32) {
        const float2 w = z[io.col0 + j];
        out[(long long)i0 * io.W + j] = w.x;
        if (has1) out[(long long)i1 * io.W + j] = w.y;
    }
    if (a.work && l == 0) atomicAdd(&a.work[PROF_CONV], (unsigned long long)f.flops_row);
}

// ------------------------------------------- one CTA per transform (small grids)
// For Nx = 32 MX and Ny = 32 MY with MX, MY in {3, 4, 5} (grids up to 160 x 160)
// the whole convolution of one channel runs in one CTA: its half spectrum
// (Ny x Kx complex values, at most 104 KB) stays in shared memory between the
// three stages, so the only global traffic is the grid read, the PSF spectrum
// read and the valid region written (in an LM trial pass, the image and sigma
// read and the chi^2 partials of the 16 x 32 output blocks written instead of
// the region).  Every transform is a warp register FFT:
//   rows     a warp per pair of grid rows, packed and unpacked as in the row
//            kernels above;
//   columns  a warp per spectrum column: forward FFT along y, product with the
//            PSF spectrum, inverse FFT; the rows [row0, row0 + H) kept in place;
//   rows     a warp per pair of output rows, inverse of the packing.
// The PSF spectrum is made by the same kernel (psf_mode): the wrapped PSF
// through the row pass and the forward column FFT, stored per column in the
// order the warp FFT leaves it in (lane l, register k2 holds bin
// k2 + MY bitrev5(l)), so that the product reads it coalesced and needs no
// reordering: hperm[k][MY l + k2] = Hhat[k2 + MY bitrev5(l)][k].
constexpr int SMALL_WARPS = 8;

struct SmallIO {
    const float* in;      // grids: problem p at in + p in_stride, rows x width, row stride ld
    long long in_stride;
    int ld, width, rows;
    float* out;           // results: problem p at out + p out_stride, H x W
    long long out_stride;
    int row0, col0, H, W;
    float2* hperm;        // per stamp Kx * Ny values (written in psf_mode)
    int nchan;
    int psf_mode;
    float flops;          // one CTA's transform work (profiling)
};

// the column transforms' register twiddles: the row set itself when Nx = Ny
template <int MX, int MY>
__device__ __forceinline__ const WarpTw<MY>& select_tw(const WarpTw<MX>& rx, const WarpTw<MY>& ry)
{
    if constexpr (MX == MY)
        return rx;
    else
        return ry;
}

// CTAs per SM that the kernel's shared memory allows (227 KB per SM), which
// its register budget is held to
constexpr size_t small_smem(int Nx, int Ny);
constexpr size_t small_part_extra(int Nx, int Ny);
template <int MX, int MY>
constexpr int small_ctas_per_sm()
{
    const int n = (int)((227u * 1024u) / small_smem(32 * MX, 32 * MY));
    return n < 1 ? 1 : (n > 5 ? 5 : n);
}

template <int MX, int MY>
__global__ void __launch_bounds__(SMALL_WARPS * 32, small_ctas_per_sm<MX, MY>()) k_conv_fft_small(SmallIO io, PassArgs a,
                                                                     const float2* tw_x,
                                                                     const float2* tw_y)
{
    pdl_entry();
    constexpr int Nx = 32 * MX, Ny = 32 * MY, Kx = Nx / 2 + 1;
    constexpr int NZ = Nx > Ny ? Nx : Ny;
    extern __shared__ __align__(16) float2 sm[];
    const int p = blockIdx.x;
    const int b = p / io.nchan;
    if (a.lm && a.lm[b].phase != a.phase) return;  // whole CTA
    float2* twx = sm;
    float2* twy = twx + warp_fft_table_len(Nx);
    float2* spec = twy + warp_fft_table_len(Ny);  // Ny x Kx (row stride Kx: odd)
    const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
    float2* z = spec + Ny * Kx + warp * NZ;       // the warp's reordering buffer
    for (int t = threadIdx.x; t < Nx; t += blockDim.x) twx[warp_fft_pad(t)] = tw_x[t];
    for (int t = threadIdx.x; t < Ny; t += blockDim.x) twy[warp_fft_pad(t)] = tw_y[t];
    __syncthreads();
    // the lane's twiddles for every transform of the CTA (one set when Nx = Ny)
    WarpTw<MX> rx;
    warp_tw_load<MX>(rx, twx);
    WarpTw<MY> ry_own;
    if constexpr (MX != MY) warp_tw_load<MY>(ry_own, twy);
    const WarpTw<MY>& ry = select_tw<MX, MY>(rx, ry_own);
    const int br = bitrev5(l);
    // rows: pairs (y0, y0 + 1) of the grid; rows >= rows are zeros
    const int npair = (io.rows + 1) / 2, hw = 2 * npair;  // spectrum rows written
    const float* in = io.in + (long long)p * io.in_stride;
    // the warp's next row pair is loaded while the current one is transformed
    auto load_pair = [&](int pr, float2 (&w)[MX]) {
        const int y0 = 2 * pr, y1 = y0 + 1;
#pragma unroll
        for (int j = 0; j < MX; ++j) {
            const int x = l + 32 * j;
            const bool cx = x < io.width;
            const float va = cx ? in[(long long)y0 * io.ld + x] : 0.0f;
            const float vb = (cx && y1 < io.rows) ? in[(long long)y1 * io.ld + x] : 0.0f;
            w[j] = make_float2(va, vb);
        }
    };
    float2 vn[MX];
    if (warp < npair) load_pair(warp, vn);
    for (int pr = warp; pr < npair; pr += SMALL_WARPS) {
        const int y0 = 2 * pr, y1 = y0 + 1;
        float2 v[MX];
#pragma unroll
        for (int j = 0; j < MX; ++j) v[j] = vn[j];
        if (pr + SMALL_WARPS < npair) load_pair(pr + SMALL_WARPS, vn);
        warp_fft_r<MX, false>(v, rx);
#pragma unroll
        for (int k2 = 0; k2 < MX; ++k2) z[k2 + MX * br] = v[k2];
        __syncwarp();
        for (int k = l; k < Kx; k += 32) {
            const float2 zk = z[k], zm = cconj(z[(Nx - k) % Nx]);
            const float2 s = cadd(zk, zm), d = csub(zk, zm);
            // A = (Z[k] + conj Z[N-k]) / 2,  B = (Z[k] - conj Z[N-k]) / (2i)
            spec[y0 * Kx + k] = make_float2(0.5f * s.x, 0.5f * s.y);
            spec[y1 * Kx + k] = make_float2(0.5f * d.y, -0.5f * d.x);
        }
        __syncwarp();
    }
    __syncthreads();
    // columns
    float2* hp = io.hperm + (long long)b * Kx * Ny;
    for (int k = warp; k < Kx; k += SMALL_WARPS) {
        float2* hk = hp + (long long)k * Ny + MY * l;
        float2 h[MY];  // the PSF spectrum's column, loaded before the transform
        if (!io.psf_mode) {
#pragma unroll
            for (int k2 = 0; k2 < MY; ++k2) h[k2] = hk[k2];
        }
        float2 v[MY];
#pragma unroll
        for (int j = 0; j < MY; ++j) {
            const int y = l + 32 * j;
            v[j] = y < hw ? spec[y * Kx + k] : make_float2(0.0f, 0.0f);
        }
        warp_fft_r<MY, false>(v, ry);
        if (io.psf_mode) {
#pragma unroll
            for (int k2 = 0; k2 < MY; ++k2) hk[k2] = v[k2];
            continue;
        }
#pragma unroll
        for (int k2 = 0; k2 < MY; ++k2) z[k2 + MY * br] = cmul(v[k2], h[k2]);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < MY; ++j) v[j] = z[l + 32 * j];
        __syncwarp();
        warp_fft_r<MY, true>(v, ry);
#pragma unroll
        for (int k2 = 0; k2 < MY; ++k2) {
            const int y = k2 + MY * br;
            if (y >= io.row0 && y < io.row0 + io.H) spec[y * Kx + k] = v[k2];
        }
    }
    if (io.psf_mode) return;
    __syncthreads();
    // rows: inverse of the packing, output rows (i0, i0 + 1).  In an LM trial
    // pass (a.conv_chi2) nothing is written: each row pair's chi^2 per 32
    // columns goes to part[pair][column block] (the twiddle tables' space,
    // free by now), and the 16 x 32 blocks' sums to the stamp's partial slots.
    float* out = io.out + (long long)p * io.out_stride;
    static_assert(sizeof(CSum) == sizeof(float2), "a partial takes one float2 slot");
    CSum* part = reinterpret_cast<CSum*>(small_part_extra(Nx, Ny) == 0 ? sm
                                         : spec + Ny * Kx + SMALL_WARPS * NZ);
    const int nbx = (io.W + 31) / 32;
    const float* img = nullptr;
    const float* sig = nullptr;
    float tmw = 0.0f, tmsky = 0.0f;
    if (a.conv_chi2) {
        const StampInfo& st = a.st[b];
        const Channel& chn = a.chan[(long long)b * a.chan_stride + (p - b * io.nchan)];
        tmw = chn.mweight;
        tmsky = chn.msky;
        img = a.img + st.pix_off;
        sig = a.sig + st.pix_off;
    }
    for (int pr = warp; 2 * pr < io.H; pr += SMALL_WARPS) {
        const int i0 = 2 * pr, i1 = i0 + 1;
        const bool has1 = i1 < io.H;
        const float2* sa = spec + (io.row0 + i0) * Kx;
        const float2* sb = spec + (io.row0 + (has1 ? i1 : i0)) * Kx;
        float2 v[MX];
#pragma unroll
        for (int j = 0; j < MX; ++j) {
            const int k = l + 32 * j;
            float2 A, Bv;
            if (k < Kx) {
                A = sa[k];
                Bv = sb[k];
            } else {
                A = cconj(sa[Nx - k]);
                Bv = cconj(sb[Nx - k]);
            }
            if (!has1) Bv = make_float2(0.0f, 0.0f);
            v[j] = make_float2(A.x - Bv.y, A.y + Bv.x);  // A + i B
        }
        warp_fft_r<MX, true>(v, rx);
#pragma unroll
        for (int k2 = 0; k2 < MX; ++k2) z[k2 + MX * br] = v[k2];
        __syncwarp();
        if (a.conv_chi2) {
            for (int t = 0; t < nbx; ++t) {
                const int j = l + 32 * t;
                CSum cs = {0.0f, 0.0f};
                if (j < io.W) {
                    const float2 w = z[io.col0 + j];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        if (r == 1 && !has1) break;
                        const long long px = (long long)(i0 + r) * io.W + j;
                        const float d = __ldg(&img[px]), sg = __ldg(&sig[px]);
                        if (isfinite(d) && isfinite(sg) && sg > 0.0f) {
                            const float zr = (d - fmaf(tmw, r ? w.y : w.x, tmsky)) / sg;
                            csum_add(cs, zr * zr);
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    CSum other;
                    other.s = __shfl_down_sync(0xffffffffu, cs.s, o);
                    other.c = __shfl_down_sync(0xffffffffu, cs.c, o);
                    cs = csum_merge(cs, other);
                }
                if (l == 0) part[pr * nbx + t] = cs;
            }
        } else {
            for (int j = l; j < io.W; j += 32) {
                const float2 w = z[io.col0 + j];
                out[(long long)i0 * io.W + j] = w.x;
                if (has1) out[(long long)i1 * io.W + j] = w.y;
            }
        }
        __syncwarp();
    }
    if (a.conv_chi2) {
        // each 16 x 32 block: its 8 row pairs' partials merged in row order
        __syncthreads();
        const int npo = (io.H + 1) / 2, nby = (io.H + 15) / 16;
        const StampInfo& st = a.st[b];
        for (int q = threadIdx.x; q < nby * nbx; q += blockDim.x) {
            const int by = q / nbx, bx = q - by * nbx;
            CSum cs = part[(8 * by) * nbx + bx];
            for (int pr = 8 * by + 1; pr < min(npo, 8 * by + 8); ++pr)
                cs = csum_merge(cs, part[pr * nbx + bx]);
            a.partial[((long long)st.wb_off + q) * io.nchan + (p - b * io.nchan)] = cs.s + cs.c;
        }
    }
    if (a.work && threadIdx.x == 0) atomicAdd(&a.work[PROF_CONV], (unsigned long long)io.flops);
}

// the trial pass's row-pair chi^2 partials, (Ny / 2) x (Nx / 32) CSum values:
// in the twiddle tables' space where they fit (no extra bytes), else in a
// region of their own after the reordering rows
constexpr size_t small_part_extra(int Nx, int Ny)
{
    const size_t need = (size_t)(Ny / 2) * (Nx / 32) * sizeof(float2);
    const size_t have = sizeof(float2) * ((size_t)warp_fft_table_len(Nx) + (size_t)warp_fft_table_len(Ny));
    return need > have ? need : 0;
}

constexpr size_t small_smem(int Nx, int Ny)
{
    // tables, the half spectrum, one reordering row per warp
    return sizeof(float2) * ((size_t)warp_fft_table_len(Nx) + (size_t)warp_fft_table_len(Ny) +
                             (size_t)Ny * (Nx / 2 + 1) + (size_t)SMALL_WARPS * (Nx > Ny ? Nx : Ny)) +
           small_part_extra(Nx, Ny);
}

template <int MX, int MY>
cudaError_t launch_small_t(const SmallIO& io, const PassArgs& a, const FFTArgs& f, int nprob,
                           cudaStream_t s)
{
    static int optin[64];
    const size_t smem = small_smem(32 * MX, 32 * MY);
    cudaError_t e = ensure_smem_optin((const void*)k_conv_fft_small<MX, MY>, (int)smem, optin);
    if (e != cudaSuccess) return e;
    GF_LAUNCH_PDL(k_conv_fft_small<MX, MY>, dim3(nprob), dim3(SMALL_WARPS * 32), smem, s, io, a,
                  (const float2*)f.tw_x, (const float2*)f.tw_y);
    GF_COUNT_LAUNCH();
    return cudaSuccess;
}

cudaError_t launch_small(const SmallIO& io, const PassArgs& a, const FFTArgs& f, int nprob,
                         cudaStream_t s)
{
    switch ((f.Nx / 32) * 8 + f.Ny / 32) {
#define SMALL_CASE(MX_, MY_) \
    case MX_ * 8 + MY_: return launch_small_t<MX_, MY_>(io, a, f, nprob, s);
        SMALL_CASE(3, 3) SMALL_CASE(3, 4) SMALL_CASE(3, 5)
        SMALL_CASE(4, 3) SMALL_CASE(4, 4) SMALL_CASE(4, 5)
        SMALL_CASE(5, 3) SMALL_CASE(5, 4) SMALL_CASE(5, 5)
#undef SMALL_CASE
    default: return cudaErrorInvalidValue;
    }
}

size_t warp_row_smem(int N) { return sizeof(float2) * ((size_t)warp_fft_table_len(N) + (size_t)WROW_WARPS * N); }

// the warp row kernels exist for these Nx
#define WARP_FFT_CASES(X) X(3) X(4) X(5) X(6) X(8) X(9) X(10) X(12) X(15) X(16) X(18) X(20)

bool warp_rows_ok(int Nx)
{
    if (Nx % 32 != 0) return false;
    switch (Nx / 32) {
#define WF_CASE(M_) case M_:
        WARP_FFT_CASES(WF_CASE)
#undef WF_CASE
        return true;
    default: return false;
    }
}

}  // namespace

size_t fft_row_smem(int Nx) { return sizeof(float2) * 3 * (size_t)Nx; }

int fft_small_len(int n)
{
    for (int M = 3; M <= 5; ++M)
        if (32 * M >= n) return 32 * M;
    return 0;
}
size_t fft_col_smem(int Ny, int cpc) { return sizeof(float2) * ((size_t)2 * Ny * cpc + Ny); }

cudaError_t launch_fft_twiddles(const FFTArgs& f, cudaStream_t s)
{
    k_twiddles<<<(f.Nx + 255) / 256, 256, 0, s>>>(f.Nx, f.tw_x);
    GF_COUNT_LAUNCH();
    k_twiddles<<<(f.Ny + 255) / 256, 256, 0, s>>>(f.Ny, f.tw_y);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

static cudaError_t optin_all(const FFTArgs& f)
{
    static int o1[64], o2[64], o3[64];
    cudaError_t e = ensure_smem_optin((const void*)k_fft_rows_fwd, (int)fft_row_smem(f.Nx), o1);
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_fft_rows_inv, (int)fft_row_smem(f.Nx), o2);
    if (e == cudaSuccess)
        e = ensure_smem_optin((const void*)k_fft_cols, (int)fft_col_smem(f.Ny, f.cpc), o3);
    return e;
}

// forward / inverse row pass over `pairs` row pairs of each of nprob problems:
// the warp kernels where Nx allows, else the shared-memory Stockham kernels
// a one-dimensional grid of nblk CTAs for each of nprob problems
static bool grid_ok(long long nblk, long long nprob) { return nblk * nprob <= 0x7fffffffLL; }

static cudaError_t rows_fwd(const FFTArgs& f, RowIO r, const PassArgs& a, int pairs,
                            int nprob, cudaStream_t s)
{
    if (warp_rows_ok(f.Nx)) {
        r.nblk = (pairs + WROW_WARPS - 1) / WROW_WARPS;
        if (!grid_ok(r.nblk, nprob)) return cudaErrorInvalidConfiguration;
        const dim3 grid((unsigned)((long long)r.nblk * nprob));
        switch (f.Nx / 32) {
#define WF_CASE(M_)                                                                          \
    case M_:                                                                                 \
        GF_LAUNCH_PDL(k_fft_rows_fwd_w<M_>, grid, dim3(WROW_WARPS * 32), warp_row_smem(f.Nx), \
                      s, f, r, a);                                                           \
        break;
            WARP_FFT_CASES(WF_CASE)
#undef WF_CASE
        default: return cudaErrorInvalidValue;
        }
    } else {
        r.nblk = pairs;
        if (!grid_ok(r.nblk, nprob)) return cudaErrorInvalidConfiguration;
        GF_LAUNCH_PDL(k_fft_rows_fwd, dim3((unsigned)((long long)pairs * nprob)), dim3(ROW_THREADS),
                      fft_row_smem(f.Nx), s, f, r, a);
    }
    GF_COUNT_LAUNCH();
    return cudaSuccess;
}

// column pass (mode 1: transform, PSF product, inverse; mode 0: forward only)
static cudaError_t cols_pass(const FFTArgs& f, ColIO c, const PassArgs& a, int nprob,
                             int mode, cudaStream_t s)
{
    const int Kx = f.Nx / 2 + 1;
    // fewer columns per CTA until the pass has four CTAs per SM (the column
    // pass waits on L2 loads: more, smaller CTAs keep more of them in flight)
    FFTArgs fc = f;
    if (mode == 1)
        while (fc.cpc > 2 && (long long)nprob * ((Kx + fc.cpc - 1) / fc.cpc) < 4 * 152) fc.cpc /= 2;
    fc.flops_col = f.flops_col * (float)fc.cpc / (float)f.cpc;
    c.nblk = (Kx + fc.cpc - 1) / fc.cpc;
    if (!grid_ok(c.nblk, nprob)) return cudaErrorInvalidConfiguration;
    GF_LAUNCH_PDL(k_fft_cols, dim3((unsigned)((long long)c.nblk * nprob)), dim3(COL_THREADS),
                  fft_col_smem(fc.Ny, fc.cpc), s, fc, c, a, mode);
    GF_COUNT_LAUNCH();
    return cudaSuccess;
}

static cudaError_t rows_inv(const FFTArgs& f, RowInvIO v, const PassArgs& a, int pairs,
                            int nprob, cudaStream_t s)
{
    if (warp_rows_ok(f.Nx)) {
        v.nblk = (pairs + WROW_WARPS - 1) / WROW_WARPS;
        if (!grid_ok(v.nblk, nprob)) return cudaErrorInvalidConfiguration;
        const dim3 grid((unsigned)((long long)v.nblk * nprob));
        switch (f.Nx / 32) {
#define WF_CASE(M_)                                                                          \
    case M_:                                                                                 \
        GF_LAUNCH_PDL(k_fft_rows_inv_w<M_>, grid, dim3(WROW_WARPS * 32), warp_row_smem(f.Nx), \
                      s, f, v, a);                                                           \
        break;
            WARP_FFT_CASES(WF_CASE)
#undef WF_CASE
        default: return cudaErrorInvalidValue;
        }
    } else {
        v.nblk = pairs;
        if (!grid_ok(v.nblk, nprob)) return cudaErrorInvalidConfiguration;
        GF_LAUNCH_PDL(k_fft_rows_inv, dim3((unsigned)((long long)pairs * nprob)), dim3(ROW_THREADS),
                      fft_row_smem(f.Nx), s, f, v, a);
    }
    GF_COUNT_LAUNCH();
    return cudaSuccess;
}

cudaError_t launch_psf_wrap(const FFTArgs& f, int count, const StampInfo* st, const float* psf,
                            cudaStream_t s)
{
    k_psf_wrap<<<dim3(8 * count), 256, 0, s>>>(f, count, st, psf);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

// PSF spectra of all stamps of a call (uniform size): wrap, row pass over all
// Ny rows, forward column pass.
cudaError_t launch_fft_psf(const FFTArgs& f, int count, const StampInfo* st, const float* psf,
                           cudaStream_t s)
{
    cudaError_t e = f.small ? cudaSuccess : optin_all(f);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(f.psfgrid, 0, sizeof(float) * (size_t)count * f.Ny * f.Nx, s);
    if (e != cudaSuccess) return e;
    k_psf_wrap<<<dim3(8 * count), 256, 0, s>>>(f, count, st, psf);
    GF_COUNT_LAUNCH();
    PassArgs none;
    memset(&none, 0, sizeof(none));
    if (f.small) {
        SmallIO io;
        memset(&io, 0, sizeof(io));
        io.in = f.psfgrid;
        io.in_stride = (long long)f.Ny * f.Nx;
        io.ld = f.Nx;
        io.width = f.Nx;
        io.rows = f.Ny;
        io.hperm = f.hhat;
        io.nchan = 1;
        io.psf_mode = 1;
        e = launch_small(io, none, f, count, s);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    const int Kx = f.Nx / 2 + 1;
    RowIO r;
    r.in = f.psfgrid;
    r.in_stride = (long long)f.Ny * f.Nx;
    r.ld = f.Nx;
    r.width = f.Nx;
    r.rows = f.Ny;
    r.spec = f.hhat;
    r.spec_stride = (long long)f.Ny * Kx;
    r.out_rows = f.Ny;
    r.nchan = 1;
    e = rows_fwd(f, r, none, (f.Ny + 1) / 2, count, s);
    if (e != cudaSuccess) return e;
    ColIO c;
    c.spec = f.hhat;
    c.spec_stride = (long long)f.Ny * Kx;
    c.rows_in = f.Ny;
    c.row0 = 0;
    c.nrows_out = f.Ny;
    c.nchan = 1;
    e = cols_pass(f, c, none, count, 0, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Convolve the pass's channel grids (a.ext) into a.y through the spectrum
// scratch `spec` (count * nchan * He * Kx complex values).
cudaError_t launch_conv_fft(const PassArgs& a, const FFTArgs& f, float2* spec, cudaStream_t s)
{
    const StampInfo& s0 = f.st0;  // uniform stamp geometry (host copy)
    const int Kx = f.Nx / 2 + 1;
    const int nprob = a.count * a.nchan;
    if (f.small) {
        SmallIO io;
        io.in = a.ext;
        io.in_stride = (long long)s0.He * s0.We;
        io.ld = s0.We;
        io.width = s0.We;
        io.rows = s0.He;
        io.out = a.y;
        io.out_stride = (long long)s0.H * s0.W;
        io.row0 = s0.c;
        io.col0 = s0.c;
        io.H = s0.H;
        io.W = s0.W;
        io.hperm = f.hhat;
        io.nchan = a.nchan;
        io.psf_mode = 0;
        io.flops = (float)(((s0.He + 1) / 2 + (s0.H + 1) / 2) * 5.0 * f.Nx * log2((double)f.Nx) +
                           Kx * (10.0 * f.Ny * log2((double)f.Ny) + 6.0 * f.Ny));
        cudaError_t e = launch_small(io, a, f, nprob, s);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    cudaError_t e = optin_all(f);
    if (e != cudaSuccess) return e;
    RowIO r;
    r.in = a.ext;
    r.in_stride = (long long)s0.He * s0.We;
    r.ld = s0.We;
    r.width = s0.We;
    r.rows = s0.He;
    r.spec = spec;
    r.spec_stride = (long long)s0.He * Kx;
    r.out_rows = s0.He;
    r.nchan = a.nchan;
    e = rows_fwd(f, r, a, (s0.He + 1) / 2, nprob, s);
    if (e != cudaSuccess) return e;
    ColIO c;
    c.spec = spec;
    c.spec_stride = (long long)s0.He * Kx;
    c.rows_in = s0.He;
    c.row0 = s0.c;
    c.nrows_out = s0.H;
    c.nchan = a.nchan;
    e = cols_pass(f, c, a, nprob, 1, s);
    if (e != cudaSuccess) return e;
    RowInvIO v;
    v.spec = spec;
    v.spec_stride = (long long)s0.He * Kx;
    v.row0 = s0.c;
    v.col0 = s0.c;
    v.H = s0.H;
    v.W = s0.W;
    v.out = a.y;
    v.out_stride = (long long)s0.H * s0.W;
    v.nchan = a.nchan;
    e = rows_inv(f, v, a, (s0.H + 1) / 2, nprob, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
