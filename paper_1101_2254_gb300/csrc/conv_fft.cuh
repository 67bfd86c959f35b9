// conv_fft.cuh -- arguments of the Fourier-space convolution kernels (conv_fft.cu).
#pragma once

#include "fft.cuh"
#include "gf_internal.cuh"

#define GF_FFT_MAX 4096

struct FFTArgs {
    int Nx, Ny;          // padded transform sizes (Nx even)
    int cpc;             // spectrum columns per CTA in the column pass
    int small;           // 1: one CTA per transform (Nx, Ny in 32 x {3, 4, 5});
                         // hhat then holds each column in warp-FFT order
    FFTPlan px, py;
    float2* tw_x;        // exp(-2 pi i k / Nx), k < Nx
    float2* tw_y;        // exp(-2 pi i k / Ny), k < Ny
    float2* hhat;        // per stamp: Ny x (Nx/2 + 1) PSF spectrum / (Ny Nx)
    float* psfgrid;      // per stamp: Ny x Nx wrapped PSF (set-up scratch)
    StampInfo st0;       // geometry shared by every stamp of the call
    float flops_row;     // 5 Nx log2 Nx: one row transform (profiling)
    float flops_col;     // one column CTA: 2 transforms of Ny per column + products
};

struct RowIO {
    const float* in;
    long long in_stride;
    int ld, width, rows;
    float2* spec;
    long long spec_stride;
    int out_rows;
    int nchan;
    int nblk;            // CTAs per problem (set by the launcher)
};

struct ColIO {
    float2* spec;
    long long spec_stride;
    int rows_in, row0, nrows_out, nchan;
    int nblk;            // CTAs per problem (set by the launcher)
};

struct RowInvIO {
    const float2* spec;
    long long spec_stride;
    int row0, col0, H, W;
    float* out;
    long long out_stride;
    int nchan;
    int nblk;            // CTAs per problem (set by the launcher)
};

size_t fft_row_smem(int Nx);
// the smallest 32 M >= n with M in {3, 4, 5} (the one-CTA transform), else 0
int fft_small_len(int n);
size_t fft_col_smem(int Ny, int cpc);
cudaError_t launch_fft_twiddles(const FFTArgs& f, cudaStream_t s);
cudaError_t launch_fft_psf(const FFTArgs& f, int count, const StampInfo* st, const float* psf,
                           cudaStream_t s);
cudaError_t launch_conv_fft(const PassArgs& a, const FFTArgs& f, float2* spec, cudaStream_t s);
// the wrapped, 1/(Ny Nx)-scaled PSF grids (zeroed by the caller)
cudaError_t launch_psf_wrap(const FFTArgs& f, int count, const StampInfo* st, const float* psf,
                            cudaStream_t s);
