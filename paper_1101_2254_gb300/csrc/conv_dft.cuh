// conv_dft.cuh -- arguments of the tensor-core DFT convolution (conv_dft.cu).
#pragma once

#include <cuda_bf16.h>

#include "gf_internal.cuh"

#define DFT_RMAX 64  // largest factor of a transform length

// One dense DFT contraction ("stage") of the four-step plan.
//   orientation A: OUT[p][l][k][q] = tw * sum_r F[k][r] IN[p][l][r][q]   (r strided by Q)
//   orientation B: OUT[p][m][k]    = tw * sum_r F[k][r] IN[p][m][r]      (r contiguous)
// F is a (conjugated for the inverse) R x R DFT matrix held as four bf16
// planes (re hi, re lo, im hi, im lo) of Rp x Rp, Rp = R rounded up to 16.
struct DftStage {
    int R, Rp;
    int L, Q;                   // orientation A: batch and contiguous extent
    int M;                      // orientation B: rows
    const __nv_bfloat16* F;     // 4 x Rp x Rp
    // twiddle: exponent e = k * ((q / tw_div) % tw_mod) (mode 1, orientation A),
    //          e = l * k (mode 2, A), e = (m % tw_mod) * k (mode 3, B); w = tw[e mod N]
    int tw_mode, tw_div, tw_mod, tw_N;
    const float2* tw;           // exp(-2 pi i e / tw_N)
    float tw_sign;              // -1 forward (tw as stored), +1 inverse (conjugate)
    // input: 0 complex buffer; 1 real grid (rows >= in_rows or cols >= in_cols are 0);
    // 2 complex buffer times the PSF spectrum hhat (per stamp, same layout)
    int in_mode;
    const float2* in;
    long long in_pstride;       // complex elements per problem
    const float* in_real;       // in_mode 1: problem p's grid at in_real + p * in_real_pstride
    long long in_real_pstride;
    int in_ld, in_rows, in_cols;   // real grid row stride and valid extent
    int in_xdigit;              // in_mode 1: element (l, r, q) is grid (l, r * in_xdigit + q)
    const float2* hhat;         // in_mode 2
    int nchan;                  // problems per stamp (hhat index = p / nchan)
    // output: 0 complex buffer; 1 real crop: element (l, r', q) -> out_real at
    // (l - crop_y0, r' * out_xdigit + q - crop_x0) when inside H x W
    int out_mode;
    float2* out;
    long long out_pstride;
    float* out_real;
    long long out_real_pstride;
    int out_xdigit, crop_y0, crop_x0, crop_H, crop_W;
    // LM phase filter: problems of stamps whose phase differs are skipped
    const LMState* lm;
    int phase;
    // set to 1 when a tensor-core wait gives up (that tile's outputs are NaN)
    int* err;
};

cudaError_t launch_dft_stage_a(const DftStage& s, int nprob, unsigned long long* work,
                               cudaStream_t st);
cudaError_t launch_dft_stage_b(const DftStage& s, int nprob, unsigned long long* work,
                               cudaStream_t st);
cudaError_t launch_dft_matrix(int R, int Rp, float sign, __nv_bfloat16* F, cudaStream_t st);
