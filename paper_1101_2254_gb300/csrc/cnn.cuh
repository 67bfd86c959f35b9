// cnn.cuh -- launchers of cnn.cu (the learned initial guess, its training data,
// the default guess and the choice between them), called from capi.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/gf.h"

#define CNN_SIDE 64
#define CNN_NOUT 8
#define CNN_NPARAM 195432

// Per-call buffers of the network inside a caller's workspace.
struct CnnBuffers {
    __nv_bfloat16 *wp, *wf, *wb;   // bf16 weights: packed, [in][tap][out], [out][tap][in]
    __nv_bfloat16 *x;              // bf16 input, B x 64 x 64
    __nv_bfloat16 *a0, *a1, *a2, *a3;  // conv outputs after ReLU
    float *h, *y;                  // fc1 output after ReLU, network output
    float *gy, *gh, *g3, *g2, *g1, *g0;  // gradients at the pre-activations
    float* part;                   // first-stage weight-gradient partials
};

// bytes of the buffers for batch B (with the gradient buffers when training);
// fills cb when ws and cb are given
size_t cnn_buffers(void* ws, int B, bool training, CnnBuffers* cb);
cudaError_t cnn_prepare(const float* w, const float* x, int B, const CnnBuffers& cb, cudaStream_t s);
cudaError_t cnn_forward(const float* w, int B, const CnnBuffers& cb, float* y, cudaStream_t s);
// the inference forward: layers 2-4 as implicit GEMMs on the tensor cores
// (cnn_tc.cu), channels-last activations; the training forward keeps cnn_forward
cudaError_t cnn_forward_tc(const float* w, int B, const CnnBuffers& cb, float* y, cudaStream_t s);
// the two fully connected layers on the conv4 output (cb.a3, NCHW) into y
cudaError_t cnn_forward_fc(const float* w, int B, const CnnBuffers& cb, float* y, cudaStream_t s);
cudaError_t cnn_backward(const float* t, int B, float* loss, float* grad, const CnnBuffers& cb,
                         cudaStream_t s);
cudaError_t cnn_adam(float* w, float* m, float* v, const float* g, int step, float lr,
                     cudaStream_t s);
cudaError_t cnn_init(float* w, unsigned long long seed, cudaStream_t s);
cudaError_t cnn_input(const float* img, const float* sig, int B, float* x, cudaStream_t s);
cudaError_t cnn_encode(const double* params, int nslots, int count, int H, int W, float* t,
                       cudaStream_t s);
cudaError_t cnn_decode(const float* y, const double* dflt, int count, int H, int W, int flags,
                       double* params, cudaStream_t s);
cudaError_t train_sample(unsigned long long seed, int count, double* params, float* psf,
                         int psf_size, cudaStream_t s);
cudaError_t noise_fill(const float* m, long long n, unsigned long long seed, float sread,
                       float gain, float* d, float* sig, cudaStream_t s);
cudaError_t philox_blocks(const unsigned* in, unsigned* out, int n, cudaStream_t s);
size_t default_guess_smem(int H, int W);
cudaError_t default_guess(int count, const int* H, const int* W, const long long* off,
                          const float* img, double* out, int nslots, size_t smem, int max_npx,
                          cudaStream_t s);
cudaError_t guess_select(int count, int nslots, const double* cand, const double* x2c,
                         const double* dflt, const double* x2d, const double* lo, const double* hi,
                         double* out, int* choice, cudaStream_t s);
