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
    size_t part_floats;            // ... and their capacity
};

// bytes of the buffers for batch B (with the gradient buffers when training);
// fills cb when ws and cb are given
size_t cnn_buffers(void* ws, int B, bool training, CnnBuffers* cb);
cudaError_t cnn_prepare(const float* w, const float* x, int B, const CnnBuffers& cb, cudaStream_t s);
// the forward (inference and training): layers 2-4 as implicit GEMMs on the
// tensor cores (cnn_tc.cu), channels-last activations
cudaError_t cnn_forward_tc(const float* w, int B, const CnnBuffers& cb, float* y, cudaStream_t s);
// the two fully connected layers on the conv4 output (cb.a3, NCHW) into y
cudaError_t cnn_forward_fc(const float* w, int B, const CnnBuffers& cb, float* y, cudaStream_t s);
cudaError_t cnn_backward(const float* t, int B, float* loss, float* grad, const CnnBuffers& cb,
                         cudaStream_t s);
// layers 4-2 of the backward on the tensor cores (cnn_bwd_tc.cu): weight and
// bias gradients into grad, input gradients (through the ReLU below) into
// gout[l - 1]; gout[l] NHWC float, ins[l] NHWC bf16, wf the [in][tap][out] copy
cudaError_t cnn_backward_tc(int B, float* grad, float* const* gout, const __nv_bfloat16* const* ins,
                            const __nv_bfloat16* wf, float* part, size_t part_floats, cudaStream_t s);
// floats of weight-gradient partials cnn_backward_tc needs for batch B
size_t cnn_bwd_tc_part_floats(int B);
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
// e2: one double of device scratch (the flux factor at n = 2, formed first)
cudaError_t default_guess(int count, const int* H, const int* W, const long long* off,
                          const float* img, double* out, int nslots, size_t smem, int max_npx,
                          double* e2, cudaStream_t s);
cudaError_t guess_select(int count, int nslots, const double* cand, const double* x2c,
                         const double* dflt, const double* x2d, const double* lo, const double* hi,
                         double* out, int* choice, cudaStream_t s);
