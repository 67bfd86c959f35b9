// peak.cu -- FMA-loop microbenchmarks that measure the FP32 and FP64 peaks the
// roofline fractions of the ALU-bound kernels are quoted against (the HBM and
// bf16 tensor peaks are measured elsewhere; these two are not).
//
// Each thread runs 8 independent FMA chains (enough independent work to cover
// the FMA latency at full occupancy), so the loop issues one FMA per lane per
// cycle when the pipe is the limit.  The chains' results are stored only if
// they reach an impossible value, which keeps the arithmetic alive without a
// per-thread store.
#include "gf_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(int iters, T seed, T* sink)
{
    T a[kChains];
    const T m = seed * (T)0.999999, c = (T)1e-7;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = a[k] * m + c;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == (T)-12345.678) *sink = s;
}

}  // namespace

// FLOPs per launch: grid * kThreads threads * iters * 16 * kChains FMAs * 2
cudaError_t launch_fma_peak(int fp64, int grid, int iters, void* sink, cudaStream_t s,
                            double* flops)
{
    if (fp64)
        k_fma_peak<double><<<grid, kThreads, 0, s>>>(iters, 1.0, static_cast<double*>(sink));
    else
        k_fma_peak<float><<<grid, kThreads, 0, s>>>(iters, 1.0f, static_cast<float*>(sink));
    GF_COUNT_LAUNCH();
    *flops = 2.0 * grid * kThreads * (double)iters * 16.0 * kChains;
    return cudaGetLastError();
}
