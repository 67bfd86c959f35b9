// chol.cuh -- the damped normal-equation solve of an LM step in FP64 (the
// paper's step 4), shared by the stamp and the spectral fitting kernels.
#pragma once

#include <cuda_runtime.h>

#include "gf.h"

// sqrt(x) and 1/sqrt(x) of a positive finite x.  A float32 seed refined by two
// Newton-Raphson steps for the reciprocal square root, y <- y (3 - x y^2) / 2
// (each step squares the relative error: ~1e-7 -> ~1e-14 -> rounding level),
// then sqrt(x) = x y: about ten dependent FP64 operations instead of a square
// root and a division, which GB300's few FP64 units run as long chains.  Values
// outside the float32 exponent range take the library square root.
__device__ __forceinline__ void sqrt_and_rsqrt(double x, double& sq, double& rs)
{
    if (x > 1e-30 && x < 1e30) {
        const double h = 0.5 * x;
        double y = (double)rsqrtf((float)x);
        y = y * fma(-h, y * y, 1.5);
        y = y * fma(-h, y * y, 1.5);
        rs = y;
        sq = x * y;
    } else {
        sq = sqrt(x);
        rs = 1.0 / sq;
    }
}

// Warp Cholesky factorisation M = L L^T of the SPD n x n matrix M (row-major,
// shared memory, n <= GF_MAX_FREE) and the solve M x = r (x in r).  Lane i holds row i of M in registers
// (the loops over columns are unrolled to GF_MAX_FREE, so the row stays in
// registers): each column step j broadcasts the pivot from lane j, scales the
// entries below it by 1/sqrt(pivot), and every lane updates its row with
// L_ij L_kj, reading L_kj from lane k by a shuffle -- independent FMAs with no
// memory round trips between them.  The forward substitution runs on the
// register rows; the factor is then written to M for the back substitution,
// which needs it by columns.  Returns false (uniformly) when a pivot is not
// positive or a result is not finite.
__device__ __forceinline__ bool warp_cholesky_solve(int n, double* M, double* r)
{
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    double row[GF_MAX_FREE];
#pragma unroll
    for (int k = 0; k < GF_MAX_FREE; ++k)
        row[k] = (lane < n && k < n && k <= lane) ? M[lane * n + k] : 0.0;
    double invd_mine = 0.0;
#pragma unroll
    for (int j = 0; j < GF_MAX_FREE; ++j) {
        if (j >= n) break;
        const double piv = __shfl_sync(kFull, row[j], j);
        if (!(piv > 0.0) || !isfinite(piv)) return false;
        double d, invd;
        sqrt_and_rsqrt(piv, d, invd);
        if (lane == j) {
            row[j] = d;
            invd_mine = invd;
        } else if (lane > j) {
            row[j] *= invd;
        }
#pragma unroll
        for (int k = j + 1; k < GF_MAX_FREE; ++k) {
            if (k >= n) break;
            const double lkj = __shfl_sync(kFull, row[j], k);
            if (lane >= k && lane < n) row[k] = fma(-row[j], lkj, row[k]);
        }
    }
    // forward substitution L y = r
    double ri = lane < n ? r[lane] : 0.0;
#pragma unroll
    for (int k = 0; k < GF_MAX_FREE; ++k) {
        if (k >= n) break;
        const double yk = __shfl_sync(kFull, ri * invd_mine, k);
        if (lane == k)
            ri = yk;
        else if (lane > k && lane < n)
            ri = fma(-row[k], yk, ri);
    }
    // the factor by rows into shared memory, then back substitution L^T x = y
    __syncwarp();
#pragma unroll
    for (int k = 0; k < GF_MAX_FREE; ++k)
        if (lane < n && k < n && k <= lane) M[lane * n + k] = row[k];
    __syncwarp();
    for (int k = n - 1; k >= 0; --k) {
        const double xk = __shfl_sync(kFull, ri * invd_mine, k);
        if (lane == k)
            ri = xk;
        else if (lane < k)
            ri = fma(-M[k * n + lane], xk, ri);
    }
    if (lane < n) r[lane] = ri;
    __syncwarp();
    return __all_sync(kFull, lane >= n || isfinite(ri));
}
