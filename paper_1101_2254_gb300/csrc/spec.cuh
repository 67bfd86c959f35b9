// spec.cuh -- spectral-line fitting: the fitting loop of Sec. 2 in one
// dimension (Sec. 5: with flexible dimensionality the same procedure fits
// spectral lines; a data cube is fitted spectrum by spectrum).
#pragma once

#include <cuda_runtime.h>

#include "gf.h"

#define GF_SPEC_MAX_PARAMS (3 + 3 * GF_SPEC_MAX_LINES)

enum { SPEC_MODEL = 0, SPEC_EVAL = 1, SPEC_NORMAL = 2, SPEC_FIT = 3 };

// Everything a spectral launch needs (passed by value as the kernel
// parameter; all pointers are device memory).
struct SpecArgs {
    int mode;                // SPEC_*
    int N, K, nc, L;         // channels, lines, continuum terms, LSF taps
    int lsf_stride;          // 0: one LSF for all spectra; L: one per spectrum
    int count, np, nf;       // spectra, parameters, free parameters
    int fs[GF_MAX_FREE];     // free slot list
    double lo[GF_SPEC_MAX_PARAMS], hi[GF_SPEC_MAX_PARAMS];
    gf_lm_opts opts;         // LM rules, jac_mode and fd_rel
    const double* p_in;      // count x np
    double* p_out;           // count x np (SPEC_FIT)
    gf_lm_result* res;       // count (SPEC_FIT)
    const float* spec;       // count x N
    const float* sig;        // count x N
    const float* lsf;        // L or count x L
    float* model;            // count x N (SPEC_MODEL; optional for SPEC_EVAL)
    double* A;               // count x nf x nf (SPEC_NORMAL)
    double* g;               // count x nf (SPEC_NORMAL)
    double* chi2;            // count (SPEC_EVAL, SPEC_NORMAL)
    unsigned long long* work;  // profiling: useful FLOPs of the passes, or null
};

cudaError_t launch_spec(const SpecArgs& a, cudaStream_t s);
