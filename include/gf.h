/*
 * gf.h -- C ABI of the GB300 galaxy-fitting library (libgf.so).
 *
 * The library runs the data-parallel core of the galaxy-fitting loop of
 * Barsdell, Barnes & Fluke, "Fitting Galaxies on GPUs" (Sec. 2, steps 1-5):
 *   step 1  evaluate the model on the pixel grid         (Sec. 3: transform)
 *   step 2  convolve it with the PSF                     (Sec. 3: FFT + transform)
 *   step 3  compare model and observation by chi^2       (Sec. 3: transform + reduce)
 *   step 4  adjust the parameters (Levenberg-Marquardt, the routine Sec. 2
 *           names for GALFIT), from finite-difference Jacobian columns
 *   step 5  check the finishing criteria
 * and keeps every image on the device for all iterations, returning only the
 * O(1) parameters (Sec. 3, the data-residency argument).
 *
 * Conventions shared by every call
 *   - Images are row-major float32, dense (row stride = width).
 *   - Pixel (row i, column j) of an H x W stamp has its centre at (x=j, y=i).
 *   - The PSF is P x P float32, P odd, centre at (c, c) with c = (P-1)/2.
 *   - The model is evaluated on the halo-extended grid of (H+2c) x (W+2c)
 *     pixels; grid pixel (ie, je) is stamp pixel (ie-c, je-c), so the PSF sees
 *     light from outside the stamp.
 *   - Convolution is the true (flipped-kernel) sum over the valid region:
 *       out(i,j) = sum_{v,u} psf[v][u] * ext[i+2c-v][j+2c-u].
 *   - Parameters are float64; slots per component, in order:
 *       GF_SERSIC  x0, y0, I_e, r_e, n, q, pa_deg, c      (8 slots)
 *       GF_EXPDISK x0, y0, I_0, r_s, q, pa_deg, c          (7 slots)
 *       GF_SKY     s0                                      (1 slot)
 *     Sersic: I_e exp(-b_n((r/r_e)^{1/n} - 1)), b_n from P(2n, b_n) = 1/2.
 *     Exponential disk: I_0 exp(-r/r_s).
 *     r = (|x'|^{c+2} + |y'/q|^{c+2})^{1/(c+2)}, x' = dx cos t + dy sin t,
 *     y' = -dx sin t + dy cos t, t = pa_deg * pi/180 (counter-clockwise from +x).
 *   - Oversampling: inside an os_box x os_box block of stamp pixels (origin
 *     os_x0, os_y0; -1 centres it) a pixel is the mean of os_factor^2 samples at
 *     x = j - 1/2 + (b + 1/2)/os_factor (same in y); elsewhere the pixel centre.
 *   - chi^2 = sum over pixels with finite image and sigma > 0 of
 *     ((image - model)/sigma)^2, accumulated in compensated float32.
 *
 * Memory and streams
 *   - The caller owns every buffer.  Pointers named *_dev are device memory;
 *     *_host are host memory.  The library allocates nothing: the scratch it
 *     needs is the caller's workspace `ws` of at least gf_workspace_size()
 *     bytes (256-byte aligned device memory).
 *   - Every call is ordered on `stream` (NULL = the legacy default stream).
 *     Calls that write host memory (gf_lm_fit, gf_lm_fit_batch) synchronise
 *     the stream before returning; the others return without synchronising.
 *   - Workspace contents do not persist between calls.
 *
 * Errors
 *   - Arguments are validated before any launch; a bad argument returns
 *     GF_EINVAL and launches nothing.  A CUDA error returns GF_ECUDA.
 *     gf_last_error() gives a message for the calling thread's last failure.
 *   - Kernels never trap: problems found on the device (non-finite chi^2,
 *     singular systems) are reported through the per-stamp LM status.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gf_stream; /* the same handle as cudaStream_t */

typedef enum {
    GF_OK = 0,
    GF_EINVAL = 1,
    GF_ECUDA = 2,
    GF_ENOCONV = 3,    /* LM: damping grew past lambda_max */
    GF_ESINGULAR = 4,
    GF_ENONFINITE = 5,
    GF_ETIMEOUT = 6,
    GF_ENOMEM = 7,     /* workspace too small */
    GF_EMAXITER = 8    /* LM: max_iter trials without meeting a criterion */
} gf_status;

typedef enum { GF_SERSIC = 1, GF_EXPDISK = 2, GF_SKY = 3 } gf_comp_kind;

typedef enum {
    GF_CONV_AUTO = 0,   /* direct for P < GF_AUTO_FFT_PSF, else FFT */
    GF_CONV_DIRECT = 1, /* tiled direct sum, PSF and halo tile in shared memory */
    GF_CONV_FFT = 2,    /* shared-memory mixed-radix FFT, 2^a 3^b 5^c sizes up to 4096;
                           the stamps of one call must share H and W */
    GF_CONV_DFT_TC = 3  /* Fourier transforms as dense DFT contractions on the tensor cores
                           (split-precision bf16 operands, float32 accumulation); sizes
                           N = R1 R2 with R1, R2 <= 64; stamps of one call share H and W */
} gf_conv_method;

#define GF_MAX_COMP 8
#define GF_MAX_SLOTS 64
#define GF_MAX_FREE 16
#define GF_DIRECT_MAX_PSF 127
#define GF_AUTO_FFT_PSF 41
#define GF_MAX_PSF 1023

/* Model structure of one stamp (or of every stamp of a batch). */
typedef struct {
    int H, W;            /* stamp rows and columns (>= 1) */
    int psf_size;        /* P, odd, 1 <= P <= GF_MAX_PSF */
    int ncomp;           /* 1 .. GF_MAX_COMP components, at most one GF_SKY */
    int kinds[GF_MAX_COMP];
    int os_factor;       /* 1 = no oversampling; else 2 .. 64 */
    int os_box;          /* block side, 0 .. min(H, W) */
    int os_x0, os_y0;    /* block origin in stamp pixels, -1 = centred */
    int conv_method;     /* gf_conv_method */
} gf_desc;

/* Levenberg-Marquardt options (Marquardt's diagonal damping). */
typedef struct {
    double lambda0;      /* initial damping */
    double lambda_up;    /* factor on a rejected trial */
    double lambda_down;  /* factor on an accepted trial */
    double lambda_min;
    double lambda_max;   /* exceeding it ends the fit with GF_ENOCONV */
    double ftol;         /* converged when an accepted trial lowers chi^2 by less than ftol*chi^2 */
    double xtol;         /* converged when max |delta_i| / max(|p_i|, scale_i) < xtol */
    double fd_rel;       /* FD step: fd_rel px for positions, fd_rel*max(|p|,1) otherwise */
    int max_iter;        /* cap on trials (accepted + rejected) */
} gf_lm_opts;

typedef struct {
    double chi2;         /* chi^2 at the returned parameters */
    double lambda;
    int iters;           /* trials taken */
    int accepted;
    int status;          /* GF_OK (converged), GF_ENOCONV, GF_EMAXITER, GF_ENONFINITE */
} gf_lm_result;

/* Stamps of a batch: one structure (gf_desc, H and W ignored), per-stamp sizes
 * and offsets into packed device arrays.  All arrays are host memory. */
typedef struct {
    int count;
    const int* H;            /* [count] */
    const int* W;            /* [count] */
    const int64_t* pix_off;  /* [count] element offset of stamp b in image/sigma */
    const int64_t* psf_off;  /* [count] element offset of PSF b */
} gf_batch;

/* Which call a workspace is sized for. */
typedef enum {
    GF_CALL_MODEL = 0,
    GF_CALL_CONVOLVE = 1,
    GF_CALL_CHI2 = 2,
    GF_CALL_EVAL = 3,
    GF_CALL_JACOBIAN = 4,
    GF_CALL_LM_FIT = 5
} gf_call;

/* Library version (major*10000 + minor*100 + patch). */
int gf_version(void);

/* Message for the calling thread's last failed call ("" if none). */
const char* gf_last_error(void);

/* Number of parameter slots of a structure (sum of the components' slots). */
int gf_nslots(const gf_desc* d);

/* Workspace bytes needed by `call` for one stamp of structure d; `fixed_host`
 * (one byte per slot, nonzero = held) matters for GF_CALL_JACOBIAN and
 * GF_CALL_LM_FIT and may be NULL (all free). */
size_t gf_workspace_size(const gf_desc* d, const uint8_t* fixed_host, int call);

/* Workspace bytes for gf_lm_fit_batch. */
size_t gf_workspace_size_batch(const gf_desc* d, const gf_batch* b, const uint8_t* fixed_host);

/* Step 1 (Sec. 2 item 1; Sec. 3 item 1, a transform): write the model
 * (sky + all components) on the extended grid, (H+2c) x (W+2c) floats. */
gf_status gf_model(const gf_desc* d, const double* params_host, float* model_ext_dev,
                   void* ws, size_t ws_bytes, gf_stream stream);

/* Step 2 (Sec. 2 item 2; Sec. 3 item 2): convolve an extended grid with the
 * PSF; out_dev receives the H x W valid region.  Method per d->conv_method. */
gf_status gf_convolve(const gf_desc* d, const float* model_ext_dev, const float* psf_dev,
                      float* out_dev, void* ws, size_t ws_bytes, gf_stream stream);

/* Step 3 (Sec. 2 item 3; Sec. 3 item 3, transform + reduce): chi^2 of an
 * H x W model against image and sigma; the float64 result is written to
 * chi2_dev (device). */
gf_status gf_chi2(const gf_desc* d, const float* model_dev, const float* image_dev,
                  const float* sigma_dev, double* chi2_dev, void* ws, size_t ws_bytes,
                  gf_stream stream);

/* Steps 1-3 for one parameter vector: chi^2 to chi2_dev and, if model_dev is
 * not NULL, the convolved H x W model. */
gf_status gf_eval(const gf_desc* d, const double* params_host, const float* image_dev,
                  const float* sigma_dev, const float* psf_dev, float* model_dev,
                  double* chi2_dev, void* ws, size_t ws_bytes, gf_stream stream);

/* Steps 1-3 for many stamps of one structure at once: params_host is
 * count x nslots, chi2_dev receives count float64 values, model_dev (may be
 * NULL) the convolved models packed like the images.  Workspace:
 * gf_workspace_size_eval_batch(). */
gf_status gf_eval_batch(const gf_desc* d, const gf_batch* b, const double* params_host,
                        const float* image_dev, const float* sigma_dev, const float* psf_dev,
                        float* model_dev, double* chi2_dev, void* ws, size_t ws_bytes,
                        gf_stream stream);

/* Workspace bytes for gf_eval_batch. */
size_t gf_workspace_size_eval_batch(const gf_desc* d, const gf_batch* b);

/* The input of step 4: Jacobian columns of the convolved model with respect to
 * the free slots, in slot order.  Amplitude and sky slots use the exact column
 * (the convolved unit-amplitude component; sum(psf) for the sky); the others
 * forward differences with the step of gf_lm_opts.fd_rel (fd_rel <= 0: 1e-3).
 * Outputs (device): J_dev nfree x H x W (may be NULL), JtWJ_dev nfree x nfree,
 * JtWr_dev nfree, chi2_dev 1, all float64 except J. */
gf_status gf_jacobian(const gf_desc* d, const double* params_host, const uint8_t* fixed_host,
                      double fd_rel, const float* image_dev, const float* sigma_dev,
                      const float* psf_dev, float* J_dev, double* JtWJ_dev,
                      double* JtWr_dev, double* chi2_dev, void* ws, size_t ws_bytes,
                      gf_stream stream);

/* Fill opts with the library defaults (lambda0 1e-3, x10 / x0.1, [1e-12, 1e12],
 * ftol 1e-8, xtol 1e-8, fd_rel 1e-3, max_iter 200). */
void gf_default_opts(gf_lm_opts* opts);

/* Steps 1-5: Levenberg-Marquardt fit of one stamp.  params_host (nslots) is
 * the start and receives the result; fixed_host (nslots bytes, may be NULL)
 * holds slots; lo_host / hi_host (nslots, may be NULL for the defaults:
 * amplitudes >= 0, radii >= 0.1, n in [0.2, 10], q in [0.05, 1], boxiness in
 * [-1.9, 2]; position angles are wrapped into [0, 180)).  opts may be NULL.
 * Synchronises `stream` before returning. */
gf_status gf_lm_fit(const gf_desc* d, double* params_host, const uint8_t* fixed_host,
                    const double* lo_host, const double* hi_host, const float* image_dev,
                    const float* sigma_dev, const float* psf_dev, const gf_lm_opts* opts,
                    gf_lm_result* result_host, void* ws, size_t ws_bytes, gf_stream stream);

/* Steps 1-5 for many independent stamps of one structure, all resident on the
 * device, advanced together; params_host is count x nslots (in/out),
 * result_host count entries.  Synchronises `stream` before returning. */
gf_status gf_lm_fit_batch(const gf_desc* d, const gf_batch* b, double* params_host,
                          const uint8_t* fixed_host, const float* image_dev,
                          const float* sigma_dev, const float* psf_dev,
                          const gf_lm_opts* opts, gf_lm_result* result_host, void* ws,
                          size_t ws_bytes, gf_stream stream);

/* ------------------------------------------------- allocation-free evaluation
 * No counterpart in the paper: an interface for callers that cannot allocate
 * device memory at all -- for example a plugin whose host application owns
 * the whole device heap, or a latency-critical pipeline that may not call
 * cudaMalloc (which can synchronise the device) once it is running, and so
 * cannot provide the workspace the other calls need.
 *
 * gf_eval_static computes exactly what gf_eval computes (steps 1-3: the
 * convolved model and chi^2 of one stamp), but keeps its scratch in a
 * fixed device array of GF_STATIC_SCRATCH_BYTES (16 MiB) inside libgf.so.
 * Every GPU that loads the library holds that array until the process exits.
 * The call allocates nothing and calls no allocating routine; the caller still
 * passes the inputs (image, sigma, PSF) and outputs (model_dev may be NULL,
 * chi2_dev one double) in its own device memory.
 *   - A stamp whose scratch (about 4 bytes per extended-grid pixel plus 4 per
 *     stamp pixel) exceeds the array is rejected with GF_ENOMEM and a message,
 *     before any launch.  A 1024x1024 stamp with a 65x65 PSF fits; 2048x2048
 *     does not.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents.
 *     Every byte a call reads is written earlier by the same call, so nothing
 *     needs clearing, but calls whose work overlaps on the GPU (different
 *     streams, or different host threads) race on the array: serialise them. */
#define GF_STATIC_SCRATCH_BYTES (16u << 20)

/* Bytes of the static scratch array (GF_STATIC_SCRATCH_BYTES). */
size_t gf_static_scratch_bytes(void);

gf_status gf_eval_static(const gf_desc* d, const double* params_host, const float* image_dev,
                         const float* sigma_dev, const float* psf_dev, float* model_dev,
                         double* chi2_dev, gf_stream stream);

/* ------------------------------------------------------------ diagnostics
 * Not part of the method; used to measure the library (no counterpart in the
 * paper).  Kernel classes: 0 model evaluation, 1 convolution, 2 reductions,
 * 3 LM and constant preparation. */
#define GF_PROF_CLASSES 4

/* Kernels launched by the library since it was loaded (all threads). */
long long gf_launch_count(void);

/* work_dev != NULL turns profiling on: work_dev is a device array of
 * GF_PROF_CLASSES zero-initialised uint64 counters to which the kernels add
 * their algorithmic work (bytes written by the model kernels, FLOPs of the
 * convolution, bytes read by the reductions), and every class launch is
 * bracketed by CUDA events on its stream.  NULL turns profiling off. */
void gf_prof_enable(unsigned long long* work_dev);

/* Waits for the recorded events and returns, per class, the launches and the
 * summed device milliseconds since the previous call (then resets).  Either
 * pointer may be NULL. */
int gf_prof_times(double* ms_out, long long* launches_out);

#ifdef __cplusplus
}
#endif
#endif
