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
 *       GF_GAUSSIAN x0, y0, I_0, fwhm, q, pa_deg, c        (7 slots)
 *       GF_MOFFAT  x0, y0, I_0, fwhm, beta, q, pa_deg, c   (8 slots)
 *       GF_KING    x0, y0, I_0, r_c, r_t, alpha, q, pa_deg, c        (9 slots)
 *       GF_NUKER   x0, y0, I_b, r_b, alpha, beta, gamma, q, pa_deg, c (10 slots)
 *       GF_PSF     x0, y0, F                                   (3 slots)
 *       GF_SKY_PLANE s0, gx, gy                                (3 slots)
 *       GF_SERSIC_F  the Sersic's 8 slots, then a1, phi1, a3, phi3, a4, phi4   (14 slots)
 *     Sersic: I_e exp(-b_n((r/r_e)^{1/n} - 1)), b_n from P(2n, b_n) = 1/2.
 *     Exponential disk: I_0 exp(-r/r_s).
 *     Gaussian: I_0 exp(-r^2 / (2 s^2)), s = fwhm / (2 sqrt(2 ln 2)).
 *     Moffat: I_0 (1 + (r/alpha)^2)^(-beta), alpha = fwhm / (2 sqrt(2^(1/beta) - 1)),
 *     beta in [0.5, 20] by default.  (The Gaussian and the Moffat are further
 *     profile families after the Sersic and the disk.)
 *     King (modified): I_0 [(w - w_t) / (1 - w_t)]^alpha for r < r_t, 0 beyond,
 *     w = (1 + (r/r_c)^2)^(-1/alpha), w_t = w(r_t); I(0) = I_0, alpha = 2 is
 *     King's 1962 law; defaults r_t >= 0.1, alpha in [0.1, 10].
 *     Nuker: I_b 2^((beta-gamma)/alpha) (r/r_b)^-gamma [1 + (r/r_b)^alpha]^((gamma-beta)/alpha),
 *     I(r_b) = I_b, radius floored at 1e-6 r_b; defaults alpha in [0.1, 10],
 *     beta in [0, 10], gamma in [0, 2].
 *     Point source (GF_PSF): flux F at (x0, y0), placed on the grid by the
 *     cubic-convolution weights of Keys (1981, a = -1/2), w(x - x0) w(y - y0),
 *     at the pixel centres (also inside the oversampled block), so that the
 *     convolved image is the PSF interpolated to the sub-pixel position.
 *     King, Nuker and point sources have finite-difference Jacobian columns
 *     only: GF_JAC_ANALYTIC with one of them is rejected (GF_EINVAL).
 *     Sky plane (GF_SKY_PLANE): s0 + gx (x - x_c) + gy (y - y_c) about each
 *     stamp's centre (x_c, y_c) = ((W-1)/2, (H-1)/2), on the extended grid
 *     like the constant sky; all three slots are linear with exact columns.
 *     A structure has at most one sky component (GF_SKY or GF_SKY_PLANE).
 *     Sersic with Fourier modes (GF_SERSIC_F): the Sersic profile of the
 *     distorted radius r (1 + sum_m a_m cos(m (t - phi_m))), m = 1, 3, 4,
 *     t = atan2(y'/q, x') the angle in the component's circularised frame
 *     (t = 0 on the major axis), phi_m in degrees; amplitudes in [-0.3, 0.3]
 *     by default, phases free.  Finite-difference columns only.
 *     r = (|x'|^{c+2} + |y'/q|^{c+2})^{1/(c+2)}, x' = dx cos t + dy sin t,
 *     y' = -dx sin t + dy cos t, t = pa_deg * pi/180 (counter-clockwise from +x).
 *   - Oversampling: inside an os_box x os_box block of stamp pixels (origin
 *     os_x0, os_y0; -1 centres it) a pixel is the mean of os_factor^2 samples at
 *     x = j - 1/2 + (b + 1/2)/os_factor (same in y); elsewhere the pixel centre.
 *   - chi^2 = sum over pixels with finite image and finite sigma > 0 of
 *     ((image - model)/sigma)^2, accumulated in compensated float32.
 *   - Bad-pixel masks: a pixel whose sigma is 0 (or negative, infinite or NaN)
 *     or whose image value is not finite has weight 0 in chi^2, J^T W J and
 *     J^T W r on every path, so a mask is passed by setting sigma to 0 at the
 *     masked pixels (the same holds for the channels of spectra).
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

typedef enum {
    GF_SERSIC = 1,
    GF_EXPDISK = 2,
    GF_SKY = 3,
    GF_GAUSSIAN = 4,
    GF_MOFFAT = 5,
    GF_KING = 6,
    GF_NUKER = 7,
    GF_PSF = 8,
    GF_SKY_PLANE = 9,
    GF_SERSIC_F = 10
} gf_comp_kind;

typedef enum {
    GF_CONV_AUTO = 0,   /* direct for P < GF_AUTO_FFT_PSF, else FFT.  (For extended
                           grids up to 160 x 160 the FFT is one CTA per transform and
                           overtakes the direct sum from about P = 15 on 64x64 and
                           96x96 stamps, P = 33 on 32x32: name GF_CONV_FFT there.) */
    GF_CONV_DIRECT = 1, /* tiled direct sum, PSF and halo tile in shared memory */
    GF_CONV_FFT = 2,    /* shared-memory mixed-radix FFT, 2^a 3^b 5^c sizes up to 4096;
                           the stamps of one call must share H and W.  Extended grids
                           up to 160 x 160 are padded to Nx, Ny in {96, 128, 160} and
                           each channel is transformed, multiplied and transformed back
                           by one CTA with its spectrum in shared memory */
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
#define GF_MAX_LADDER 4

/* How the Jacobian columns of the nonlinear slots are formed. */
#define GF_JAC_FD 0        /* forward differences of the model (step fd_rel) */
#define GF_JAC_ANALYTIC 1  /* the convolved analytic derivative of the model grid */

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
    int jac_mode;        /* GF_JAC_FD: forward-difference columns for the nonlinear slots
                            (the default); GF_JAC_ANALYTIC: their analytic derivatives */
    int ladder;          /* trials evaluated together in one pass: the steps for lambda,
                            lambda*up, ... (1 .. GF_MAX_LADDER; 0 = automatic: 1 when the
                            call has at least as many stamps as the device has SMs, else
                            2).  The fit takes
                            exactly the steps of the one-trial-at-a-time rule: the trials
                            after the first are the ones that rule would try next after
                            rejections, and only those it reaches are used. */
    double time_budget_s; /* wall-clock budget of a stamp fit on the device, measured
                             by the GPU's global timer from the start of the LM loop;
                             0 = none.  When it runs out, every stamp still fitting
                             stops with status GF_ETIMEOUT and keeps its last
                             accepted parameters.  Used by the stamp fits
                             (gf_lm_fit, gf_lm_fit_batch, gf_lm_fit_multistart). */
} gf_lm_opts;

typedef struct {
    double chi2;         /* chi^2 at the returned parameters */
    double lambda;
    int iters;           /* trials taken */
    int accepted;
    int status;          /* GF_OK (converged), GF_ENOCONV, GF_EMAXITER, GF_ENONFINITE,
                            GF_ETIMEOUT (the options' time budget ran out) */
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
 * GF_CALL_LM_FIT and may be NULL (all free).  The GF_CALL_LM_FIT size holds for
 * any gf_lm_opts.ladder (it provides GF_MAX_LADDER trial channels); a smaller
 * workspace is accepted when it covers the ladder of the call (GF_ENOMEM
 * otherwise). */
size_t gf_workspace_size(const gf_desc* d, const uint8_t* fixed_host, int call);

/* Workspace bytes for gf_lm_fit_multistart with `starts` starts per stamp. */
size_t gf_workspace_size_multistart(const gf_desc* d, const gf_batch* b, int starts,
                                    const uint8_t* fixed_host);

/* Workspace bytes for gf_lm_fit_batch (for any ladder, as gf_workspace_size). */
size_t gf_workspace_size_batch(const gf_desc* d, const gf_batch* b, const uint8_t* fixed_host);

/* Step 1 (Sec. 2 item 1; Sec. 3 item 1, a transform): write the model
 * (sky + all components) on the extended grid, (H+2c) x (W+2c) floats. */
gf_status gf_model(const gf_desc* d, const double* params_host, float* model_ext_dev,
                   void* ws, size_t ws_bytes, gf_stream stream);

/* Step 1 for many stamps of one structure in one launch: params_host is
 * count x nslots; model_ext_dev receives the extended grids packed stamp after
 * stamp ((H_b+2c) x (W_b+2c) floats each, in batch order; b->pix_off and
 * b->psf_off are not used).  Workspace: gf_workspace_size_model_batch(). */
gf_status gf_model_batch(const gf_desc* d, const gf_batch* b, const double* params_host,
                         float* model_ext_dev, void* ws, size_t ws_bytes, gf_stream stream);
size_t gf_workspace_size_model_batch(const gf_desc* d, const gf_batch* b);

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

/* Workspace bytes for gf_eval_batch and gf_eval_batch_dev. */
size_t gf_workspace_size_eval_batch(const gf_desc* d, const gf_batch* b);

/* gf_eval_batch with the parameters already in device memory (params_dev,
 * count x nslots float64, read on the stream).  With image_dev, sigma_dev and
 * chi2_dev all NULL the call only renders: model_dev (required) receives the
 * convolved models and no chi^2 is formed. */
gf_status gf_eval_batch_dev(const gf_desc* d, const gf_batch* b, const double* params_dev,
                            const float* image_dev, const float* sigma_dev, const float* psf_dev,
                            float* model_dev, double* chi2_dev, void* ws, size_t ws_bytes,
                            gf_stream stream);

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

/* As gf_jacobian, with the nonlinear columns formed from the analytic
 * derivatives of the model (the chain rule through the generalised radius, the
 * rotation and the Sersic index; db_n/dn from the b_n table) instead of finite
 * differences.  The paper names the finite-difference Jacobian as the routine's
 * own (Sec. 2 item 4: "routine-specific"); this is the next step after it:
 * no step-size noise, one evaluation of each component per sample instead of
 * one per finite-difference channel.  Arguments as gf_jacobian without fd_rel;
 * the workspace is gf_workspace_size(d, fixed_host, GF_CALL_JACOBIAN). */
gf_status gf_jacobian_analytic(const gf_desc* d, const double* params_host,
                               const uint8_t* fixed_host, const float* image_dev,
                               const float* sigma_dev, const float* psf_dev, float* J_dev,
                               double* JtWJ_dev, double* JtWr_dev, double* chi2_dev, void* ws,
                               size_t ws_bytes, gf_stream stream);

/* Fill opts with the library defaults (lambda0 1e-3, x10 / x0.1, [1e-12, 1e12],
 * ftol 1e-8, xtol 1e-8, fd_rel 1e-3, max_iter 200, jac_mode GF_JAC_FD,
 * ladder 0 = automatic, no time budget). */
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
 * result_host count entries.  Synchronises `stream` before returning.
 *
 * Residency (Sec. 3): on a capturable stream (not the legacy default stream)
 * the whole LM loop is one CUDA-graph launch.  The loop body (work lists,
 * Jacobian pass, damped solves, trial pass, accept/reject) sits inside a
 * conditional WHILE node, and the body's last kernel decides on the device
 * whether to run it again: while any stamp is still fitting, fewer than
 * max_iter + 2 bodies have run and the time budget (opts->time_budget_s) is
 * not spent.  The host waits once, for the final parameters.  The executable
 * graph is kept per host thread and updated in place when the next call has
 * the same shape.  A call on the legacy default stream (NULL), which cannot
 * be captured, runs on a blocking stream the library keeps per host thread
 * and device; the legacy stream's implicit synchronisation orders it with
 * the caller's work.  Profiled calls (gf_prof_enable) launch the same body
 * directly and the host reads the active-stamp count every few bodies. */
gf_status gf_lm_fit_batch(const gf_desc* d, const gf_batch* b, double* params_host,
                          const uint8_t* fixed_host, const float* image_dev,
                          const float* sigma_dev, const float* psf_dev,
                          const gf_lm_opts* opts, gf_lm_result* result_host, void* ws,
                          size_t ws_bytes, gf_stream stream);

/* Multi-start fitting: each of the b->count stamps is fitted from `starts`
 * starting points, and the fit with the lowest finite chi^2 is kept (the
 * earliest start on ties).  This spends the GPU's speed-up on robustness
 * against local minima: Sec. 5 names costlier, more robust routines as the use
 * of the speed-up.  All count x starts fits advance together in one batched
 * fit; the copies of a stamp share its image, sigma and PSF (nothing is
 * copied).
 *   starts_host: count x starts x nslots float64, start k of stamp i at
 *     (i * starts + k) * nslots;
 *   params_out: count x nslots, the kept fits;
 *   result_out: count entries;
 *   best_out (may be NULL): count ints, the start each stamp kept.
 * Each fit is the one gf_lm_fit_batch gives for that start.  Workspace:
 * gf_workspace_size_multistart().  Synchronises `stream` before returning. */
gf_status gf_lm_fit_multistart(const gf_desc* d, const gf_batch* b, int starts,
                               const double* starts_host, const uint8_t* fixed_host,
                               const float* image_dev, const float* sigma_dev,
                               const float* psf_dev, const gf_lm_opts* opts, double* params_out,
                               gf_lm_result* result_out, int* best_out, void* ws,
                               size_t ws_bytes, gf_stream stream);

/* ------------------------------------------------------------ tile tuning
 * No counterpart in the paper.  The direct convolution covers each stamp with
 * TY x TX output tiles on a persistent grid.  The shape is kept per device:
 *   - the tile width TX (64 or 32) per PSF side P and class ceil(W / 32).  The
 *     widths differ only for classes with ceil(W / 32) odd: there the narrow
 *     tile saves a 32-column strip per tile row but stages more halo per
 *     output.  Untuned odd classes use the narrow tile, even ones the wide;
 *   - the tile height TY (32 or 16) and the persistent grid (CTAs per SM) per
 *     P, for every stamp of a call; untuned: 32 and 8.
 * Results do not depend on the shape (every output sums its taps in the same
 * order).
 *
 * gf_autotune times the candidates on the call's stamps over the Jacobian
 * pass's channels and the caller's PSFs, and keeps the fastest: the two widths
 * per odd class, then the six (TY, CTAs per SM) pairs in {32, 16} x {4, 8, 16}
 * on the whole batch, then the widths again under the chosen pair (12 shapes
 * per odd class, 6 per even one).  It synchronises the stream, must not run
 * under stream capture, and needs a workspace of gf_workspace_size_batch()
 * bytes.  It does nothing for Fourier-space convolution. */
gf_status gf_autotune(const gf_desc* d, const gf_batch* b, const float* psf_dev, void* ws,
                      size_t ws_bytes, gf_stream stream);
/* The tile width (64 or 32) the current device uses for PSF side P and width W. */
int gf_conv_tile_width(int psf_size, int width);
/* Set it for the class of W (a class with ceil(W / 32) even accepts only 64). */
gf_status gf_set_conv_tile_width(int psf_size, int width, int tile_w);
/* The whole shape the current device uses for PSF side P and width W (any
 * pointer may be NULL). */
gf_status gf_conv_tile_shape(int psf_size, int width, int* tile_w, int* tile_h, int* ctas_per_sm);
/* Set the tile height (16 or 32) and CTAs per SM (1 .. 32) for PSF side P. */
gf_status gf_set_conv_tile_shape(int psf_size, int tile_h, int ctas_per_sm);

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
 *   - A stamp is accepted exactly when gf_workspace_size(d, NULL,
 *     GF_CALL_EVAL) <= GF_STATIC_SCRATCH_BYTES; otherwise the call returns
 *     GF_ENOMEM with a message, before any launch.  The scratch depends on the
 *     convolution method (He x We = extended grid, Ny x Nx = transform size,
 *     each array rounded up to 256 bytes, plus a few KB of tables):
 *       direct:  4 He We + 4 H W
 *       FFT:     the direct terms + 8 Ny (Nx/2+1) + 4 Ny Nx + 8 He (Nx/2+1)
 *                + 8 (Nx + Ny); without the 8 He (Nx/2+1) spectrum scratch when
 *                He, We <= 160 (one CTA per transform, Nx, Ny in {96, 128, 160})
 *       DFT_TC:  the direct terms + 8 Ny Nx + 4 Ny Nx + 2 x 8 Ny Nx
 *                + 8 (Nx + Ny) + 256 KiB of DFT matrices
 *     With a 65x65 PSF, GF_CONV_AUTO takes the FFT (P >= GF_AUTO_FFT_PSF):
 *     square stamps up to 836x836 fit and 1024x1024 (24.4 MB) does not; with
 *     GF_CONV_DIRECT named, 1024x1024 fits (8.9 MB) and 2048x2048 does not.
 *     A 33x33 PSF (direct under GF_CONV_AUTO) fits up to 1431x1431.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and (like the first
 *     model-evaluating call of any kind) fills the library's static b_n table
 *     with one kernel and a synchronisation of the stream; make that first
 *     call before any stream capture.
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

/* ------------------------------------------------- learned initial guess
 * No counterpart in the paper's text, which needs a starting point for step 4
 * (Sec. 2 item 4) but does not say where it comes from, and names more robust
 * fitting as the use of the speed-up (Sec. 5).  A convolutional network maps
 * a 64x64 stamp to a start for a single Sersic + sky fit (9 slots: x0, y0, I_e,
 * r_e, n, q, pa_deg, c, sky); a moments-based default guess is the fallback.
 *
 * Network: input x = asinh(img / a), a = median sigma over the stamp's outer
 * ring; conv 3x3 stride 2 padding 1 1->32->64->64->128 (64 -> 4 pixels), fc
 * 2048->32, fc 32->8, ReLU after all but the last layer.  Parameters: float32
 * masters, GF_CNN_NPARAM of them, packed per layer as weights [out][in][ky][kx]
 * (fc [out][in]) then biases.  Arithmetic: bf16 weights and activations, float32
 * accumulation, fixed-order (deterministic) reductions.
 * Outputs / targets (8, each scaled to about [-1, 1] over the training prior):
 *   x0 - 31.5, y0 - 31.5, (ln F - 3.5 ln 10) / (1.5 ln 10),
 *   (ln r_e - ln 80 / 2) / (ln 20 / 2), (n - 3.25) / 2.75, (q - 0.6) / 0.4,
 *   cos 2 pa, sin 2 pa;   F = closed-form Sersic flux.
 * All buffers are device memory owned by the caller; calls are stream-ordered
 * and do not synchronise. */
#define GF_CNN_SIDE 64
#define GF_CNN_NOUT 8
#define GF_CNN_NPARAM 195432

size_t gf_cnn_nparams(void);
/* Workspace bytes of gf_cnn_forward (training = 0) or gf_cnn_loss_grad
 * (training = 1) for a batch. */
size_t gf_cnn_workspace_size(int batch, int training);

/* He-normal weights N(0, 2 / fan_in) from Philox4x32-10 keyed by seed, zero
 * biases, into w_dev (GF_CNN_NPARAM floats). */
gf_status gf_cnn_init(float* w_dev, unsigned long long seed, gf_stream stream);

/* Network input of `batch` 64x64 stamps: x_dev = asinh(img / a) per stamp. */
gf_status gf_cnn_input(const float* image_dev, const float* sigma_dev, int batch, float* x_dev,
                       gf_stream stream);

/* y_dev (batch x 8) = network(x_dev (batch x 64 x 64, rounded to bf16)). */
gf_status gf_cnn_forward(const float* w_dev, const float* x_dev, int batch, float* y_dev,
                         void* ws, size_t ws_bytes, gf_stream stream);

/* Mean squared error over batch x 8 against t_dev, into loss_dev (1 float),
 * and its gradient with respect to every parameter, into grad_dev. */
gf_status gf_cnn_loss_grad(const float* w_dev, const float* x_dev, const float* t_dev, int batch,
                           float* loss_dev, float* grad_dev, void* ws, size_t ws_bytes,
                           gf_stream stream);

/* One Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) on the
 * masters w_dev with moments m_dev, v_dev (zero before step 1); step >= 1. */
gf_status gf_cnn_adam(float* w_dev, float* m_dev, float* v_dev, const float* grad_dev, int step,
                      float lr, gf_stream stream);

/* Targets (count x 8 float) of the Sersic slots 0..6 of count parameter
 * vectors of nslots float64 each (64x64 stamps). */
gf_status gf_cnn_encode(const double* params_dev, int nslots, int count, float* t_dev,
                        gf_stream stream);

/* Inverse of gf_cnn_encode: count x 9 slots, c = 0, sky copied from slot 8 of
 * dflt_dev (count x 9, e.g. gf_default_guess); I_e is NaN where n leaves
 * [0.2, 10] or q leaves (0, 1].  flags: 0, or GF_DECODE_MOMENT_CENTRE to take
 * x0, y0 from dflt_dev instead of the network. */
#define GF_DECODE_MOMENT_CENTRE 1
gf_status gf_cnn_decode(const float* y_dev, const double* dflt_dev, int count, int flags,
                        double* params_dev, gf_stream stream);

/* Training batch keyed by seed: count x 9 parameters drawn from the prior
 * (centre 31.5 + U[-1, 1], n ~ U[0.5, 6], r_e log-uniform [2, 40],
 * q ~ U[0.2, 1], pa ~ U[0, 180), flux log-uniform [1e2, 1e5], c = 0,
 * sky 0.05) and count Moffat PSFs (beta 3, FWHM ~ U[2, 5], sum 1) of
 * psf_size^2 floats.  Deterministic in (seed, stamp index). */
gf_status gf_train_sample(unsigned long long seed, int count, int psf_size, double* params_dev,
                          float* psf_dev, gf_stream stream);

/* Noise on n model pixels: sigma = sqrt(sigma_read^2 + max(m, 0) / gain),
 * image = m + sigma z, z standard normal by Box-Muller from Philox4x32-10
 * (counter = pixel index, key = seed). */
gf_status gf_noise(const float* model_dev, int64_t n, unsigned long long seed, float sigma_read,
                   float gain, float* image_dev, float* sigma_dev, gf_stream stream);

/* Philox4x32-10 (Salmon et al., SC 2011) of n blocks: in_dev holds per block
 * the counter (4 words) then the key (2 words); out_dev 4 words per block.
 * Exposed so the generator can be checked against its published vectors. */
gf_status gf_philox4x32_10(const uint32_t* in_dev, uint32_t* out_dev, int n, gf_stream stream);

/* Workspace bytes of gf_default_guess / gf_guess_select for count stamps. */
size_t gf_workspace_size_guess(int count);

/* Moments-based start of a single Sersic + sky fit for every stamp of a batch
 * (any sizes; stamp ring at most 8192 pixels), params_dev count x 9:
 *   sky = median of the outer ring of pixels;
 *   x0, y0 = first moments of the sky-subtracted positive pixels;
 *   q, pa = from their second moments;
 *   r_e = semi-major axis of the smallest elliptical aperture (0.25 px steps)
 *         holding half their summed flux;  n = 2;  c = 0;
 *   I_e = summed flux / closed-form flux of unit I_e. */
gf_status gf_default_guess(const gf_batch* b, const float* image_dev, double* params_dev,
                           void* ws, size_t ws_bytes, gf_stream stream);

/* Per stamp, out_dev = cand_dev where every slot is finite and inside the
 * bounds (lo_host / hi_host, 9 each, NULL = the defaults of gf_lm_fit) and
 * chi2_cand is finite and no larger than chi2_dflt; else dflt_dev.  choice_dev
 * (may be NULL) receives 1 where the candidate was taken. */
gf_status gf_guess_select(int count, const double* cand_dev, const double* chi2_cand_dev,
                          const double* dflt_dev, const double* chi2_dflt_dev,
                          const double* lo_host, const double* hi_host, double* out_dev,
                          int* choice_dev, void* ws, size_t ws_bytes, gf_stream stream);

/* ------------------------------------------------------ spectral lines, cubes
 * The fitting loop in one dimension (Sec. 5: with a flexible dimensionality
 * the same procedure fits spectral lines or data cubes; a cube is fitted
 * spectrum by spectrum, each spaxel's spectrum one entry of a batch).
 *
 * A spectrum has n_chan channels; channel i has its centre at x = i.  Its
 * model on the extended grid x = -c .. n_chan-1+c,
 *     E(x) = sum_{j < n_cont} a_j t^j + sum_k A_k exp(-(x - mu_k)^2 / (2 s_k^2)),
 *     t = (x - (n_chan-1)/2) / h,  h = (n_chan-1)/2 (1 when n_chan = 1),
 * is convolved with an odd line-spread function (LSF) of lsf_len = 2c+1 taps
 * by the flipped-kernel sum m_i = sum_u lsf[u] E(i + c - u), the stamp
 * convention in one dimension.  chi^2 as for stamps (finite data, sigma > 0).
 * Parameters (float64) of a spectrum, in order:
 *     a_0 .. a_{n_cont-1}, then A_k, mu_k, s_k for each line k
 * (mu and s in channels).  Default box: s_k >= 0.25, the rest free.
 * The amplitude and continuum columns of the Jacobian are exact (convolved
 * basis functions); the centre and width columns are forward differences
 * (GF_JAC_FD, step fd_rel channels for mu, fd_rel*max(|s|,1) for s) or
 * analytic derivatives (GF_JAC_ANALYTIC).  The LM rules are those of
 * gf_lm_fit taken one trial at a time (opts.ladder is not used).
 * All arrays are device memory unless named *_host; spectra, sigma maps and
 * models are packed count x n_chan float32, parameters count x nparams
 * float64.  Nothing is allocated: these calls need no workspace. */
#define GF_SPEC_MAX_LINES 5
#define GF_SPEC_MAX_CONT 3
#define GF_SPEC_MAX_LSF 129
#define GF_SPEC_MAX_CHAN (1 << 24)

typedef struct {
    int n_chan;            /* 1 .. GF_SPEC_MAX_CHAN */
    int n_lines;           /* 0 .. GF_SPEC_MAX_LINES */
    int n_cont;            /* 0 .. GF_SPEC_MAX_CONT */
    int lsf_len;           /* odd, 1 .. GF_SPEC_MAX_LSF */
    int lsf_per_spectrum;  /* 0: one LSF (lsf_len floats) for all; 1: count x lsf_len */
} gf_spec_desc;

/* n_cont + 3 n_lines, or -1 for an invalid description. */
int gf_spec_nparams(const gf_spec_desc* d);

/* Convolved models (count x n_chan) at params_dev. */
gf_status gf_spec_model(const gf_spec_desc* d, int count, const double* params_dev,
                        const float* lsf_dev, float* model_dev, gf_stream stream);

/* chi^2 of each spectrum (chi2_dev, count float64) and, if model_dev is not
 * NULL, its convolved model. */
gf_status gf_spec_eval(const gf_spec_desc* d, int count, const double* params_dev,
                       const float* spec_dev, const float* sig_dev, const float* lsf_dev,
                       double* chi2_dev, float* model_dev, gf_stream stream);

/* Normal equations at params_dev over the free slots (fixed_host: nparams
 * bytes shared by all spectra, nonzero = held; NULL = all free; at most
 * GF_MAX_FREE free): A_dev count x nf x nf, g_dev count x nf (J^T W r),
 * chi2_dev count.  jac_mode and fd_rel as in gf_lm_opts. */
gf_status gf_spec_normal(const gf_spec_desc* d, int count, const double* params_dev,
                         const uint8_t* fixed_host, const float* spec_dev,
                         const float* sig_dev, const float* lsf_dev, int jac_mode,
                         double fd_rel, double* A_dev, double* g_dev, double* chi2_dev,
                         gf_stream stream);

/* Batched LM: every spectrum fitted independently from its row of params_dev
 * (projected into the box first) into params_out_dev (may equal params_dev);
 * result_dev receives count gf_lm_result.  lo_host / hi_host: nparams bounds
 * or NULL for the defaults.  A spectrum's result does not depend on the
 * batch around it.  Returns once the launch is queued; the results are ready
 * when the stream is. */
gf_status gf_spec_fit(const gf_spec_desc* d, int count, const double* params_dev,
                      const uint8_t* fixed_host, const double* lo_host, const double* hi_host,
                      const float* spec_dev, const float* sig_dev, const float* lsf_dev,
                      const gf_lm_opts* opts, double* params_out_dev, gf_lm_result* result_dev,
                      gf_stream stream);

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

/* Measured FMA peak of the current device, the denominator of the ALU-bound
 * kernels' roofline fractions: an FMA loop (8 independent chains per thread,
 * 8 CTAs of 256 threads per SM) in float32 (fp64 = 0) or float64 (fp64 = 1),
 * timed by CUDA events on `stream` over `reps` launches after one warm-up
 * launch.  sink_dev: 8 bytes of device memory the kernel may write (it does
 * not in practice).  *tflops_out = FLOPs (2 per FMA) / seconds / 1e12.
 * Synchronises the stream.  Diagnostic only. */
gf_status gf_fma_peak(int fp64, int reps, void* sink_dev, double* tflops_out, gf_stream stream);

#ifdef __cplusplus
}
#endif
#endif
