/*
 * gfo.h -- FP64 CPU oracle for the galaxy-fitting loop of Barsdell, Barnes &
 * Fluke, "Fitting Galaxies on GPUs" (Sec. 2, steps 1-5; Sec. 3, items 1-3).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct statement of what the GPU path computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no source, header, table or helper with the CUDA library, and neither side
 * includes or links the other.
 *
 * Everything is double precision, plain loops, no blocking or fusion.
 * OpenMP is used only across independent stamps (gfo_lm_fit_batch).
 *
 * Conventions (the paper names the steps only; these are the readings taken):
 *   - pixel (row i, column j) of an H x W stamp has its centre at (x=j, y=i);
 *   - the model is evaluated on the halo-extended grid E of
 *     (H+2c) x (W+2c) pixels, c = (P-1)/2 for an odd P x P PSF; grid pixel
 *     (ie, je) is stamp pixel (ie-c, je-c);
 *   - the convolved image on the stamp is the true (flipped-kernel) sum
 *     out(i,j) = sum_{v,u} psf[v][u] * E[i+2c-v][j+2c-u].
 *
 * Parameter slots per component, in order:
 *   Sersic  (kind 1): x0, y0, I_e, r_e, n, q, pa_deg, c     (8 slots)
 *   ExpDisk (kind 2): x0, y0, I_0, r_s, q, pa_deg, c         (7 slots)
 *   Sky     (kind 3): s0                                     (1 slot)
 *   Gaussian(kind 4): x0, y0, I_0, FWHM, q, pa_deg, c        (7 slots)
 *   Moffat  (kind 5): x0, y0, I_0, FWHM, beta, q, pa_deg, c  (8 slots)
 *   King    (kind 6): x0, y0, I_0, r_c, r_t, alpha, q, pa_deg, c        (9 slots)
 *   Nuker   (kind 7): x0, y0, I_b, r_b, alpha, beta, gamma, q, pa_deg, c (10 slots)
 *   Point   (kind 8): x0, y0, F                                (3 slots)
 *   Sky plane (kind 9): s0, gx, gy                             (3 slots)
 *   Sersic + Fourier modes (kind 10): the Sersic's 8 slots, then a1, phi1,
 *             a3, phi3, a4, phi4 (14 slots; phases in degrees)
 * The King, Nuker and point-source kinds have finite-difference Jacobian
 * columns only (no analytic gradient).
 */
#ifndef GFO_H
#define GFO_H
#include <stdint.h>

#define GFO_SERSIC 1
#define GFO_EXPDISK 2
#define GFO_SKY 3
#define GFO_GAUSSIAN 4  /* I_0 exp(-r^2 / (2 sigma^2)), sigma = FWHM / (2 sqrt(2 ln 2)) */
#define GFO_MOFFAT 5    /* I_0 (1 + (r/alpha)^2)^(-beta), alpha = FWHM / (2 sqrt(2^(1/beta) - 1)) */
#define GFO_KING 6      /* I_0 [(w - w_t) / (1 - w_t)]^alpha inside r_t, w = (1 + (r/r_c)^2)^(-1/alpha) */
#define GFO_NUKER 7     /* I_b 2^((beta-gamma)/alpha) (r/r_b)^-gamma [1 + (r/r_b)^alpha]^((gamma-beta)/alpha) */
#define GFO_PSF 8       /* point source: F, placed by cubic-convolution weights (see gfo.c) */
#define GFO_SKYPLANE 9  /* sky s0 + gx (x - x_c) + gy (y - y_c) about the stamp centre */
#define GFO_SERSIC_F 10 /* Sersic with Fourier modes m = 1, 3, 4 of its isophotes */
#define GFO_COMP_MAXSLOTS 14
#define GFO_MAX_COMP 8
#define GFO_MAX_SLOTS 64
#define GFO_MAX_FREE 16

/* LM status words */
#define GFO_CONVERGED 0
#define GFO_MAXITER 8
#define GFO_NOCONV 3
#define GFO_BADINPUT 1

typedef struct {
    int H, W;        /* stamp rows, columns */
    int P;           /* PSF side, odd */
    int ncomp;
    int kinds[GFO_MAX_COMP];
    int os_factor;   /* s: s x s sub-samples per pixel inside the block (1 = off) */
    int os_box;      /* B: block side in pixels */
    int os_x0, os_y0;/* block origin in stamp pixels; -1 = centred on the stamp */
} gfo_desc;

/* Jacobian columns of the nonlinear slots */
#define GFO_JAC_FORWARD 0   /* forward differences (the LM default) */
#define GFO_JAC_CENTRAL 1   /* central differences */
#define GFO_JAC_ANALYTIC 2  /* convolved analytic derivatives of the model */

typedef struct {
    double lambda0, lambda_up, lambda_down, lambda_min, lambda_max;
    double ftol, xtol, fd_rel;
    int max_iter;
    int jac_mode;    /* GFO_JAC_FORWARD or GFO_JAC_ANALYTIC */
} gfo_lm_opts;

typedef struct {
    double chi2;
    double lambda;
    int iters;       /* trial steps taken (accepted + rejected) */
    int accepted;
    int status;
} gfo_lm_result;

/* A least-squares problem as the LM core sees it: nslots parameters of which
 * the nfree listed in free_slots move; normal() returns chi^2 at p and fills
 * A = J^T W J (nfree x nfree) and g = J^T W r; eval() returns chi^2 at p;
 * project() moves p into the box; xscale(s) is the floor of |p_s| in the
 * scaled step test. */
typedef struct {
    int nslots, nfree;
    const int* free_slots;
    double (*normal)(void* ctx, const double* p, double* A, double* g);
    double (*eval)(void* ctx, const double* p);
    void (*project)(void* ctx, double* p);
    double (*xscale)(void* ctx, int slot);
    void* ctx;
} gfo_lm_problem;

/* Levenberg-Marquardt over any such problem (the rules of gfo_lm_fit). */
int gfo_lm_core(const gfo_lm_problem* P, double* params, const gfo_lm_opts* o,
                gfo_lm_result* res);

int gfo_comp_nslots(int kind);
int gfo_nslots(const gfo_desc* d);

/* b_n: the root of P(2n, b) = 1/2 (regularised lower incomplete gamma). */
double gfo_bn(double n);
/* regularised lower incomplete gamma P(a, x), series form */
double gfo_gammainc_lower(double a, double x);
/* closed-form total flux of an elliptical (c = 0) Sersic component */
double gfo_sersic_flux(double Ie, double re, double n, double q);
/* alpha / FWHM of a Moffat profile of index beta */
double gfo_moffat_alpha_per_fwhm(double beta);

/* surface brightness of one component at a point (amplitude taken from p) */
double gfo_comp_value(int kind, const double* p, double x, double y, double bn);

/* value of one component averaged over stamp pixel (i, j) with the desc's
 * oversampling rule; i, j may lie in the halo. */
double gfo_comp_pixel(const gfo_desc* d, int kind, const double* p, int i, int j);

/* db_n/dn (central differences of gfo_bn) */
double gfo_bn_deriv(double n);
/* value of a component at (x, y) and its derivative with respect to each of
 * its slots (grad: one entry per slot) */
double gfo_comp_grad(int kind, const double* p, double x, double y, double bn, double dbdn,
                     double* grad);
/* derivative of the extended-grid model with respect to slot `slot` */
int gfo_model_ext_grad(const gfo_desc* d, const double* params, int slot, double* out);

/* Step 1: the model on the extended grid; out has (H+2c)*(W+2c) entries.
 * comp = -1: all components summed; comp = k >= 0: component k only.
 * unit_amp = 1: component k with its amplitude slot set to 1. */
int gfo_model_ext(const gfo_desc* d, const double* params, int comp, int unit_amp,
                  double* out);
/* The extended-grid basis function of linear slot `slot` (its exact column
 * before the convolution). */
int gfo_model_ext_basis(const gfo_desc* d, const double* params, int slot, double* out);

/* Step 2, by the definition: out (H*W) from ext ((H+2c)*(W+2c)) */
void gfo_convolve_direct(int H, int W, int P, const double* ext, const double* psf,
                         double* out);
/* Step 2, via the oracle's own FP64 mixed-radix FFT (circular at the padded
 * size, exact on the valid region) */
void gfo_convolve_fft(int H, int W, int P, const double* ext, const double* psf,
                      double* out);
/* one complex DFT of length n by the oracle's FFT (sign -1 forward, +1 inverse,
 * unnormalised); re/im in place */
void gfo_fft(int n, double* re, double* im, int sign);
int gfo_fft_size(int n); /* smallest 2^a 3^b 5^c >= n */

/* Step 3: chi^2 over pixels with finite d, sigma > 0 (Neumaier sum) */
double gfo_chi2(int npix, const double* d, const double* sigma, const double* m);

/* Steps 1-3 for one parameter vector: convolved model on the stamp and chi^2.
 * method 0 = direct, 1 = FFT. */
double gfo_eval(const gfo_desc* d, const double* params, const double* psf,
                const double* img, const double* sigma, int method, double* model_out);

/* Step 4 input: Jacobian columns for the free slots (fixed[s] == 0).
 * J: nfree x H*W (may be NULL), A: nfree^2, g: nfree, returns chi^2 at params.
 * mode: GFO_JAC_FORWARD / GFO_JAC_CENTRAL differences, or GFO_JAC_ANALYTIC
 * (the convolution of the analytic derivative grid) for the nonlinear slots. */
double gfo_jacobian(const gfo_desc* d, const double* params, const uint8_t* fixed,
                    const double* psf, const double* img, const double* sigma,
                    int method, double fd_rel, int mode, double* J, double* A,
                    double* g, double* model_out);

/* default bounds for every slot */
void gfo_default_bounds(const gfo_desc* d, double* lo, double* hi);
void gfo_default_opts(gfo_lm_opts* o);
/* the FD step for slot s at value v (absolute) */
double gfo_fd_step(const gfo_desc* d, int slot, double v, double fd_rel);
int gfo_slot_is_linear(const gfo_desc* d, int slot);

/* Steps 4-5: Levenberg-Marquardt from params (in/out) */
int gfo_lm_fit(const gfo_desc* d, double* params, const uint8_t* fixed,
               const double* lo, const double* hi, const double* psf,
               const double* img, const double* sigma, int method,
               const gfo_lm_opts* opts, gfo_lm_result* res);

/* independent stamps, OpenMP across stamps.  Stamp b uses desc ds[b],
 * params + b*nslots, fixed + b*nslots (NULL = all free), psf + psf_off[b],
 * img/sigma + pix_off[b]. */
int gfo_lm_fit_batch(int nb, const gfo_desc* ds, double* params, const uint8_t* fixed,
                     const double* psf, const int64_t* psf_off, const double* img,
                     const double* sigma, const int64_t* pix_off, int method,
                     const gfo_lm_opts* opts, gfo_lm_result* res);

int gfo_num_threads(void);
void gfo_set_num_threads(int n);
/* Single-precision storage emulation (experiment; 0 = off, the default):
 * component pixel values and convolved model pixels rounded to float32. */
void gfo_set_f32_emulation(int on);

/* cubic-convolution interpolation weight (Keys 1981, a = -1/2) of offset x */
double gfo_keys_weight(double x);

/* ---- initial-guess network and default guess (gfo_cnn.c) ---- */
long gfo_cnn_nparams(void);
/* outputs y (nb x 8) of the network with parameters w for inputs x (nb x 64 x 64);
 * round_act = 1 stores the convolution outputs as bfloat16 */
void gfo_cnn_forward(const double* w, const double* x, int nb, double* y, int round_act);
/* mean squared error against targets t (nb x 8) and its gradient (nparams) */
double gfo_cnn_loss_grad(const double* w, const double* x, const double* t, int nb, double* grad,
                         int round_act);
/* nearest bfloat16, ties to even */
double gfo_bf16_round(double v);
/* moments-based start of a Sersic + sky fit: x0, y0, I_e, r_e, n, q, pa, c, sky */
void gfo_default_guess(const double* img, int H, int W, double* out);
/* network input asinh(img / a), a = median sigma over the outer ring */
void gfo_cnn_input(const double* img, const double* sigma, int H, int W, double* x);
/* regression targets (8) of Sersic slots p (7 used), and the inverse */
void gfo_cnn_encode(const double* p, int H, int W, double* t);
void gfo_cnn_decode(const double* t, int H, int W, double* p);

/* ------------------------------------------------ spectral lines (gfo_spec.c)
 * One-dimensional form of the loop: spectra of n_chan channels, a continuum
 * polynomial of n_cont terms and n_lines Gaussian lines (A, mu, s each),
 * convolved with an odd line-spread function of lsf_len taps.  Parameters
 * [a_0 .. a_{n_cont-1}, A_0, mu_0, s_0, A_1, ...]. */
typedef struct {
    int n_chan, n_lines, n_cont, lsf_len;
} gfo_spec_desc;

int gfo_spec_nparams(const gfo_spec_desc* d);
int gfo_spec_slot_is_linear(const gfo_spec_desc* d, int s);
double gfo_spec_value(const gfo_spec_desc* d, const double* p, double x);
double gfo_spec_grad(const gfo_spec_desc* d, const double* p, int s, double x);
void gfo_spec_model_ext(const gfo_spec_desc* d, const double* p, int slot, double* E);
void gfo_spec_convolve(const gfo_spec_desc* d, const double* E, const double* lsf, double* m);
double gfo_spec_eval(const gfo_spec_desc* d, const double* p, const double* lsf,
                     const double* spec, const double* sig, double* m_out);
double gfo_spec_fd_step(const gfo_spec_desc* d, int s, double v, double fd_rel);
double gfo_spec_jacobian(const gfo_spec_desc* d, const double* p, const uint8_t* fixed,
                         const double* lsf, const double* spec, const double* sig, int mode,
                         double fd_rel, double* J, double* A, double* g);
void gfo_spec_default_bounds(const gfo_spec_desc* d, double* lo, double* hi);
int gfo_spec_fit(const gfo_spec_desc* d, double* params, const uint8_t* fixed,
                 const double* lo, const double* hi, const double* lsf, const double* spec,
                 const double* sig, const gfo_lm_opts* opts, gfo_lm_result* res);
int gfo_spec_fit_batch(int count, const gfo_spec_desc* d, double* params, const uint8_t* fixed,
                       const double* lsf, int lsf_per_spectrum, const double* spec,
                       const double* sig, const gfo_lm_opts* opts, gfo_lm_result* res);

#endif
