/*
 * gfo_cnn.c -- FP64 CPU oracle of the initial-guess network and of the
 * moments-based default guess.  TEST INFRASTRUCTURE ONLY (see gfo.c).
 *
 * Network (one 64x64 input channel, NCHW, zero padding 1, stride 2, ReLU after
 * every layer except the last):
 *   conv1 3x3  1 -> 32   64x64 -> 32x32
 *   conv2 3x3 32 -> 64   32x32 -> 16x16
 *   conv3 3x3 64 -> 64   16x16 ->  8x8
 *   conv4 3x3 64 -> 128   8x8  ->  4x4
 *   fc1   2048 -> 32 (flattened c, y, x)
 *   fc2   32 -> 8
 * Parameters are packed layer by layer as weights [out][in][ky][kx] (or
 * [out][in] for the fully connected layers) followed by biases [out].
 * Loss: mean over the batch and the 8 outputs of (y - t)^2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "gfo.h"

typedef struct {
    int cin, cout, hin, hout; /* conv layers; fc: hin = hout = 1 */
    int conv;
} layer_t;

static const layer_t LAYERS[6] = {
    {1, 32, 64, 32, 1}, {32, 64, 32, 16, 1}, {64, 64, 16, 8, 1},
    {64, 128, 8, 4, 1}, {2048, 32, 1, 1, 0}, {32, 8, 1, 1, 0},
};

static long layer_wcount(const layer_t* L) { return (long)L->cout * L->cin * (L->conv ? 9 : 1); }

long gfo_cnn_nparams(void)
{
    long n = 0;
    for (int i = 0; i < 6; ++i) n += layer_wcount(&LAYERS[i]) + LAYERS[i].cout;
    return n;
}

static long layer_size(const layer_t* L, int out)
{
    return L->conv ? (long)(out ? L->cout : L->cin) * (out ? L->hout : L->hin) * (out ? L->hout : L->hin)
                   : (out ? L->cout : L->cin);
}

/* Round to the nearest bfloat16 (8 significant bits), ties to even: first to
 * the nearest float32, then the low 16 bits of its encoding are dropped with
 * round-to-nearest-even on them. */
double gfo_bf16_round(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof(u));
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf, nan */
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    memcpy(&f, &u, sizeof(f));
    return (double)f;
}

/* one sample's forward; acts[i] = output of layer i after ReLU (pre-ReLU kept
 * in pre[i]); acts[-1] is the input.  round_act = 1 stores the outputs of the
 * four convolution layers as bfloat16, the precision the network is specified
 * in; the derivative of that rounding is taken as 1. */
static void forward1(const double* w, const double* x, double** pre, double** act, int round_act)
{
    const double* in = x;
    long off = 0;
    for (int li = 0; li < 6; ++li) {
        const layer_t* L = &LAYERS[li];
        const double* W = w + off;
        const double* b = W + layer_wcount(L);
        off += layer_wcount(L) + L->cout;
        if (L->conv) {
            for (int co = 0; co < L->cout; ++co)
                for (int oy = 0; oy < L->hout; ++oy)
                    for (int ox = 0; ox < L->hout; ++ox) {
                        double s = b[co];
                        for (int ci = 0; ci < L->cin; ++ci)
                            for (int ky = 0; ky < 3; ++ky)
                                for (int kx = 0; kx < 3; ++kx) {
                                    int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
                                    if (iy < 0 || ix < 0 || iy >= L->hin || ix >= L->hin) continue;
                                    s += W[((co * L->cin + ci) * 3 + ky) * 3 + kx] *
                                         in[(ci * L->hin + iy) * L->hin + ix];
                                }
                        long o = (co * L->hout + oy) * L->hout + ox;
                        pre[li][o] = s;
                        act[li][o] = s > 0.0 ? s : 0.0;
                        if (round_act) act[li][o] = gfo_bf16_round(act[li][o]);
                    }
        } else {
            for (int co = 0; co < L->cout; ++co) {
                double s = b[co];
                for (int ci = 0; ci < L->cin; ++ci) s += W[co * L->cin + ci] * in[ci];
                pre[li][co] = s;
                act[li][co] = (li == 5) ? s : (s > 0.0 ? s : 0.0);
            }
        }
        in = act[li];
    }
}

/* Forward of nb samples x (nb x 4096), outputs y (nb x 8). */
void gfo_cnn_forward(const double* w, const double* x, int nb, double* y, int round_act)
{
    double* pre[6];
    double* act[6];
    for (int i = 0; i < 6; ++i) {
        pre[i] = (double*)malloc(sizeof(double) * layer_size(&LAYERS[i], 1));
        act[i] = (double*)malloc(sizeof(double) * layer_size(&LAYERS[i], 1));
    }
    for (int s = 0; s < nb; ++s) {
        forward1(w, x + (long)s * 4096, pre, act, round_act);
        memcpy(y + (long)s * 8, act[5], sizeof(double) * 8);
    }
    for (int i = 0; i < 6; ++i) {
        free(pre[i]);
        free(act[i]);
    }
}

/* Loss (mean squared error over nb x 8) and its gradient with respect to every
 * parameter, by reverse-mode differentiation of forward1 (chain rule through
 * each layer in reverse order). */
double gfo_cnn_loss_grad(const double* w, const double* x, const double* t, int nb, double* grad,
                         int round_act)
{
    const long np = gfo_cnn_nparams();
    memset(grad, 0, sizeof(double) * np);
    double* pre[6];
    double* act[6];
    double* gact[6];
    for (int i = 0; i < 6; ++i) {
        long n = layer_size(&LAYERS[i], 1);
        pre[i] = (double*)malloc(sizeof(double) * n);
        act[i] = (double*)malloc(sizeof(double) * n);
        gact[i] = (double*)malloc(sizeof(double) * n);
    }
    double* gin = (double*)malloc(sizeof(double) * 32 * 32 * 32);
    long offs[6];
    long off = 0;
    for (int i = 0; i < 6; ++i) {
        offs[i] = off;
        off += layer_wcount(&LAYERS[i]) + LAYERS[i].cout;
    }
    double loss = 0.0;
    const double scale = 1.0 / (8.0 * nb);
    for (int s = 0; s < nb; ++s) {
        const double* xs = x + (long)s * 4096;
        forward1(w, xs, pre, act, round_act);
        for (int j = 0; j < 8; ++j) {
            double e = act[5][j] - t[(long)s * 8 + j];
            loss += e * e * scale;
            gact[5][j] = 2.0 * e * scale; /* dL/d(pre of fc2) */
        }
        for (int li = 5; li >= 0; --li) {
            const layer_t* L = &LAYERS[li];
            const double* W = w + offs[li];
            double* gW = grad + offs[li];
            double* gb = gW + layer_wcount(L);
            const double* in = li == 0 ? xs : act[li - 1];
            long nout = layer_size(L, 1);
            /* gradient at the pre-activation */
            for (long o = 0; o < nout; ++o)
                if (li != 5 && pre[li][o] <= 0.0) gact[li][o] = 0.0;
            double* gprev = li == 0 ? NULL : gact[li - 1];
            long nin = layer_size(L, 0);
            if (gprev) memset(gprev, 0, sizeof(double) * nin);
            if (L->conv) {
                for (int co = 0; co < L->cout; ++co)
                    for (int oy = 0; oy < L->hout; ++oy)
                        for (int ox = 0; ox < L->hout; ++ox) {
                            double g = gact[li][(co * L->hout + oy) * L->hout + ox];
                            if (g == 0.0) continue;
                            gb[co] += g;
                            for (int ci = 0; ci < L->cin; ++ci)
                                for (int ky = 0; ky < 3; ++ky)
                                    for (int kx = 0; kx < 3; ++kx) {
                                        int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
                                        if (iy < 0 || ix < 0 || iy >= L->hin || ix >= L->hin) continue;
                                        long wi = ((co * L->cin + ci) * 3 + ky) * 3 + kx;
                                        long ii = (ci * L->hin + iy) * L->hin + ix;
                                        gW[wi] += g * in[ii];
                                        if (gprev) gprev[ii] += g * W[wi];
                                    }
                        }
            } else {
                for (int co = 0; co < L->cout; ++co) {
                    double g = gact[li][co];
                    gb[co] += g;
                    for (int ci = 0; ci < L->cin; ++ci) {
                        gW[co * L->cin + ci] += g * in[ci];
                        if (gprev) gprev[ci] += g * W[co * L->cin + ci];
                    }
                }
            }
        }
    }
    for (int i = 0; i < 6; ++i) {
        free(pre[i]);
        free(act[i]);
        free(gact[i]);
    }
    free(gin);
    return loss;
}

/* ----------------------------------------------------------- default guess */

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Moments-based start for a single Sersic + sky fit of an H x W stamp:
 *   sky   = median of the border pixels (outermost ring);
 *   x0,y0 = first moments of the sky-subtracted positive pixels;
 *   q, pa = from the second moments (eigen-decomposition of the 2x2 matrix);
 *   r_e   = semi-major axis of the elliptical aperture (axis ratio q, angle
 *           pa), grown in 0.25 px steps, that first holds half the summed flux;
 *   n     = 2;  I_e from the summed flux by the closed-form Sersic flux.
 * Output slots: x0, y0, I_e, r_e, n, q, pa_deg, c(=0), sky. */
void gfo_default_guess(const double* img, int H, int W, double* out)
{
    int nb = 2 * W + 2 * (H - 2);
    if (nb < 1) nb = 1;
    double* border = (double*)malloc(sizeof(double) * nb);
    int k = 0;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j)
            if (i == 0 || j == 0 || i == H - 1 || j == W - 1) border[k++] = img[(long)i * W + j];
    qsort(border, k, sizeof(double), cmp_double);
    double sky = (k % 2) ? border[k / 2] : 0.5 * (border[k / 2 - 1] + border[k / 2]);
    free(border);
    double s0 = 0.0, sx = 0.0, sy = 0.0;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double v = img[(long)i * W + j] - sky;
            if (v <= 0.0) continue;
            s0 += v;
            sx += v * j;
            sy += v * i;
        }
    double x0 = s0 > 0.0 ? sx / s0 : 0.5 * (W - 1), y0 = s0 > 0.0 ? sy / s0 : 0.5 * (H - 1);
    double mxx = 0.0, myy = 0.0, mxy = 0.0;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double v = img[(long)i * W + j] - sky;
            if (v <= 0.0) continue;
            double dx = j - x0, dy = i - y0;
            mxx += v * dx * dx;
            myy += v * dy * dy;
            mxy += v * dx * dy;
        }
    if (s0 > 0.0) {
        mxx /= s0;
        myy /= s0;
        mxy /= s0;
    }
    double tr = mxx + myy, det = mxx * myy - mxy * mxy;
    double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
    double l1 = 0.5 * tr + disc, l2 = 0.5 * tr - disc;
    double q = (l1 > 0.0 && l2 > 0.0) ? sqrt(l2 / l1) : 1.0;
    if (q < 0.05) q = 0.05;
    if (q > 1.0) q = 1.0;
    double pa = 0.5 * atan2(2.0 * mxy, mxx - myy) * 180.0 / M_PI;
    pa = fmod(pa, 180.0);
    if (pa < 0.0) pa += 180.0;
    /* curve of growth in elliptical apertures (semi-major a) */
    double th = pa * M_PI / 180.0, cs = cos(th), sn = sin(th);
    double half = 0.5 * s0, a_half = 1.0;
    double amax = (double)(H > W ? H : W);
    for (double a = 0.25; a <= amax; a += 0.25) {
        double enc = 0.0;
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double v = img[(long)i * W + j] - sky;
                if (v <= 0.0) continue;
                double dx = j - x0, dy = i - y0;
                double xp = dx * cs + dy * sn, yp = (-dx * sn + dy * cs) / q;
                if (xp * xp + yp * yp <= a * a) enc += v;
            }
        if (enc >= half) {
            a_half = a;
            break;
        }
    }
    double re = a_half;
    if (re < 0.5) re = 0.5;
    double n = 2.0, b = gfo_bn(n);
    double F = s0 > 0.0 ? s0 : 1.0;
    double ie = F / (2.0 * M_PI * q * re * re * n * exp(b + lgamma(2.0 * n) - 2.0 * n * log(b)));
    out[0] = x0;
    out[1] = y0;
    out[2] = ie;
    out[3] = re;
    out[4] = n;
    out[5] = q;
    out[6] = pa;
    out[7] = 0.0;
    out[8] = sky;
}

/* ------------------------------------------- network input and targets */

/* Input scaling of one H x W stamp: x = asinh(img / a), a = median of sigma
 * over the outermost ring of pixels (mean of the two middle values when the
 * ring has an even count). */
void gfo_cnn_input(const double* img, const double* sigma, int H, int W, double* x)
{
    int nb = (H == 1 || W == 1) ? H * W : 2 * W + 2 * (H - 2);
    double* ring = (double*)malloc(sizeof(double) * nb);
    int k = 0;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j)
            if (i == 0 || j == 0 || i == H - 1 || j == W - 1) ring[k++] = sigma[(long)i * W + j];
    qsort(ring, k, sizeof(double), cmp_double);
    double a = (k % 2) ? ring[k / 2] : 0.5 * (ring[k / 2 - 1] + ring[k / 2]);
    free(ring);
    if (!(a > 0.0)) a = 1.0;
    for (long p = 0; p < (long)H * W; ++p) x[p] = asinh(img[p] / a);
}

/* Targets of one Sersic component in an H x W stamp (slots x0, y0, I_e, r_e,
 * n, q, pa_deg), each scaled so the training prior spans about [-1, 1]:
 *   t0, t1 = offsets of the centre from the stamp centre ((W-1)/2, (H-1)/2)
 *   t2 = (ln F - 3.5 ln 10) / (1.5 ln 10),  F the closed-form total flux
 *   t3 = (ln r_e - ln 80 / 2) / (ln 20 / 2)
 *   t4 = (n - 3.25) / 2.75,   t5 = (q - 0.6) / 0.4
 *   t6, t7 = cos 2 pa, sin 2 pa  (the angle is defined modulo 180 degrees) */
void gfo_cnn_encode(const double* p, int H, int W, double* t)
{
    const double l10 = log(10.0);
    double F = gfo_sersic_flux(p[2], p[3], p[4], p[5]);
    double th = 2.0 * p[6] * M_PI / 180.0;
    t[0] = p[0] - 0.5 * (W - 1);
    t[1] = p[1] - 0.5 * (H - 1);
    t[2] = (log(F) - 3.5 * l10) / (1.5 * l10);
    t[3] = (log(p[3]) - 0.5 * log(80.0)) / (0.5 * log(20.0));
    t[4] = (p[4] - 3.25) / 2.75;
    t[5] = (p[5] - 0.6) / 0.4;
    t[6] = cos(th);
    t[7] = sin(th);
}

/* Inverse of gfo_cnn_encode: Sersic slots x0, y0, I_e, r_e, n, q, pa_deg, c
 * (c = 0).  I_e is NaN where n leaves [0.2, 10] or q leaves (0, 1], the domain
 * of the closed-form flux. */
void gfo_cnn_decode(const double* t, int H, int W, double* p)
{
    const double l10 = log(10.0);
    double F = exp(3.5 * l10 + 1.5 * l10 * t[2]);
    double re = exp(0.5 * log(80.0) + 0.5 * log(20.0) * t[3]);
    double n = 3.25 + 2.75 * t[4];
    double q = 0.6 + 0.4 * t[5];
    double pa = 0.5 * atan2(t[7], t[6]) * 180.0 / M_PI;
    if (pa < 0.0) pa += 180.0;
    p[0] = 0.5 * (W - 1) + t[0];
    p[1] = 0.5 * (H - 1) + t[1];
    p[2] = (n >= 0.2 && n <= 10.0 && q > 0.0 && q <= 1.0) ? F / gfo_sersic_flux(1.0, re, n, q) : NAN;
    p[3] = re;
    p[4] = n;
    p[5] = q;
    p[6] = pa;
    p[7] = 0.0;
}
