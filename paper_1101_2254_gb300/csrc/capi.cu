// capi.cu -- the extern "C" boundary of libgf.so (declared in include/gf.h).
//
// Host code only: argument validation, the workspace layout, the per-stamp
// block tables, and the order of kernel launches.  Every step of the fitting
// loop runs in the kernels of model.cu, conv_*.cu, reduce.cu and lm.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cnn.cuh"
#include "conv_dft.cuh"
#include "conv_fft.cuh"
#include "gf_internal.cuh"
#include "spec.cuh"

std::atomic<long long> g_launch_count{0};

static thread_local std::string g_err;

static gf_status fail(gf_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

#define GF_CUDA(expr)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(GF_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

cudaError_t ensure_smem_optin(const void* func, int bytes, int* cache)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && cache[dev] >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) cache[dev] = bytes;
    return e;
}

// ------------------------------------------------------------ profiling
// Off unless gf_prof_enable() received a device counter array.  When on, each
// kernel class launch is bracketed by CUDA events on its stream, and the
// kernels add their algorithmic work to the caller's counters.
namespace prof {
struct Rec {
    int cls;
    long long launches;
    cudaEvent_t e0, e1;
};
std::mutex mu;
unsigned long long* work_dev = nullptr;
std::vector<Rec> pending;
std::vector<cudaEvent_t> pool;
double ms[PROF_CLASSES];
long long launches[PROF_CLASSES];

cudaEvent_t get_event()
{
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
        e = pool.back();
        pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}
}  // namespace prof

struct ProfScope {
    int cls;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr;
    long long n0 = 0;
    ProfScope(int c, cudaStream_t st) : cls(c), s(st)
    {
        if (!prof::work_dev) return;
        std::lock_guard<std::mutex> g(prof::mu);
        e0 = prof::get_event();
        if (e0) cudaEventRecord(e0, s);
        n0 = g_launch_count.load();
    }
    ~ProfScope()
    {
        if (!e0) return;
        std::lock_guard<std::mutex> g(prof::mu);
        cudaEvent_t e1 = prof::get_event();
        if (!e1) return;
        cudaEventRecord(e1, s);
        prof::pending.push_back({cls, g_launch_count.load() - n0, e0, e1});
    }
};

namespace {

int comp_slots(int kind)
{
    switch (kind) {
    case GF_SERSIC: return 8;
    case GF_EXPDISK: return 7;
    case GF_SKY: return 1;
    case GF_GAUSSIAN: return 7;
    case GF_MOFFAT: return 8;
    case GF_KING: return 9;
    case GF_NUKER: return 10;
    case GF_PSF: return 3;
    case GF_SKY_PLANE: return 3;
    case GF_SERSIC_F: return 14;
    default: return -1;
    }
}

int resolve_method(const gf_desc* d)
{
    if (d->conv_method == GF_CONV_AUTO)
        return d->psf_size < GF_AUTO_FFT_PSF ? GF_CONV_DIRECT : GF_CONV_FFT;
    return d->conv_method;
}

// Structure checks shared by every call; H and W are checked per stamp.
gf_status check_structure(const gf_desc* d)
{
    if (!d) return fail(GF_EINVAL, "desc is NULL");
    const int P = d->psf_size;
    if (P < 1 || P > GF_MAX_PSF || P % 2 == 0)
        return fail(GF_EINVAL, "psf_size must be odd and in [1, " + std::to_string(GF_MAX_PSF) + "]");
    if (d->ncomp < 1 || d->ncomp > GF_MAX_COMP) return fail(GF_EINVAL, "ncomp out of range");
    int nsky = 0, nprof = 0;
    for (int k = 0; k < d->ncomp; ++k) {
        if (comp_slots(d->kinds[k]) < 0) return fail(GF_EINVAL, "unknown component kind");
        if (is_sky_kind(d->kinds[k]))
            ++nsky;
        else
            ++nprof;
    }
    if (nsky > 1) return fail(GF_EINVAL, "at most one sky component");
    if (nprof < 1) return fail(GF_EINVAL, "at least one profile component (Sersic, disk, Gaussian)");
    if (d->os_factor < 1 || d->os_factor > 64) return fail(GF_EINVAL, "os_factor out of [1, 64]");
    if (d->os_box < 0) return fail(GF_EINVAL, "os_box < 0");
    const int m = resolve_method(d);
    if (m != GF_CONV_DIRECT && m != GF_CONV_FFT && m != GF_CONV_DFT_TC)
        return fail(GF_EINVAL, "unknown conv_method");
    if (m == GF_CONV_DIRECT && P > GF_DIRECT_MAX_PSF)
        return fail(GF_EINVAL, "direct convolution supports psf_size <= " +
                                   std::to_string(GF_DIRECT_MAX_PSF));
    return GF_OK;
}

// smallest 2^a 3^b 5^c >= n (even: a >= 1)
int fft_len(int n, bool even)
{
    for (int m = n > 1 ? n : 1;; ++m) {
        if (even && (m & 1)) continue;
        int r = m;
        while (r % 2 == 0) r /= 2;
        while (r % 3 == 0) r /= 3;
        while (r % 5 == 0) r /= 5;
        if (r == 1) return m;
    }
}

FFTPlan make_fft_plan(int n)
{
    FFTPlan p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    int m = n;
    while (m % 8 == 0 && p.nst < FFT_MAX_STAGES) p.radix[p.nst++] = 8, m /= 8;
    while (m % 4 == 0 && p.nst < FFT_MAX_STAGES) p.radix[p.nst++] = 4, m /= 4;
    while (m % 2 == 0 && p.nst < FFT_MAX_STAGES) p.radix[p.nst++] = 2, m /= 2;
    while (m % 3 == 0 && p.nst < FFT_MAX_STAGES) p.radix[p.nst++] = 3, m /= 3;
    while (m % 5 == 0 && p.nst < FFT_MAX_STAGES) p.radix[p.nst++] = 5, m /= 5;
    int ns = 1;
    for (int t = 0; t < p.nst; ++t) {
        p.ns[t] = ns;
        p.mag[t] = ns > 1 ? (unsigned)((((unsigned long long)1 << 32) + ns - 1) / ns) : 0u;
        p.twstep[t] = n / (ns * p.radix[t]);
        ns *= p.radix[t];
    }
    return p;
}

// Transform length for the DFT-contraction path: the smallest N >= n that
// factors as R1 R2 with R1, R2 <= DFT_RMAX, and the factorisation with the
// least padding work.  `inner_tile` marks the x axis, whose first stage runs
// over R2 contiguous columns in tiles of 64 (a short R2 wastes tile width).
struct DftFactor {
    int N, R1, R2;
};

DftFactor dft_factor(int n, bool inner_tile)
{
    for (int N = n > 1 ? n : 1; N <= DFT_RMAX * DFT_RMAX; ++N) {
        double best = 1e30;
        DftFactor f = {0, 0, 0};
        for (int R2 = 1; R2 <= DFT_RMAX; ++R2) {
            if (N % R2) continue;
            const int R1 = N / R2;
            if (R1 > DFT_RMAX) continue;
            const double p1 = (double)((R1 + 15) / 16 * 16) / R1, p2 = (double)((R2 + 15) / 16 * 16) / R2;
            const double tile = inner_tile ? (double)((R2 + 63) / 64 * 64) / R2 : 1.0;
            const double cost = p1 * tile + p2;
            if (cost < best) {
                best = cost;
                f = {N, R1, R2};
            }
        }
        if (f.N) return f;
    }
    return {0, 0, 0};
}

// columns per CTA of the column pass: the largest power of two <= 16 whose two
// buffers and twiddles stay within ~100 KB of shared memory
int choose_cpc(int Ny)
{
    int cpc = 16;
    while (cpc > 1 && fft_col_smem(Ny, cpc) > 100 * 1024) cpc /= 2;
    return cpc;
}

// the FFT method needs one geometry for the whole call and sizes within limits
gf_status check_fft(const gf_desc* d, int count, const int* H, const int* W)
{
    const int m = resolve_method(d);
    if (m == GF_CONV_DFT_TC) {
        for (int b = 1; b < count; ++b)
            if (H[b] != H[0] || W[b] != W[0])
                return fail(GF_EINVAL, "DFT convolution needs stamps of one size per call");
        return GF_OK;
    }
    if (m != GF_CONV_FFT) return GF_OK;
    const int c = (d->psf_size - 1) / 2;
    for (int b = 1; b < count; ++b)
        if (H[b] != H[0] || W[b] != W[0])
            return fail(GF_EINVAL, "FFT convolution needs stamps of one size per call");
    if (fft_len(H[0] + 2 * c, false) > GF_FFT_MAX || fft_len(W[0] + 2 * c, true) > GF_FFT_MAX)
        return fail(GF_EINVAL, "FFT size exceeds " + std::to_string(GF_FFT_MAX));
    return GF_OK;
}

int fft_len(int n, bool even);

gf_status check_stamp(const gf_desc* d, int H, int W)
{
    if (H < 1 || W < 1) return fail(GF_EINVAL, "stamp H and W must be >= 1");
    if (resolve_method(d) == GF_CONV_FFT) {
        const int c = (d->psf_size - 1) / 2;
        if (fft_len(H + 2 * c, false) > GF_FFT_MAX || fft_len(W + 2 * c, true) > GF_FFT_MAX)
            return fail(GF_EINVAL, "FFT size exceeds " + std::to_string(GF_FFT_MAX));
    }
    if (resolve_method(d) == GF_CONV_DFT_TC) {
        const int c = (d->psf_size - 1) / 2;
        if (H + 2 * c > DFT_RMAX * DFT_RMAX || W + 2 * c > DFT_RMAX * DFT_RMAX)
            return fail(GF_EINVAL, "DFT size exceeds " + std::to_string(DFT_RMAX * DFT_RMAX));
    }
    if ((long long)H * W > (1LL << 31) - 1) return fail(GF_EINVAL, "stamp too large");
    if (d->os_factor > 1 && d->os_box > 0) {
        if (d->os_box > H || d->os_box > W) return fail(GF_EINVAL, "os_box exceeds the stamp");
        const int x0 = d->os_x0 >= 0 ? d->os_x0 : (W - d->os_box) / 2;
        const int y0 = d->os_y0 >= 0 ? d->os_y0 : (H - d->os_box) / 2;
        if (x0 + d->os_box > W || y0 + d->os_box > H)
            return fail(GF_EINVAL, "oversampling block leaves the stamp");
    }
    return GF_OK;
}

int nslots_of(const gf_desc* d)
{
    int n = 0;
    for (int k = 0; k < d->ncomp; ++k) n += comp_slots(d->kinds[k]);
    return n;
}

void default_opts(gf_lm_opts* o)
{
    o->lambda0 = 1e-3;
    o->lambda_up = 10.0;
    o->lambda_down = 0.1;
    o->lambda_min = 1e-12;
    o->lambda_max = 1e12;
    o->ftol = 1e-8;
    o->xtol = 1e-8;
    o->fd_rel = 1e-3;
    o->max_iter = 200;
    o->jac_mode = GF_JAC_FD;
    o->ladder = 0;  // automatic: see auto_ladder
    o->time_budget_s = 0.0;
}

// The trial ladder of a fit left to the library (gf_lm_opts.ladder 0): one rung
// when the call has at least as many stamps as the device has SMs (its passes
// fill the GPU, and a second rung's model and convolution are mostly extra
// work: it is used only after a rejection), else two (a few stamps are latency
// bound, and a rejection followed by an acceptance then takes one LM body
// instead of two).  The fits are the same for any ladder.
int auto_ladder(int count)
{
    static int sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 2;
    if (sms[dev] <= 0 &&
        cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 2;
    return count >= sms[dev] ? 1 : 2;
}

gf_status make_structure(const gf_desc* d, const uint8_t* fixed, const double* lo,
                         const double* hi, const gf_lm_opts* opts, Structure* S)
{
    memset(S, 0, sizeof(*S));
    S->ncomp = d->ncomp;
    S->sky_slot = -1;
    S->sky_jcol = -1;
    S->tilt_slot[0] = S->tilt_slot[1] = -1;
    S->tilt_jcol[0] = S->tilt_jcol[1] = -1;
    S->nplane = 0;
    int s = 0;
    for (int k = 0; k < d->ncomp; ++k) {
        const int kind = d->kinds[k];
        S->kinds[k] = kind;
        S->slot0[k] = s;
        if (!is_sky_kind(kind)) S->nprofile++;
        if (kind == GF_SKY_PLANE) S->nplane = 2;
        const int ns = comp_slots(kind);
        for (int l = 0; l < ns; ++l, ++s) {
            int role;
            if (kind == GF_SKY || (kind == GF_SKY_PLANE && l == 0)) {
                role = R_SKY;
                S->sky_slot = s;
            } else if (kind == GF_SKY_PLANE) {
                role = l == 1 ? R_TILTX : R_TILTY;
                S->tilt_slot[l - 1] = s;
            } else if (l <= 1) {
                role = R_POS;
            } else if (l == 2) {
                role = R_AMP;
            } else if (l == 3) {
                role = R_RAD;
            } else if (kind == GF_SERSIC) {
                static const int r[8] = {0, 0, 1, 2, R_N, R_Q, R_PA, R_BOXY};
                role = r[l];
            } else if (kind == GF_SERSIC_F) {
                static const int r[14] = {0,      0,      1,      2,      R_N,    R_Q,    R_PA,
                                          R_BOXY, R_FAMP, R_FPHI, R_FAMP, R_FPHI, R_FAMP, R_FPHI};
                role = r[l];
            } else if (kind == GF_MOFFAT) {
                static const int r[8] = {0, 0, 1, 2, R_BETA, R_Q, R_PA, R_BOXY};
                role = r[l];
            } else if (kind == GF_KING) {
                static const int r[9] = {0, 0, 1, 2, R_RT, R_KALPHA, R_Q, R_PA, R_BOXY};
                role = r[l];
            } else if (kind == GF_NUKER) {
                static const int r[10] = {0, 0, 1, 2, R_NALPHA, R_NBETA, R_NGAMMA, R_Q, R_PA, R_BOXY};
                role = r[l];
            } else {
                static const int r[7] = {0, 0, 1, 2, R_Q, R_PA, R_BOXY};
                role = r[l];
            }
            S->role[s] = role;
            S->owner[s] = k;
            double l0 = -INFINITY, h0 = INFINITY;
            switch (role) {
            case R_AMP: l0 = 0.0; break;
            case R_RAD: l0 = 0.1; break;
            case R_N: l0 = 0.2; h0 = 10.0; break;
            case R_Q: l0 = 0.05; h0 = 1.0; break;
            case R_BOXY: l0 = -1.9; h0 = 2.0; break;
            case R_BETA: l0 = 0.5; h0 = 20.0; break;
            case R_RT: l0 = 0.1; break;
            case R_KALPHA: l0 = 0.1; h0 = 10.0; break;
            case R_NALPHA: l0 = 0.1; h0 = 10.0; break;
            case R_NBETA: l0 = 0.0; h0 = 10.0; break;
            case R_NGAMMA: l0 = 0.0; h0 = 2.0; break;
            case R_FAMP: l0 = -0.3; h0 = 0.3; break;
            default: break;
            }
            S->lo[s] = lo ? lo[s] : l0;
            S->hi[s] = hi ? hi[s] : h0;
        }
    }
    S->nslots = s;
    if (s > GF_MAX_SLOTS) return fail(GF_EINVAL, "too many parameter slots");
    int nf = 0, nfd = 0;
    for (int t = 0; t < s; ++t) {
        if (fixed && fixed[t]) continue;
        if (nf >= GF_MAX_FREE)
            return fail(GF_EINVAL, "more than " + std::to_string(GF_MAX_FREE) + " free slots");
        if (S->role[t] == R_SKY) S->sky_jcol = nf;
        if (S->role[t] == R_TILTX) S->tilt_jcol[0] = nf;
        if (S->role[t] == R_TILTY) S->tilt_jcol[1] = nf;
        if (S->role[t] != R_AMP && S->role[t] != R_SKY && S->role[t] != R_TILTX &&
            S->role[t] != R_TILTY)
            ++nfd;
        S->freeslot[nf++] = t;
    }
    S->nfree = nf;
    S->nchan = S->nprofile + S->nplane + nfd;
    if (S->nchan > GF_MAX_CHAN) return fail(GF_EINVAL, "too many channels");
    S->nacc = nf * (nf + 1) / 2 + nf + 1;
    if (opts)
        S->opts = *opts;
    else
        default_opts(&S->opts);
    if (!(S->opts.fd_rel > 0.0)) S->opts.fd_rel = 1e-3;
    if (S->opts.jac_mode != GF_JAC_FD && S->opts.jac_mode != GF_JAC_ANALYTIC)
        return fail(GF_EINVAL, "jac_mode must be GF_JAC_FD or GF_JAC_ANALYTIC");
    if (S->opts.jac_mode == GF_JAC_ANALYTIC)
        for (int k = 0; k < S->ncomp; ++k)
            if (S->kinds[k] == GF_KING || S->kinds[k] == GF_NUKER || S->kinds[k] == GF_PSF ||
                S->kinds[k] == GF_SERSIC_F)
                return fail(GF_EINVAL, "analytic Jacobian columns are not available for King, Nuker, "
                                       "point-source or Fourier-mode components (use GF_JAC_FD)");
    if (S->opts.ladder < 0 || S->opts.ladder > GF_MAX_LADDER)
        return fail(GF_EINVAL, "LM ladder must be 0 (automatic) or 1 .. " + std::to_string(GF_MAX_LADDER));
    return GF_OK;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

enum { NEED_JAC = 1, NEED_TRIAL = 2, NEED_LM = 4, NEED_CHI2 = 8 };

// ------------------------------------------------------ tile-width choice
// Direct-convolution tile width per stamp: 64 (4 warps) or 32 (2 warps).  The
// two cover a stamp's columns in the same number of 64-wide steps unless
// ceil(W / 32) is odd, when the 32-wide tile saves a 32-column strip per tile
// row but stages more halo per output.  Which wins for a given PSF side and
// width class is measured by gf_autotune and kept per device; until then the
// smaller padded width wins.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tune[64];  // (P, ceil(W / 32)) -> tile width
// per PSF side: direct-convolution tile height and persistent CTAs per SM
struct ConvShape {
    int ty, ctas_per_sm;
};
std::map<int, ConvShape> g_tune_shape[64];
constexpr ConvShape kConvShapeDefault = {CONV_TY, 8};

ConvShape conv_shape(int P)
{
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        const auto it = g_tune_shape[dev].find(P);
        if (it != g_tune_shape[dev].end()) return it->second;
    }
    return kConvShapeDefault;
}

int conv_tile_width(int P, int W)
{
    const int cls = (W + 31) / 32;
    if ((cls & 1) == 0) return 64;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        const auto it = g_tune[dev].find({P, cls});
        if (it != g_tune[dev].end()) return it->second;
    }
    return 32;
}

struct Layout {
    size_t S, st, pre, params, chan_jac, chan_trial, lm, psum, ext_jac, ext_trial, y_jac,
        y_trial, part_jac, part_trial, active, exp, ctl, blob_end, total;
    size_t ids_static, n_static;            // the all-stamps work list (in the blob)
    size_t wl_n[2], wl_ids[2], wl_pre[2];   // LM work lists: 0 Jacobian pass, 1 trial pass
    size_t wl_blk;                          // their per-CTA sums
    size_t tw_x, tw_y, hhat, psfgrid, spec_jac, spec_trial;
    size_t dft_buf[2], dft_mat;  // DFT path: ping-pong complex buffers, bf16 DFT matrices
    int count, nchan, nacc, nslots;
    int rungs;  // channels of the trial pass: 1, or the LM ladder's rungs
    int tot_model, tot_os, tot_conv, tot_red, tot_conv32;
    int max_red;  // most reduction blocks of one stamp
    long long tot_wb;  // 16 x 32 output blocks of all stamps (the fused trial chi^2's partials)
    long long max_wb;  // ... and the most of one stamp
    int conv_ty, conv_cap;  // direct convolution: tile height, persistent CTAs per SM
    int eval_variant;  // the model kernels' evaluator: 0 Sersic / disk / Gaussian,
                       // 1 with Moffat, 2 with King, Nuker or point sources
    int os_ns;         // sub-samples per oversampled pixel (os_factor^2; 1 without a block)
};

struct Plan {
    Layout L;
    std::vector<StampInfo> st;
    std::vector<int> pre;  // 4 * (count + 1): model, os, conv, red
    int method;            // GF_CONV_DIRECT, GF_CONV_FFT or GF_CONV_DFT_TC
    int Nx, Ny, cpc;       // FFT geometry (method FFT)
    int small = 0;         // FFT: one CTA per transform (Nx, Ny in 32 x {3, 4, 5})
    DftFactor fx, fy;      // DFT geometry (method DFT_TC)
};

// Build the stamp table, the block tables and the workspace layout.
void plan_batch(const gf_desc* d, const Structure& S, int count, const int* H, const int* W,
                const int64_t* pix_off, const int64_t* psf_off, int need, Plan* pl)
{
    const int P = d->psf_size, c = (P - 1) / 2;
    pl->st.resize(count);
    pl->pre.assign(WK_KINDS * (count + 1), 0);
    int* pm = pl->pre.data() + WK_MODEL * (count + 1);
    int* po = pl->pre.data() + WK_OS * (count + 1);
    int* pc = pl->pre.data() + WK_CONV * (count + 1);
    int* pr = pl->pre.data() + WK_RED * (count + 1);
    int* pc32 = pl->pre.data() + WK_CONV32 * (count + 1);
    int max_red = 0;
    long long e1 = 0, y1 = 0, wb = 0, max_wb = 0;
    const ConvShape shape = conv_shape(P);
    for (int b = 0; b < count; ++b) {
        StampInfo& s = pl->st[b];
        memset(&s, 0, sizeof(s));
        s.H = H[b];
        s.W = W[b];
        s.P = P;
        s.c = c;
        s.He = s.H + 2 * c;
        s.We = s.W + 2 * c;
        s.os_factor = d->os_factor;
        s.os_box = (d->os_factor > 1) ? d->os_box : 0;
        if (s.os_box == 0) s.os_factor = 1;
        s.os_x0 = d->os_x0 >= 0 ? d->os_x0 : (s.W - s.os_box) / 2;
        s.os_y0 = d->os_y0 >= 0 ? d->os_y0 : (s.H - s.os_box) / 2;
        s.nchan = S.nchan;
        s.pix_off = pix_off ? pix_off[b] : y1;
        s.psf_off = psf_off ? psf_off[b] : 0;
        s.ext1_off = e1;
        s.y1_off = y1;
        e1 += (long long)s.He * s.We;
        y1 += (long long)s.H * s.W;
        const long long ne = (long long)s.He * s.We;
        pm[b + 1] = pm[b] + (int)((ne + MODEL_THREADS - 1) / MODEL_THREADS);
        const int nb2 = s.os_factor > 1 ? s.os_box * s.os_box : 0;
        po[b + 1] = po[b] + (nb2 + OS_WARPS - 1) / OS_WARPS;
        s.conv_tw = conv_tile_width(P, s.W);
        const int conv_tiles = ((s.H + shape.ty - 1) / shape.ty) * ((s.W + s.conv_tw - 1) / s.conv_tw);
        pc[b + 1] = pc[b] + (s.conv_tw == 64 ? conv_tiles : 0);
        pc32[b + 1] = pc32[b] + (s.conv_tw == 32 ? conv_tiles : 0);
        pr[b + 1] = pr[b] + (int)(((long long)s.H * s.W + RED_PIX - 1) / RED_PIX);
        s.wb_off = (int)std::min<long long>(wb, INT32_MAX);
        const long long nwb = (long long)((s.H + 15) / 16) * ((s.W + 31) / 32);
        wb += nwb;
        max_wb = std::max<long long>(max_wb, nwb);
        max_red = std::max(max_red, pr[b + 1] - pr[b]);
    }
    Layout& L = pl->L;
    memset(&L, 0, sizeof(L));
    L.max_red = max_red;
    L.max_wb = max_wb;
    L.tot_wb = wb;
    L.conv_ty = shape.ty;
    L.conv_cap = shape.ctas_per_sm;
    L.count = count;
    L.nchan = S.nchan;
    L.eval_variant = 0;
    L.os_ns = (d->os_factor > 1 && d->os_box > 0) ? d->os_factor * d->os_factor : 1;
    for (int k = 0; k < S.ncomp; ++k) {
        const int kd = S.kinds[k];
        if (kd == GF_MOFFAT) L.eval_variant = std::max(L.eval_variant, 1);
        if (kd == GF_KING || kd == GF_NUKER || kd == GF_PSF || kd == GF_SERSIC_F) L.eval_variant = 2;
    }
    L.nacc = S.nacc;
    L.nslots = S.nslots;
    L.tot_model = pm[count];
    L.tot_os = po[count];
    L.tot_conv = pc[count];
    L.tot_conv32 = pc32[count];
    L.tot_red = pr[count];
    size_t o = 0;
    L.S = o;
    o += al(sizeof(Structure));
    L.st = o;
    o += al(sizeof(StampInfo) * count);
    L.pre = o;
    o += al(sizeof(int) * WK_KINDS * (count + 1));
    L.params = o;
    o += al(sizeof(double) * (size_t)count * S.nslots);
    L.ids_static = o;
    o += al(sizeof(int) * (size_t)count);
    L.n_static = o;
    o += al(sizeof(int));
    L.blob_end = o;
    // the trial pass: one channel per stamp, or one per rung of the LM ladder
    const int R = (need & NEED_LM) ? (S.opts.ladder > 0 ? S.opts.ladder : auto_ladder(count)) : 1;
    L.rungs = R;
    L.chan_trial = o;
    o += al(sizeof(Channel) * (size_t)count * R);
    L.psum = o;
    o += al(sizeof(float) * (size_t)count);
    L.active = o;
    o += al(sizeof(int) * 4);
    if (need & (NEED_JAC | NEED_LM)) {
        L.chan_jac = o;
        o += al(sizeof(Channel) * (size_t)count * S.nchan);
        L.ext_jac = o;
        o += al(sizeof(float) * (size_t)S.nchan * e1);
        L.y_jac = o;
        o += al(sizeof(float) * (size_t)S.nchan * y1);
        L.part_jac = o;
        o += al(sizeof(float) * (size_t)L.tot_red * S.nacc);
    }
    if (need & (NEED_TRIAL | NEED_LM)) {
        L.ext_trial = o;
        o += al(sizeof(float) * (size_t)R * e1);
        L.y_trial = o;
        o += al(sizeof(float) * (size_t)R * y1);
    }
    if (need & (NEED_TRIAL | NEED_LM | NEED_CHI2)) {
        // per rung: one partial per reduce block, or (LM on the direct path)
        // one per 16 x 32 output block
        L.part_trial = o;
        o += al(sizeof(float) * (size_t)R * std::max<long long>(L.tot_red, L.tot_wb));
    }
    if (need & NEED_LM) {
        L.lm = o;
        o += al(sizeof(LMState) * (size_t)count);
        L.exp = o;
        o += al(sizeof(double) * (size_t)count * (S.nslots + 5));
        L.ctl = o;
        o += al(sizeof(LoopCtl));
        for (int w = 0; w < 2; ++w) {
            L.wl_n[w] = o;
            o += al(sizeof(int));
            L.wl_ids[w] = o;
            o += al(sizeof(int) * (size_t)count);
            L.wl_pre[w] = o;
            o += al(sizeof(int) * (size_t)WK_KINDS * (count + 1));
        }
        L.wl_blk = o;
        o += al(sizeof(int) * (size_t)worklist_blocks(count) * (1 + WK_KINDS));
    }
    pl->method = resolve_method(d);
    if (pl->method == GF_CONV_FFT) {
        const StampInfo& s0 = pl->st[0];
        pl->Nx = fft_len(s0.We, true);
        pl->Ny = fft_len(s0.He, false);
        pl->cpc = choose_cpc(pl->Ny);
        // grids up to 160 x 160: padded to 32 M and transformed one CTA each,
        // the spectrum kept in shared memory (no spectrum scratch)
        const int sx = fft_small_len(s0.We), sy = fft_small_len(s0.He);
        pl->small = sx > 0 && sy > 0;
        if (pl->small) {
            pl->Nx = sx;
            pl->Ny = sy;
        }
        const size_t Kx = pl->Nx / 2 + 1;
        L.tw_x = o;
        o += al(sizeof(float2) * pl->Nx);
        L.tw_y = o;
        o += al(sizeof(float2) * pl->Ny);
        L.hhat = o;
        o += al(sizeof(float2) * (size_t)count * pl->Ny * Kx);
        L.psfgrid = o;
        o += al(sizeof(float) * (size_t)count * pl->Ny * pl->Nx);
        const size_t spec_rows = pl->small ? 0 : (size_t)s0.He * Kx;
        if (need & (NEED_JAC | NEED_LM)) {
            L.spec_jac = o;
            o += al(sizeof(float2) * (size_t)count * S.nchan * spec_rows);
        }
        // gf_eval and gf_convolve use one channel per stamp, the LM trial pass
        // one per rung
        L.spec_trial = o;
        o += al(sizeof(float2) * (size_t)count * R * spec_rows);
    }
    if (pl->method == GF_CONV_DFT_TC) {
        const StampInfo& s0 = pl->st[0];
        pl->fx = dft_factor(s0.We, true);
        pl->fy = dft_factor(s0.He, false);
        pl->Nx = pl->fx.N;
        pl->Ny = pl->fy.N;
        const size_t nn = (size_t)pl->Ny * pl->Nx;
        const int nch = (need & (NEED_JAC | NEED_LM)) ? std::max(S.nchan, R) : 1;
        L.tw_x = o;
        o += al(sizeof(float2) * pl->Nx);
        L.tw_y = o;
        o += al(sizeof(float2) * pl->Ny);
        L.hhat = o;
        o += al(sizeof(float2) * (size_t)count * nn);
        L.psfgrid = o;
        o += al(sizeof(float) * (size_t)count * nn);
        for (int w = 0; w < 2; ++w) {
            L.dft_buf[w] = o;
            o += al(sizeof(float2) * (size_t)count * nch * nn);
        }
        L.dft_mat = o;
        o += al(sizeof(__nv_bfloat16) * 8 * 4 * DFT_RMAX * DFT_RMAX);
    }
    L.total = o;
}

// the host image of [0, blob_end): Structure, stamp table, block tables, params
std::vector<uint8_t> make_blob(const Plan& pl, const Structure& S, const double* params)
{
    const Layout& L = pl.L;
    std::vector<uint8_t> blob(L.blob_end, 0);
    memcpy(blob.data() + L.S, &S, sizeof(S));
    memcpy(blob.data() + L.st, pl.st.data(), sizeof(StampInfo) * L.count);
    memcpy(blob.data() + L.pre, pl.pre.data(), sizeof(int) * pl.pre.size());
    if (params) memcpy(blob.data() + L.params, params, sizeof(double) * (size_t)L.count * S.nslots);
    int* ids = reinterpret_cast<int*>(blob.data() + L.ids_static);
    for (int b = 0; b < L.count; ++b) ids[b] = b;
    *reinterpret_cast<int*>(blob.data() + L.n_static) = L.count;
    return blob;
}

template <class T>
T* at(void* ws, size_t off)
{
    return reinterpret_cast<T*>(static_cast<uint8_t*>(ws) + off);
}

// Persistent launch grids: the work items of a pass (all stamps' blocks times
// the pass's channels) or a few waves of resident CTAs, whichever is smaller.
void set_grids(PassArgs& a, const Layout& L, int nchan)
{
    const long long items[WK_KINDS] = {(long long)L.tot_model * nchan, (long long)L.tot_os * nchan,
                                       (long long)L.tot_conv * nchan, (long long)L.tot_red,
                                       (long long)L.tot_conv32 * nchan};
    const long long cc = 152LL * L.conv_cap;  // the direct convolution's persistent grid
    const long long cap[WK_KINDS] = {152LL * 16, 152LL * 8, cc, 152LL * 6, cc};
    for (int k = 0; k < WK_KINDS; ++k) {
        a.maxitems[k] = (int)std::min<long long>(items[k], INT32_MAX);
        a.grid[k] = (int)std::min(items[k], cap[k]);
    }
}

PassArgs base_args(void* ws, const Layout& L, const float* psf, const float* img,
                   const float* sig, int P)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.count = L.count;
    a.st = at<StampInfo>(ws, L.st);
    a.S = at<Structure>(ws, L.S);
    const int* pre = at<int>(ws, L.pre);
    a.pre_static = pre;
    a.max_red = L.max_red;
    a.max_trial_slots = L.max_red;
    a.wl.n = at<int>(ws, L.n_static);
    a.wl.ids = at<int>(ws, L.ids_static);
    a.wl.pre = pre;
    set_grids(a, L, 1);
    a.psf = psf;
    a.psf_sum = at<float>(ws, L.psum);
    a.img = img;
    a.sig = sig;
    a.P = P;
    a.phase = PH_NONE;
    a.work = prof::work_dev;
    a.eval_variant = L.eval_variant;
    a.os_ns = L.os_ns;
    a.conv_ty = L.conv_ty;
    return a;
}

PassArgs jac_args(void* ws, const Layout& L, const PassArgs& base)
{
    PassArgs a = base;
    set_grids(a, L, L.nchan);
    a.chan = at<Channel>(ws, L.chan_jac);
    a.chan_stride = L.nchan;
    a.nchan = L.nchan;
    a.jac_pass = 1;
    a.ext = at<float>(ws, L.ext_jac);
    a.y = at<float>(ws, L.y_jac);
    a.partial = at<float>(ws, L.part_jac);
    a.nacc = L.nacc;
    return a;
}

PassArgs trial_args(void* ws, const Layout& L, const PassArgs& base)
{
    PassArgs a = base;
    a.chan = at<Channel>(ws, L.chan_trial);
    a.chan_stride = 1;
    a.nchan = 1;
    a.ext = at<float>(ws, L.ext_trial);
    a.y = at<float>(ws, L.y_trial);
    a.partial = at<float>(ws, L.part_trial);
    a.nacc = 1;
    return a;
}

gf_status check_ws(void* ws, size_t bytes, size_t need)
{
    if (!ws) return fail(GF_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
        return fail(GF_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < need)
        return fail(GF_ENOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
    return GF_OK;
}

gf_status upload(void* ws, const std::vector<uint8_t>& blob, cudaStream_t s)
{
    GF_CUDA(cudaMemcpyAsync(ws, blob.data(), blob.size(), cudaMemcpyHostToDevice, s));
    return GF_OK;
}

FFTArgs fft_args(void* ws, const Plan& pl)
{
    FFTArgs f;
    memset(&f, 0, sizeof(f));
    f.Nx = pl.Nx;
    f.Ny = pl.Ny;
    f.cpc = pl.cpc;
    f.small = pl.small;
    f.px = make_fft_plan(pl.Nx);
    f.py = make_fft_plan(pl.Ny);
    f.tw_x = at<float2>(ws, pl.L.tw_x);
    f.tw_y = at<float2>(ws, pl.L.tw_y);
    f.hhat = at<float2>(ws, pl.L.hhat);
    f.psfgrid = at<float>(ws, pl.L.psfgrid);
    f.st0 = pl.st[0];
    f.flops_row = (float)(5.0 * pl.Nx * log2((double)pl.Nx));
    f.flops_col = (float)(pl.cpc * (2.0 * 5.0 * pl.Ny * log2((double)pl.Ny) + 6.0 * pl.Ny));
    return f;
}

// ------------------------------------------------ DFT-contraction convolution
int rpad16(int R) { return (R + 15) / 16 * 16; }

// DFT matrix table t (0..7): axis x/y, digit 1/2, forward/inverse
__nv_bfloat16* dft_matrix(void* ws, const Plan& pl, int axis, int digit, int inverse)
{
    const int t = (axis * 2 + digit) * 2 + inverse;
    return at<__nv_bfloat16>(ws, pl.L.dft_mat) + (size_t)t * 4 * DFT_RMAX * DFT_RMAX;
}

DftStage dft_base(void* ws, const Plan& pl, const PassArgs& a)
{
    DftStage g;
    memset(&g, 0, sizeof(g));
    g.lm = a.lm;
    g.phase = a.phase;
    g.nchan = a.nchan > 0 ? a.nchan : 1;
    return g;
}

void dft_set(DftStage& g, int R, const __nv_bfloat16* F)
{
    g.R = R;
    g.Rp = rpad16(R);
    g.F = F;
}

// the four forward stages: real grid(s) -> digit-reversed spectrum in `out`
gf_status dft_forward(void* ws, const Plan& pl, DftStage g, const float* real, long long real_ps,
                      int ld, int rows, int cols, float2* out, int nprob, unsigned long long* work,
                      cudaStream_t s)
{
    const int Nx = pl.Nx, Ny = pl.Ny;
    const long long nn = (long long)Ny * Nx;
    float2* B0 = at<float2>(ws, pl.L.dft_buf[0]);
    float2* B1 = at<float2>(ws, pl.L.dft_buf[1]);
    g.in_pstride = g.out_pstride = nn;
    // x axis, digit 1 (stride R2x), twiddle W_Nx^{k1 x2}
    DftStage f1 = g;
    dft_set(f1, pl.fx.R1, dft_matrix(ws, pl, 0, 0, 0));
    f1.L = Ny;
    f1.Q = pl.fx.R2;
    f1.tw_mode = 1;
    f1.tw_div = 1;
    f1.tw_mod = pl.fx.R2;
    f1.tw_N = Nx;
    f1.tw = at<float2>(ws, pl.L.tw_x);
    f1.tw_sign = -1.0f;
    f1.in_mode = 1;
    f1.in_real = real;
    f1.in_real_pstride = real_ps;
    f1.in_ld = ld;
    f1.in_rows = rows;
    f1.in_cols = cols;
    f1.in_xdigit = pl.fx.R2;
    f1.out = B0;
    GF_CUDA(launch_dft_stage_a(f1, nprob, work, s));
    // x axis, digit 2 (contiguous)
    DftStage f2 = g;
    dft_set(f2, pl.fx.R2, dft_matrix(ws, pl, 0, 1, 0));
    f2.M = Ny * pl.fx.R1;
    f2.in = B0;
    f2.out = B1;
    GF_CUDA(launch_dft_stage_b(f2, nprob, work, s));
    // y axis, digit 1 (stride R2y * Nx), twiddle W_Ny^{k1 y2}, y2 = (q / Nx) % R2y
    DftStage f3 = g;
    dft_set(f3, pl.fy.R1, dft_matrix(ws, pl, 1, 0, 0));
    f3.L = 1;
    f3.Q = pl.fy.R2 * Nx;
    f3.tw_mode = 1;
    f3.tw_div = Nx;
    f3.tw_mod = pl.fy.R2;
    f3.tw_N = Ny;
    f3.tw = at<float2>(ws, pl.L.tw_y);
    f3.tw_sign = -1.0f;
    f3.in = B1;
    f3.out = B0;
    GF_CUDA(launch_dft_stage_a(f3, nprob, work, s));
    // y axis, digit 2 (stride Nx)
    DftStage f4 = g;
    dft_set(f4, pl.fy.R2, dft_matrix(ws, pl, 1, 1, 0));
    f4.L = pl.fy.R1;
    f4.Q = Nx;
    f4.in = B0;
    f4.out = out;
    GF_CUDA(launch_dft_stage_a(f4, nprob, work, s));
    return GF_OK;
}

gf_status run_conv_dft(const PassArgs& a, const Plan& pl, void* ws, cudaStream_t s)
{
    const StampInfo& s0 = pl.st[0];
    const int Nx = pl.Nx, Ny = pl.Ny;
    const long long nn = (long long)Ny * Nx;
    const int nprob = a.count * a.nchan;
    if (nprob > 65535) return fail(GF_EINVAL, "DFT convolution: stamps x channels must be <= 65535");
    float2* B0 = at<float2>(ws, pl.L.dft_buf[0]);
    float2* B1 = at<float2>(ws, pl.L.dft_buf[1]);
    DftStage g = dft_base(ws, pl, a);
    gf_status r = dft_forward(ws, pl, g, a.ext, (long long)s0.He * s0.We, s0.We, s0.He, s0.We,
                              B1, nprob, a.work ? &a.work[PROF_CONV] : nullptr, s);
    if (r != GF_OK) return r;
    unsigned long long* work = a.work ? &a.work[PROF_CONV] : nullptr;
    g.in_pstride = g.out_pstride = nn;
    // inverse y, digit 2, with the PSF spectrum product and twiddle W_Ny^{+k1 y2}
    DftStage i1 = g;
    dft_set(i1, pl.fy.R2, dft_matrix(ws, pl, 1, 1, 1));
    i1.L = pl.fy.R1;
    i1.Q = Nx;
    i1.tw_mode = 2;
    i1.tw_N = Ny;
    i1.tw = at<float2>(ws, pl.L.tw_y);
    i1.tw_sign = 1.0f;
    i1.in_mode = 2;
    i1.in = B1;
    i1.hhat = at<float2>(ws, pl.L.hhat);
    i1.out = B0;
    GF_CUDA(launch_dft_stage_a(i1, nprob, work, s));
    // inverse y, digit 1
    DftStage i2 = g;
    dft_set(i2, pl.fy.R1, dft_matrix(ws, pl, 1, 0, 1));
    i2.L = 1;
    i2.Q = pl.fy.R2 * Nx;
    i2.in = B0;
    i2.out = B1;
    GF_CUDA(launch_dft_stage_a(i2, nprob, work, s));
    // inverse x, digit 2 (contiguous), twiddle W_Nx^{+k1 x2}, k1 = m mod R1x
    DftStage i3 = g;
    dft_set(i3, pl.fx.R2, dft_matrix(ws, pl, 0, 1, 1));
    i3.M = Ny * pl.fx.R1;
    i3.tw_mode = 3;
    i3.tw_mod = pl.fx.R1;
    i3.tw_N = Nx;
    i3.tw = at<float2>(ws, pl.L.tw_x);
    i3.tw_sign = 1.0f;
    i3.in = B1;
    i3.out = B0;
    GF_CUDA(launch_dft_stage_b(i3, nprob, work, s));
    // inverse x, digit 1, real part of the valid region into the pass output
    DftStage i4 = g;
    dft_set(i4, pl.fx.R1, dft_matrix(ws, pl, 0, 0, 1));
    i4.L = Ny;
    i4.Q = pl.fx.R2;
    i4.in = B0;
    i4.out_mode = 1;
    i4.out_real = a.y;
    i4.out_real_pstride = (long long)s0.H * s0.W;
    i4.out_xdigit = pl.fx.R2;
    i4.crop_y0 = s0.c;
    i4.crop_x0 = s0.c;
    i4.crop_H = s0.H;
    i4.crop_W = s0.W;
    GF_CUDA(launch_dft_stage_a(i4, nprob, work, s));
    return GF_OK;
}

gf_status setup_conv_dft(void* ws, const Plan& pl, const float* psf, cudaStream_t s)
{
    FFTArgs f;
    memset(&f, 0, sizeof(f));
    f.Nx = pl.Nx;
    f.Ny = pl.Ny;
    f.tw_x = at<float2>(ws, pl.L.tw_x);
    f.tw_y = at<float2>(ws, pl.L.tw_y);
    f.psfgrid = at<float>(ws, pl.L.psfgrid);
    GF_CUDA(launch_fft_twiddles(f, s));
    const int Rs[4] = {pl.fx.R1, pl.fx.R2, pl.fy.R1, pl.fy.R2};
    for (int axis = 0; axis < 2; ++axis)
        for (int digit = 0; digit < 2; ++digit)
            for (int inv = 0; inv < 2; ++inv) {
                const int R = Rs[axis * 2 + digit];
                GF_CUDA(launch_dft_matrix(R, rpad16(R), inv ? 1.0f : -1.0f,
                                          dft_matrix(ws, pl, axis, digit, inv), s));
            }
    GF_CUDA(cudaMemsetAsync(f.psfgrid, 0, sizeof(float) * (size_t)pl.L.count * pl.Ny * pl.Nx, s));
    GF_CUDA(launch_psf_wrap(f, pl.L.count, at<StampInfo>(ws, pl.L.st), psf, s));
    PassArgs none;
    memset(&none, 0, sizeof(none));
    none.nchan = 1;
    DftStage g = dft_base(ws, pl, none);
    return dft_forward(ws, pl, g, f.psfgrid, (long long)pl.Ny * pl.Nx, pl.Nx, pl.Ny, pl.Nx,
                       at<float2>(ws, pl.L.hhat), pl.L.count, nullptr, s);
}

// per-call set-up of the convolution: twiddles and PSF spectra (FFT method)
gf_status setup_conv(void* ws, const Plan& pl, const float* psf, cudaStream_t s)
{
    if (pl.method == GF_CONV_DFT_TC) {
        ProfScope ps(PROF_CONV, s);
        return setup_conv_dft(ws, pl, psf, s);
    }
    if (pl.method != GF_CONV_FFT) return GF_OK;
    ProfScope ps(PROF_CONV, s);
    const FFTArgs f = fft_args(ws, pl);
    GF_CUDA(launch_fft_twiddles(f, s));
    GF_CUDA(launch_fft_psf(f, pl.L.count, at<StampInfo>(ws, pl.L.st), psf, s));
    return GF_OK;
}

// step 2 for the pass `a`; spec is the pass's spectrum scratch (FFT method)
gf_status run_conv(const PassArgs& a, const Plan& pl, void* ws, size_t spec_off, cudaStream_t s)
{
    ProfScope ps(PROF_CONV, s);
    if (pl.method == GF_CONV_DIRECT) {
        GF_CUDA(launch_conv_direct(a, s));
        return GF_OK;
    }
    if (pl.method == GF_CONV_DFT_TC) return run_conv_dft(a, pl, ws, s);
    GF_CUDA(launch_conv_fft(a, fft_args(ws, pl), at<float2>(ws, spec_off), s));
    return GF_OK;
}

gf_status jac_pass(const PassArgs& a, const Plan& pl, void* ws, const double* params, double* A,
                   double* g, double* x2, cudaStream_t s)
{
    {
        ProfScope ps(PROF_LM, s);
        GF_CUDA(launch_prep_jac(a, params, s));
    }
    {
        ProfScope ps(PROF_MODEL, s);
        GF_CUDA(launch_model(a, s));
    }
    gf_status r = run_conv(a, pl, ws, pl.L.spec_jac, s);
    if (r != GF_OK) return r;
    ProfScope ps(PROF_REDUCE, s);
    GF_CUDA(launch_reduce_jac(a, s));
    GF_CUDA(launch_final_jac(a, A, g, x2, s));
    return GF_OK;
}

gf_status trial_pass(const PassArgs& a, const Plan& pl, void* ws, cudaStream_t s, double* x2)
{
    {
        ProfScope ps(PROF_MODEL, s);
        GF_CUDA(launch_model(a, s));
    }
    gf_status r = run_conv(a, pl, ws, pl.L.spec_trial, s);
    if (r != GF_OK) return r;
    ProfScope ps(PROF_REDUCE, s);
    if (a.lm) {
        // the LM body: one chi^2 per rung of the trial ladder, summed by
        // k_final_update (on the direct path already reduced per tile by the
        // convolution)
        if (!a.conv_chi2) GF_CUDA(launch_reduce_rungs(a, s));
        return GF_OK;
    }
    GF_CUDA(launch_reduce_chi2(a, s));
    // a render (no image) has no chi^2
    if (x2) GF_CUDA(launch_final_chi2(a, x2, s));
    return GF_OK;
}

// The b_n table of the LM kernels, built once per device on the first call
// that evaluates a model (a one-time synchronisation of that call's stream).
// Under stream capture it is left for a later call: until it exists the
// kernels solve for b_n directly.
std::mutex g_bn_mu;
bool g_bn_built[64];

gf_status ensure_bn_table(cudaStream_t s)
{
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GF_OK;
    std::lock_guard<std::mutex> g(g_bn_mu);
    if (g_bn_built[dev]) return GF_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GF_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return GF_OK;
    GF_CUDA(launch_bn_table(s));
    GF_CUDA(cudaStreamSynchronize(s));
    g_bn_built[dev] = true;
    return GF_OK;
}

// Make every per-kernel attribute call (shared-memory opt-in) before a stream
// capture begins.
gf_status prepare_conv(const Plan& pl)
{
    if (pl.method == GF_CONV_DIRECT) {
        static int optin[64];
        GF_CUDA(ensure_smem_optin_conv_direct(pl.st[0].P, optin));
    }
    return GF_OK;
}

// The batched LM loop as one CUDA graph per host thread: a conditional WHILE
// node whose body graph holds one LM body (captured from the stream), and whose
// condition the body's last kernel (k_loop_ctl) sets on the device.  The outer
// graph, its node and the condition handle are made once per thread and
// device; each call empties the body, captures its own body into it and
// updates the executable in place (cudaGraphExecUpdate), or instantiates it
// again when the body's shape changed.
// A blocking stream per host thread and device (created on first use, kept
// until exit) for LM fits the caller queues on the legacy default stream.
thread_local cudaStream_t t_loop_stream[64];

gf_status loop_stream(cudaStream_t* out)
{
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GF_ECUDA, "device ordinal out of range");
    if (!t_loop_stream[dev]) GF_CUDA(cudaStreamCreateWithFlags(&t_loop_stream[dev], cudaStreamDefault));
    *out = t_loop_stream[dev];
    return GF_OK;
}

struct LoopGraph {
    cudaGraph_t g = nullptr;
    cudaGraph_t body = nullptr;
    cudaGraphNode_t cond = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaGraphExec_t exec = nullptr;
    int dev = -1;
};
thread_local LoopGraph t_loop;

void loop_graph_reset(LoopGraph& G)
{
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
    G = LoopGraph();
}

// capture(h) launches one LM body on the stream (k_loop_ctl given handle h)
template <typename F>
gf_status loop_graph(cudaStream_t s, F&& capture, cudaGraphExec_t* out)
{
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    LoopGraph& G = t_loop;
    if (G.g && G.dev != dev) loop_graph_reset(G);
    if (!G.g) {
        GF_CUDA(cudaGraphCreate(&G.g, 0));
        G.dev = dev;
        cudaError_t e = cudaGraphConditionalHandleCreate(&G.h, G.g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {};
        if (e == cudaSuccess) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = G.h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            e = cudaGraphAddNode(&G.cond, G.g, nullptr, nullptr, 0, &np);
        }
        if (e != cudaSuccess) {
            loop_graph_reset(G);
            return fail(GF_ECUDA, std::string("conditional graph node: ") + cudaGetErrorString(e));
        }
        G.body = np.conditional.phGraph_out[0];
    } else {
        size_t n = 0;
        GF_CUDA(cudaGraphGetNodes(G.body, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        if (n) GF_CUDA(cudaGraphGetNodes(G.body, nodes.data(), &n));
        for (cudaGraphNode_t nd : nodes) GF_CUDA(cudaGraphDestroyNode(nd));
    }
    GF_CUDA(cudaStreamBeginCaptureToGraph(s, G.body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    const gf_status rb = capture(G.h);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &captured);
    if (rb != GF_OK) return rb;
    GF_CUDA(ce);
    if (G.exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(G.exec, G.g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
    }
    if (!G.exec) {
        const cudaError_t e = cudaGraphInstantiate(&G.exec, G.g, 0);
        if (e != cudaSuccess) {
            G.exec = nullptr;
            return fail(GF_ECUDA, std::string("loop graph instantiation: ") + cudaGetErrorString(e));
        }
    }
    *out = G.exec;
    return GF_OK;
}

}  // namespace

// ================================================================ the C ABI

extern "C" {

int gf_version(void) { return 100; }

long long gf_launch_count(void) { return g_launch_count.load(); }

void gf_prof_enable(unsigned long long* work_dev)
{
    std::lock_guard<std::mutex> g(prof::mu);
    prof::work_dev = work_dev;
}

int gf_prof_times(double* ms_out, long long* launches_out)
{
    std::lock_guard<std::mutex> g(prof::mu);
    int st = GF_OK;
    for (auto& r : prof::pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            prof::ms[r.cls] += ms;
            prof::launches[r.cls] += r.launches;
        } else {
            st = GF_ECUDA;
        }
        prof::pool.push_back(r.e0);
        prof::pool.push_back(r.e1);
    }
    prof::pending.clear();
    for (int c = 0; c < PROF_CLASSES; ++c) {
        if (ms_out) ms_out[c] = prof::ms[c];
        if (launches_out) launches_out[c] = prof::launches[c];
        prof::ms[c] = 0.0;
        prof::launches[c] = 0;
    }
    return st;
}

const char* gf_last_error(void) { return g_err.c_str(); }

gf_status gf_fma_peak(int fp64, int reps, void* sink, double* tflops, gf_stream stream)
{
    if (!sink || !tflops || reps < 1 || reps > 1000 || (fp64 != 0 && fp64 != 1))
        return fail(GF_EINVAL, "gf_fma_peak: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    GF_CUDA(cudaGetDevice(&dev));
    GF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // about 10 ms per float32 launch at full rate; float64 runs far slower, so
    // it takes fewer iterations
    const int grid = sms * 8, iters = fp64 ? 64 : 4096;
    double flops = 0.0;
    GF_CUDA(launch_fma_peak(fp64, grid, iters, sink, s, &flops));
    cudaEvent_t e0, e1;
    GF_CUDA(cudaEventCreate(&e0));
    GF_CUDA(cudaEventCreate(&e1));
    cudaError_t err = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && err == cudaSuccess; ++r)
        err = launch_fma_peak(fp64, grid, iters, sink, s, &flops);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GF_CUDA(err);
    *tflops = flops * reps / (ms * 1e-3) / 1e12;
    return GF_OK;
}

int gf_nslots(const gf_desc* d)
{
    if (check_structure(d) != GF_OK) return -1;
    return nslots_of(d);
}

void gf_default_opts(gf_lm_opts* opts)
{
    if (opts) default_opts(opts);
}

static int need_of(int call)
{
    switch (call) {
    case GF_CALL_CHI2: return NEED_CHI2;
    case GF_CALL_EVAL: return NEED_TRIAL;
    case GF_CALL_JACOBIAN: return NEED_JAC;
    case GF_CALL_LM_FIT: return NEED_LM;
    default: return 0;
    }
}

size_t gf_workspace_size(const gf_desc* d, const uint8_t* fixed, int call)
{
    if (check_structure(d) != GF_OK || check_stamp(d, d->H, d->W) != GF_OK) return 0;
    Structure S;
    if (make_structure(d, fixed, nullptr, nullptr, nullptr, &S) != GF_OK) return 0;
    S.opts.ladder = GF_MAX_LADDER;  // an LM fit's size holds for any ladder
    Plan pl;
    plan_batch(d, S, 1, &d->H, &d->W, nullptr, nullptr, need_of(call), &pl);
    return pl.L.total;
}

size_t gf_workspace_size_eval_batch(const gf_desc* d, const gf_batch* b)
{
    if (!b || b->count < 1 || !b->H || !b->W) return 0;
    if (check_structure(d) != GF_OK) return 0;
    for (int i = 0; i < b->count; ++i)
        if (check_stamp(d, b->H[i], b->W[i]) != GF_OK) return 0;
    if (check_fft(d, b->count, b->H, b->W) != GF_OK) return 0;
    Structure S;
    if (make_structure(d, nullptr, nullptr, nullptr, nullptr, &S) != GF_OK) return 0;
    Plan pl;
    plan_batch(d, S, b->count, b->H, b->W, b->pix_off, b->psf_off, NEED_TRIAL, &pl);
    return pl.L.total;
}

size_t gf_workspace_size_batch(const gf_desc* d, const gf_batch* b, const uint8_t* fixed)
{
    if (!b || b->count < 1 || !b->H || !b->W) return 0;
    if (check_structure(d) != GF_OK) return 0;
    for (int i = 0; i < b->count; ++i)
        if (check_stamp(d, b->H[i], b->W[i]) != GF_OK) return 0;
    Structure S;
    if (make_structure(d, fixed, nullptr, nullptr, nullptr, &S) != GF_OK) return 0;
    S.opts.ladder = GF_MAX_LADDER;  // an LM fit's size holds for any ladder
    Plan pl;
    plan_batch(d, S, b->count, b->H, b->W, b->pix_off, b->psf_off, NEED_LM, &pl);
    return pl.L.total;
}

gf_status gf_model(const gf_desc* d, const double* params, float* out, void* ws, size_t ws_bytes,
                   gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if ((r = check_stamp(d, d->H, d->W)) != GF_OK) return r;
    if (!params || !out) return fail(GF_EINVAL, "params or output is NULL");
    Structure S;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, &S)) != GF_OK) return r;
    Plan pl;
    plan_batch(d, S, 1, &d->H, &d->W, nullptr, nullptr, 0, &pl);
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = ensure_bn_table(s)) != GF_OK) return r;
    if ((r = upload(ws, make_blob(pl, S, params), s)) != GF_OK) return r;
    PassArgs a = base_args(ws, pl.L, nullptr, nullptr, nullptr, d->psf_size);
    a.chan = at<Channel>(ws, pl.L.chan_trial);
    a.chan_stride = 1;
    a.nchan = 1;
    a.ext = out;
    GF_CUDA(launch_prep_sum(a, at<double>(ws, pl.L.params), 0, s));
    GF_CUDA(launch_model(a, s));
    return GF_OK;
}

static gf_status model_batch_plan(const gf_desc* d, const gf_batch* b, Structure* S, Plan* pl)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if (!b || b->count < 1 || !b->H || !b->W) return fail(GF_EINVAL, "bad batch");
    for (int i = 0; i < b->count; ++i)
        if ((r = check_stamp(d, b->H[i], b->W[i])) != GF_OK) return r;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, S)) != GF_OK) return r;
    plan_batch(d, *S, b->count, b->H, b->W, nullptr, nullptr, 0, pl);
    return GF_OK;
}

size_t gf_workspace_size_model_batch(const gf_desc* d, const gf_batch* b)
{
    Structure S;
    Plan pl;
    if (model_batch_plan(d, b, &S, &pl) != GF_OK) return 0;
    return pl.L.total;
}

gf_status gf_model_batch(const gf_desc* d, const gf_batch* b, const double* params, float* out,
                         void* ws, size_t ws_bytes, gf_stream stream)
{
    Structure S;
    Plan pl;
    gf_status r = model_batch_plan(d, b, &S, &pl);
    if (r != GF_OK) return r;
    if (!params || !out) return fail(GF_EINVAL, "params or output is NULL");
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = ensure_bn_table(s)) != GF_OK) return r;
    if ((r = upload(ws, make_blob(pl, S, params), s)) != GF_OK) return r;
    PassArgs a = base_args(ws, pl.L, nullptr, nullptr, nullptr, d->psf_size);
    a.chan = at<Channel>(ws, pl.L.chan_trial);
    a.chan_stride = 1;
    a.nchan = 1;
    a.ext = out;
    GF_CUDA(launch_prep_sum(a, at<double>(ws, pl.L.params), 0, s));
    GF_CUDA(launch_model(a, s));
    return GF_OK;
}

gf_status gf_convolve(const gf_desc* d, const float* ext, const float* psf, float* out, void* ws,
                      size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if ((r = check_stamp(d, d->H, d->W)) != GF_OK) return r;
    if (!ext || !psf || !out) return fail(GF_EINVAL, "NULL buffer");
    Structure S;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, &S)) != GF_OK) return r;
    Plan pl;
    plan_batch(d, S, 1, &d->H, &d->W, nullptr, nullptr, 0, &pl);
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = upload(ws, make_blob(pl, S, nullptr), s)) != GF_OK) return r;
    PassArgs a = base_args(ws, pl.L, psf, nullptr, nullptr, d->psf_size);
    a.nchan = 1;
    a.chan_stride = 1;
    a.ext = const_cast<float*>(ext);
    a.y = out;
    if ((r = setup_conv(ws, pl, psf, s)) != GF_OK) return r;
    return run_conv(a, pl, ws, pl.L.spec_trial, s);
}

gf_status gf_chi2(const gf_desc* d, const float* model, const float* img, const float* sig,
                  double* chi2, void* ws, size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if ((r = check_stamp(d, d->H, d->W)) != GF_OK) return r;
    if (!model || !img || !sig || !chi2) return fail(GF_EINVAL, "NULL buffer");
    Structure S;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, &S)) != GF_OK) return r;
    Plan pl;
    plan_batch(d, S, 1, &d->H, &d->W, nullptr, nullptr, NEED_CHI2, &pl);
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    // the given model as one channel of weight 1
    std::vector<uint8_t> blob = make_blob(pl, S, nullptr);
    if ((r = upload(ws, blob, s)) != GF_OK) return r;
    Channel ch;
    memset(&ch, 0, sizeof(ch));
    ch.type = CH_SUM;
    ch.jcol = -1;
    ch.mweight = 1.0f;
    GF_CUDA(cudaMemcpyAsync(at<Channel>(ws, pl.L.chan_trial), &ch, sizeof(ch),
                            cudaMemcpyHostToDevice, s));
    PassArgs a = base_args(ws, pl.L, nullptr, img, sig, d->psf_size);
    a.chan = at<Channel>(ws, pl.L.chan_trial);
    a.chan_stride = 1;
    a.nchan = 1;
    a.y = const_cast<float*>(model);
    a.partial = at<float>(ws, pl.L.part_trial);
    GF_CUDA(launch_reduce_chi2(a, s));
    GF_CUDA(launch_final_chi2(a, chi2, s));
    return GF_OK;
}

gf_status gf_eval(const gf_desc* d, const double* params, const float* img, const float* sig,
                  const float* psf, float* model_out, double* chi2, void* ws, size_t ws_bytes,
                  gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if ((r = check_stamp(d, d->H, d->W)) != GF_OK) return r;
    if (!params || !img || !sig || !psf || !chi2) return fail(GF_EINVAL, "NULL argument");
    Structure S;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, &S)) != GF_OK) return r;
    Plan pl;
    plan_batch(d, S, 1, &d->H, &d->W, nullptr, nullptr, NEED_TRIAL, &pl);
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = ensure_bn_table(s)) != GF_OK) return r;
    if ((r = upload(ws, make_blob(pl, S, params), s)) != GF_OK) return r;
    PassArgs a = trial_args(ws, pl.L, base_args(ws, pl.L, psf, img, sig, d->psf_size));
    a.m_out = model_out;
    if ((r = setup_conv(ws, pl, psf, s)) != GF_OK) return r;
    GF_CUDA(launch_prep_sum(a, at<double>(ws, pl.L.params), 0, s));
    return trial_pass(a, pl, ws, s, chi2);
}

static gf_status eval_batch_impl(const gf_desc* d, const gf_batch* b, const double* params,
                                 bool params_on_device, const float* img, const float* sig,
                                 const float* psf, float* model_out, double* chi2, void* ws,
                                 size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if (!b || b->count < 1 || !b->H || !b->W) return fail(GF_EINVAL, "bad batch");
    for (int i = 0; i < b->count; ++i)
        if ((r = check_stamp(d, b->H[i], b->W[i])) != GF_OK) return r;
    if ((r = check_fft(d, b->count, b->H, b->W)) != GF_OK) return r;
    const bool render = params_on_device && !img && !sig && !chi2;
    if (!params || !psf || (!render && (!img || !sig || !chi2)) || (render && !model_out))
        return fail(GF_EINVAL, "NULL argument");
    Structure S;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, &S)) != GF_OK) return r;
    Plan pl;
    plan_batch(d, S, b->count, b->H, b->W, b->pix_off, b->psf_off, NEED_TRIAL, &pl);
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = ensure_bn_table(s)) != GF_OK) return r;
    if ((r = upload(ws, make_blob(pl, S, params_on_device ? nullptr : params), s)) != GF_OK) return r;
    if (params_on_device)
        GF_CUDA(cudaMemcpyAsync(at<double>(ws, pl.L.params), params,
                                sizeof(double) * (size_t)b->count * S.nslots,
                                cudaMemcpyDeviceToDevice, s));
    PassArgs a = trial_args(ws, pl.L, base_args(ws, pl.L, psf, img, sig, d->psf_size));
    a.m_out = model_out;
    if ((r = setup_conv(ws, pl, psf, s)) != GF_OK) return r;
    GF_CUDA(launch_prep_sum(a, at<double>(ws, pl.L.params), 0, s));
    return trial_pass(a, pl, ws, s, chi2);
}

gf_status gf_eval_batch(const gf_desc* d, const gf_batch* b, const double* params,
                        const float* img, const float* sig, const float* psf, float* model_out,
                        double* chi2, void* ws, size_t ws_bytes, gf_stream stream)
{
    return eval_batch_impl(d, b, params, false, img, sig, psf, model_out, chi2, ws, ws_bytes,
                           stream);
}

gf_status gf_eval_batch_dev(const gf_desc* d, const gf_batch* b, const double* params_dev,
                            const float* img, const float* sig, const float* psf,
                            float* model_out, double* chi2, void* ws, size_t ws_bytes,
                            gf_stream stream)
{
    return eval_batch_impl(d, b, params_dev, true, img, sig, psf, model_out, chi2, ws, ws_bytes,
                           stream);
}

static gf_status jacobian_impl(const gf_desc* d, const double* params, const uint8_t* fixed,
                               double fd_rel, int jac_mode, const float* img, const float* sig,
                               const float* psf, float* J_out, double* A, double* g,
                               double* chi2, void* ws, size_t ws_bytes, gf_stream stream);

gf_status gf_jacobian(const gf_desc* d, const double* params, const uint8_t* fixed, double fd_rel,
                      const float* img, const float* sig, const float* psf, float* J_out,
                      double* A, double* g, double* chi2, void* ws, size_t ws_bytes,
                      gf_stream stream)
{
    return jacobian_impl(d, params, fixed, fd_rel, GF_JAC_FD, img, sig, psf, J_out, A, g, chi2,
                         ws, ws_bytes, stream);
}

gf_status gf_jacobian_analytic(const gf_desc* d, const double* params, const uint8_t* fixed,
                               const float* img, const float* sig, const float* psf,
                               float* J_out, double* A, double* g, double* chi2, void* ws,
                               size_t ws_bytes, gf_stream stream)
{
    return jacobian_impl(d, params, fixed, 0.0, GF_JAC_ANALYTIC, img, sig, psf, J_out, A, g, chi2,
                         ws, ws_bytes, stream);
}

static gf_status jacobian_impl(const gf_desc* d, const double* params, const uint8_t* fixed,
                               double fd_rel, int jac_mode, const float* img, const float* sig,
                               const float* psf, float* J_out, double* A, double* g,
                               double* chi2, void* ws, size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if ((r = check_stamp(d, d->H, d->W)) != GF_OK) return r;
    if (!params || !img || !sig || !psf || !A || !g || !chi2)
        return fail(GF_EINVAL, "NULL argument");
    gf_lm_opts o;
    default_opts(&o);
    if (fd_rel > 0.0) o.fd_rel = fd_rel;
    o.jac_mode = jac_mode;
    Structure S;
    if ((r = make_structure(d, fixed, nullptr, nullptr, &o, &S)) != GF_OK) return r;
    if (S.nfree < 1) return fail(GF_EINVAL, "no free slots");
    Plan pl;
    plan_batch(d, S, 1, &d->H, &d->W, nullptr, nullptr, NEED_JAC, &pl);
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = ensure_bn_table(s)) != GF_OK) return r;
    if ((r = upload(ws, make_blob(pl, S, params), s)) != GF_OK) return r;
    PassArgs a = jac_args(ws, pl.L, base_args(ws, pl.L, psf, img, sig, d->psf_size));
    a.jac_analytic = jac_mode == GF_JAC_ANALYTIC;
    a.J_out = J_out;
    GF_CUDA(launch_psf_sum(1, a.st, psf, const_cast<float*>(a.psf_sum), s));
    if ((r = setup_conv(ws, pl, psf, s)) != GF_OK) return r;
    return jac_pass(a, pl, ws, at<double>(ws, pl.L.params), A, g, chi2, s);
}

static gf_status lm_fit_impl(const gf_desc* d, const gf_batch* b, double* params,
                             const uint8_t* fixed, const double* lo, const double* hi,
                             const float* img, const float* sig, const float* psf,
                             const gf_lm_opts* opts, gf_lm_result* res, void* ws, size_t ws_bytes,
                             gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if (!b || b->count < 1 || !b->H || !b->W) return fail(GF_EINVAL, "bad batch");
    for (int i = 0; i < b->count; ++i)
        if ((r = check_stamp(d, b->H[i], b->W[i])) != GF_OK) return r;
    if (!params || !img || !sig || !psf || !res) return fail(GF_EINVAL, "NULL argument");
    if (opts && !(opts->max_iter >= 1 && opts->lambda_up > 1.0 && opts->lambda_down > 0.0 &&
                  opts->lambda_down < 1.0 && opts->lambda0 > 0.0 &&
                  opts->time_budget_s >= 0.0 && opts->time_budget_s < 1e6))
        return fail(GF_EINVAL, "bad LM options");
    Structure S;
    if ((r = make_structure(d, fixed, lo, hi, opts, &S)) != GF_OK) return r;
    if (S.nfree < 1) return fail(GF_EINVAL, "no free slots");
    if ((r = check_fft(d, b->count, b->H, b->W)) != GF_OK) return r;
    Plan pl;
    plan_batch(d, S, b->count, b->H, b->W, b->pix_off, b->psf_off, NEED_LM, &pl);
    if ((r = check_ws(ws, ws_bytes, pl.L.total)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    // the legacy default stream cannot be captured: a call on it runs on the
    // thread's own blocking stream, which the legacy stream's semantics order
    // after the legacy stream's earlier work and before its later work
    if (s == nullptr && !prof::work_dev && (r = loop_stream(&s)) != GF_OK) return r;
    if ((r = ensure_bn_table(s)) != GF_OK) return r;
    const Layout& L = pl.L;
    if ((r = upload(ws, make_blob(pl, S, params), s)) != GF_OK) return r;
    if ((r = setup_conv(ws, pl, psf, s)) != GF_OK) return r;
    PassArgs base = base_args(ws, L, psf, img, sig, d->psf_size);
    LMState* lm = at<LMState>(ws, L.lm);
    PassArgs aj = jac_args(ws, L, base);
    aj.jac_analytic = S.opts.jac_mode == GF_JAC_ANALYTIC;
    aj.lm = lm;
    aj.phase = PH_NEED_JAC;
    PassArgs at_ = trial_args(ws, L, base);
    at_.lm = lm;
    at_.phase = PH_TRIAL;
    at_.nchan = at_.chan_stride = L.rungs;  // one trial channel per rung of the ladder
    set_grids(at_, L, L.rungs);
    // the direct path and the one-CTA FFT reduce the trial chi^2 inside the
    // convolution (no convolved trial model written)
    at_.conv_chi2 = (pl.method == GF_CONV_DIRECT || (pl.method == GF_CONV_FFT && pl.small)) ? 1 : 0;
    if (at_.conv_chi2) at_.max_trial_slots = (int)std::min<long long>(L.max_wb, INT32_MAX);
    // each pass walks the list of stamps in its phase, rebuilt every body
    aj.wl.n = at<int>(ws, L.wl_n[0]);
    aj.wl.ids = at<int>(ws, L.wl_ids[0]);
    aj.wl.pre = at<int>(ws, L.wl_pre[0]);
    at_.wl.n = at<int>(ws, L.wl_n[1]);
    at_.wl.ids = at<int>(ws, L.wl_ids[1]);
    at_.wl.pre = at<int>(ws, L.wl_pre[1]);
    int* active = at<int>(ws, L.active);
    GF_CUDA(launch_psf_sum(L.count, base.st, psf, const_cast<float*>(base.psf_sum), s));
    GF_CUDA(launch_lm_init(L.count, base.S, lm, at<double>(ws, L.params), s));
    // One LM "body": the Jacobian pass (stamps that need it), the damped solve,
    // the trial pass, accept/reject, and the loop's control kernel (stamps
    // still active, bodies run, time budget).
    LoopCtl* ctl = at<LoopCtl>(ws, L.ctl);
    auto body = [&](cudaGraphConditionalHandle h, int use_handle) -> gf_status {
        {
            ProfScope ps(PROF_LM, s);
            GF_CUDA(launch_worklist(L.count, lm, PH_NEED_JAC, base.pre_static,
                                    at<int>(ws, L.wl_n[0]), at<int>(ws, L.wl_ids[0]),
                                    at<int>(ws, L.wl_pre[0]), at<int>(ws, L.wl_blk), s));
        }
        gf_status rr = jac_pass(aj, pl, ws, nullptr, nullptr, nullptr, nullptr, s);
        if (rr != GF_OK) return rr;
        {
            ProfScope ps(PROF_LM, s);
            GF_CUDA(launch_final_solve(aj, at<Channel>(ws, L.chan_trial), active, L.rungs, s));
            GF_CUDA(launch_worklist(L.count, lm, PH_TRIAL, base.pre_static,
                                    at<int>(ws, L.wl_n[1]), at<int>(ws, L.wl_ids[1]),
                                    at<int>(ws, L.wl_pre[1]), at<int>(ws, L.wl_blk), s));
        }
        if ((rr = trial_pass(at_, pl, ws, s, nullptr)) != GF_OK) return rr;
        ProfScope ps(PROF_LM, s);
        GF_CUDA(launch_final_update(at_, active, s));
        GF_CUDA(launch_loop_ctl(L.count, lm, active, ctl, h, use_handle, s));
        return GF_OK;
    };
    const int max_bodies = S.opts.max_iter + 2;
    const unsigned long long budget_ns =
        S.opts.time_budget_s > 0.0 ? (unsigned long long)(S.opts.time_budget_s * 1e9) + 1ull : 0ull;
    GF_CUDA(launch_loop_start(ctl, budget_ns, max_bodies, s));
    // With a capturable stream and no profiling, the whole loop is one graph
    // launch: the body inside a conditional WHILE node that k_loop_ctl drives.
    long long per_body = 0;
    if (s != nullptr && !prof::work_dev) {
        if ((r = prepare_conv(pl)) != GF_OK) return r;
        cudaGraphExec_t exec = nullptr;
        const long long n0 = g_launch_count.load();
        r = loop_graph(s, [&](cudaGraphConditionalHandle h) { return body(h, 1); }, &exec);
        if (r != GF_OK) return r;
        per_body = g_launch_count.load() - n0;
        GF_CUDA(cudaGraphLaunch(exec, s));
    } else {
        // profiled calls need host-recorded events around each kernel class:
        // the body is launched directly and the host reads the active count
        // every few bodies
        int bodies = 0;
        for (;;) {
            const int K = bodies < 8 ? 2 : 4;
            for (int k = 0; k < K && bodies < max_bodies; ++k, ++bodies)
                if ((r = body(0, 0)) != GF_OK) return r;
            int h_active = 0;
            GF_CUDA(cudaMemcpyAsync(&h_active, active, sizeof(int), cudaMemcpyDeviceToHost, s));
            GF_CUDA(cudaStreamSynchronize(s));
            if (h_active == 0 || bodies >= max_bodies) break;
        }
    }
    double* ex = at<double>(ws, L.exp);
    GF_CUDA(launch_lm_export(L.count, base.S, lm, ex, s));
    const int stride = S.nslots + 5;
    std::vector<double> hx((size_t)L.count * stride);
    LoopCtl hc;
    GF_CUDA(cudaMemcpyAsync(hx.data(), ex, sizeof(double) * hx.size(), cudaMemcpyDeviceToHost, s));
    GF_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
    GF_CUDA(cudaStreamSynchronize(s));
    // the capture counted one body's launches; the graph ran hc.bodies of them
    if (per_body > 0 && hc.bodies > 1) g_launch_count.fetch_add(per_body * (hc.bodies - 1));
    for (int i = 0; i < L.count; ++i) {
        const double* o = hx.data() + (size_t)i * stride;
        memcpy(params + (size_t)i * S.nslots, o, sizeof(double) * S.nslots);
        res[i].chi2 = o[S.nslots];
        res[i].lambda = o[S.nslots + 1];
        res[i].iters = (int)o[S.nslots + 2];
        res[i].accepted = (int)o[S.nslots + 3];
        res[i].status = (int)o[S.nslots + 4];
    }
    return GF_OK;
}

// The direct convolution's launch shape, tuned on the device per PSF side P:
//   tile width TX (64 or 32) per width class ceil(W / 32), for the odd
//   classes (the only ones where the widths differ);
//   tile height TY (32 or 16) and the persistent grid (4, 8 or 16 CTAs per
//   SM), for all stamps of side P.
// Candidates are timed on the call's own stamps over the Jacobian pass's
// channels (best of three launches after a warm-up), coordinate-wise: widths
// per class, then the 6 (TY, grid) pairs on the whole batch, then the widths
// again under the chosen pair.  So each class sees 2 x 2 x 3 = 12 shapes (6
// for even classes).  Results do not depend on the shape: every output sums
// its taps in the same order.
gf_status gf_autotune(const gf_desc* d, const gf_batch* b, const float* psf, void* ws,
                      size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if (!b || b->count < 1 || !b->H || !b->W || !psf) return fail(GF_EINVAL, "bad batch or PSF");
    for (int i = 0; i < b->count; ++i)
        if ((r = check_stamp(d, b->H[i], b->W[i])) != GF_OK) return r;
    if (resolve_method(d) != GF_CONV_DIRECT) return GF_OK;  // nothing to choose
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GF_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return fail(GF_EINVAL, "gf_autotune cannot run under capture");
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GF_ECUDA, "device ordinal out of range");
    Structure S;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, &S)) != GF_OK) return r;
    const int P = d->psf_size;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GF_CUDA(cudaEventCreate(&e0));
    GF_CUDA(cudaEventCreate(&e1));
    gf_status out = GF_OK;
    // time the Jacobian-pass convolution of stamps idx under the current table;
    // tile_w > 0 launches that width's kind alone
    auto time_conv = [&](const std::vector<int>& idx, int tile_w, float* best) -> gf_status {
        std::vector<int> H, W;
        std::vector<int64_t> psf_off;
        for (int i : idx) {
            H.push_back(b->H[i]);
            W.push_back(b->W[i]);
            psf_off.push_back(b->psf_off ? b->psf_off[i] : (int64_t)i * P * P);
        }
        Plan pl;
        plan_batch(d, S, (int)H.size(), H.data(), W.data(), nullptr, psf_off.data(), NEED_JAC, &pl);
        gf_status rr = check_ws(ws, ws_bytes, pl.L.total);
        if (rr != GF_OK) return rr;
        if ((rr = upload(ws, make_blob(pl, S, nullptr), s)) != GF_OK) return rr;
        PassArgs a = jac_args(ws, pl.L, base_args(ws, pl.L, psf, nullptr, nullptr, P));
        auto launch = [&]() {
            return tile_w > 0 ? launch_conv_direct_width(a, tile_w, s) : launch_conv_direct(a, s);
        };
        if (cudaMemsetAsync(a.ext, 0, sizeof(float) * (size_t)pl.L.nchan *
                                          (pl.st.back().ext1_off +
                                           (long long)pl.st.back().He * pl.st.back().We),
                            s) != cudaSuccess ||
            launch() != cudaSuccess)
            return fail(GF_ECUDA, "autotune launch failed");
        *best = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
            float ms = 0.0f;
            if (cudaEventRecord(e0, s) != cudaSuccess || launch() != cudaSuccess ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                return fail(GF_ECUDA, "autotune timing failed");
            *best = std::min(*best, ms);
        }
        return GF_OK;
    };
    std::map<int, std::vector<int>> classes;  // odd class -> stamps
    std::vector<int> all(b->count);
    for (int i = 0; i < b->count; ++i) {
        all[i] = i;
        const int cls = (b->W[i] + 31) / 32;
        if (cls & 1) classes[cls].push_back(i);
    }
    auto tune_widths = [&]() -> gf_status {
        for (const auto& kv : classes) {
            const int widths[2] = {64, 32};
            float ms[2] = {INFINITY, INFINITY};
            for (int v = 0; v < 2; ++v) {
                {
                    std::lock_guard<std::mutex> g(g_tune_mu);
                    g_tune[dev][{P, kv.first}] = widths[v];
                }
                gf_status rr = time_conv(kv.second, widths[v], &ms[v]);
                if (rr != GF_OK) return rr;
            }
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune[dev][{P, kv.first}] = ms[1] < ms[0] ? 32 : 64;
        }
        return GF_OK;
    };
    if ((out = tune_widths()) == GF_OK) {
        const ConvShape cand[6] = {{32, 8}, {32, 4}, {32, 16}, {16, 8}, {16, 4}, {16, 16}};
        float best = INFINITY;
        ConvShape pick = kConvShapeDefault;
        for (const ConvShape& c : cand) {
            {
                std::lock_guard<std::mutex> g(g_tune_mu);
                g_tune_shape[dev][P] = c;
            }
            float ms = INFINITY;
            if ((out = time_conv(all, 0, &ms)) != GF_OK) break;
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_shape[dev][P] = pick;
    }
    if (out == GF_OK) out = tune_widths();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return out;
}

int gf_conv_tile_width(int psf_size, int width) { return conv_tile_width(psf_size, width); }

gf_status gf_conv_tile_shape(int psf_size, int width, int* tile_w, int* tile_h, int* ctas_per_sm)
{
    if (psf_size < 1 || psf_size > GF_DIRECT_MAX_PSF || (psf_size & 1) == 0 || width < 1)
        return fail(GF_EINVAL, "bad PSF side or width");
    const ConvShape c = conv_shape(psf_size);
    if (tile_w) *tile_w = conv_tile_width(psf_size, width);
    if (tile_h) *tile_h = c.ty;
    if (ctas_per_sm) *ctas_per_sm = c.ctas_per_sm;
    return GF_OK;
}

gf_status gf_set_conv_tile_shape(int psf_size, int tile_h, int ctas_per_sm)
{
    if (psf_size < 1 || psf_size > GF_DIRECT_MAX_PSF || (psf_size & 1) == 0)
        return fail(GF_EINVAL, "bad PSF side");
    if (tile_h != 16 && tile_h != 32) return fail(GF_EINVAL, "tile height must be 16 or 32");
    if (ctas_per_sm < 1 || ctas_per_sm > 32) return fail(GF_EINVAL, "CTAs per SM must be 1 .. 32");
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GF_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_shape[dev][psf_size] = ConvShape{tile_h, ctas_per_sm};
    return GF_OK;
}

gf_status gf_set_conv_tile_width(int psf_size, int width, int tile_w)
{
    if (tile_w != 32 && tile_w != 64) return fail(GF_EINVAL, "tile width must be 32 or 64");
    if (psf_size < 1 || width < 1) return fail(GF_EINVAL, "bad PSF side or width");
    const int cls = (width + 31) / 32;
    if ((cls & 1) == 0) return tile_w == 64 ? GF_OK : fail(GF_EINVAL, "even width classes use 64");
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GF_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[dev][{psf_size, cls}] = tile_w;
    return GF_OK;
}

gf_status gf_lm_fit_batch(const gf_desc* d, const gf_batch* b, double* params,
                          const uint8_t* fixed, const float* img, const float* sig,
                          const float* psf, const gf_lm_opts* opts, gf_lm_result* res, void* ws,
                          size_t ws_bytes, gf_stream stream)
{
    return lm_fit_impl(d, b, params, fixed, nullptr, nullptr, img, sig, psf, opts, res, ws,
                       ws_bytes, stream);
}

// The batch of a multi-start fit: stamp i repeated `starts` times (entry
// i * starts + k), every copy pointing at the stamp's own image, sigma and PSF.
struct MultiBatch {
    std::vector<int> H, W;
    std::vector<int64_t> pix, psf;
    gf_batch b;
};

static gf_status make_multi(const gf_batch* b, int starts, MultiBatch* m)
{
    if (!b || b->count < 1 || !b->H || !b->W) return fail(GF_EINVAL, "bad batch");
    if (starts < 1) return fail(GF_EINVAL, "starts must be >= 1");
    const long long n = (long long)b->count * starts;
    if (n > INT32_MAX) return fail(GF_EINVAL, "count x starts too large");
    m->H.resize(n);
    m->W.resize(n);
    m->pix.resize(n);
    m->psf.resize(n);
    long long packed = 0;
    for (int i = 0; i < b->count; ++i) {
        const int64_t po = b->pix_off ? b->pix_off[i] : packed;
        const int64_t fo = b->psf_off ? b->psf_off[i] : 0;
        packed += (long long)b->H[i] * b->W[i];
        for (int k = 0; k < starts; ++k) {
            const long long e = (long long)i * starts + k;
            m->H[e] = b->H[i];
            m->W[e] = b->W[i];
            m->pix[e] = po;
            m->psf[e] = fo;
        }
    }
    m->b.count = (int)n;
    m->b.H = m->H.data();
    m->b.W = m->W.data();
    m->b.pix_off = m->pix.data();
    m->b.psf_off = m->psf.data();
    return GF_OK;
}

size_t gf_workspace_size_multistart(const gf_desc* d, const gf_batch* b, int starts,
                                    const uint8_t* fixed)
{
    MultiBatch m;
    if (make_multi(b, starts, &m) != GF_OK) return 0;
    return gf_workspace_size_batch(d, &m.b, fixed);
}

gf_status gf_lm_fit_multistart(const gf_desc* d, const gf_batch* b, int starts,
                               const double* starts_host, const uint8_t* fixed, const float* img,
                               const float* sig, const float* psf, const gf_lm_opts* opts,
                               double* params_out, gf_lm_result* res_out, int* best_out, void* ws,
                               size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    MultiBatch m;
    if ((r = make_multi(b, starts, &m)) != GF_OK) return r;
    if (!starts_host || !params_out || !res_out) return fail(GF_EINVAL, "NULL argument");
    const int ns = nslots_of(d);
    const long long n = m.b.count;
    std::vector<double> p(starts_host, starts_host + (size_t)n * ns);
    std::vector<gf_lm_result> res((size_t)n);
    if ((r = lm_fit_impl(d, &m.b, p.data(), fixed, nullptr, nullptr, img, sig, psf, opts, res.data(),
                         ws, ws_bytes, stream)) != GF_OK)
        return r;
    // per stamp the fit with the lowest finite chi^2, the earliest start on ties
    for (int i = 0; i < b->count; ++i) {
        int best = -1;
        for (int k = 0; k < starts; ++k) {
            const gf_lm_result& q = res[(size_t)i * starts + k];
            if (!std::isfinite(q.chi2)) continue;
            if (best < 0 || q.chi2 < res[(size_t)i * starts + best].chi2) best = k;
        }
        if (best < 0) best = 0;
        const size_t e = (size_t)i * starts + best;
        memcpy(params_out + (size_t)i * ns, p.data() + e * ns, sizeof(double) * ns);
        res_out[i] = res[e];
        if (best_out) best_out[i] = best;
    }
    return GF_OK;
}

gf_status gf_lm_fit(const gf_desc* d, double* params, const uint8_t* fixed, const double* lo,
                    const double* hi, const float* img, const float* sig, const float* psf,
                    const gf_lm_opts* opts, gf_lm_result* res, void* ws, size_t ws_bytes,
                    gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    int H = d->H, W = d->W;
    int64_t zero = 0;
    gf_batch b;
    b.count = 1;
    b.H = &H;
    b.W = &W;
    b.pix_off = &zero;
    b.psf_off = &zero;
    return lm_fit_impl(d, &b, params, fixed, lo, hi, img, sig, psf, opts, res, ws, ws_bytes,
                       stream);
}

}  // extern "C"

// ======================================================= allocation-free eval
// gf_eval_static: steps 1-3 like gf_eval, with its scratch in a file-scope
// device array instead of a caller workspace (see include/gf.h).
static __device__ __align__(256) unsigned char g_static_scratch[GF_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kStaticBlobMax = 4096;

// the call's tables and parameters, passed by value so that no host-to-device
// copy is needed
struct StaticBlob {
    unsigned char bytes[kStaticBlobMax];
};

__global__ void k_static_blob(StaticBlob blob, int n, unsigned char* dst)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = blob.bytes[i];
}

std::mutex g_static_mu;
void* g_static_addr[64];

// Device address of g_static_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself: on the host it only names a
// stand-in object, not device memory).
gf_status static_scratch_address(void** out)
{
    int dev = 0;
    GF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GF_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        GF_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return GF_OK;
}

}  // namespace

extern "C" size_t gf_static_scratch_bytes(void) { return GF_STATIC_SCRATCH_BYTES; }

extern "C" gf_status gf_eval_static(const gf_desc* d, const double* params, const float* img,
                                    const float* sig, const float* psf, float* model_out,
                                    double* chi2, gf_stream stream)
{
    gf_status r = check_structure(d);
    if (r != GF_OK) return r;
    if ((r = check_stamp(d, d->H, d->W)) != GF_OK) return r;
    if (!params || !img || !sig || !psf || !chi2) return fail(GF_EINVAL, "NULL argument");
    Structure S;
    if ((r = make_structure(d, nullptr, nullptr, nullptr, nullptr, &S)) != GF_OK) return r;
    Plan pl;
    plan_batch(d, S, 1, &d->H, &d->W, nullptr, nullptr, NEED_TRIAL, &pl);
    if (pl.L.total > GF_STATIC_SCRATCH_BYTES)
        return fail(GF_ENOMEM, "gf_eval_static: this stamp needs " + std::to_string(pl.L.total) +
                                   " bytes of scratch; the static scratch holds " +
                                   std::to_string((size_t)GF_STATIC_SCRATCH_BYTES) +
                                   " bytes (use gf_eval with a workspace)");
    if (pl.L.blob_end > (size_t)kStaticBlobMax)
        return fail(GF_ENOMEM, "gf_eval_static: call tables exceed the by-value limit");
    void* ws = nullptr;
    if ((r = static_scratch_address(&ws)) != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = ensure_bn_table(s)) != GF_OK) return r;
    const std::vector<uint8_t> blob = make_blob(pl, S, params);
    StaticBlob sb;
    memcpy(sb.bytes, blob.data(), blob.size());
    k_static_blob<<<1, 256, 0, s>>>(sb, (int)blob.size(), static_cast<unsigned char*>(ws));
    GF_COUNT_LAUNCH();
    GF_CUDA(cudaGetLastError());
    PassArgs a = trial_args(ws, pl.L, base_args(ws, pl.L, psf, img, sig, d->psf_size));
    a.m_out = model_out;
    if ((r = setup_conv(ws, pl, psf, s)) != GF_OK) return r;
    GF_CUDA(launch_prep_sum(a, at<double>(ws, pl.L.params), 0, s));
    return trial_pass(a, pl, ws, s, chi2);
}

// ==================================================== learned initial guess

namespace {

// the start of a single-Sersic + sky fit: 9 slots
constexpr int kGuessSlots = 9;

gf_status check_cnn_batch(int batch)
{
    if (batch < 1 || batch > (1 << 20)) return fail(GF_EINVAL, "batch out of range [1, 2^20]");
    return GF_OK;
}

// a guess call's tables in its workspace: H, W (int), offsets (int64), lo, hi
struct GuessLayout {
    size_t H, W, off, lo, hi, e2, total;
};

GuessLayout guess_layout(int count)
{
    GuessLayout g;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    g.H = take(sizeof(int) * (size_t)count);
    g.W = take(sizeof(int) * (size_t)count);
    g.off = take(sizeof(long long) * (size_t)count);
    g.lo = take(sizeof(double) * kGuessSlots);
    g.hi = take(sizeof(double) * kGuessSlots);
    g.e2 = take(sizeof(double));  // the Sersic flux factor at n = 2
    g.total = o;
    return g;
}

}  // namespace

extern "C" {

size_t gf_cnn_nparams(void) { return CNN_NPARAM; }

size_t gf_cnn_workspace_size(int batch, int training)
{
    if (batch < 1) return 0;
    return cnn_buffers(nullptr, batch, training != 0, nullptr);
}

gf_status gf_cnn_init(float* w, unsigned long long seed, gf_stream stream)
{
    if (!w) return fail(GF_EINVAL, "NULL argument");
    GF_CUDA(cnn_init(w, seed, (cudaStream_t)stream));
    return GF_OK;
}

gf_status gf_cnn_input(const float* img, const float* sig, int batch, float* x, gf_stream stream)
{
    gf_status r = check_cnn_batch(batch);
    if (r != GF_OK) return r;
    if (!img || !sig || !x) return fail(GF_EINVAL, "NULL argument");
    GF_CUDA(cnn_input(img, sig, batch, x, (cudaStream_t)stream));
    return GF_OK;
}

gf_status gf_cnn_forward(const float* w, const float* x, int batch, float* y, void* ws,
                         size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_cnn_batch(batch);
    if (r != GF_OK) return r;
    if (!w || !x || !y) return fail(GF_EINVAL, "NULL argument");
    if ((r = check_ws(ws, ws_bytes, cnn_buffers(nullptr, batch, false, nullptr))) != GF_OK) return r;
    CnnBuffers cb;
    cnn_buffers(ws, batch, false, &cb);
    cudaStream_t s = (cudaStream_t)stream;
    GF_CUDA(cnn_prepare(w, x, batch, cb, s));
    GF_CUDA(cnn_forward_tc(w, batch, cb, y, s));
    return GF_OK;
}

gf_status gf_cnn_loss_grad(const float* w, const float* x, const float* t, int batch, float* loss,
                           float* grad, void* ws, size_t ws_bytes, gf_stream stream)
{
    gf_status r = check_cnn_batch(batch);
    if (r != GF_OK) return r;
    if (!w || !x || !t || !loss || !grad) return fail(GF_EINVAL, "NULL argument");
    if ((r = check_ws(ws, ws_bytes, cnn_buffers(nullptr, batch, true, nullptr))) != GF_OK) return r;
    CnnBuffers cb;
    cnn_buffers(ws, batch, true, &cb);
    cudaStream_t s = (cudaStream_t)stream;
    GF_CUDA(cnn_prepare(w, x, batch, cb, s));
    GF_CUDA(cnn_forward_tc(w, batch, cb, nullptr, s));
    GF_CUDA(cnn_backward(t, batch, loss, grad, cb, s));
    return GF_OK;
}

gf_status gf_cnn_adam(float* w, float* m, float* v, const float* grad, int step, float lr,
                      gf_stream stream)
{
    if (!w || !m || !v || !grad) return fail(GF_EINVAL, "NULL argument");
    if (step < 1 || !(lr > 0.0f)) return fail(GF_EINVAL, "Adam step must be >= 1 and lr > 0");
    GF_CUDA(cnn_adam(w, m, v, grad, step, lr, (cudaStream_t)stream));
    return GF_OK;
}

gf_status gf_cnn_encode(const double* params, int nslots, int count, float* t, gf_stream stream)
{
    gf_status r = check_cnn_batch(count);
    if (r != GF_OK) return r;
    if (!params || !t) return fail(GF_EINVAL, "NULL argument");
    if (nslots < 7) return fail(GF_EINVAL, "a Sersic component needs slots 0..6");
    GF_CUDA(cnn_encode(params, nslots, count, CNN_SIDE, CNN_SIDE, t, (cudaStream_t)stream));
    return GF_OK;
}

gf_status gf_cnn_decode(const float* y, const double* dflt, int count, int flags, double* params,
                        gf_stream stream)
{
    gf_status r = check_cnn_batch(count);
    if (r != GF_OK) return r;
    if (!y || !dflt || !params) return fail(GF_EINVAL, "NULL argument");
    if (flags & ~GF_DECODE_MOMENT_CENTRE) return fail(GF_EINVAL, "unknown decode flags");
    GF_CUDA(cnn_decode(y, dflt, count, CNN_SIDE, CNN_SIDE, flags, params, (cudaStream_t)stream));
    return GF_OK;
}

gf_status gf_train_sample(unsigned long long seed, int count, int psf_size, double* params,
                          float* psf, gf_stream stream)
{
    gf_status r = check_cnn_batch(count);
    if (r != GF_OK) return r;
    if (!params || !psf) return fail(GF_EINVAL, "NULL argument");
    if (psf_size < 1 || psf_size % 2 == 0 || psf_size > GF_MAX_PSF)
        return fail(GF_EINVAL, "PSF side must be odd and <= GF_MAX_PSF");
    GF_CUDA(train_sample(seed, count, params, psf, psf_size, (cudaStream_t)stream));
    return GF_OK;
}

gf_status gf_noise(const float* model, int64_t n, unsigned long long seed, float sigma_read,
                   float gain, float* img, float* sig, gf_stream stream)
{
    if (!model || !img || !sig) return fail(GF_EINVAL, "NULL argument");
    if (n < 0 || !(gain > 0.0f) || !(sigma_read >= 0.0f))
        return fail(GF_EINVAL, "need n >= 0, gain > 0, sigma_read >= 0");
    if (n == 0) return GF_OK;
    GF_CUDA(noise_fill(model, n, seed, sigma_read, gain, img, sig, (cudaStream_t)stream));
    return GF_OK;
}

gf_status gf_philox4x32_10(const uint32_t* in, uint32_t* out, int n, gf_stream stream)
{
    if (!in || !out || n < 0) return fail(GF_EINVAL, "bad argument");
    if (n == 0) return GF_OK;
    GF_CUDA(philox_blocks(in, out, n, (cudaStream_t)stream));
    return GF_OK;
}

size_t gf_workspace_size_guess(int count)
{
    if (count < 1) return 0;
    return guess_layout(count).total;
}

gf_status gf_default_guess(const gf_batch* b, const float* img, double* params, void* ws,
                           size_t ws_bytes, gf_stream stream)
{
    if (!b || b->count < 1 || !b->H || !b->W) return fail(GF_EINVAL, "bad batch");
    if (!img || !params) return fail(GF_EINVAL, "NULL argument");
    const int count = b->count;
    std::vector<int> H(b->H, b->H + count), W(b->W, b->W + count);
    std::vector<long long> off(count);
    size_t smem = 0;
    long long run = 0;
    int max_npx = 0;
    for (int i = 0; i < count; ++i) {
        if (H[i] < 1 || W[i] < 1 || (long long)H[i] * W[i] > (1LL << 30))
            return fail(GF_EINVAL, "stamp size out of range");
        smem = std::max(smem, default_guess_smem(H[i], W[i]));
        max_npx = (int)std::min<long long>(std::max<long long>(max_npx, (long long)H[i] * W[i]), INT_MAX);
        off[i] = b->pix_off ? (long long)b->pix_off[i] : run;
        run += (long long)H[i] * W[i];
    }
    if (smem > 64 * 1024) return fail(GF_EINVAL, "default guess: stamp ring longer than 8192 pixels");
    const GuessLayout g = guess_layout(count);
    gf_status r = check_ws(ws, ws_bytes, g.total);
    if (r != GF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint8_t> blob(g.lo, 0);
    memcpy(blob.data() + g.H, H.data(), sizeof(int) * count);
    memcpy(blob.data() + g.W, W.data(), sizeof(int) * count);
    memcpy(blob.data() + g.off, off.data(), sizeof(long long) * count);
    if ((r = upload(ws, blob, s)) != GF_OK) return r;
    GF_CUDA(default_guess(count, at<int>(ws, g.H), at<int>(ws, g.W), at<long long>(ws, g.off), img,
                          params, kGuessSlots, smem, max_npx, at<double>(ws, g.e2), s));
    return GF_OK;
}

gf_status gf_guess_select(int count, const double* cand, const double* chi2_cand,
                          const double* dflt, const double* chi2_dflt, const double* lo,
                          const double* hi, double* out, int* choice, void* ws, size_t ws_bytes,
                          gf_stream stream)
{
    gf_status r = check_cnn_batch(count);
    if (r != GF_OK) return r;
    if (!cand || !chi2_cand || !dflt || !chi2_dflt || !out) return fail(GF_EINVAL, "NULL argument");
    const GuessLayout g = guess_layout(1);
    if ((r = check_ws(ws, ws_bytes, g.total)) != GF_OK) return r;
    std::vector<uint8_t> blob(g.total, 0);
    double* blo = reinterpret_cast<double*>(blob.data() + g.lo);
    double* bhi = reinterpret_cast<double*>(blob.data() + g.hi);
    gf_desc d;
    memset(&d, 0, sizeof(d));
    d.H = d.W = CNN_SIDE;
    d.psf_size = 1;
    d.ncomp = 2;
    d.kinds[0] = GF_SERSIC;
    d.kinds[1] = GF_SKY;
    Structure S;
    if ((r = make_structure(&d, nullptr, lo, hi, nullptr, &S)) != GF_OK) return r;
    for (int k = 0; k < kGuessSlots; ++k) {
        blo[k] = S.lo[k];
        bhi[k] = S.hi[k];
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((r = upload(ws, blob, s)) != GF_OK) return r;
    GF_CUDA(guess_select(count, kGuessSlots, cand, chi2_cand, dflt, chi2_dflt, at<double>(ws, g.lo),
                         at<double>(ws, g.hi), out, choice, s));
    return GF_OK;
}

}  // extern "C"

// ------------------------------------------------------ spectral lines, cubes

namespace {

gf_status check_spec(const gf_spec_desc* d, int count)
{
    if (!d) return fail(GF_EINVAL, "NULL spectral description");
    if (d->n_chan < 1 || d->n_chan > GF_SPEC_MAX_CHAN)
        return fail(GF_EINVAL, "n_chan must be 1 .. " + std::to_string(GF_SPEC_MAX_CHAN));
    if (d->n_lines < 0 || d->n_lines > GF_SPEC_MAX_LINES)
        return fail(GF_EINVAL, "n_lines must be 0 .. " + std::to_string(GF_SPEC_MAX_LINES));
    if (d->n_cont < 0 || d->n_cont > GF_SPEC_MAX_CONT)
        return fail(GF_EINVAL, "n_cont must be 0 .. " + std::to_string(GF_SPEC_MAX_CONT));
    if (d->n_cont + d->n_lines < 1) return fail(GF_EINVAL, "a spectrum needs a continuum or a line");
    if (d->lsf_len < 1 || d->lsf_len > GF_SPEC_MAX_LSF || (d->lsf_len & 1) == 0)
        return fail(GF_EINVAL, "lsf_len must be odd, 1 .. " + std::to_string(GF_SPEC_MAX_LSF));
    if (d->lsf_per_spectrum != 0 && d->lsf_per_spectrum != 1)
        return fail(GF_EINVAL, "lsf_per_spectrum must be 0 or 1");
    if (count < 0) return fail(GF_EINVAL, "count must be >= 0");
    return GF_OK;
}

SpecArgs spec_args(const gf_spec_desc* d, int count, int mode)
{
    SpecArgs a;
    memset(&a, 0, sizeof(a));
    a.mode = mode;
    a.N = d->n_chan;
    a.K = d->n_lines;
    a.nc = d->n_cont;
    a.L = d->lsf_len;
    a.lsf_stride = d->lsf_per_spectrum ? d->lsf_len : 0;
    a.count = count;
    a.np = d->n_cont + 3 * d->n_lines;
    default_opts(&a.opts);
    for (int s = 0; s < a.np; ++s) {
        const bool width = s >= a.nc && (s - a.nc) % 3 == 2;
        a.lo[s] = width ? 0.25 : -INFINITY;
        a.hi[s] = INFINITY;
    }
    return a;
}

gf_status spec_free(SpecArgs& a, const uint8_t* fixed)
{
    a.nf = 0;
    for (int s = 0; s < a.np; ++s) {
        if (fixed && fixed[s]) continue;
        if (a.nf >= GF_MAX_FREE)
            return fail(GF_EINVAL, "more than " + std::to_string(GF_MAX_FREE) + " free slots");
        a.fs[a.nf++] = s;
    }
    if (a.nf < 1) return fail(GF_EINVAL, "no free slots");
    return GF_OK;
}

gf_status spec_launch(SpecArgs a, gf_stream stream)
{
    // profiled as the convolution class: the LSF sums are most of its work
    ProfScope ps(PROF_CONV, (cudaStream_t)stream);
    a.work = prof::work_dev ? prof::work_dev + PROF_CONV : nullptr;
    GF_CUDA(launch_spec(a, (cudaStream_t)stream));
    return GF_OK;
}

}  // namespace

int gf_spec_nparams(const gf_spec_desc* d)
{
    if (check_spec(d, 0) != GF_OK) return -1;
    return d->n_cont + 3 * d->n_lines;
}

gf_status gf_spec_model(const gf_spec_desc* d, int count, const double* params_dev,
                        const float* lsf_dev, float* model_dev, gf_stream stream)
{
    gf_status r = check_spec(d, count);
    if (r != GF_OK) return r;
    if (count == 0) return GF_OK;
    if (!params_dev || !lsf_dev || !model_dev) return fail(GF_EINVAL, "NULL argument");
    SpecArgs a = spec_args(d, count, SPEC_MODEL);
    a.p_in = params_dev;
    a.lsf = lsf_dev;
    a.model = model_dev;
    return spec_launch(a, stream);
}

gf_status gf_spec_eval(const gf_spec_desc* d, int count, const double* params_dev,
                       const float* spec_dev, const float* sig_dev, const float* lsf_dev,
                       double* chi2_dev, float* model_dev, gf_stream stream)
{
    gf_status r = check_spec(d, count);
    if (r != GF_OK) return r;
    if (count == 0) return GF_OK;
    if (!params_dev || !spec_dev || !sig_dev || !lsf_dev || !chi2_dev)
        return fail(GF_EINVAL, "NULL argument");
    SpecArgs a = spec_args(d, count, SPEC_EVAL);
    a.p_in = params_dev;
    a.spec = spec_dev;
    a.sig = sig_dev;
    a.lsf = lsf_dev;
    a.chi2 = chi2_dev;
    a.model = model_dev;
    return spec_launch(a, stream);
}

gf_status gf_spec_normal(const gf_spec_desc* d, int count, const double* params_dev,
                         const uint8_t* fixed_host, const float* spec_dev,
                         const float* sig_dev, const float* lsf_dev, int jac_mode,
                         double fd_rel, double* A_dev, double* g_dev, double* chi2_dev,
                         gf_stream stream)
{
    gf_status r = check_spec(d, count);
    if (r != GF_OK) return r;
    if (jac_mode != GF_JAC_FD && jac_mode != GF_JAC_ANALYTIC)
        return fail(GF_EINVAL, "jac_mode must be GF_JAC_FD or GF_JAC_ANALYTIC");
    SpecArgs a = spec_args(d, count, SPEC_NORMAL);
    if ((r = spec_free(a, fixed_host)) != GF_OK) return r;
    if (count == 0) return GF_OK;
    if (!params_dev || !spec_dev || !sig_dev || !lsf_dev || !A_dev || !g_dev || !chi2_dev)
        return fail(GF_EINVAL, "NULL argument");
    a.opts.jac_mode = jac_mode;
    if (fd_rel > 0.0) a.opts.fd_rel = fd_rel;
    a.p_in = params_dev;
    a.spec = spec_dev;
    a.sig = sig_dev;
    a.lsf = lsf_dev;
    a.A = A_dev;
    a.g = g_dev;
    a.chi2 = chi2_dev;
    return spec_launch(a, stream);
}

gf_status gf_spec_fit(const gf_spec_desc* d, int count, const double* params_dev,
                      const uint8_t* fixed_host, const double* lo_host, const double* hi_host,
                      const float* spec_dev, const float* sig_dev, const float* lsf_dev,
                      const gf_lm_opts* opts, double* params_out_dev, gf_lm_result* result_dev,
                      gf_stream stream)
{
    gf_status r = check_spec(d, count);
    if (r != GF_OK) return r;
    SpecArgs a = spec_args(d, count, SPEC_FIT);
    if ((r = spec_free(a, fixed_host)) != GF_OK) return r;
    if (opts) a.opts = *opts;
    if (!(a.opts.fd_rel > 0.0)) a.opts.fd_rel = 1e-3;
    if (a.opts.jac_mode != GF_JAC_FD && a.opts.jac_mode != GF_JAC_ANALYTIC)
        return fail(GF_EINVAL, "jac_mode must be GF_JAC_FD or GF_JAC_ANALYTIC");
    if (a.opts.max_iter < 0) return fail(GF_EINVAL, "max_iter must be >= 0");
    for (int s = 0; s < a.np; ++s) {
        if (lo_host) a.lo[s] = lo_host[s];
        if (hi_host) a.hi[s] = hi_host[s];
        if (!(a.lo[s] <= a.hi[s])) return fail(GF_EINVAL, "bounds: lo > hi");
    }
    if (count == 0) return GF_OK;
    if (!params_dev || !spec_dev || !sig_dev || !lsf_dev || !params_out_dev || !result_dev)
        return fail(GF_EINVAL, "NULL argument");
    a.p_in = params_dev;
    a.p_out = params_out_dev;
    a.res = result_dev;
    a.spec = spec_dev;
    a.sig = sig_dev;
    a.lsf = lsf_dev;
    return spec_launch(a, stream);
}
