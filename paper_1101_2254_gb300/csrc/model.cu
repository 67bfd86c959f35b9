// model.cu -- step 1 of the fitting loop (Sec. 2 item 1): the analytic surface
// brightness on the halo-extended pixel grid, a per-pixel "transform" (Sec. 3).
//
// Two kernels write a channel grid:
//   k_model     one thread per grid pixel, the profile at the pixel centre;
//               pixels inside the oversampling block are left to
//   k_model_os  one warp per block pixel: the os_factor^2 sub-samples are spread
//               over the lanes and averaged by a shuffle tree.
// Splitting the block off keeps every warp of k_model uniform (a block pixel
// costs os_factor^2 evaluations, 100x a plain one for 10x10 sampling).
//
// A Jacobian pass (unit-amplitude shape channels and finite-difference channels
// that all share the same components) uses k_model_jac / k_model_os_jac: a
// thread (or warp) covers every channel of its pixel and evaluates each
// component at p once, so an FD channel costs one evaluation (at p + h) instead
// of two.  The values written are the same floats as channel_value gives.
#include <algorithm>

#include "gf_internal.cuh"

namespace {

__device__ __forceinline__ void load_channel(Channel* dst, const Channel* src)
{
    static_assert(sizeof(Channel) % 16 == 0, "Channel must be a multiple of 16 bytes");
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Channel) / 16); i += blockDim.x) d[i] = s[i];
}

// channels [0, nch) of a stamp (contiguous) into shared memory: four 16-byte
// loads per thread in flight before their stores, so the copy takes a couple of
// L2 round trips instead of one per channel
__device__ __forceinline__ void load_channels(Channel* dst, const Channel* src, int nch)
{
    const int n = nch * (int)(sizeof(Channel) / 16);
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    for (int i0 = threadIdx.x; i0 < n; i0 += 4 * blockDim.x) {
        int4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) v[u] = s[i];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) d[i] = v[u];
        }
    }
}

// ceil(2^32 / d) for d > 1 (0 for d = 1): with it, div_mag gives floor(x / d)
// by a multiply-high and one correction instead of a division
__device__ __forceinline__ unsigned mag_of(int d)
{
    return d > 1 ? (unsigned)(((1ull << 32) + (unsigned long long)d - 1ull) / (unsigned long long)d) : 0u;
}
// floor(x / d) for 0 <= x < 2^31: the multiply-high is floor(x / d) or one more
__device__ __forceinline__ int div_mag(int x, int d, unsigned mag)
{
    if (mag == 0u) return x;
    int q = (int)__umulhi((unsigned)x, mag);
    if ((long long)q * d > (long long)x) --q;
    return q;
}

// Grid pixel pix of the stamp's extended grid: its stamp coordinates (i, j),
// and whether the plain body evaluates it (false inside the oversampling
// block, which the block bodies evaluate).
__device__ __forceinline__ bool grid_pixel(const StampInfo& st, unsigned mag, int pix, int& i, int& j)
{
    const int ie = div_mag(pix, st.We, mag), je = pix - ie * st.We;
    i = ie - st.c;
    j = je - st.c;
    return !(st.os_factor > 1 && i >= st.os_y0 && i < st.os_y0 + st.os_box && j >= st.os_x0 &&
             j < st.os_x0 + st.os_box);
}

// Work item = (channel, block of MODEL_THREADS grid pixels of a listed stamp).
// A CTA's items are consecutive, so the (channel, block) pair advances by a
// counter instead of a division per item.
template <int EV>
__device__ __forceinline__ void body_model(const PassArgs& a, int vb, int vg)
{
    __shared__ __align__(16) Channel ch;
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_MODEL * (a.count + 1);
    const int tot = pre[n];
    const long long items = (long long)tot * a.nchan;
    int hint = -1, cur_b = -1, cur_k = -1;
    StampInfo st;
    unsigned mag = 0u;
    const long long chunk = (items + vg - 1) / vg;
    const long long it0 = (long long)vb * chunk, it1 = min(items, it0 + chunk);
    int k = 0, blk = 0;
    if (it0 < it1) {
        k = (int)(it0 / tot);
        blk = (int)(it0 - (long long)k * tot);
    }
    // Two consecutive items of the same stamp and channel are evaluated
    // together (a thread's two pixels are independent chains the scheduler
    // interleaves); a lone item at a stamp's end or the range's end alone.
    for (long long it = it0; it < it1;) {
        if (blk == tot) {
            blk = 0;
            ++k;
        }
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        if (b != cur_b || k != cur_k) {
            if (b != cur_b) {  // the stamp's geometry, kept while it lasts
                st = a.st[b];
                mag = mag_of(st.We);
            }
            __syncthreads();
            load_channel(&ch, &a.chan[(long long)b * a.chan_stride + k]);
            __syncthreads();
            cur_b = b;
            cur_k = k;
        }
        const bool two = it + 1 < it1 && blk + 1 < pre[li + 1];
        const int npix = st.He * st.We;  // stamps are validated below 2^31 pixels
        const int pix0 = (blk - pre[li]) * MODEL_THREADS + threadIdx.x;
        const int pix1 = pix0 + MODEL_THREADS;
        int i0 = 0, j0 = 0, i1 = 0, j1 = 0;
        const bool w0 = pix0 < npix && grid_pixel(st, mag, pix0, i0, j0);
        const bool w1 = two && pix1 < npix && grid_pixel(st, mag, pix1, i1, j1);
        if (w0 || w1) {
            float v0, v1;
            channel_value2<EV>(ch, (float)j0, (float)i0, (float)j1, (float)i1, v0, v1);
            float* E = a.ext + ext_index(st, a.nchan, k);
            if (w0) E[pix0] = v0;
            if (w1) E[pix1] = v1;
        }
        if (a.work) {
            const int cnt = __syncthreads_count(w0) + __syncthreads_count(w1);
            if (threadIdx.x == 0) atomicAdd(&a.work[PROF_MODEL], 4ull * (unsigned long long)cnt);
        }
        it += two ? 2 : 1;
        blk += two ? 2 : 1;
    }
}

// Work item = (channel, OS_WARPS pixels of a listed stamp's oversampling block).
template <int EV>
__device__ __forceinline__ void body_model_os(const PassArgs& a, int vb, int vg)
{
    __shared__ __align__(16) Channel ch;
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_OS * (a.count + 1);
    const int tot = pre[n];
    const long long items = (long long)tot * a.nchan;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int hint = -1, cur_b = -1, cur_k = -1;
    const long long chunk = (items + vg - 1) / vg;
    const long long it0 = (long long)vb * chunk, it1 = min(items, it0 + chunk);
    int k = 0, blk = 0;
    if (it0 < it1) {
        k = (int)(it0 / tot);
        blk = (int)(it0 - (long long)k * tot);
    }
    for (long long it = it0; it < it1; ++it, ++blk) {
        if (blk == tot) {
            blk = 0;
            ++k;
        }
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        const StampInfo st = a.st[b];
        if (b != cur_b || k != cur_k) {
            __syncthreads();
            load_channel(&ch, &a.chan[(long long)b * a.chan_stride + k]);
            __syncthreads();
            cur_b = b;
            cur_k = k;
        }
        const int q = (blk - pre[li]) * OS_WARPS + warp;
        const int B = st.os_box;
        if (q >= B * B) continue;
        const int i = st.os_y0 + q / B, j = st.os_x0 + q % B;
        const int s = st.os_factor, ns = s * s;
        const float fs = (float)s;
        float v = 0.0f;
        for (int t = lane; t < ns; t += 32) {
            const int ay = t / s, bx = t - ay * s;
            const float oy = ((float)ay + 0.5f) / fs - 0.5f;
            const float ox = ((float)bx + 0.5f) / fs - 0.5f;
            v += channel_value<EV>(ch, (float)j, (float)i, ox, oy);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            const long long pix = (long long)(i + st.c) * st.We + (j + st.c);
            a.ext[ext_index(st, a.nchan, k) + pix] = v / (float)ns;
            if (a.work) atomicAdd(&a.work[PROF_MODEL], 4ull);
        }
    }
}

// Jacobian-pass value of channel c given the components at p (base)
template <int EV>
__device__ __forceinline__ float jac_channel(const Channel& ch, const float* base, float xi, float yi,
                                             float ox, float oy)
{
    float b = 0.0f;
#pragma unroll
    for (int k = 0; k < GF_MAX_COMP; ++k)
        if (k == ch.comp) b = base[k];
    if (ch.type == CH_SHAPE) return b;
    if (ch.type == CH_PLANE) return ch.dslot == 0 ? xi - ch.pxc : yi - ch.pyc;  // pixel centre
    if (ch.type == CH_DERIV) {
        float g[8];
        comp_grad(ch.cc[ch.comp], xi, yi, ox, oy, ch.dbdn, g);
        return grad_pick(g, ch.dslot) * ch.scale;
    }
    return (comp_eval<EV>(ch.pert, xi, yi, ox, oy) - b) * ch.scale;
}

template <int EV>
__device__ __forceinline__ void comp_base(const Channel& c0, float* base, float xi, float yi,
                                          float ox, float oy)
{
#pragma unroll
    for (int k = 0; k < GF_MAX_COMP; ++k)
        base[k] = (k < c0.ncomp && !is_sky_kind(c0.cc[k].kind)) ? comp_eval<EV>(c0.cc[k], xi, yi, ox, oy)
                                                                 : 0.0f;
}

// Jacobian-pass value of channel c.  The cursor holds the last component
// evaluated at p (with its radius and log2 t): a channel of the same component
// reuses it, and a finite-difference channel reuses as much of it as its
// perturbed slot leaves unchanged (lvl, from fd_reuse_level).  Every value is
// the float a full evaluation gives.
template <int EV>
__device__ __forceinline__ float jac_value(const Channel* chs, int c, int lvl, EvalCursor& e,
                                           float xi, float yi, float ox, float oy)
{
    const Channel& ch = chs[c];
    if (ch.type == CH_PLANE) return ch.dslot == 0 ? xi - ch.pxc : yi - ch.pyc;  // pixel centre
    if (ch.type == CH_DERIV) {
        float g[8];
        comp_grad(ch.cc[ch.comp], xi, yi, ox, oy, ch.dbdn, g);
        return grad_pick(g, ch.dslot) * ch.scale;
    }
    if (ch.comp != e.comp) {
        e.comp = ch.comp;
        const CompConst& k = chs[0].cc[ch.comp];
        if (ch.comp < chs[0].ncomp && !is_sky_kind(k.kind))
            comp_eval_keep<EV>(k, xi, yi, ox, oy, e);
        else
            e.v = 0.0f;
    }
    if (ch.type == CH_SHAPE) return e.v;
    float pv;
    if (lvl == 2) {
        pv = comp_tail<EV>(ch.pert, e.t, e.lt);
    } else if (lvl == 1) {
        const float t = e.r * ch.pert.invr;
        pv = comp_tail<EV>(ch.pert, t, comp_log_t<EV>(ch.pert, t));
    } else {
        pv = comp_eval<EV>(ch.pert, xi, yi, ox, oy);
    }
    return (pv - e.v) * ch.scale;
}

// the reuse level of each channel of a Jacobian pass (after its channels are
// in shared memory; one barrier)
__device__ __forceinline__ void fd_levels(const Channel* chs, int nch, int* lvl)
{
    const int c = threadIdx.x;
    if (c < nch) {
        const Channel& ch = chs[c];
        lvl[c] = (ch.type == CH_FD && ch.comp < chs[0].ncomp) ? fd_reuse_level(chs[0].cc[ch.comp], ch.pert)
                                                              : 0;
    }
    __syncthreads();
}

// Work item = block of MODEL_THREADS grid pixels of a listed stamp (all channels).
template <int EV>
__device__ __forceinline__ void body_model_jac(const PassArgs& a, int vb, int vg)
{
    __shared__ __align__(16) Channel chs[GF_MAX_CHAN];
    __shared__ int lvl[GF_MAX_CHAN];  // finite-difference reuse level per channel
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_MODEL * (a.count + 1);
    const int tot = pre[n];
    const int nch = a.nchan;
    int hint = -1, cur_b = -1;
    unsigned mag = 0u;  // the stamp width's reciprocal for div_mag
    const int chunk = (tot + vg - 1) / vg;
    const int it0 = vb * chunk, it1 = min(tot, it0 + chunk);
    for (int blk = it0; blk < it1; ++blk) {
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        const StampInfo st = a.st[b];
        if (b != cur_b) {
            mag = mag_of(st.We);
            __syncthreads();
            load_channels(chs, &a.chan[(long long)b * a.chan_stride], nch);
            __syncthreads();
            fd_levels(chs, nch, lvl);
            cur_b = b;
        }
        const int npix = st.He * st.We;
        const int pix = (blk - pre[li]) * MODEL_THREADS + threadIdx.x;
        bool write = pix < npix;
        int i = 0, j = 0;
        if (write) {
            const int ie = div_mag(pix, st.We, mag), je = pix - ie * st.We;
            i = ie - st.c;
            j = je - st.c;
            write = !(st.os_factor > 1 && i >= st.os_y0 && i < st.os_y0 + st.os_box &&
                      j >= st.os_x0 && j < st.os_x0 + st.os_box);
        }
        if (write) {
            EvalCursor e;
            e.comp = -1;
            float* E = a.ext + ext_index(st, nch, 0) + pix;
            const long long cs = (long long)st.He * st.We;
            for (int c = 0; c < nch; ++c)
                E[c * cs] = jac_value<EV>(chs, c, lvl[c], e, (float)j, (float)i, 0.0f, 0.0f);
        }
        if (a.work) {
            const int cnt = __syncthreads_count(write);
            if (threadIdx.x == 0)
                atomicAdd(&a.work[PROF_MODEL], 4ull * (unsigned long long)cnt * (unsigned long long)nch);
        }
    }
}

// Work item = block of MODEL_THREADS grid pixels of a listed stamp (all
// channels) of an analytic Jacobian pass: each component's value and gradient
// once per pixel (comp_grad), its shape channel and every derivative channel
// of it written from them.
template <int EV>
__device__ __forceinline__ void body_model_jac_an(const PassArgs& a, int vb, int vg)
{
    __shared__ __align__(16) Channel chs[GF_MAX_CHAN];
    __shared__ int shape_c[GF_MAX_COMP], d0[GF_MAX_COMP], d1[GF_MAX_COMP];
    __shared__ float dbdn_c[GF_MAX_COMP];
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_MODEL * (a.count + 1);
    const int tot = pre[n];
    const int nch = a.nchan;
    int hint = -1, cur_b = -1;
    unsigned mag = 0u;  // the stamp width's reciprocal for div_mag
    StampInfo st;
    const int chunk = (tot + vg - 1) / vg;
    const int it0 = vb * chunk, it1 = min(tot, it0 + chunk);
    for (int blk = it0; blk < it1; ++blk) {
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        if (b != cur_b) {
            st = a.st[b];
            mag = mag_of(st.We);
            __syncthreads();
            load_channels(chs, &a.chan[(long long)b * a.chan_stride], nch);
            __syncthreads();
            if (threadIdx.x == 0) {  // the channel ranges of each component
                for (int k = 0; k < GF_MAX_COMP; ++k) {
                    shape_c[k] = -1;
                    d0[k] = d1[k] = 0;
                    dbdn_c[k] = 0.0f;
                }
                for (int c = nch - 1; c >= 0; --c) {
                    const int k = chs[c].comp;
                    if (chs[c].type == CH_SHAPE) shape_c[k] = c;
                    if (chs[c].type == CH_DERIV) {
                        if (d1[k] == 0) d1[k] = c + 1;
                        d0[k] = c;
                        dbdn_c[k] = chs[c].dbdn;
                    }
                }
            }
            __syncthreads();
            cur_b = b;
        }
        const int npix = st.He * st.We;
        const int pix = (blk - pre[li]) * MODEL_THREADS + threadIdx.x;
        bool write = pix < npix;
        int i = 0, j = 0;
        if (write) {
            const int ie = div_mag(pix, st.We, mag), je = pix - ie * st.We;
            i = ie - st.c;
            j = je - st.c;
            write = !(st.os_factor > 1 && i >= st.os_y0 && i < st.os_y0 + st.os_box &&
                      j >= st.os_x0 && j < st.os_x0 + st.os_box);
        }
        if (write) {
            float* E = a.ext + ext_index(st, nch, 0) + pix;
            const long long cs = (long long)st.He * st.We;
            const Channel& c0 = chs[0];
            for (int k = 0; k < c0.ncomp; ++k) {
                if (is_sky_kind(c0.cc[k].kind)) continue;
                float g[8];
                const float v = comp_grad(c0.cc[k], (float)j, (float)i, 0.0f, 0.0f, dbdn_c[k], g);
                if (shape_c[k] >= 0) E[shape_c[k] * cs] = v;
                for (int c = d0[k]; c < d1[k]; ++c)
                    E[c * cs] = grad_pick(g, chs[c].dslot) * chs[c].scale;
            }
            for (int c = 0; c < nch; ++c)  // a sky plane's slope bases
                if (chs[c].type == CH_PLANE)
                    E[c * cs] = chs[c].dslot == 0 ? (float)j - chs[c].pxc : (float)i - chs[c].pyc;
        }
        if (a.work) {
            const int cnt = __syncthreads_count(write);
            if (threadIdx.x == 0)
                atomicAdd(&a.work[PROF_MODEL], 4ull * (unsigned long long)cnt * (unsigned long long)nch);
        }
    }
}

// Work item = OS_WARPS pixels of a listed stamp's oversampling block (all
// channels) for blocks of at most 32 sub-samples (os_factor <= 5): one
// sub-sample per lane, the components at p once, then a runtime loop over the
// channels, each reduced across the lanes as soon as it is evaluated.  Kept apart
// from the general body below, whose per-lane accumulators for every channel
// would otherwise set this one's register count (and occupancy) too.
template <int EV>
__device__ __forceinline__ void body_model_os_jac32(const PassArgs& a, int vb, int vg)
{
    __shared__ __align__(16) Channel chs[GF_MAX_CHAN];
    __shared__ int lvl[GF_MAX_CHAN];  // finite-difference reuse level per channel
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_OS * (a.count + 1);
    const int tot = pre[n];
    const int nch = a.nchan;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int hint = -1, cur_b = -1;
    const int chunk = (tot + vg - 1) / vg;
    const int it0 = vb * chunk, it1 = min(tot, it0 + chunk);
    for (int blk = it0; blk < it1; ++blk) {
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        const StampInfo st = a.st[b];
        if (b != cur_b) {
            __syncthreads();
            load_channels(chs, &a.chan[(long long)b * a.chan_stride], nch);
            __syncthreads();
            fd_levels(chs, nch, lvl);
            cur_b = b;
        }
        const int q = (blk - pre[li]) * OS_WARPS + warp;
        const int B = st.os_box;
        if (q >= B * B) continue;
        const int i = st.os_y0 + q / B, j = st.os_x0 + q % B;
        const int s = st.os_factor, ns = s * s;
        const float fs = (float)s;
        const long long pix = (long long)(i + st.c) * st.We + (j + st.c);
        const long long cs = (long long)st.He * st.We;
        float* E = a.ext + ext_index(st, nch, 0) + pix;
        const bool on = lane < ns;
        float ox = 0.0f, oy = 0.0f;
        if (on) {
            const int ay = lane / s, bx = lane - ay * s;
            oy = ((float)ay + 0.5f) / fs - 0.5f;
            ox = ((float)bx + 0.5f) / fs - 0.5f;
        }
        EvalCursor e;
        e.comp = -1;
        for (int c = 0; c < nch; ++c) {
            // (the same sums, in the same order, as the general body's)
            float v = on ? jac_value<EV>(chs, c, lvl[c], e, (float)j, (float)i, ox, oy) : 0.0f;
            v += 0.0f;  // an idle lane adds +0, as the general body's accumulator
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) E[c * cs] = v / (float)ns;
        }
        if (a.work && lane == 0) atomicAdd(&a.work[PROF_MODEL], 4ull * (unsigned long long)nch);
    }
}

// Work item = OS_WARPS pixels of a listed stamp's oversampling block (all
// channels), any block size: lanes take sub-samples, each lane keeps every
// channel's sum.
template <int EV>
__device__ __forceinline__ void body_model_os_jac(const PassArgs& a, int vb, int vg)
{
    __shared__ __align__(16) Channel chs[GF_MAX_CHAN];
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_OS * (a.count + 1);
    const int tot = pre[n];
    const int nch = a.nchan;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int hint = -1, cur_b = -1;
    const int chunk = (tot + vg - 1) / vg;
    const int it0 = vb * chunk, it1 = min(tot, it0 + chunk);
    for (int blk = it0; blk < it1; ++blk) {
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        const StampInfo st = a.st[b];
        if (b != cur_b) {
            __syncthreads();
            load_channels(chs, &a.chan[(long long)b * a.chan_stride], nch);
            __syncthreads();
            cur_b = b;
        }
        const int q = (blk - pre[li]) * OS_WARPS + warp;
        const int B = st.os_box;
        if (q >= B * B) continue;
        const int i = st.os_y0 + q / B, j = st.os_x0 + q % B;
        const int s = st.os_factor, ns = s * s;
        const float fs = (float)s;
        const long long pix = (long long)(i + st.c) * st.We + (j + st.c);
        const long long cs = (long long)st.He * st.We;
        float* E = a.ext + ext_index(st, nch, 0) + pix;
        float acc[GF_MAX_CHAN];
#pragma unroll
        for (int c = 0; c < GF_MAX_CHAN; ++c) acc[c] = 0.0f;
        for (int t = lane; t < ns; t += 32) {
            const int ay = t / s, bx = t - ay * s;
            const float oy = ((float)ay + 0.5f) / fs - 0.5f;
            const float ox = ((float)bx + 0.5f) / fs - 0.5f;
            float base[GF_MAX_COMP];
            comp_base<EV>(chs[0], base, (float)j, (float)i, ox, oy);
#pragma unroll
            for (int c = 0; c < GF_MAX_CHAN; ++c)
                if (c < nch) acc[c] += jac_channel<EV>(chs[c], base, (float)j, (float)i, ox, oy);
        }
#pragma unroll
        for (int c = 0; c < GF_MAX_CHAN; ++c) {
            if (c >= nch) break;
            float v = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) E[c * cs] = v / (float)ns;
        }
        if (a.work && lane == 0) atomicAdd(&a.work[PROF_MODEL], 4ull * (unsigned long long)nch);
    }
}

// The oversampled blocks of an analytic Jacobian pass, all channels per warp:
// per sub-sample each component's value and gradient once (comp_grad), then
// every channel of that component takes its entry.
template <int EV>
__device__ __forceinline__ void body_model_os_jac_an(const PassArgs& a, int vb, int vg)
{
    __shared__ __align__(16) Channel chs[GF_MAX_CHAN];
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_OS * (a.count + 1);
    const int tot = pre[n];
    const int nch = a.nchan;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int hint = -1, cur_b = -1;
    const int chunk = (tot + vg - 1) / vg;
    const int it0 = vb * chunk, it1 = min(tot, it0 + chunk);
    for (int blk = it0; blk < it1; ++blk) {
        const int li = wl_locate(pre, n, blk, hint);
        const int b = a.wl.ids[li];
        const StampInfo st = a.st[b];
        if (b != cur_b) {
            __syncthreads();
            load_channels(chs, &a.chan[(long long)b * a.chan_stride], nch);
            __syncthreads();
            cur_b = b;
        }
        const int q = (blk - pre[li]) * OS_WARPS + warp;
        const int B = st.os_box;
        if (q >= B * B) continue;
        const int i = st.os_y0 + q / B, j = st.os_x0 + q % B;
        const int s = st.os_factor, ns = s * s;
        const float fs = (float)s;
        float acc[GF_MAX_CHAN];
#pragma unroll
        for (int c = 0; c < GF_MAX_CHAN; ++c) acc[c] = 0.0f;
        const Channel& c0 = chs[0];
        for (int t = lane; t < ns; t += 32) {
            const int ay = t / s, bx = t - ay * s;
            const float oy = ((float)ay + 0.5f) / fs - 0.5f;
            const float ox = ((float)bx + 0.5f) / fs - 0.5f;
            for (int k = 0; k < c0.ncomp; ++k) {
                if (is_sky_kind(c0.cc[k].kind)) continue;
                float dbdn = 0.0f;
                for (int c = 0; c < nch; ++c)
                    if (chs[c].comp == k && chs[c].type == CH_DERIV) dbdn = chs[c].dbdn;
                float g[8];
                const float v = comp_grad(c0.cc[k], (float)j, (float)i, ox, oy, dbdn, g);
#pragma unroll
                for (int c = 0; c < GF_MAX_CHAN; ++c) {
                    if (c < nch && chs[c].comp == k)
                        acc[c] += chs[c].type == CH_SHAPE ? v
                                                          : grad_pick(g, chs[c].dslot) * chs[c].scale;
                }
            }
#pragma unroll
            for (int c = 0; c < GF_MAX_CHAN; ++c)  // a sky plane's slope bases (pixel centre)
                if (c < nch && chs[c].type == CH_PLANE)
                    acc[c] += chs[c].dslot == 0 ? (float)j - chs[c].pxc : (float)i - chs[c].pyc;
        }
        const long long pix = (long long)(i + st.c) * st.We + (j + st.c);
        const long long cs = (long long)st.He * st.We;
        float* E = a.ext + ext_index(st, nch, 0) + pix;
#pragma unroll
        for (int c = 0; c < GF_MAX_CHAN; ++c) {
            if (c >= nch) break;
            float v = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) E[c * cs] = v / (float)ns;
        }
        if (a.work && lane == 0) atomicAdd(&a.work[PROF_MODEL], 4ull * (unsigned long long)nch);
    }
}

// One launch per pass for all of step 1: blocks [0, g_os) evaluate the
// oversampled blocks (the heavy items, scheduled first), the others the plain
// grid pixels, so that the two kinds of work overlap instead of running as two
// dependent launches.  PIX: 0 one channel per item, 1 every channel of a
// Jacobian pass per pixel, 2 the same with analytic derivative channels, 3 none
// (a launch of oversampled blocks alone).  OS: 0 none, 1 a warp per (channel,
// block pixel), 2 a warp per block pixel with every channel, 3 the same with
// analytic channels, 4 as 2 for blocks of at most 32 sub-samples.
// CTAs per SM the register budget is held to: four for the plain and the
// oversampled Jacobian passes (64 registers; the latter spills 8 bytes), five
// for the one-channel pass with its oversampled blocks (48 registers, 48 bytes
// spilled): measured faster than the counts their free allocation gives
template <int PIX, int OS, int EV>
constexpr int model_min_blocks()
{
    return (PIX == 1 && OS == 0 && EV <= 1) || (PIX == 3 && OS == 4 && EV <= 1) ? 4
           : (PIX == 0 && OS == 1 && EV == 0)                                   ? 5
                                                                                : 0;  // 0: no minimum
}

template <int PIX, int OS, int EV>
__global__ void __launch_bounds__(MODEL_THREADS, (model_min_blocks<PIX, OS, EV>())) k_model_pass(PassArgs a, int g_os)
{
    static_assert(MODEL_THREADS == OS_WARPS * 32, "one block size for both kinds of item");
    pdl_entry();
    if (OS != 0 && (int)blockIdx.x < g_os) {
        if (OS == 1)
            body_model_os<EV>(a, blockIdx.x, g_os);
        else if (OS == 2)
            body_model_os_jac<EV>(a, blockIdx.x, g_os);
        else if (OS == 3)
            body_model_os_jac_an<EV>(a, blockIdx.x, g_os);
        else
            body_model_os_jac32<EV>(a, blockIdx.x, g_os);
        return;
    }
    if (PIX == 3) return;
    const int vb = blockIdx.x - (OS != 0 ? g_os : 0), vg = gridDim.x - (OS != 0 ? g_os : 0);
    if (PIX == 0)
        body_model<EV>(a, vb, vg);
    else if (PIX == 1)
        body_model_jac<EV>(a, vb, vg);
    else
        body_model_jac_an<EV>(a, vb, vg);
}

template <int PIX, int OS>
cudaError_t launch_pass(const PassArgs& a, int g_pix, int g_os, cudaStream_t s)
{
    if (a.eval_variant == 2)
        GF_LAUNCH_PDL((k_model_pass<PIX, OS, 2>), dim3(g_pix + g_os), dim3(MODEL_THREADS), 0, s,
                      a, g_os);
    else if (a.eval_variant == 1)
        GF_LAUNCH_PDL((k_model_pass<PIX, OS, 1>), dim3(g_pix + g_os), dim3(MODEL_THREADS), 0, s,
                      a, g_os);
    else
        GF_LAUNCH_PDL((k_model_pass<PIX, OS, 0>), dim3(g_pix + g_os), dim3(MODEL_THREADS), 0,
                      s, a, g_os);
    GF_COUNT_LAUNCH();
    return cudaSuccess;
}

}  // namespace

// The oversampled blocks share the plain pixels' launch when they are few (one
// large stamp: the two kinds of work then overlap); many of them (batches of
// stamps) take a launch of their own, so that the plain pixels keep the lower
// register count and full occupancy.
constexpr long long MERGE_OS_MAX = 152LL * 8;

cudaError_t launch_model(const PassArgs& a, cudaStream_t s)
{
    cudaError_t e;
    if (a.jac_pass && a.nchan > 1) {  // a Jacobian pass: all channels of a pixel together
        const int cap[2] = {152 * 16, 152 * 8};
        const int g_pix = a.maxitems[WK_MODEL] > 0
                              ? std::max(1, (int)std::min<long long>(a.maxitems[WK_MODEL] / a.nchan, cap[0]))
                              : 0;
        // the oversampled blocks: all channels per warp when there are enough
        // block pixels to fill the GPU (many stamps), else a warp per channel
        // and pixel (one large stamp)
        const long long os_groups = a.maxitems[WK_OS] / a.nchan;
        const int g_os2 = std::max(1, (int)std::min<long long>(os_groups, cap[1]));
        if (a.jac_analytic) {
            if (os_groups * OS_WARPS >= 152LL * 32) {
                if (g_pix > 0 && (e = launch_pass<2, 0>(a, g_pix, 0, s)) != cudaSuccess) return e;
                return launch_pass<3, 3>(a, 0, g_os2, s);
            }
            if (a.maxitems[WK_OS] == 0) return g_pix > 0 ? launch_pass<2, 0>(a, g_pix, 0, s) : cudaSuccess;
            if (a.grid[WK_OS] <= MERGE_OS_MAX) return launch_pass<2, 1>(a, g_pix, a.grid[WK_OS], s);
            if (g_pix > 0 && (e = launch_pass<2, 0>(a, g_pix, 0, s)) != cudaSuccess) return e;
            return launch_pass<0, 1>(a, 0, a.grid[WK_OS], s);
        }
        if (os_groups * OS_WARPS >= 152LL * 32) {
            if (g_pix > 0 && (e = launch_pass<1, 0>(a, g_pix, 0, s)) != cudaSuccess) return e;
            return a.os_ns <= 32 ? launch_pass<3, 4>(a, 0, g_os2, s) : launch_pass<3, 2>(a, 0, g_os2, s);
        }
        if (a.maxitems[WK_OS] == 0) return g_pix > 0 ? launch_pass<1, 0>(a, g_pix, 0, s) : cudaSuccess;
        if (a.grid[WK_OS] <= MERGE_OS_MAX) return launch_pass<1, 1>(a, g_pix, a.grid[WK_OS], s);
        if (g_pix > 0 && (e = launch_pass<1, 0>(a, g_pix, 0, s)) != cudaSuccess) return e;
        return launch_pass<0, 1>(a, 0, a.grid[WK_OS], s);
    }
    const int g_pix = a.maxitems[WK_MODEL] > 0 ? a.grid[WK_MODEL] : 0;
    if (a.maxitems[WK_OS] == 0) return g_pix > 0 ? launch_pass<0, 0>(a, g_pix, 0, s) : cudaSuccess;
    if (a.grid[WK_OS] <= MERGE_OS_MAX) return launch_pass<0, 1>(a, g_pix, a.grid[WK_OS], s);
    if (g_pix > 0 && (e = launch_pass<0, 0>(a, g_pix, 0, s)) != cudaSuccess) return e;
    return launch_pass<0, 1>(a, 0, a.grid[WK_OS], s);
}
