// reduce.cu -- step 3 of the fitting loop (Sec. 2 item 3; Sec. 3 item 3,
// transform + reduce) and the normal equations of step 4.
//
// Per pixel (a transform): the model m = sum_ch mweight_ch Y_ch + msky, the
// residual r = d - m, the weight 1/sigma^2 on valid pixels (finite d and sigma,
// sigma > 0), and the Jacobian columns (convolved channels; sum(psf) for the
// sky).  Then the reduce:
//   chi^2 = sum (r/sigma)^2,  A_ij = sum w J_i J_j,  g_i = sum w J_i r.
// All sums are compensated float32 (Neumaier per thread, error-free TwoSum when
// partial sums merge) in a fixed order, so results are deterministic.
//
// Two stages: each block of 256 threads reduces RED_PIX = 1024 pixels of one
// stamp into `nacc` partials; a final kernel, one block per stamp, sums the
// partials of the stamp in block order.
#include <math.h>

#include <algorithm>

#include "gf_internal.cuh"

namespace {

struct ChanInfo {
    float mw[GF_MAX_CHAN];
    int jc[GF_MAX_CHAN];
};

__device__ __forceinline__ void load_chan_info(ChanInfo& ci, float& msky, const PassArgs& a,
                                               int b)
{
    const Channel* c = a.chan + (long long)b * a.chan_stride;
    if (threadIdx.x < a.nchan) {
        ci.mw[threadIdx.x] = c[threadIdx.x].mweight;
        ci.jc[threadIdx.x] = c[threadIdx.x].jcol;
    }
    if (threadIdx.x == 0) msky = c[0].msky;
}

// The normal equations as one bordered matrix: with v = (J_0 .. J_{nf-1}, r)
// per pixel and weight w, M = sum w v v^T holds A (i, j < nf), g (j = nf) and
// chi^2 (i = j = nf).  Its upper triangle is covered by T = nt (nt + 1) / 2
// tiles of 4 x 4 (nt = ceil((nf + 1) / 4)).  The pixels of each 256-pixel chunk
// are split into G = 256 / T contiguous groups, and thread (group, tile) with
// tid = group T + tile sums its tile over its group's pixels (two 16-byte
// shared loads feed 16 FMAs), so every thread but 256 - G T has a tile.  Sums
// over a group's pixels are plain float32; they are added to the thread's
// compensated totals, and the G groups of a tile are merged in group order, so
// the partials are deterministic.
constexpr int VSTR = 20;  // row stride of the staged pixel vectors: >= 4 nt for nf <= 19
static_assert(GF_MAX_FREE + 1 <= VSTR, "bordered vector longer than the staged row");
constexpr int RSTR = 17;  // row stride of the per-thread tile sums (odd: the 16 stores of a
                          // thread's row land in distinct banks across the warp)

// PF > 0 (passes of at most PF channels): each thread loads its next chunk's
// image, sigma and channel values into registers before the current chunk's
// tile sums, so the loads of one chunk overlap the arithmetic of the last; and
// three CTAs share an SM (80 registers, a few spilled, against 121 for two).
// The values and the order of every sum are the same either way.
// TS: the tile side, 4 or 3.  Both cover the bordered matrix with the same
// number of tiles per side where the host picks 3 (ceil(nv/3) = ceil(nv/4),
// e.g. nv = 9), so the groups and every entry's sums are the same and only
// fewer padded products are formed.
template <int PF, int TS>
__global__ void __launch_bounds__(RED_THREADS, PF > 0 ? 3 : 2) k_reduce_jac(PassArgs a)
{
    pdl_entry();
    __shared__ __align__(16) float V[RED_THREADS][VSTR];  // pixel vectors v = (J, r)
    __shared__ float Wt[RED_THREADS];                     // weights 1/sigma^2
    __shared__ ChanInfo ci;
    __shared__ float msky;
    __shared__ float red[RED_THREADS][RSTR];  // per (group, tile), its TS x TS sums
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_RED * (a.count + 1);
    const int tot = pre[n];
    const int nf = a.S->nfree, skyc = a.S->sky_jcol;
    const int nv = nf + 1;                 // bordered size
    const int nt = (nv + TS - 1) / TS;     // tiles per side
    int hint = -1;
    const int chunk = (tot + gridDim.x - 1) / gridDim.x;
    const int it0 = blockIdx.x * chunk, it1 = min(tot, it0 + chunk);
    for (int it = it0; it < it1; ++it) {
    const int li = wl_locate(pre, n, it, hint);
    const int b = a.wl.ids[li];
    const int local = it - pre[li];
    const int blk = a.pre_static[WK_RED * (a.count + 1) + b] + local;  // partial slot
    const StampInfo st = a.st[b];
    __syncthreads();  // the previous item is done with the shared arrays
    load_chan_info(ci, msky, a, b);
    __syncthreads();
    const float psum = a.psf_sum[b];
    const long long HW = (long long)st.H * st.W;
    const float* img = a.img + st.pix_off;
    const float* sig = a.sig + st.pix_off;
    const float* Y = a.y + y_index(st, a.nchan, 0);
    const int tid = threadIdx.x;
    // this thread's tile (upper triangle, row-major over tile pairs) and group
    const int T = nt * (nt + 1) / 2, G = RED_THREADS / T;
    const int tslot = tid % T, grp = tid / T;
    int ti = 0, tj = 0;
    {
        int k = 0;
        for (int I = 0; I < nt; ++I)
            for (int J = I; J < nt; ++J, ++k)
                if (k == tslot) {
                    ti = I;
                    tj = J;
                }
    }
    const bool active_tile = grp < G;
    const int pg0 = grp * RED_THREADS / G, pg1 = (grp + 1) * RED_THREADS / G;  // the group's pixels
    CSum acc[TS][TS];
#pragma unroll
    for (int x = 0; x < TS; ++x)
#pragma unroll
        for (int y = 0; y < TS; ++y) acc[x][y] = CSum{0.0f, 0.0f};
    const long long base = (long long)local * RED_PIX;
    constexpr int NPF = PF > 0 ? PF : 1;
    float nd = 0.0f, ns = 0.0f, ny[NPF];  // the next chunk's pixel (PF > 0)
    auto fetch = [&](int q) {
        const long long px = base + (long long)q * RED_THREADS + tid;
        if (px < HW) {
            nd = img[px];
            ns = sig[px];
#pragma unroll
            for (int k = 0; k < NPF; ++k)
                if (k < a.nchan) ny[k] = Y[(long long)k * HW + px];
        }
    };
    if (PF > 0) fetch(0);
    for (int q = 0; q < RED_CHUNKS; ++q) {
        const long long px = base + (long long)q * RED_THREADS + tid;
        if (px < HW) {
            const float d = PF > 0 ? nd : img[px], s = PF > 0 ? ns : sig[px];
            const bool valid = isfinite(d) && isfinite(s) && s > 0.0f;
            float m = msky;
            if (PF > 0) {
#pragma unroll
                for (int k = 0; k < NPF; ++k) {
                    if (k >= a.nchan) break;
                    const float yk = ny[k];
                    if (ci.mw[k] != 0.0f) m = fmaf(ci.mw[k], yk, m);
                    if (ci.jc[k] >= 0) V[tid][ci.jc[k]] = yk;
                }
            } else {
                for (int k = 0; k < a.nchan; ++k) {
                    const float yk = Y[(long long)k * HW + px];
                    if (ci.mw[k] != 0.0f) m = fmaf(ci.mw[k], yk, m);
                    if (ci.jc[k] >= 0) V[tid][ci.jc[k]] = yk;
                }
            }
            if (skyc >= 0) V[tid][skyc] = psum;
            V[tid][nf] = valid ? d - m : 0.0f;
            Wt[tid] = valid ? 1.0f / (s * s) : 0.0f;
            if (a.m_out) a.m_out[st.pix_off + px] = m;
            if (a.J_out)
                for (int f = 0; f < nf; ++f) a.J_out[(long long)f * HW + px] = V[tid][f];
        } else {
            for (int f = 0; f < nv; ++f) V[tid][f] = 0.0f;
            Wt[tid] = 0.0f;
        }
        for (int f = nv; f < VSTR; ++f) V[tid][f] = 0.0f;
        if (PF > 0 && q + 1 < RED_CHUNKS) fetch(q + 1);
        __syncthreads();
        if (active_tile) {
            float sum[TS][TS];
#pragma unroll
            for (int x = 0; x < TS; ++x)
#pragma unroll
                for (int y = 0; y < TS; ++y) sum[x][y] = 0.0f;
            const int i0 = TS * ti, j0 = TS * tj;
            for (int p = pg0; p < pg1; ++p) {
                const float w = Wt[p];
                float vi[TS], vj[TS];
                if constexpr (TS == 4) {
                    const float4 a4 = *reinterpret_cast<const float4*>(&V[p][i0]);
                    const float4 b4 = *reinterpret_cast<const float4*>(&V[p][j0]);
                    vi[0] = w * a4.x, vi[1] = w * a4.y, vi[2] = w * a4.z, vi[3] = w * a4.w;
                    vj[0] = b4.x, vj[1] = b4.y, vj[2] = b4.z, vj[3] = b4.w;
                } else {
#pragma unroll
                    for (int x = 0; x < TS; ++x) {
                        vi[x] = w * V[p][i0 + x];
                        vj[x] = V[p][j0 + x];
                    }
                }
#pragma unroll
                for (int x = 0; x < TS; ++x)
#pragma unroll
                    for (int y = 0; y < TS; ++y) sum[x][y] = fmaf(vi[x], vj[y], sum[x][y]);
            }
#pragma unroll
            for (int x = 0; x < TS; ++x)
#pragma unroll
                for (int y = 0; y < TS; ++y) csum_add(acc[x][y], sum[x][y]);
        }
        __syncthreads();
    }
    // merge the G groups of each tile in group order, then write the partials
    // in the accumulator order of decode_acc (A pairs, g, chi^2)
    if (active_tile)
#pragma unroll
        for (int x = 0; x < TS; ++x)
#pragma unroll
            for (int y = 0; y < TS; ++y) red[tid][x * TS + y] = acc[x][y].s + acc[x][y].c;
    __syncthreads();
    for (int t = tid; t < a.nacc; t += RED_THREADS) {
        int i, j;
        const int kind = decode_acc(t, nf, i, j);
        int r_, c_;
        if (kind == 0) {
            r_ = i;
            c_ = j;
        } else if (kind == 1) {
            r_ = i;
            c_ = nf;
        } else {
            r_ = nf;
            c_ = nf;
        }
        const int I = r_ / TS, J = c_ / TS;
        int slot = 0;
        for (int II = 0; II < I; ++II) slot += nt - II;
        slot += J - I;
        CSum tot = {0.0f, 0.0f};
        for (int gq = 0; gq < G; ++gq) csum_add(tot, red[gq * T + slot][(r_ % TS) * TS + (c_ % TS)]);
        a.partial[(long long)blk * a.nacc + t] = tot.s + tot.c;
    }
    if (a.work && tid == 0) {
        const long long np = min((long long)RED_PIX, HW - base);
        atomicAdd(&a.work[PROF_REDUCE], (unsigned long long)np * (4ull * a.nchan + 8ull));
    }
    }
}

// Where the chi^2 pass's current item sits: its stamp, the stamp's offsets and
// the end of the stamp's item range, kept in registers so that the next item of
// the same stamp is found without the dependent loads of the work-list search.
struct Chi2Loc {
    int b, end, blk0, local;
    long long HW, pix_off, yoff;
};

__device__ __forceinline__ void chi2_locate(Chi2Loc& L, const PassArgs& a, const int* pre, int n,
                                            int it, int& hint)
{
    const int li = wl_locate(pre, n, it, hint);
    L.b = a.wl.ids[li];
    L.end = pre[li + 1];
    L.local = it - pre[li];
    L.blk0 = a.pre_static[WK_RED * (a.count + 1) + L.b];
    const StampInfo& st = a.st[L.b];
    L.HW = (long long)st.H * st.W;
    L.pix_off = st.pix_off;
    L.yoff = y_index(st, a.nchan, 0);
}

// the item after L's, in the work list's order
__device__ __forceinline__ void chi2_advance(Chi2Loc& L, const PassArgs& a, const int* pre, int n,
                                             int it, int& hint)
{
    if (it < L.end)
        ++L.local;
    else
        chi2_locate(L, a, pre, n, it, hint);
}

// The values one thread reads for one item: RED_CHUNKS consecutive pixels
// base + RED_CHUNKS t + e of the image, sigma and model.  Where the stamp's
// arrays are 16-byte aligned and its pixel count a multiple of 4 they come in
// one 16-byte load each; otherwise by single loads.  The values are not used
// here, so the loads stay in flight while the caller finishes the previous
// item.
struct Chi2Vals {
    float m[RED_CHUNKS], dv[RED_CHUNKS], sv[RED_CHUNKS];
};

__device__ __forceinline__ void chi2_fetch(Chi2Vals& q, const Chi2Loc& L, const PassArgs& a)
{
    const long long p0 = (long long)L.local * RED_PIX + (long long)RED_CHUNKS * threadIdx.x;
    const float* Y = a.y + L.yoff;
    const float* img = a.img + L.pix_off;
    const float* sig = a.sig + L.pix_off;
    const bool has_img = a.img != nullptr;
    const bool vec = ((L.pix_off | L.HW | L.yoff) & 3) == 0 && p0 < L.HW;
    if (vec) {
        const float4 y4 = __ldg(reinterpret_cast<const float4*>(Y + p0));
        q.m[0] = y4.x; q.m[1] = y4.y; q.m[2] = y4.z; q.m[3] = y4.w;
        if (has_img) {
            const float4 d4 = __ldg(reinterpret_cast<const float4*>(img + p0));
            const float4 s4 = __ldg(reinterpret_cast<const float4*>(sig + p0));
            q.dv[0] = d4.x; q.dv[1] = d4.y; q.dv[2] = d4.z; q.dv[3] = d4.w;
            q.sv[0] = s4.x; q.sv[1] = s4.y; q.sv[2] = s4.z; q.sv[3] = s4.w;
        } else {
#pragma unroll
            for (int e = 0; e < RED_CHUNKS; ++e) q.dv[e] = q.sv[e] = 0.0f;
        }
    } else {
#pragma unroll
        for (int e = 0; e < RED_CHUNKS; ++e) {
            const long long px = p0 + e;
            const bool in = px < L.HW;
            q.m[e] = in ? __ldg(&Y[px]) : 0.0f;
            q.dv[e] = (in && has_img) ? __ldg(&img[px]) : 0.0f;
            q.sv[e] = (in && has_img) ? __ldg(&sig[px]) : 0.0f;
        }
    }
}

// chi^2 partials, one per work item of RED_PIX pixels.  A block walks its
// contiguous range of items with the loads of item i + 1 issued before the
// reduction tree of item i, so the tree, its barrier and the partial's store
// hide under the next item's memory latency.  Each item is summed in the same
// per-thread order and the same tree whatever its neighbours, so a stamp's
// chi^2 does not depend on the batch around it.
__global__ void __launch_bounds__(RED_THREADS, 4) k_reduce_chi2(PassArgs a)
{
    pdl_entry();
    __shared__ CSum wsum[2][RED_THREADS / 32];  // by item parity: one barrier per item
    static_assert(RED_CHUNKS == 4, "one float4 per thread and array");
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_RED * (a.count + 1);
    const int tot = pre[n];
    int hint = -1;
    const int chunk = (tot + gridDim.x - 1) / gridDim.x;
    const int it0 = blockIdx.x * chunk, it1 = min(tot, it0 + chunk);
    const bool has_img = a.img != nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (it0 >= it1) return;
    Chi2Loc cl, nl;
    Chi2Vals cv, nv;
    chi2_locate(cl, a, pre, n, it0, hint);
    chi2_fetch(cv, cl, a);
    for (int it = it0; it < it1; ++it) {
        nl = cl;
        if (it + 1 < it1) {
            chi2_advance(nl, a, pre, n, it + 1, hint);
            chi2_fetch(nv, nl, a);
        }
        const long long p0 = (long long)cl.local * RED_PIX + (long long)RED_CHUNKS * threadIdx.x;
        // the model: channel weights of this stamp (read through the cache;
        // every thread of the block reads the same words)
        const Channel* ch = a.chan + (long long)cl.b * a.chan_stride;
        const float msky = ch[0].msky, mw0 = ch[0].mweight;
        float m[RED_CHUNKS];
#pragma unroll
        for (int e = 0; e < RED_CHUNKS; ++e) m[e] = fmaf(mw0, cv.m[e], msky);
        if (a.nchan > 1) {
            const float* Y = a.y + cl.yoff;
#pragma unroll
            for (int e = 0; e < RED_CHUNKS; ++e) {
                const long long px = p0 + e;
                for (int k = 1; k < a.nchan; ++k)
                    if (px < cl.HW) m[e] = fmaf(ch[k].mweight, Y[(long long)k * cl.HW + px], m[e]);
            }
        }
        float* m_out = a.m_out ? a.m_out + cl.pix_off : nullptr;
        CSum acc = {0.0f, 0.0f};
#pragma unroll
        for (int e = 0; e < RED_CHUNKS; ++e) {
            const long long px = p0 + e;
            if (px >= cl.HW) break;
            if (m_out) m_out[px] = m[e];
            if (!has_img) continue;  // model only
            const float d = cv.dv[e], s = cv.sv[e];
            if (isfinite(d) && isfinite(s) && s > 0.0f) {
                const float z = (d - m[e]) / s;
                csum_add(acc, z * z);
            }
        }
        // deterministic shuffle tree, then across warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            CSum other;
            other.s = __shfl_down_sync(0xffffffffu, acc.s, o);
            other.c = __shfl_down_sync(0xffffffffu, acc.c, o);
            acc = csum_merge(acc, other);
        }
        CSum* ws = wsum[it & 1];
        if (lane == 0) ws[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            CSum t = ws[0];
            for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, ws[w]);
            a.partial[cl.blk0 + cl.local] = t.s + t.c;
            if (a.work) {
                const long long np = min((long long)RED_PIX, cl.HW - (long long)cl.local * RED_PIX);
                atomicAdd(&a.work[PROF_REDUCE], (unsigned long long)np * (4ull * a.nchan + 8ull));
            }
        }
        cl = nl;
        cv = nv;
    }
}

// The trial pass of an LM body evaluates the rungs of the trial ladder (one
// channel each, each its own model): per work item and channel k, the chi^2
// partial of channel k goes to partial[item * nchan + k].  Each channel is
// summed exactly as k_reduce_chi2 sums a one-channel pass (same per-thread
// order, same tree), so a rung's chi^2 does not depend on the other rungs.
__global__ void __launch_bounds__(RED_THREADS) k_reduce_rungs(PassArgs a)
{
    pdl_entry();
    __shared__ ChanInfo ci;
    __shared__ float mskys[GF_MAX_LADDER];
    __shared__ CSum wsum[GF_MAX_LADDER][RED_THREADS / 32];
    const int n = *a.wl.n;
    const int* pre = a.wl.pre + WK_RED * (a.count + 1);
    const int tot = pre[n];
    const int nch = a.nchan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int hint = -1;
    const int chunk = (tot + gridDim.x - 1) / gridDim.x;
    const int it0 = blockIdx.x * chunk, it1 = min(tot, it0 + chunk);
    for (int it = it0; it < it1; ++it) {
        const int li = wl_locate(pre, n, it, hint);
        const int b = a.wl.ids[li];
        const int local = it - pre[li];
        const int blk = a.pre_static[WK_RED * (a.count + 1) + b] + local;  // partial slot
        const StampInfo st = a.st[b];
        __syncthreads();
        {
            const Channel* c = a.chan + (long long)b * a.chan_stride;
            if (threadIdx.x < nch) {
                ci.mw[threadIdx.x] = c[threadIdx.x].mweight;
                mskys[threadIdx.x] = c[threadIdx.x].msky;
            }
        }
        __syncthreads();
        const long long HW = (long long)st.H * st.W;
        const float* img = a.img + st.pix_off;
        const float* sig = a.sig + st.pix_off;
        const long long base = (long long)local * RED_PIX;
        float dv[RED_CHUNKS], sv[RED_CHUNKS];
#pragma unroll
        for (int q = 0; q < RED_CHUNKS; ++q) {
            const long long px = base + (long long)q * RED_THREADS + threadIdx.x;
            const bool in = px < HW;
            dv[q] = in ? __ldg(&img[px]) : 0.0f;
            sv[q] = in ? __ldg(&sig[px]) : 0.0f;
        }
        for (int k = 0; k < nch; ++k) {
            const float* Y = a.y + y_index(st, nch, k);
            float m[RED_CHUNKS];
#pragma unroll
            for (int q = 0; q < RED_CHUNKS; ++q) {
                const long long px = base + (long long)q * RED_THREADS + threadIdx.x;
                m[q] = px < HW ? __ldg(&Y[px]) : 0.0f;
            }
            CSum acc = {0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < RED_CHUNKS; ++q) {
                const long long px = base + (long long)q * RED_THREADS + threadIdx.x;
                if (px >= HW) break;
                const float mq = fmaf(ci.mw[k], m[q], mskys[k]);
                const float d = dv[q], s = sv[q];
                if (isfinite(d) && isfinite(s) && s > 0.0f) {
                    const float z = (d - mq) / s;
                    csum_add(acc, z * z);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                CSum other;
                other.s = __shfl_down_sync(0xffffffffu, acc.s, o);
                other.c = __shfl_down_sync(0xffffffffu, acc.c, o);
                acc = csum_merge(acc, other);
            }
            if (lane == 0) wsum[k][warp] = acc;
        }
        __syncthreads();
        if (threadIdx.x < nch) {
            const int k = threadIdx.x;
            CSum t = wsum[k][0];
            for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, wsum[k][w]);
            a.partial[(long long)blk * nch + k] = t.s + t.c;
        }
        if (a.work && threadIdx.x == 0) {
            const long long np = min((long long)RED_PIX, HW - base);
            atomicAdd(&a.work[PROF_REDUCE], (unsigned long long)np * (4ull * nch + 8ull));
        }
    }
}

// one block per stamp: sum the stamp's partials in block order
// Final sums of the Jacobian pass.  Block (stamp b, group y) owns accumulators
// 32y .. 32y + 31, one per lane, so each warp reads whole 128-byte rows of the
// partials; the warps split the stamp's partials into nseg interleaved
// segments (nseg from the stamp's own partial count, so a stamp is summed in
// the same order in any batch), merged in segment order.  Writes A, g and chi^2
// into the stamp's LM state, or into A_out, g_out, chi2_out.
constexpr int FINAL_SEG_MAX = 16;

__host__ __device__ __forceinline__ int final_nseg(int nred)
{
    return nred / 4 < 1 ? 1 : (nred / 4 > FINAL_SEG_MAX ? FINAL_SEG_MAX : nred / 4);
}

__global__ void __launch_bounds__(32 * FINAL_SEG_MAX) k_final_jac(PassArgs a, double* A_out,
                                                                  double* g_out, double* chi2_out)
{
    pdl_entry();
    __shared__ CSum part[FINAL_SEG_MAX][32];
    const int b = blockIdx.x;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const int nacc = a.nacc, lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int t = blockIdx.y * 32 + lane;
    const int* pst = a.pre_static + WK_RED * (a.count + 1);
    const int b0 = pst[b], b1 = pst[b + 1];
    const int nseg = final_nseg(b1 - b0);
    CSum acc = {0.0f, 0.0f};
    if (t < nacc && seg < nseg) {
        const float* src = a.partial + t;
        int k = b0 + seg;
        for (; k + 3 * nseg < b1; k += 4 * nseg) {
            const float v0 = src[(long long)k * nacc];
            const float v1 = src[(long long)(k + nseg) * nacc];
            const float v2 = src[(long long)(k + 2 * nseg) * nacc];
            const float v3 = src[(long long)(k + 3 * nseg) * nacc];
            csum_add(acc, v0);
            csum_add(acc, v1);
            csum_add(acc, v2);
            csum_add(acc, v3);
        }
        for (; k < b1; k += nseg) csum_add(acc, src[(long long)k * nacc]);
    }
    part[seg][lane] = acc;
    __syncthreads();
    if (seg != 0 || t >= nacc) return;
    CSum tot = part[0][lane];
    for (int q = 1; q < nseg; ++q) tot = csum_merge(tot, part[q][lane]);
    const double v = (double)tot.s + (double)tot.c;
    const int nf = a.S->nfree;
    int i, j;
    const int kind = decode_acc(t, nf, i, j);
    double* A = a.lm ? a.lm[b].A : A_out + (long long)b * nf * nf;
    double* g = a.lm ? a.lm[b].g : g_out + (long long)b * nf;
    if (kind == 0) {
        A[i * nf + j] = v;
        A[j * nf + i] = v;
    } else if (kind == 1) {
        g[i] = v;
    } else {
        if (a.lm)
            a.lm[b].chi2 = v;
        else
            chi2_out[b] = v;
    }
}

// k_final_jac for batches whose stamps all sum in one segment (fewer than 8
// reduce blocks each): a warp per (stamp, 32 accumulators), 8 stamps per CTA,
// each summed in the order of the one-segment case above (the same bits).
__global__ void __launch_bounds__(256) k_final_jac_w(PassArgs a, double* A_out, double* g_out,
                                                     double* chi2_out)
{
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (b >= a.count) return;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const int nacc = a.nacc;
    const int t = blockIdx.y * 32 + lane;
    if (t >= nacc) return;
    const int* pst = a.pre_static + WK_RED * (a.count + 1);
    const int b0 = pst[b], b1 = pst[b + 1];
    CSum acc = {0.0f, 0.0f};
    const float* src = a.partial + t;
    int k = b0;
    for (; k + 3 < b1; k += 4) {
        const float v0 = src[(long long)k * nacc];
        const float v1 = src[(long long)(k + 1) * nacc];
        const float v2 = src[(long long)(k + 2) * nacc];
        const float v3 = src[(long long)(k + 3) * nacc];
        csum_add(acc, v0);
        csum_add(acc, v1);
        csum_add(acc, v2);
        csum_add(acc, v3);
    }
    for (; k < b1; ++k) csum_add(acc, src[(long long)k * nacc]);
    const double v = (double)acc.s + (double)acc.c;
    const int nf = a.S->nfree;
    int i, j;
    const int kind = decode_acc(t, nf, i, j);
    double* A = a.lm ? a.lm[b].A : A_out + (long long)b * nf * nf;
    double* g = a.lm ? a.lm[b].g : g_out + (long long)b * nf;
    if (kind == 0) {
        A[i * nf + j] = v;
        A[j * nf + i] = v;
    } else if (kind == 1) {
        g[i] = v;
    } else {
        if (a.lm)
            a.lm[b].chi2 = v;
        else
            chi2_out[b] = v;
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_final_chi2(PassArgs a, double* chi2_out)
{
    pdl_entry();
    __shared__ CSum wsum[RED_THREADS / 32];
    const int b = blockIdx.x;
    if (a.lm && a.lm[b].phase != a.phase) return;
    const int* pst = a.pre_static + WK_RED * (a.count + 1);
    const int b0 = pst[b], b1 = pst[b + 1];
    CSum acc = {0.0f, 0.0f};
    for (int k = b0 + threadIdx.x; k < b1; k += RED_THREADS) csum_add(acc, a.partial[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CSum other;
        other.s = __shfl_down_sync(0xffffffffu, acc.s, o);
        other.c = __shfl_down_sync(0xffffffffu, acc.c, o);
        acc = csum_merge(acc, other);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        CSum t = wsum[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, wsum[w]);
        const double v = (double)t.s + (double)t.c;
        if (a.lm)
            a.lm[b].chi2t = v;
        else
            chi2_out[b] = v;
    }
}

// sum of each PSF (the sky column and the sky's share of the model)
__global__ void __launch_bounds__(RED_THREADS) k_psf_sum(int count, const StampInfo* st,
                                                         const float* psf, float* out)
{
    __shared__ CSum wsum[RED_THREADS / 32];
    const int b = blockIdx.x;
    if (b >= count) return;
    const int n = st[b].P * st[b].P;
    const float* p = psf + st[b].psf_off;
    CSum acc = {0.0f, 0.0f};
    for (int k = threadIdx.x; k < n; k += RED_THREADS) csum_add(acc, p[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CSum other;
        other.s = __shfl_down_sync(0xffffffffu, acc.s, o);
        other.c = __shfl_down_sync(0xffffffffu, acc.c, o);
        acc = csum_merge(acc, other);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        CSum t = wsum[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) t = csum_merge(t, wsum[w]);
        out[b] = t.s + t.c;
    }
}

}  // namespace

cudaError_t launch_reduce_jac(const PassArgs& a, cudaStream_t s)
{
    if (a.maxitems[WK_RED] > 0) {
        // tiles of side 3 where they need no more tiles per side than 4 does
        int nv = 1;  // the bordered size: nacc = nv (nv + 1) / 2
        while (nv * (nv + 1) / 2 < a.nacc) ++nv;
        const bool ts3 = (nv + 2) / 3 == (nv + 3) / 4;
        const dim3 g(a.grid[WK_RED]), t(RED_THREADS);
        if (a.nchan <= 8) {
            if (ts3)
                GF_LAUNCH_PDL((k_reduce_jac<8, 3>), g, t, 0, s, a);
            else
                GF_LAUNCH_PDL((k_reduce_jac<8, 4>), g, t, 0, s, a);
        } else {
            if (ts3)
                GF_LAUNCH_PDL((k_reduce_jac<0, 3>), g, t, 0, s, a);
            else
                GF_LAUNCH_PDL((k_reduce_jac<0, 4>), g, t, 0, s, a);
        }
        GF_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_chi2(const PassArgs& a, cudaStream_t s)
{
    if (a.maxitems[WK_RED] > 0) {
        // one wave: four CTAs per SM are resident (64 registers a thread), and
        // each keeps two items' loads in flight
        const int g = (int)std::min<long long>(a.maxitems[WK_RED], 152LL * 4);
        GF_LAUNCH_PDL(k_reduce_chi2, dim3(g), dim3(RED_THREADS), 0, s, a);
        GF_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_rungs(const PassArgs& a, cudaStream_t s)
{
    if (a.nchan > GF_MAX_LADDER) return cudaErrorInvalidValue;
    if (a.maxitems[WK_RED] > 0) {
        GF_LAUNCH_PDL(k_reduce_rungs, dim3(a.grid[WK_RED]), dim3(RED_THREADS), 0, s, a);
        GF_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

cudaError_t launch_final_jac(const PassArgs& a, double* A_out, double* g_out, double* chi2_out,
                             cudaStream_t s)
{
    if (final_nseg(a.max_red) == 1) {
        const dim3 grid((a.count + 7) / 8, (a.nacc + 31) / 32);
        GF_LAUNCH_PDL(k_final_jac_w, dim3(grid), dim3(256), 0, s, a, A_out, g_out, chi2_out);
        GF_COUNT_LAUNCH();
        return cudaGetLastError();
    }
    const dim3 grid(a.count, (a.nacc + 31) / 32);
    GF_LAUNCH_PDL(k_final_jac, dim3(grid), dim3(32 * final_nseg(a.max_red)), 0, s, a, A_out, g_out, chi2_out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_final_chi2(const PassArgs& a, double* chi2_out, cudaStream_t s)
{
    GF_LAUNCH_PDL(k_final_chi2, dim3(a.count), dim3(RED_THREADS), 0, s, a, chi2_out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}

cudaError_t launch_psf_sum(int count, const StampInfo* st, const float* psf, float* out,
                           cudaStream_t s)
{
    k_psf_sum<<<count, RED_THREADS, 0, s>>>(count, st, psf, out);
    GF_COUNT_LAUNCH();
    return cudaGetLastError();
}
