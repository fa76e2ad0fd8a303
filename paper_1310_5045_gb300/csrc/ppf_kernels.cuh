// ppf_kernels.cuh -- per-particle device code shared by the single-filter and
// batched SIS steps: the online log-sum-exp accumulator, the Gaussian PSF
// samples and the eq. 3 / eq. 4 patch likelihood.
#pragma once

#include <cmath>

#include "ppf_device.cuh"
#include "ppf_internal.h"

namespace ppf {

// Online log-sum-exp accumulator of the weight statistics.
struct Acc {
    float m, s0, s[5], s2, mp, sp;
    __device__ __forceinline__ void init()
    {
        m = mp = -INFINITY;
        s0 = s2 = sp = 0.0f;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            s[c] = 0.0f;
    }
    __device__ __forceinline__ void add(float lw, float lwp, const float v[5])
    {
        add_cur(lw, v);
        add_prev(lwp);
    }
    __device__ __forceinline__ void add_cur(float lw, const float v[5])
    {
        if (lw > m) {
            const float sc = __expf(m - lw);
            s0 *= sc;
            s2 *= sc * sc;
#pragma unroll
            for (int c = 0; c < 5; ++c)
                s[c] *= sc;
            m = lw;
        }
        if (lw > -INFINITY) {
            const float e = __expf(lw - m);
            s0 += e;
            s2 = fmaf(e, e, s2);
#pragma unroll
            for (int c = 0; c < 5; ++c)
                s[c] = fmaf(e, v[c], s[c]);
        }
    }
    __device__ __forceinline__ void add_prev(float lwp)
    {
        if (lwp > mp) {
            sp *= __expf(mp - lwp);
            mp = lwp;
        }
        if (lwp > -INFINITY)
            sp += __expf(lwp - mp);
    }
    // add_prev(0) after a resample to equal weights: the same bits without
    // the exponentials (mp = 0, sp counts the particles)
    __device__ __forceinline__ void add_prev_zero()
    {
        mp = 0.0f;
        sp += 1.0f;
    }
    __device__ __forceinline__ void merge(const Acc &o)
    {
        const float nm = fmaxf(m, o.m);
        const float fa = (m == -INFINITY) ? 0.0f : __expf(m - nm);
        const float fb = (o.m == -INFINITY) ? 0.0f : __expf(o.m - nm);
        s0 = s0 * fa + o.s0 * fb;
        s2 = s2 * fa * fa + o.s2 * fb * fb;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            s[c] = s[c] * fa + o.s[c] * fb;
        m = (nm == -INFINITY) ? -INFINITY : nm;
        const float nmp = fmaxf(mp, o.mp);
        const float ga = (mp == -INFINITY) ? 0.0f : __expf(mp - nmp);
        const float gb = (o.mp == -INFINITY) ? 0.0f : __expf(o.mp - nmp);
        sp = sp * ga + o.sp * gb;
        mp = nmp;
    }
    __device__ __forceinline__ void shfl_merge(int o)
    {
        Acc b;
        b.m = __shfl_xor_sync(0xffffffffu, m, o);
        b.s0 = __shfl_xor_sync(0xffffffffu, s0, o);
        b.s2 = __shfl_xor_sync(0xffffffffu, s2, o);
#pragma unroll
        for (int c = 0; c < 5; ++c)
            b.s[c] = __shfl_xor_sync(0xffffffffu, s[c], o);
        b.mp = __shfl_xor_sync(0xffffffffu, mp, o);
        b.sp = __shfl_xor_sync(0xffffffffu, sp, o);
        merge(b);
    }
};

// Point samples g(k) = exp(-a (k + f)^2), k = -R..R, f in (-1/2, 1/2]: the
// centre by one exponential, the rest by the exact ratios
// g(k+1) / g(k) = exp(-a (2k+1)) exp(-2 a f) and
// g(-k-1) / g(-k) = exp(-a (2k+1)) exp(2 a f), k >= 0,
// with the constants Kc[k] = exp(-a (2k+1)) precomputed per model.
template <int R>
__device__ __forceinline__ void gauss_samples(float f, float a, const float *Kc, float g[2 * R + 1])
{
    g[R] = __expf(-a * f * f);
    if (R > 0) {
        const float up = __expf(-2.0f * a * f), dn = __expf(2.0f * a * f);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            g[R + k + 1] = g[R + k] * (Kc[k] * up);
            g[R - k - 1] = g[R - k] * (Kc[k] * dn);
        }
    }
}

// Eq. 4 over S_x with the eq. 3 model, pixels outside S_x modelled as
// background: l = -sum_{S_x} [(Zb - a)^2 - Zb^2] / (2 sigma_xi^2) with
// Zb = Z - I_bg and a = I0 g, g separable: g = gx(col) gy(row).  Expanded,
// l = I0 (B - I0 C / 2) / sigma_xi^2 with B = sum gy_j sum_i gx_i Zb and
// C = sum gx_i^2 sum gy_j^2.  Samples of columns / rows outside the image are
// zeroed (only for patches that cross the border); Zp is zero there as well.
struct PatchGeom {
    const float *Zp;   // padded frame minus background, as pixel pairs (see patch_loglik)
    int W, H, Wp, pad;
    float inv2s2;      // 1 / (2 sigma_PSF^2)
    float inv_sxi2;    // 1 / sigma_xi^2
    const float *Kc;   // exp(-(2k+1) inv2s2), k = 0..R-1
    int Hp = 0;                      // padded frame height (the debug build's window check)
    const int32_t *flags = nullptr;  // debug build: where a failed window check is reported
};

// The anchor c = floor(x + 1/2), the PSF samples of the patch columns and
// rows (zero outside the image) and C = sum gx^2 sum gy^2.  Returns false when
// no patch sum is needed, with the log-likelihood in *l: -inf for a
// non-finite particle, 0 for a patch entirely outside the image.
template <int R>
__device__ __forceinline__ bool patch_setup(const PatchGeom &a, float x, float y, float I0, int &cx, int &cy,
                                            float gx[2 * R + 1], float gy[2 * R + 1], float &C, float *l)
{
    if (!isfinite(x) || !isfinite(y) || !isfinite(I0)) {
        *l = -INFINITY;
        return false;
    }
    const float cxf = floorf(x + 0.5f), cyf = floorf(y + 0.5f);
    if (cxf < -(float)R || cxf > (float)(a.W - 1 + R) || cyf < -(float)R || cyf > (float)(a.H - 1 + R)) {
        *l = 0.0f;
        return false;
    }
    cx = (int)cxf;
    cy = (int)cyf;
    constexpr int P = 2 * R + 1;
    gauss_samples<R>(cxf - x, a.inv2s2, a.Kc, gx);
    gauss_samples<R>(cyf - y, a.inv2s2, a.Kc, gy);
    if (cx < R || cx > a.W - 1 - R || cy < R || cy > a.H - 1 - R) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int px = cx + i - R, py = cy + i - R;
            gx[i] = (px >= 0 && px < a.W) ? gx[i] : 0.0f;
            gy[i] = (py >= 0 && py < a.H) ? gy[i] : 0.0f;
        }
    }
    float sxx = 0.0f, syy = 0.0f;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        sxx = fmaf(gx[i], gx[i], sxx);
        syy = fmaf(gy[i], gy[i], syy);
    }
    C = sxx * syy;
    return true;
}

// The patch sum B = sum_j gy_j sum_i gx_i Zb(i, j), read two pixels at a
// time: a.Zp holds the prepared frame as pixel pairs, element (row, col) of
// the float2 array (row pitch a.Wp) being (Zb(row, col), Zb(row, col + 1)).
// The pair starting at any column is then one aligned float2 load, and lanes
// whose patches start at neighbouring columns read neighbouring words.
//
// The even and the odd columns are summed apart: for every row,
// r_j = (sum_k gx_2k Zb(2k, j) + gx_P-1 Zb(P-1, j), sum_k gx_2k+1 Zb(2k+1, j)),
// k over the P / 2 full column pairs; then b = sum_j gy_j r_j lane by lane and
// B = b.x + b.y.  PACKED computes the two lanes with packed two-lane FMAs
// over the pixel pairs; the scalar form (kept by the batched step, whose
// warp-per-unit kernel ran slower with packed FMAs) performs the same
// roundings in the same order, so both give the same bits.
//
// patch_rows takes the first pair of the window's first row and the row pitch
// (in pairs); SMEM reads a window staged in shared memory with plain loads,
// otherwise the prepared frame through the read-only path.  Both forms do the
// same arithmetic, so a particle's likelihood has the same bits either way.
template <int R, bool PACKED, bool SMEM = false>
__device__ __forceinline__ float patch_rows(const float2 *row, int pitch, const float gx[2 * R + 1],
                                            const float gy[2 * R + 1])
{
    constexpr int P = 2 * R + 1;
    constexpr int Q = P / 2;  // full column pairs; column P - 1 is the odd one out
    auto ld = [](const float2 *q) -> float2 {
        if constexpr (SMEM)
            return *q;
        else
            return __ldg(q);
    };
    float2 b = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < P; ++j) {
        float2 r = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const float2 z = ld(row + 2 * k);
            if constexpr (PACKED) {
                r = (k == 0) ? __fmul2_rn(make_float2(gx[0], gx[1]), z)
                             : __ffma2_rn(make_float2(gx[2 * k], gx[2 * k + 1]), z, r);
            } else {
                r.x = (k == 0) ? __fmul_rn(gx[0], z.x) : __fmaf_rn(gx[2 * k], z.x, r.x);
                r.y = (k == 0) ? __fmul_rn(gx[1], z.y) : __fmaf_rn(gx[2 * k + 1], z.y, r.y);
            }
        }
        r.x = __fmaf_rn(gx[P - 1], ld(row + 2 * Q).x, r.x);
        if constexpr (PACKED) {
            b = (j == 0) ? __fmul2_rn(make_float2(gy[0], gy[0]), r) : __ffma2_rn(make_float2(gy[j], gy[j]), r, b);
        } else {
            b.x = (j == 0) ? __fmul_rn(gy[0], r.x) : __fmaf_rn(gy[j], r.x, b.x);
            b.y = (j == 0) ? __fmul_rn(gy[0], r.y) : __fmaf_rn(gy[j], r.y, b.y);
        }
        row += pitch;
    }
    return __fadd_rn(b.x, b.y);
}

template <int R, bool PACKED>
__device__ __forceinline__ float patch_sum(const PatchGeom &a, int cx, int cy, const float gx[2 * R + 1],
                                           const float gy[2 * R + 1])
{
    constexpr int Q = R;  // (2R + 1) / 2 full column pairs
    // the window: 2R + 1 rows from cy - R, pairs from column cx - R up to
    // 2Q + 1 columns on (inside the padded frame by the anchor's range)
    if (a.flags && !PPF_DCHECK(cy - R + a.pad >= 0 && cy + R + a.pad < a.Hp && cx - R + a.pad >= 0 &&
                                   cx - R + a.pad + 2 * Q < a.Wp,
                               a.flags, FLAG_INTERNAL))
        return 0.0f;
    const float2 *row = reinterpret_cast<const float2 *>(a.Zp) + (int64_t)(cy - R + a.pad) * a.Wp +
                        (cx - R + a.pad);
    return patch_rows<R, PACKED, false>(row, a.Wp, gx, gy);
}

template <int R, bool PACKED = true>
__device__ __forceinline__ float patch_loglik(const PatchGeom &a, float x, float y, float I0)
{
    constexpr int P = 2 * R + 1;
    int cx, cy;
    float gx[P], gy[P], C, l;
    if (!patch_setup<R>(a, x, y, I0, cx, cy, gx, gy, C, &l))
        return l;
    const float B = patch_sum<R, PACKED>(a, cx, cy, gx, gy);
    return I0 * fmaf(-0.5f * I0, C, B) * a.inv_sxi2;
}

// pcSIR (Sec. 6): the likelihood held constant on every pixel cell, at its
// value for the cell centre c = floor((x, y) + 1/2).  lmap holds (B, C) of the
// patch sum at every anchor c (row pitch W + 2R, c shifted by R), so a
// particle costs one lookup: l = I0 (B - I0 C / 2) / sigma_xi^2.
template <int R>
__device__ __forceinline__ float cell_loglik(const PatchGeom &a, const float2 *__restrict__ lmap, float x, float y,
                                             float I0)
{
    if (!isfinite(x) || !isfinite(y) || !isfinite(I0))
        return -INFINITY;
    const float cxf = floorf(x + 0.5f), cyf = floorf(y + 0.5f);
    if (cxf < -(float)R || cxf > (float)(a.W - 1 + R) || cyf < -(float)R || cyf > (float)(a.H - 1 + R))
        return 0.0f;
    const float2 bc = __ldg(lmap + (int64_t)((int)cyf + R) * (a.W + 2 * R) + ((int)cxf + R));
    return I0 * fmaf(-0.5f * I0, bc.y, bc.x) * a.inv_sxi2;
}

// ------------------------------------------------------------ the finaliser
// Cross-block totals in FP64 (the paper's global sum for normalisation):
// estimate, N_eff, log-evidence, from n per-block partials.  Run by the last
// block of the kernel that produced them.  It also decides which likelihood
// path the next step takes (the binned path when more than a quarter of the
// warps of this step saw their particles spread wider than BIN_SPREAD_PX)
// and clears the counters of that decision.
__device__ __forceinline__ void finalize_block(const Partial *part, int n, DevSummary *sum, int32_t frame)
{
    __shared__ float smf[32];
    __shared__ double smd[32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float m = -INFINITY, mp = -INFINITY;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        m = fmaxf(m, __ldcg(&part[b].m));
        mp = fmaxf(mp, __ldcg(&part[b].mp));
    }
    m = warp_max(m);
    if (lane == 0)
        smf[warp] = m;
    __syncthreads();
    float M = -INFINITY;
    for (int w = 0; w < nw; ++w)
        M = fmaxf(M, smf[w]);
    __syncthreads();
    mp = warp_max(mp);
    if (lane == 0)
        smf[warp] = mp;
    __syncthreads();
    float Mp = -INFINITY;
    for (int w = 0; w < nw; ++w)
        Mp = fmaxf(Mp, smf[w]);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // s0, s[5], s2, sp
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const float qm = __ldcg(&part[b].m), qmp = __ldcg(&part[b].mp);
        if (qm > -INFINITY) {
            const double f = (double)expf(qm - M);  // scale factor to 1 ulp; sums in FP64
            acc[0] += __ldcg(&part[b].s0) * f;
            for (int c = 0; c < 5; ++c)
                acc[1 + c] += __ldcg(&part[b].s[c]) * f;
            acc[6] += __ldcg(&part[b].s2) * f * f;
        }
        if (qmp > -INFINITY)
            acc[7] += __ldcg(&part[b].sp) * (double)expf(qmp - Mp);
    }
    for (int c = 0; c < 8; ++c)
        acc[c] = warp_sum_d(acc[c]);
    if (lane == 0)
        for (int c = 0; c < 8; ++c)
            smd[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < nw; ++w)
            for (int c = 0; c < 8; ++c)
                t[c] += smd[w][c];
        for (int c = 0; c < 5; ++c)
            sum->mean[c] = t[1 + c] / t[0];
        sum->ess = t[0] * t[0] / t[6];
        sum->log_total = (double)M + log(t[0]);
        sum->log_evidence = sum->log_total - ((double)Mp + log(t[7]));
        sum->max_lw = (double)M;
        sum->M = M;
        sum->frame = frame;
        if (!(t[0] > 0.0))
            sum->flags |= FLAG_DEGENERATE;
        const uint32_t spread = sum->spread_warps, total = sum->total_warps;
        sum->bin_next = (4ull * spread > (uint64_t)total) ? 1 : 0;
        sum->spread_warps = 0u;
        sum->total_warps = 0u;
    }
}

// ------------------------------------------------------- input-space bins
// The binned likelihood path (Sec. 6.3's input-space decomposition): the
// particles are binned by the image tile that holds their patch anchor, and
// each tile's window (the tile plus the patch halo) is staged in shared
// memory once for all the particles of its bin.  Anchors u = cx + R in
// [0, W + 2R) and v = cy + R in [0, H + 2R) (the range with a nonempty
// patch) are tiled by T x T; the last bin holds the particles that need no
// patch sum (non-finite, or no pixel of the patch inside the image).
struct BinGeom {
    int T, nx, nbins;  // tile edge, tiles per row, bins (tiles + 1)
};

template <int R>
__device__ __forceinline__ uint32_t bin_of(const BinGeom &g, int W, int H, float x, float y, float I0)
{
    if (!isfinite(x) || !isfinite(y) || !isfinite(I0))
        return (uint32_t)(g.nbins - 1);
    const float cxf = floorf(x + 0.5f), cyf = floorf(y + 0.5f);
    if (cxf < -(float)R || cxf > (float)(W - 1 + R) || cyf < -(float)R || cyf > (float)(H - 1 + R))
        return (uint32_t)(g.nbins - 1);
    const int u = (int)cxf + R, v = (int)cyf + R;
    return (uint32_t)((v / g.T) * g.nx + u / g.T);
}

// warps whose particles' anchors span more than this many pixels in x or y
// count as spread (their patch reads touch a separate cache line per lane)
constexpr int BIN_SPREAD_PX = 64;

// Per warp: the extent of the anchors of the lanes' sampled particles (one
// iteration of the step's loop per block; lanes without a sample pass
// active = false); one count per warp into the counters (lane 0).  Called by
// all 32 lanes after the loop: the decision needs a fraction, not a census.
__device__ __forceinline__ void spread_tally(float x, float y, bool active, unsigned &n_spread, unsigned &n_total)
{
    const bool fin = active && isfinite(x) && isfinite(y) && fabsf(x) < 1e9f && fabsf(y) < 1e9f;
    const int cx = fin ? (int)floorf(x + 0.5f) : 0, cy = fin ? (int)floorf(y + 0.5f) : 0;
    const unsigned m = 0xffffffffu;
    const int lox = __reduce_min_sync(m, fin ? cx : INT32_MAX), hix = __reduce_max_sync(m, fin ? cx : INT32_MIN);
    const int loy = __reduce_min_sync(m, fin ? cy : INT32_MAX), hiy = __reduce_max_sync(m, fin ? cy : INT32_MIN);
    const bool any_fin = __any_sync(m, fin);
    if ((threadIdx.x & 31) == 0 && any_fin) {
        n_total += 1u;
        if (lox <= hix && ((int64_t)hix - lox > BIN_SPREAD_PX || (int64_t)hiy - loy > BIN_SPREAD_PX))
            n_spread += 1u;
    }
}

}  // namespace ppf
