// ppf_grad.cu -- gradient of the log marginal likelihood estimate
//   L(theta) = sum_k [log sum_i exp(l_k^i) - log N]
// (the per-frame log-evidences of Alg. 1, systematic resampling every frame)
// with respect to theta = (sigma_PSF, A, I_bg, sigma_m), the intensity fixed
// at I0 = A.  Resampling is a stop-gradient (ancestors held fixed), and so
// are the patch anchors (L is piecewise smooth in the positions).
//
// sigma_PSF, A and I_bg enter only through the frame-k likelihood:
//   dL/dtheta = sum_k sum_i w_k^i dl_k^i/dtheta,  w_k = softmax(l_k).
// sigma_m enters the dynamics, x_k = x_{k-1}^{a} + vx_{k-1}^{a} + sigma_m e,
// so dx_k/dsigma_m = dx_{k-1}^{a}/dsigma_m + e: a two-float tangent per
// particle, carried forward with its ancestor (forward mode; with a single
// dynamics parameter this needs no stored states and no reverse sweep), and
// dl/dsigma_m = dl/dx tx + dl/dy ty.
#include <cmath>
#include <cstring>

#include "ppf_device.cuh"
#include "ppf_internal.h"

namespace ppf {

struct GradArgs {
    int64_t N;
    int W, H, Wp, Hp, pad;
    float sigma, inv2s2, inv_sxi2, A, sm, sv;
    float Kc[MAX_RADIUS];
    uint64_t seed;
    PhiloxKeys rk;     // round keys of seed
    uint32_t fid, frame;
    int first;                       // first frame: identity ancestry, zero tangents
    const float *__restrict__ src;   // 6 x N
    float *__restrict__ dst;
    const float *__restrict__ tsrc;  // 2 x N tangents (dx, dy) / dsigma_m
    float *__restrict__ tdst;
    const int32_t *__restrict__ anc;
    const int32_t *__restrict__ degenerate;  // last resample kept every particle
    const float *__restrict__ Zp;    // prepared frame as pixel pairs (float2, row pitch Wp)
    int32_t *__restrict__ anchors;   // optional 2 x N export (cx, cy)
    GradPartial *__restrict__ part;
    unsigned int *done;
    DevSummary *sum;
};

// Gaussian samples by the exact ratio recurrence (as in the step kernel)
template <int R>
__device__ __forceinline__ void gauss_row(float f, float a, const float *Kc, float g[2 * R + 1])
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

// l and dl/d(sigma, I0, bg, x, y) of one particle, separable over the patch:
// with Zb = Z - I_bg, h = Zb - I0 g, g = gx gy, dx = px - x, dy = py - y,
//   l      = (I0 B - I0^2 C / 2) / sxi^2,  B = sum gy R0, C = Sx0 Sy0
//   dl/dI0 = (B - I0 C) / sxi^2
//   dl/dbg = -(I0 / sxi^2) Gx Gy
//   dl/dx  = I0 / (sxi^2 s^2) [sum gy R1 - I0 Sx1 Sy0]
//   dl/dy  = I0 / (sxi^2 s^2) [sum gy dy R0 - I0 Sx0 Sy1]
//   dl/ds  = I0 / (sxi^2 s^3) [sum gy (R2 + dy^2 R0) - I0 (Sx2 Sy0 + Sx0 Sy2)]
// with row sums Rm_j = sum_i gx dx^m Zb, moments Sxm = sum gx^2 dx^m,
// Sym = sum gy^2 dy^m, Gx = sum gx, Gy = sum gy (all over in-image pixels).
template <int R>
__device__ __forceinline__ void grad_patch(const GradArgs &a, float x, float y, float I0, float out[6], int &cxo,
                                           int &cyo)
{
#pragma unroll
    for (int c = 0; c < 6; ++c)
        out[c] = 0.0f;
    if (!isfinite(x) || !isfinite(y) || !isfinite(I0)) {
        out[0] = -INFINITY;
        cxo = cyo = INT32_MIN;
        return;
    }
    const float cxf = floorf(x + 0.5f), cyf = floorf(y + 0.5f);
    cxo = (int)fmaxf(fminf(cxf, 2.0e9f), -2.0e9f);
    cyo = (int)fmaxf(fminf(cyf, 2.0e9f), -2.0e9f);
    if (cxf < -(float)R || cxf > (float)(a.W - 1 + R) || cyf < -(float)R || cyf > (float)(a.H - 1 + R))
        return;
    const int cx = (int)cxf, cy = (int)cyf;
    constexpr int P = 2 * R + 1;
    const float fx = cxf - x, fy = cyf - y;
    float gx[P], gy[P];
    gauss_row<R>(fx, a.inv2s2, a.Kc, gx);
    gauss_row<R>(fy, a.inv2s2, a.Kc, gy);
    if (cx < R || cx > a.W - 1 - R || cy < R || cy > a.H - 1 - R) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int px = cx + i - R, py = cy + i - R;
            gx[i] = (px >= 0 && px < a.W) ? gx[i] : 0.0f;
            gy[i] = (py >= 0 && py < a.H) ? gy[i] : 0.0f;
        }
    }
    float Sx0 = 0, Sx1 = 0, Sx2 = 0, Sy0 = 0, Sy1 = 0, Sy2 = 0, Gx = 0, Gy = 0;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const float dx = fx + (float)(i - R), dy = fy + (float)(i - R);
        const float gx2 = gx[i] * gx[i], gy2 = gy[i] * gy[i];
        Sx0 += gx2;
        Sx1 = fmaf(gx2, dx, Sx1);
        Sx2 = fmaf(gx2 * dx, dx, Sx2);
        Sy0 += gy2;
        Sy1 = fmaf(gy2, dy, Sy1);
        Sy2 = fmaf(gy2 * dy, dy, Sy2);
        Gx += gx[i];
        Gy += gy[i];
    }
    // per-column weights gx, gx dx, gx dx^2; the row sums read the frame as
    // pixel pairs (one aligned float2 per two columns) and run as packed
    // two-lane FMAs over the full column pairs, the odd last column on the
    // even lane
    constexpr int Q = P / 2;
    float w0[P], w1[P], w2[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const float dx = fx + (float)(i - R);
        w0[i] = gx[i];
        w1[i] = gx[i] * dx;
        w2[i] = w1[i] * dx;
    }
    const float2 *row = reinterpret_cast<const float2 *>(a.Zp) + (int64_t)(cy - R + a.pad) * a.Wp +
                        (cx - R + a.pad);
    float B = 0, By1 = 0, Bx1 = 0, Bs = 0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        float2 p0 = make_float2(0.0f, 0.0f), p1 = p0, p2 = p0;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const float2 z = __ldg(row + 2 * k);
            p0 = __ffma2_rn(make_float2(w0[2 * k], w0[2 * k + 1]), z, p0);
            p1 = __ffma2_rn(make_float2(w1[2 * k], w1[2 * k + 1]), z, p1);
            p2 = __ffma2_rn(make_float2(w2[2 * k], w2[2 * k + 1]), z, p2);
        }
        const float zl = __ldg(row + 2 * Q).x;
        const float r0 = fmaf(w0[P - 1], zl, p0.x) + p0.y;
        const float r1 = fmaf(w1[P - 1], zl, p1.x) + p1.y;
        const float r2 = fmaf(w2[P - 1], zl, p2.x) + p2.y;
        const float dy = fy + (float)(j - R);
        B = fmaf(gy[j], r0, B);
        By1 = fmaf(gy[j] * dy, r0, By1);
        Bx1 = fmaf(gy[j], r1, Bx1);
        Bs = fmaf(gy[j], fmaf(dy * dy, r0, r2), Bs);
        row += a.Wp;
    }
    const float C = Sx0 * Sy0;
    const float k2 = I0 * a.inv_sxi2 * a.inv2s2 * 2.0f;  // I0 / (sxi^2 s^2)
    out[0] = I0 * fmaf(-0.5f * I0, C, B) * a.inv_sxi2;
    out[1] = k2 / a.sigma * (Bs - I0 * fmaf(Sx2, Sy0, Sx0 * Sy2));
    out[2] = fmaf(-I0, C, B) * a.inv_sxi2;
    out[3] = -I0 * a.inv_sxi2 * Gx * Gy;
    out[4] = k2 * (Bx1 - I0 * Sx1 * Sy0);
    out[5] = k2 * (By1 - I0 * Sx0 * Sy1);
}

// online log-sum-exp of l with the weighted sums of the four derivatives
struct GAcc {
    float m, s0, s[4];
    __device__ __forceinline__ void init()
    {
        m = -INFINITY;
        s0 = 0.0f;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            s[c] = 0.0f;
    }
    __device__ __forceinline__ void add(float l, const float d[4])
    {
        if (!(l > -INFINITY))
            return;
        if (l > m) {
            const float sc = __expf(m - l);
            s0 *= sc;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                s[c] *= sc;
            m = l;
        }
        const float e = __expf(l - m);
        s0 += e;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            s[c] = fmaf(e, d[c], s[c]);
    }
    __device__ __forceinline__ void merge(const GAcc &o)
    {
        const float nm = fmaxf(m, o.m);
        const float fa = (m == -INFINITY) ? 0.0f : __expf(m - nm);
        const float fb = (o.m == -INFINITY) ? 0.0f : __expf(o.m - nm);
        s0 = s0 * fa + o.s0 * fb;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            s[c] = s[c] * fa + o.s[c] * fb;
        m = nm;
    }
    __device__ __forceinline__ void shfl_merge(int o)
    {
        GAcc b;
        b.m = __shfl_xor_sync(0xffffffffu, m, o);
        b.s0 = __shfl_xor_sync(0xffffffffu, s0, o);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            b.s[c] = __shfl_xor_sync(0xffffffffu, s[c], o);
        merge(b);
    }
};

__device__ void grad_finalize(const GradPartial *part, int n, DevSummary *sum, int64_t N, int32_t frame)
{
    __shared__ float smf[32];
    __shared__ double smd[32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float m = -INFINITY;
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        m = fmaxf(m, __ldcg(&part[b].m));
    m = warp_max(m);
    if (lane == 0)
        smf[warp] = m;
    __syncthreads();
    float M = -INFINITY;
    for (int w = 0; w < nw; ++w)
        M = fmaxf(M, smf[w]);
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const float qm = __ldcg(&part[b].m);
        if (qm > -INFINITY) {
            const double f = (double)expf(qm - M);
            acc[0] += __ldcg(&part[b].s0) * f;
            for (int c = 0; c < 4; ++c)
                acc[1 + c] += __ldcg(&part[b].s[c]) * f;
        }
    }
    for (int c = 0; c < 5; ++c)
        acc[c] = warp_sum_d(acc[c]);
    if (lane == 0)
        for (int c = 0; c < 5; ++c)
            smd[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < nw; ++w)
            for (int c = 0; c < 5; ++c)
                t[c] += smd[w][c];
        const double le = (double)M + log(t[0]) - log((double)N);
        sum->log_total = (double)M + log(t[0]);
        sum->log_evidence = le;
        sum->max_lw = (double)M;
        sum->M = M;
        sum->frame = frame;
        sum->grad_L += le;
        for (int c = 0; c < 4; ++c)
            sum->grad_g[c] += t[1 + c] / t[0];
        if (!(t[0] > 0.0))
            sum->flags |= FLAG_DEGENERATE;
    }
}

template <int R>
__global__ void __launch_bounds__(256) grad_step_kernel(GradArgs a)
{
    const int64_t N = a.N;
    const bool ident = a.first || *a.degenerate;
    GAcc acc;
    acc.init();
    // the ancestor of the next slot is loaded one iteration ahead
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t pn = (i0 < N) ? (ident ? i0 : (int64_t)__ldg(a.anc + i0)) : 0;
    for (int64_t i = i0; i < N; i += stride) {
        int64_t p = pn;
        if (i + stride < N)
            pn = ident ? i + stride : (int64_t)__ldg(a.anc + i + stride);
        if ((uint64_t)p >= (uint64_t)N)
            p = i;
        const float x = __ldg(a.src + p), y = __ldg(a.src + N + p);
        const float vx = __ldg(a.src + 2 * N + p), vy = __ldg(a.src + 3 * N + p);
        const float tx = a.first ? 0.0f : __ldg(a.tsrc + p), ty = a.first ? 0.0f : __ldg(a.tsrc + N + p);
        uint32_t f[6];
        prop_fields(philox_rk(make_uint4((uint32_t)i, a.frame, a.fid, PURPOSE_PROP << 8), a.rk), f);
        float e0, e1, e2, e3;
        box_muller(u21(f[0]), u21(f[1]), e0, e1);
        box_muller(u21(f[2]), u21(f[3]), e2, e3);
        const float nx = fmaf(a.sm, e0, x + vx), ny = fmaf(a.sm, e1, y + vy);
        const float ntx = tx + e0, nty = ty + e1;
        float d[6];
        int cx, cy;
        grad_patch<R>(a, nx, ny, a.A, d, cx, cy);
        a.dst[i] = nx;
        a.dst[N + i] = ny;
        a.dst[2 * N + i] = fmaf(a.sv, e2, vx);
        a.dst[3 * N + i] = fmaf(a.sv, e3, vy);
        a.dst[4 * N + i] = a.A;
        a.dst[5 * N + i] = d[0];
        a.tdst[i] = ntx;
        a.tdst[N + i] = nty;
        if (a.anchors) {
            a.anchors[i] = cx;
            a.anchors[N + i] = cy;
        }
        const float g4[4] = {d[1], d[2], d[3], fmaf(d[4], ntx, d[5] * nty)};
        acc.add(d[0], g4);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc.shfl_merge(o);
    __shared__ GAcc sh[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        sh[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        if (lane < nw)
            acc = sh[lane];
        else
            acc.init();
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)
            acc.shfl_merge(o);
        if (lane == 0) {
            GradPartial q;
            q.m = acc.m;
            q.s0 = acc.s0;
            for (int c = 0; c < 4; ++c)
                q.s[c] = acc.s[c];
            a.part[blockIdx.x] = q;
        }
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(a.done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        grad_finalize(a.part, gridDim.x, a.sum, a.N, (int32_t)a.frame);
        if (threadIdx.x == 0)
            *a.done = 0u;
    }
}

template <int R>
static void launch_grad_r(const GradArgs &a, int grid, cudaStream_t s)
{
    grad_step_kernel<R><<<grid, 256, 0, s>>>(a);
}

cudaError_t launch_grad_step(ppf_ctx *c, int32_t k, bool first, int32_t *anchors)
{
    GradArgs a;
    a.N = c->N;
    a.W = c->m.width;
    a.H = c->m.height;
    a.Wp = c->Wp;
    a.Hp = c->Hp;
    a.pad = c->pad;
    a.sigma = c->m.psf_sigma;
    a.inv2s2 = 1.0f / (2.0f * c->m.psf_sigma * c->m.psf_sigma);
    for (int q = 0; q < MAX_RADIUS; ++q)
        a.Kc[q] = (float)exp(-(2.0 * q + 1.0) * (double)a.inv2s2);
    a.inv_sxi2 = 1.0f / (c->m.sigma_xi * c->m.sigma_xi);
    a.A = c->m.amplitude;
    a.sm = c->m.sigma_m;
    a.sv = c->m.sigma_v;
    a.seed = c->m.seed;
    a.rk = philox_keys(c->m.seed);
    a.fid = c->m.filter_id;
    a.frame = (uint32_t)k;
    a.first = first ? 1 : 0;
    a.src = c->state[c->cur];
    a.dst = c->state[c->cur ^ 1];
    a.tsrc = c->tang[c->tcur];
    a.tdst = c->tang[c->tcur ^ 1];
    a.anc = c->anc;
    a.degenerate = &c->sum->degenerate;
    a.Zp = c->Zp;
    a.anchors = anchors;
    a.part = c->gpart;
    a.done = &c->sum->blocks_done;
    a.sum = c->sum;
    const int grid = c->n_part;
    switch (c->m.patch_radius) {
    case 0: launch_grad_r<0>(a, grid, c->stream); break;
    case 1: launch_grad_r<1>(a, grid, c->stream); break;
    case 2: launch_grad_r<2>(a, grid, c->stream); break;
    case 3: launch_grad_r<3>(a, grid, c->stream); break;
    case 4: launch_grad_r<4>(a, grid, c->stream); break;
    case 5: launch_grad_r<5>(a, grid, c->stream); break;
    case 6: launch_grad_r<6>(a, grid, c->stream); break;
    case 7: launch_grad_r<7>(a, grid, c->stream); break;
    default: launch_grad_r<8>(a, grid, c->stream); break;
    }
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace ppf
