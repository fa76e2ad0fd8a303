// ppf_step.cu -- S0 initialisation and the fused SIS step of Alg. 1:
// propagation (Sec. 7.1 NCV dynamics, bootstrap proposal), patch likelihood
// (eq. 3 appearance, eq. 4 likelihood over the (2r+1)^2 box S_x) and the
// normalisation statistics (log-sum-exp partials per block, FP64 total).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "ppf_device.cuh"
#include "ppf_internal.h"
#include "ppf_kernels.cuh"

namespace ppf {

// ------------------------------------------------------------------- S0 init
// Alg. 1 initialisation: equal weights, particles drawn uniformly (Sec. 7.3).
__global__ void init_kernel(float *__restrict__ st, int64_t N, uint64_t seed, uint32_t fid, float W,
                            float H, float v0, float A)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 a = draw(seed, (uint32_t)i, 0u, fid, PURPOSE_INIT, 0);
        const uint4 b = draw(seed, (uint32_t)i, 0u, fid, PURPOSE_INIT, 1);
        st[i] = -0.5f + W * u01(a.x);
        st[N + i] = -0.5f + H * u01(a.y);
        st[2 * N + i] = v0 * (2.0f * u01(a.z) - 1.0f);
        st[3 * N + i] = v0 * (2.0f * u01(a.w) - 1.0f);
        st[4 * N + i] = A * (0.5f + u01(b.x));
        st[5 * N + i] = 0.0f;
    }
}

// --------------------------------------------------------- frame preparation
// Zb = Z - I_bg inside the image, 0 in a border of width pad = 2r, so that a
// patch anchored up to r pixels outside the image never leaves the buffer.
template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename T>
__global__ void prepare_frame_kernel(const T *__restrict__ Z, float *__restrict__ Zp, int W, int H, int Wp,
                                     int Hp, int pad, float bg)
{
    // pixel pairs: element (row, col) = (Zb(row, col), Zb(row, col + 1)) with
    // Zb = Z - bg inside the image and 0 in the border of `pad` (pitch Wp)
    const int n = Wp * Hp;
    auto px_at = [&](int py, int px) -> float {
        return (px >= 0 && px < W && py >= 0 && py < H) ? to_f32<T>(Z[(int64_t)py * W + px]) - bg : 0.0f;
    };
    float2 *__restrict__ out = reinterpret_cast<float2 *>(Zp);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int py = idx / Wp - pad, px = idx % Wp - pad;
        out[idx] = make_float2(px_at(py, px), px_at(py, px + 1));
    }
}

// ------------------------------------------------------------ the SIS step
struct StepArgs {
    int64_t N;
    int W, H, Wp, Hp, pad;
    float inv2s2;      // 1 / (2 sigma_PSF^2)
    float Kc[MAX_RADIUS];  // exp(-(2k+1) / (2 sigma_PSF^2)), k = 0..R-1
    float inv_sxi2;    // 1 / sigma_xi^2
    float sm, sv, sI;
    uint64_t seed;
    PhiloxKeys rk;     // round keys of seed
    uint32_t fid, frame;
    const float *__restrict__ src;
    float *__restrict__ dst;
    const int32_t *__restrict__ anc;
    const float *__restrict__ lwp;
    const int32_t *__restrict__ degenerate;
    int32_t *flags;
    int mode;
    const float *__restrict__ Zp;
    const float2 *__restrict__ lmap;  // pcSIR cell map, or nullptr (eq. 4 at the particle)
    Partial *__restrict__ part;
    unsigned int *done;    // blocks finished (reset by the last one)
    DevSummary *sum;
};

// --------------------------------------------------------------- finalise
// Cross-block totals in FP64 (the paper's global sum for normalisation):
// estimate, N_eff, log-evidence.  Run by the last block of the step.
__device__ void finalize_block(const Partial *part, int n, DevSummary *sum, int32_t frame)
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
    }
}

// PC: pcSIR (cell map lookup) instead of the patch sum at the particle
template <int R, bool PC>
__global__ void __launch_bounds__(256) step_kernel(StepArgs a)
{
    int mode = a.mode;
    if (mode != MODE_CARRY && *a.degenerate)
        mode = MODE_CARRY;  // the last resample kept every particle
    const PatchGeom geom{a.Zp, a.W, a.H, a.Wp, a.pad, a.inv2s2, a.inv_sxi2, a.Kc, a.Hp, a.flags};
    // N < 2^31: 32-bit slot indices into per-component planes
    const int32_t N = (int32_t)a.N;
    const float *__restrict__ sx = a.src, *__restrict__ sy = a.src + a.N, *__restrict__ svx = a.src + 2 * a.N;
    const float *__restrict__ svy = a.src + 3 * a.N, *__restrict__ sI = a.src + 4 * a.N;
    const float *__restrict__ slw = a.src + 5 * a.N;
    float *__restrict__ dplane[6];
#pragma unroll
    for (int c = 0; c < 6; ++c)
        dplane[c] = a.dst + c * a.N;
    Acc acc;
    acc.init();
    // unsigned: i + stride stays below 2^32 for any N < 2^31.  The ancestor of
    // the next slot is loaded one iteration ahead, so the parent-state gather
    // does not wait on a dependent load.
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t pn = (i0 < (uint32_t)N) ? ((mode == MODE_CARRY) ? i0 : (uint32_t)__ldg(a.anc + i0)) : 0u;
    for (uint32_t i = i0; i < (uint32_t)N; i += stride) {
        uint32_t p = pn;
        if (i + stride < (uint32_t)N)
            pn = (mode == MODE_CARRY) ? i + stride : (uint32_t)__ldg(a.anc + i + stride);
        if (p >= (uint32_t)N) {  // caller-supplied ancestors are checked, never trusted
            atomicOr(a.flags, FLAG_BAD_ANCESTOR);
            p = i;
        }
        const float x = __ldg(sx + p), y = __ldg(sy + p);
        const float vx = __ldg(svx + p), vy = __ldg(svy + p);
        const float I0 = __ldg(sI + p);
        float lwp;
        if (mode == MODE_CARRY)
            lwp = __ldg(slw + p);
        else if (mode == MODE_UNIFORM)
            lwp = 0.0f;
        else
            lwp = __ldg(a.lwp + i);
        uint32_t f[6];
        prop_fields(philox_rk(make_uint4((uint32_t)i, a.frame, a.fid, PURPOSE_PROP << 8), a.rk), f);
        float e0, e1, e2, e3, e4, e5;
        box_muller(u21(f[0]), u21(f[1]), e0, e1);
        box_muller(u21(f[2]), u21(f[3]), e2, e3);
        box_muller(u21(f[4]), u21(f[5]), e4, e5);
        float v[5];
        v[0] = fmaf(a.sm, e0, x + vx);
        v[1] = fmaf(a.sm, e1, y + vy);
        v[2] = fmaf(a.sv, e2, vx);
        v[3] = fmaf(a.sv, e3, vy);
        v[4] = fmaf(a.sI, e4, I0);
        const float l = PC ? cell_loglik<R>(geom, a.lmap, v[0], v[1], v[4]) : patch_loglik<R>(geom, v[0], v[1], v[4]);
        const float lw = lwp + l;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            dplane[c][i] = v[c];
        dplane[5][i] = lw;
        acc.add_cur(lw, v);
        if (mode == MODE_UNIFORM)
            acc.add_prev_zero();
        else
            acc.add_prev(lwp);
    }
    // block reduction of the partial statistics
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc.shfl_merge(o);
    __shared__ Acc sh[8];
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
            Partial q;
            q.m = acc.m;
            q.s0 = acc.s0;
            q.s2 = acc.s2;
#pragma unroll
            for (int c = 0; c < 5; ++c)
                q.s[c] = acc.s[c];
            q.mp = acc.mp;
            q.sp = acc.sp;
            a.part[blockIdx.x] = q;
        }
    }
    // the last block to finish combines every block's partials (no waiting:
    // it only runs once all the others have published theirs)
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(a.done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        finalize_block(a.part, gridDim.x, a.sum, (int32_t)a.frame);
        if (threadIdx.x == 0)
            *a.done = 0u;
    }
}

// --------------------------------------------------------------- launchers
int step_grid(ppf_ctx *c)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<5, false>, 256, 0);
    if (per_sm < 1)
        per_sm = 1;
    int64_t need = (c->N + 255) / 256;
    int64_t g = (int64_t)c->num_sms * per_sm;
    return (int)(need < g ? need : g);
}

// pcSIR cell map: (B, C) of the patch sum at every anchor c in
// [-R, W-1+R] x [-R, H-1+R], PSF samples at the cell centre (offset 0); the
// same arithmetic as patch_loglik for a particle at the centre
struct KcArr {
    float v[MAX_RADIUS];
};

template <int R>
__global__ void cell_map_kernel(PatchGeom geom, KcArr kc, float2 *__restrict__ lmap)
{
    constexpr int P = 2 * R + 1;
    geom.Kc = kc.v;
    const int lw = geom.W + 2 * R, lh = geom.H + 2 * R;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < lw * lh; idx += gridDim.x * blockDim.x) {
        const int cx = idx % lw - R, cy = idx / lw - R;
        int ax, ay;
        float gx[P], gy[P], C, l;
        const bool inside = patch_setup<R>(geom, (float)cx, (float)cy, 1.0f, ax, ay, gx, gy, C, &l);
        lmap[idx] = inside ? make_float2(patch_sum<R, true>(geom, ax, ay, gx, gy), C) : make_float2(0.0f, 0.0f);
    }
}

template <int R>
static void launch_cell_map_r(const PatchGeom &g, const KcArr &kc, float2 *lmap, int n, cudaStream_t s)
{
    const int grid = (n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048;
    cell_map_kernel<R><<<grid, 256, 0, s>>>(g, kc, lmap);
}

cudaError_t launch_cell_map(ppf_ctx *c)
{
    const int R = c->m.patch_radius;
    PatchGeom g{c->Zp, c->m.width, c->m.height, c->Wp, c->pad, 0.0f, 0.0f, nullptr, c->Hp, &c->sum->flags};
    g.inv2s2 = 1.0f / (2.0f * c->m.psf_sigma * c->m.psf_sigma);
    g.inv_sxi2 = 1.0f / (c->m.sigma_xi * c->m.sigma_xi);
    KcArr kc;
    for (int k = 0; k < MAX_RADIUS; ++k)
        kc.v[k] = (float)exp(-(2.0 * k + 1.0) * (double)g.inv2s2);
    const int n = (c->m.width + 2 * R) * (c->m.height + 2 * R);
    switch (R) {
    case 0: launch_cell_map_r<0>(g, kc, c->lmap, n, c->stream); break;
    case 1: launch_cell_map_r<1>(g, kc, c->lmap, n, c->stream); break;
    case 2: launch_cell_map_r<2>(g, kc, c->lmap, n, c->stream); break;
    case 3: launch_cell_map_r<3>(g, kc, c->lmap, n, c->stream); break;
    case 4: launch_cell_map_r<4>(g, kc, c->lmap, n, c->stream); break;
    case 5: launch_cell_map_r<5>(g, kc, c->lmap, n, c->stream); break;
    case 6: launch_cell_map_r<6>(g, kc, c->lmap, n, c->stream); break;
    case 7: launch_cell_map_r<7>(g, kc, c->lmap, n, c->stream); break;
    default: launch_cell_map_r<8>(g, kc, c->lmap, n, c->stream); break;
    }
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_init(ppf_ctx *c)
{
    const int grid = (int)((c->N + 255) / 256 < 65536 ? (c->N + 255) / 256 : 65536);
    init_kernel<<<grid, 256, 0, c->stream>>>(c->state[c->cur], c->N, c->m.seed, c->m.filter_id,
                                              (float)c->m.width, (float)c->m.height, c->m.v0_max,
                                              c->m.amplitude);
    return cudaGetLastError();
}

cudaError_t launch_prepare_frame(ppf_ctx *c, const void *frame)
{
    prof_mark(c, PH_PREPARE, 0);
    c->launches += 1;
    const int64_t n = (int64_t)c->Wp * c->Hp;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    const float bg = c->m.background;
    switch (c->m.frame_dtype) {
    case PPF_BF16:
        prepare_frame_kernel<__nv_bfloat16><<<grid, 256, 0, c->stream>>>(
            (const __nv_bfloat16 *)frame, c->Zp, c->m.width, c->m.height, c->Wp, c->Hp, c->pad, bg);
        break;
    case PPF_F16:
        prepare_frame_kernel<__half><<<grid, 256, 0, c->stream>>>(
            (const __half *)frame, c->Zp, c->m.width, c->m.height, c->Wp, c->Hp, c->pad, bg);
        break;
    default:
        prepare_frame_kernel<float><<<grid, 256, 0, c->stream>>>(
            (const float *)frame, c->Zp, c->m.width, c->m.height, c->Wp, c->Hp, c->pad, bg);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c->lmap)
        e = launch_cell_map(c);  // pcSIR: the patch sums of every anchor of this frame
    prof_mark(c, PH_PREPARE, 1);
    return e;
}

template <int R>
static void launch_step_r(const StepArgs &a, int grid, cudaStream_t s)
{
    if (a.lmap)
        step_kernel<R, true><<<grid, 256, 0, s>>>(a);
    else
        step_kernel<R, false><<<grid, 256, 0, s>>>(a);
}

cudaError_t launch_step(ppf_ctx *c, int32_t k)
{
    StepArgs a;
    a.N = c->N;
    a.W = c->m.width;
    a.H = c->m.height;
    a.Wp = c->Wp;
    a.Hp = c->Hp;
    a.pad = c->pad;
    a.inv2s2 = 1.0f / (2.0f * c->m.psf_sigma * c->m.psf_sigma);
    for (int k = 0; k < MAX_RADIUS; ++k)
        a.Kc[k] = (float)exp(-(2.0 * k + 1.0) * (double)a.inv2s2);
    a.inv_sxi2 = 1.0f / (c->m.sigma_xi * c->m.sigma_xi);
    a.sm = c->m.sigma_m;
    a.sv = c->m.sigma_v;
    a.sI = c->m.sigma_I;
    a.seed = c->m.seed;
    a.rk = philox_keys(c->m.seed);
    a.fid = c->m.filter_id;
    a.frame = (uint32_t)k;
    a.src = c->state[c->cur];
    a.dst = c->state[c->cur ^ 1];
    a.anc = c->anc;
    a.lwp = c->lwp;
    a.degenerate = &c->sum->degenerate;
    a.flags = &c->sum->flags;
    a.mode = c->mode;
    a.Zp = c->Zp;
    a.lmap = c->lmap;
    a.part = c->part;
    a.done = &c->sum->blocks_done;
    a.sum = c->sum;
    const int grid = step_grid(c);
    prof_mark(c, PH_STEP, 0);
    switch (c->m.patch_radius) {
    case 0: launch_step_r<0>(a, grid, c->stream); break;
    case 1: launch_step_r<1>(a, grid, c->stream); break;
    case 2: launch_step_r<2>(a, grid, c->stream); break;
    case 3: launch_step_r<3>(a, grid, c->stream); break;
    case 4: launch_step_r<4>(a, grid, c->stream); break;
    case 5: launch_step_r<5>(a, grid, c->stream); break;
    case 6: launch_step_r<6>(a, grid, c->stream); break;
    case 7: launch_step_r<7>(a, grid, c->stream); break;
    default: launch_step_r<8>(a, grid, c->stream); break;
    }
    prof_mark(c, PH_STEP, 1);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace ppf
