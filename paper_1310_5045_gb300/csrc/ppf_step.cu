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
                                     int Hp, int pad, float bg, DevSummary *sum, int force,
                                     uint32_t *__restrict__ bin_tot, int nbins)
{
    // the likelihood path of this step: the caller's choice, else the one the
    // previous step's finaliser decided; and the binned path's counts cleared
    if (blockIdx.x == 0 && threadIdx.x == 0 && sum)
        sum->bin_this = force >= 0 ? force : sum->bin_next;
    if (bin_tot)  // the bin sizes and the scatter's cursors
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * (nbins + 1); t += gridDim.x * blockDim.x)
            bin_tot[t] = 0u;
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
    // binned path: the bin of every slot (then its place in bin order), the
    // bin sizes, and every record's l in bin order
    uint32_t *__restrict__ bin_key;
    uint32_t *__restrict__ bin_tot;
    const float *__restrict__ bin_l;
    BinGeom bg;
};

// PC: pcSIR (cell map lookup) instead of the patch sum at the particle
// The propagation of slot i (Sec. 7.1 NCV dynamics, bootstrap proposal):
// parent p, its state, the starting log-weight, the five propagated values.
struct Propagated {
    float v[5];
    float lwp;
};

__device__ __forceinline__ Propagated propagate_slot(const StepArgs &a, int mode, uint32_t i, uint32_t p)
{
    const float *__restrict__ src = a.src;
    const int64_t n = a.N;
    const float x = __ldg(src + p), y = __ldg(src + n + p);
    const float vx = __ldg(src + 2 * n + p), vy = __ldg(src + 3 * n + p);
    const float I0 = __ldg(src + 4 * n + p);
    Propagated r;
    if (mode == MODE_CARRY)
        r.lwp = __ldg(src + 5 * n + p);
    else if (mode == MODE_UNIFORM)
        r.lwp = 0.0f;
    else
        r.lwp = __ldg(a.lwp + i);
    uint32_t f[6];
    prop_fields(philox_rk(make_uint4(i, a.frame, a.fid, PURPOSE_PROP << 8), a.rk), f);
    float e0, e1, e2, e3, e4, e5;
    box_muller(u21(f[0]), u21(f[1]), e0, e1);
    box_muller(u21(f[2]), u21(f[3]), e2, e3);
    box_muller(u21(f[4]), u21(f[5]), e4, e5);
    r.v[0] = fmaf(a.sm, e0, x + vx);
    r.v[1] = fmaf(a.sm, e1, y + vy);
    r.v[2] = fmaf(a.sv, e2, vx);
    r.v[3] = fmaf(a.sv, e3, vy);
    r.v[4] = fmaf(a.sI, e4, I0);
    return r;
}

// the warps' spread counts of this block into the step's counters
__device__ __forceinline__ void publish_spread(DevSummary *sum, unsigned ns, unsigned nt)
{
    ns = __reduce_add_sync(0xffffffffu, ns);
    nt = __reduce_add_sync(0xffffffffu, nt);
    if ((threadIdx.x & 31) == 0 && nt) {
        atomicAdd(&sum->spread_warps, ns);
        atomicAdd(&sum->total_warps, nt);
    }
}

// The binned path's first pass: propagate every slot, write its state (the
// log-weight plane is filled by the sums of phase 1), its bin, and count the
// bin sizes (a shared-memory histogram per block, added to the global one).
// Particles of one bin may land in any order: the likelihood of each does not
// depend on it, and the sums are taken in slot order.
template <int R>
__device__ __forceinline__ void bin_propagate(const StepArgs &a, int mode)
{
    __shared__ uint32_t shist[BIN_MAX_BINS];
    const int nb = a.bg.nbins;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        shist[t] = 0u;
    __syncthreads();
    const int32_t N = (int32_t)a.N;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned ns = 0, nt = 0, it = 0;
    const uint32_t ts = blockIdx.x % (((uint32_t)N / stride) > 0 ? ((uint32_t)N / stride) : 1u);
    float tx = 0.0f, ty = 0.0f;
    bool tok = false;
    uint32_t pn = (i0 < (uint32_t)N) ? ((mode == MODE_CARRY) ? i0 : (uint32_t)__ldg(a.anc + i0)) : 0u;
    for (uint32_t i = i0; i < (uint32_t)N; i += stride, ++it) {
        uint32_t p = pn;
        if (i + stride < (uint32_t)N)
            pn = (mode == MODE_CARRY) ? i + stride : (uint32_t)__ldg(a.anc + i + stride);
        if (p >= (uint32_t)N) {  // caller-supplied ancestors are checked, never trusted
            atomicOr(a.flags, FLAG_BAD_ANCESTOR);
            p = i;
        }
        const Propagated q = propagate_slot(a, mode, i, p);
#pragma unroll
        for (int c = 0; c < 5; ++c)
            a.dst[c * a.N + i] = q.v[c];
        const uint32_t key = bin_of<R>(a.bg, a.W, a.H, q.v[0], q.v[1], q.v[4]);
        a.bin_key[i] = key;
        atomicAdd(&shist[key], 1u);
        if (it == ts) {
            tx = q.v[0];
            ty = q.v[1];
            tok = true;
        }
    }
    spread_tally(tx, ty, tok, ns, nt);
    publish_spread(a.sum, ns, nt);
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        if (shist[t])
            atomicAdd(a.bin_tot + t, shist[t]);
}

// PC: pcSIR (cell map lookup) instead of the patch sum at the particle.
// Phase 0: with the binned path chosen for this step (bin_this), only
// propagate and bin (bin_propagate); otherwise the whole direct step.
// Phase 1 (launched after the binned likelihood; returns at once on the
// direct path): the binned path's sums.  It visits the slots in the direct
// path's order, reads each slot's state and its l, forms lw = lw_prev + l and
// accumulates exactly as the direct path does, so both paths give the same
// bits for every result of the step.
template <int R, bool PC>
__global__ void __launch_bounds__(256, 3) step_kernel(StepArgs a, int phase)
{
    if (phase == 1)
        pdl_wait();  // the binned likelihood's l (launched as a dependent of it)
    else
        pdl_trigger();  // the binned path's kernels may be scheduled meanwhile
    int mode = a.mode;
    if (mode != MODE_CARRY && *a.degenerate)
        mode = MODE_CARRY;  // the last resample kept every particle
    const bool binned = !PC && a.bin_key && __ldcg(&a.sum->bin_this) != 0;
    if (phase == 0 && binned) {
        bin_propagate<R>(a, mode);
        return;
    }
    if (phase == 1 && !binned)
        return;
    const PatchGeom geom{a.Zp, a.W, a.H, a.Wp, a.pad, a.inv2s2, a.inv_sxi2, a.Kc, a.Hp, a.flags};
    // N < 2^31: 32-bit slot indices into per-component planes
    const int32_t N = (int32_t)a.N;
    float *__restrict__ dplane[6];
#pragma unroll
    for (int c = 0; c < 6; ++c)
        dplane[c] = a.dst + c * a.N;
    Acc acc;
    acc.init();
    unsigned ns = 0, nt = 0;
    // unsigned: i + stride stays below 2^32 for any N < 2^31.  The ancestor of
    // the next slot is loaded one iteration ahead, so the parent-state gather
    // does not wait on a dependent load.
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const float *__restrict__ sx = a.src, *__restrict__ sy = a.src + a.N, *__restrict__ svx = a.src + 2 * a.N;
    const float *__restrict__ svy = a.src + 3 * a.N, *__restrict__ sI = a.src + 4 * a.N;
    const float *__restrict__ slw = a.src + 5 * a.N;
    if (phase == 1) {
        // l of slot i sits in bin order at the place its key entry now holds
        for (uint32_t i = i0; i < (uint32_t)N; i += stride) {
            float v[5];
#pragma unroll
            for (int c = 0; c < 5; ++c)
                v[c] = __ldcg(dplane[c] + i);
            const float l = __ldcg(a.bin_l + __ldcg(a.bin_key + i));
            float lwp;
            if (mode == MODE_CARRY)
                lwp = __ldg(slw + i);  // identity ancestry
            else if (mode == MODE_UNIFORM)
                lwp = 0.0f;
            else
                lwp = __ldg(a.lwp + i);
            const float lw = lwp + l;
            dplane[5][i] = lw;
            acc.add_cur(lw, v);
            if (mode == MODE_UNIFORM)
                acc.add_prev_zero();
            else
                acc.add_prev(lwp);
        }
    } else {
        uint32_t pn = (i0 < (uint32_t)N) ? ((mode == MODE_CARRY) ? i0 : (uint32_t)__ldg(a.anc + i0)) : 0u;
        // the spread statistic samples one iteration per block, blocks spread
        // over the slots; its anchors are kept and tallied after the loop
        const uint32_t ts = blockIdx.x % (((uint32_t)N / stride) > 0 ? ((uint32_t)N / stride) : 1u);
        float tx = 0.0f, ty = 0.0f;
        bool tok = false;
        unsigned it = 0;
        for (uint32_t i = i0; i < (uint32_t)N; i += stride, ++it) {
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
            if (it == ts) {
                tx = v[0];
                ty = v[1];
                tok = true;
            }
        }
        if (!PC) {
            spread_tally(tx, ty, tok, ns, nt);
            publish_spread(a.sum, ns, nt);
        }
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
    // pcSIR and contexts without the binned path take the direct path
    const int force = c->bin_key ? c->bin_force : 0;
    switch (c->m.frame_dtype) {
    case PPF_BF16:
        prepare_frame_kernel<__nv_bfloat16><<<grid, 256, 0, c->stream>>>(
            (const __nv_bfloat16 *)frame, c->Zp, c->m.width, c->m.height, c->Wp, c->Hp, c->pad, bg, c->sum, force, c->bin_tot,
            c->bin_nbins);
        break;
    case PPF_F16:
        prepare_frame_kernel<__half><<<grid, 256, 0, c->stream>>>(
            (const __half *)frame, c->Zp, c->m.width, c->m.height, c->Wp, c->Hp, c->pad, bg, c->sum, force, c->bin_tot,
            c->bin_nbins);
        break;
    default:
        prepare_frame_kernel<float><<<grid, 256, 0, c->stream>>>(
            (const float *)frame, c->Zp, c->m.width, c->m.height, c->Wp, c->Hp, c->pad, bg, c->sum, force, c->bin_tot,
            c->bin_nbins);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c->lmap)
        e = launch_cell_map(c);  // pcSIR: the patch sums of every anchor of this frame
    prof_mark(c, PH_PREPARE, 1);
    return e;
}

template <int R>
static void launch_step_r(const StepArgs &a, int grid, int phase, cudaStream_t s)
{
    if (phase == 1)  // the binned path's sums: a dependent launch (it waits for the likelihood)
        launch_pdl(step_kernel<R, false>, grid, 256, 0, s, a, phase);
    else if (a.lmap)
        step_kernel<R, true><<<grid, 256, 0, s>>>(a, phase);
    else
        step_kernel<R, false><<<grid, 256, 0, s>>>(a, phase);
}

static void launch_step_phase(const StepArgs &a, int R, int grid, int phase, cudaStream_t s)
{
    switch (R) {
    case 0: launch_step_r<0>(a, grid, phase, s); break;
    case 1: launch_step_r<1>(a, grid, phase, s); break;
    case 2: launch_step_r<2>(a, grid, phase, s); break;
    case 3: launch_step_r<3>(a, grid, phase, s); break;
    case 4: launch_step_r<4>(a, grid, phase, s); break;
    case 5: launch_step_r<5>(a, grid, phase, s); break;
    case 6: launch_step_r<6>(a, grid, phase, s); break;
    case 7: launch_step_r<7>(a, grid, phase, s); break;
    default: launch_step_r<8>(a, grid, phase, s); break;
    }
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
    a.bin_key = c->bin_key;
    a.bin_tot = c->bin_tot;
    a.bin_l = c->bin_l;
    a.bg = BinGeom{c->bin_T, c->bin_nx, c->bin_nbins};
    const int grid = step_grid(c);
    prof_mark(c, PH_STEP, 0);
    launch_step_phase(a, c->m.patch_radius, grid, 0, c->stream);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c->bin_key && c->bin_force != 0) {  // (a forced direct path needs none of them)
        // the binned path's scatter and likelihood, then its sums; all three
        // return at once when this step takes the direct path
        e = launch_binned(c);
        if (e == cudaSuccess) {
            launch_step_phase(a, c->m.patch_radius, grid, 1, c->stream);
            c->launches += 1;
            e = cudaGetLastError();
        }
    }
    prof_mark(c, PH_STEP, 1);
    return e;
}

}  // namespace ppf
