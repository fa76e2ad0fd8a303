// ppf_batch.cu -- F independent SIR filters (the paper's bank of particle
// filters, Sec. 3 "MPF") with uneven particle counts, stepped together:
//   * all particles of all filters live in one concatenated 6 x Ntot SoA
//     state; filter f owns slots [off_f, off_f + n_f);
//   * one persistent kernel per frame walks work units (filter, run of at most
//     `unit` particles) and writes per-unit weight statistics;
//   * a per-filter FP64 finalisation (one warp per filter) gives each
//     filter's estimate, N_eff and log-evidence;
//   * one block per filter resamples it systematically (Alg. 1) on 64-bit
//     fixed point, exactly as a single filter with filter id f would;
//   * a whole movie of K frames can be captured in one CUDA graph;
//   * an autotuner times launch shapes (block size, blocks per SM, unit size)
//     on the caller's data and keeps the fastest.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ppf_device.cuh"
#include "ppf_internal.h"
#include "ppf_kernels.cuh"
#include "ppf_tiles.cuh"
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace ppf {

struct FilterParams {
    int64_t off, n;
    uint64_t seed;
    Divisor ndiv;             // n as a divisor of the ticket grid
    double ess_thr;           // Alg. 1's test: resample only while N_eff < ess_thr (+inf: always)
    uint32_t fid;
    float inv2s2, inv_sxi2, sm, sv, sI, bg;
    float Kc[MAX_RADIUS];
};

// same layout as ppf_filter_estimate_t
struct FilterSummary {
    double mean[5];
    double log_evidence;
    double ess;
    float M;
    int32_t degenerate;
};
static_assert(sizeof(FilterSummary) == sizeof(ppf_filter_estimate_t), "layout");

// Device-resident position in a frame sequence: the kernels of one frame
// iteration read their frame index, frame and estimate slot from here, so a
// single captured iteration can be replayed frame after frame.
struct BatchCursor {
    const char *frames;       // K x F x H x W (or one F x H x W frame)
    int64_t frame_bytes;      // bytes of one F x H x W frame
    FilterSummary *est;       // optional K x F estimates
    int32_t k;                // frame index of the current iteration
    int32_t t;                // position in the sequence
    int32_t cur;              // state buffer holding the particles the step starts from
    int32_t first;            // the step starts from the prior draw (identity ancestry)
};

}  // namespace ppf

struct ppf_batch {
    int32_t F;
    int64_t Ntot;
    int32_t W, H, r, Wp, Hp, pad;
    int32_t dtype;
    size_t frame_bytes;                // one filter's frame
    cudaStream_t stream;
    int num_sms;
    std::vector<ppf_model> models;
    std::vector<int64_t> n, off;
    ppf::FilterParams *fp;             // device [F]
    std::vector<ppf::FilterParams> hp; // host copy of fp
    int32_t *fkeep;                    // device [F]: the last resample kept the filter's particles
    float *state[2];
    int cur;
    int32_t *anc;
    float *Zp;                         // F x Hp x Wp pixel pairs (float2): (Z(col), Z(col + 1))
    // work units
    int32_t unit, block, bps;          // tuned launch shape
    int32_t U;
    int32_t *unit_f;                   // device [U]
    int64_t *unit_lo;
    int32_t *unit_n;
    int32_t *fu_off;                   // device [F + 1]: units of filter f
    // resampling tiles: every filter cut into runs of at most TILE particles
    int32_t T;
    int32_t *tile_f;                   // device [T]
    int64_t *tile_lo;
    int32_t *tile_n;
    int32_t *ft_off;                   // device [F + 1]: tiles of filter f
    uint64_t *tQ;                      // device [T] tile totals
    uint64_t *tC;                      // device [T] exclusive prefix within the filter
    int64_t *tT;                       // device [T + 1]: first ticket of the tile (filter-local)
    uint64_t *fQu;                     // device [4F]: per filter Q_f, u_f, Q_f / n_f, Q_f mod n_f
    ppf::Partial *upart;               // device [U]
    ppf::FilterSummary *fsum;          // device [F]
    ppf::FilterSummary *fsum_host;     // pinned [F]
    ppf::FilterSummary *fsum_run;      // device [K x F] of the last graph run
    int64_t fsum_run_cap;
    int32_t *flags;                    // device: FLAG_DEGENERATE (a degenerate filter), FLAG_INTERNAL (a debug check)
    ppf::BatchCursor *cursor;          // device
    cudaStream_t gstream;              // stream the cached graph runs on
    cudaGraphExec_t gexec;             // cached one-frame iteration
    bool first;                        // next step starts from the prior draw
    bool weighted;
    int32_t last_k;
    int64_t launches;
    char err[256];
};

namespace ppf {
namespace {

// ------------------------------------------------------------------ kernels
__global__ void batch_init_kernel(float *__restrict__ st, int64_t Ntot, const FilterParams *__restrict__ fp,
                                  const int32_t *__restrict__ unit_f, const int64_t *__restrict__ unit_lo,
                                  const int32_t *__restrict__ unit_n, int32_t U, float W, float H,
                                  const float *__restrict__ v0A)
{
    for (int32_t u = blockIdx.x; u < U; u += gridDim.x) {
        const int32_t f = unit_f[u];
        const FilterParams P = fp[f];
        const float v0 = v0A[2 * f], A = v0A[2 * f + 1];
        for (int32_t j = threadIdx.x; j < unit_n[u]; j += blockDim.x) {
            const int64_t i = unit_lo[u] + j;
            const uint32_t slot = (uint32_t)(i - P.off);
            const uint4 a = draw(P.seed, slot, 0u, P.fid, PURPOSE_INIT, 0);
            const uint4 b = draw(P.seed, slot, 0u, P.fid, PURPOSE_INIT, 1);
            st[i] = -0.5f + W * u01(a.x);
            st[Ntot + i] = -0.5f + H * u01(a.y);
            st[2 * Ntot + i] = v0 * (2.0f * u01(a.z) - 1.0f);
            st[3 * Ntot + i] = v0 * (2.0f * u01(a.w) - 1.0f);
            st[4 * Ntot + i] = A * (0.5f + u01(b.x));
            st[5 * Ntot + i] = 0.0f;
        }
    }
}

// frames F x H x W -> padded F x Hp x Wp, minus each filter's background
template <typename T>
__device__ __forceinline__ float tof(T v);
template <>
__device__ __forceinline__ float tof<float>(float v) { return v; }
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float tof<__half>(__half v) { return __half2float(v); }

__global__ void batch_set_cursor(BatchCursor *c, const char *frames, int64_t frame_bytes, FilterSummary *est,
                                 int32_t k, int32_t t, int32_t cur, int32_t first)
{
    c->frames = frames;
    c->frame_bytes = frame_bytes;
    c->est = est;
    c->k = k;
    c->t = t;
    c->cur = cur;
    c->first = first;
}

// start of one frame iteration of a sequence: next frame; after the first
// iteration the particles of the previous one are current and resampled
__global__ void batch_advance(BatchCursor *c)
{
    c->k += 1;
    c->t += 1;
    if (c->t > 0) {
        c->cur ^= 1;
        c->first = 0;
    }
}

template <typename T>
__global__ void batch_prepare_kernel(const BatchCursor *__restrict__ cur, float *__restrict__ Zp, int32_t F, int W,
                                     int H, int Wp, int Hp, int pad, const FilterParams *__restrict__ fp)
{
    // one warp per padded row (F * Hp rows), lanes across its columns; each
    // element is the pixel pair (Z(col), Z(col + 1)) minus the background
    const T *Z = reinterpret_cast<const T *>(cur->frames + cur->frame_bytes * cur->t);
    const int lane = threadIdx.x & 31;
    const int32_t rows = F * Hp;
    const int32_t nw = (int32_t)(gridDim.x * (blockDim.x >> 5));
    for (int32_t row = (int32_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); row < rows; row += nw) {
        const int32_t f = row / Hp;
        const int py = row - f * Hp - pad;
        const float bg = fp[f].bg;
        float2 *__restrict__ out = reinterpret_cast<float2 *>(Zp) + (int64_t)row * Wp;
        const bool in_row = py >= 0 && py < H;
        const T *zrow = Z + ((int64_t)f * H + (in_row ? py : 0)) * W;
        for (int c = lane; c < Wp; c += 32) {
            const int px = c - pad;
            out[c] = make_float2((in_row && px >= 0 && px < W) ? tof<T>(zrow[px]) - bg : 0.0f,
                                 (in_row && px + 1 >= 0 && px + 1 < W) ? tof<T>(zrow[px + 1]) - bg : 0.0f);
        }
    }
}

struct BatchStepArgs {
    int64_t Ntot;
    int W, H, Wp, Hp, pad;
    const BatchCursor *cur;
    const FilterParams *__restrict__ fp;
    const int32_t *__restrict__ unit_f;
    const int64_t *__restrict__ unit_lo;
    const int32_t *__restrict__ unit_n;
    int32_t U;
    float *st0, *st1;           // the two state buffers; the cursor says which is current
    const int32_t *__restrict__ anc;
    const int32_t *__restrict__ fkeep;
    const float *__restrict__ Zp;
    Partial *__restrict__ part;
    int32_t *flags;             // FLAG_INTERNAL from a failed debug check
};

// Persistent SIS step over all work units of all filters.  A unit is a run
// of at most `unit` particles of one filter and belongs to one warp: the warp
// steps its particles (the next slot's ancestor loaded one iteration ahead)
// and reduces their weight statistics with shuffles into the unit's partial,
// with no block-wide synchronisation.
template <int R>
__global__ void batch_step_kernel(BatchStepArgs a)
{
    const uint32_t N = (uint32_t)a.Ntot;  // < 2^31
    const uint32_t frame = (uint32_t)a.cur->k;
    const bool first = a.cur->first != 0;
    const float *__restrict__ src = a.cur->cur ? a.st1 : a.st0;
    float *__restrict__ dst = a.cur->cur ? a.st0 : a.st1;
    const float *__restrict__ sx = src, *__restrict__ sy = src + N, *__restrict__ svx = src + 2 * (size_t)N;
    const float *__restrict__ svy = src + 3 * (size_t)N, *__restrict__ sI = src + 4 * (size_t)N;
    const float *__restrict__ slw = src + 5 * (size_t)N;
    __shared__ float kcs[32][MAX_RADIUS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int32_t nwarps = (int32_t)(gridDim.x * (blockDim.x >> 5));
    for (int32_t u = (int32_t)(blockIdx.x * (blockDim.x >> 5)) + wib; u < a.U; u += nwarps) {
        const int32_t f = a.unit_f[u];
        const FilterParams *__restrict__ P = a.fp + f;
        const uint32_t off = (uint32_t)P->off, nf = (uint32_t)P->n;
        const uint64_t seed = P->seed;
        const uint32_t fid = P->fid;
        const float sm = P->sm, sv = P->sv, sIn = P->sI;
        __syncwarp();
        if (lane < R)
            kcs[wib][lane] = P->Kc[lane];
        __syncwarp();
        const PatchGeom geom{a.Zp + (int64_t)f * 2 * a.Wp * a.Hp, a.W, a.H, a.Wp, a.pad, P->inv2s2, P->inv_sxi2,
                             kcs[wib], a.Hp, a.flags};
        // after the prior draw, or when the last resample kept this filter's
        // particles, every slot continues its own particle with its weight
        const bool carry = first || a.fkeep[f] != 0;
        Acc acc;
        acc.init();
        const uint32_t lo = (uint32_t)a.unit_lo[u];
        const int32_t n = a.unit_n[u];
        uint32_t pn = (lane < n) ? (carry ? lo + lane : (uint32_t)__ldg(a.anc + lo + lane)) : 0u;
        for (int32_t j = lane; j < n; j += 32) {
            const uint32_t i = lo + (uint32_t)j;
            uint32_t p = pn;
            if (j + 32 < n)
                pn = carry ? i + 32 : (uint32_t)__ldg(a.anc + i + 32);
            if (p < off || p >= off + nf)
                p = i;  // ancestors never cross filters
            const float x = __ldg(sx + p), y = __ldg(sy + p);
            const float vx = __ldg(svx + p), vy = __ldg(svy + p);
            const float I0 = __ldg(sI + p);
            const float lwp = carry ? __ldg(slw + p) : 0.0f;
            uint32_t fl[6];
            prop_fields(draw(seed, i - off, frame, fid, PURPOSE_PROP, 0), fl);
            float e0, e1, e2, e3, e4, e5;
            box_muller(u21(fl[0]), u21(fl[1]), e0, e1);
            box_muller(u21(fl[2]), u21(fl[3]), e2, e3);
            box_muller(u21(fl[4]), u21(fl[5]), e4, e5);
            float v[5];
            v[0] = fmaf(sm, e0, x + vx);
            v[1] = fmaf(sm, e1, y + vy);
            v[2] = fmaf(sv, e2, vx);
            v[3] = fmaf(sv, e3, vy);
            v[4] = fmaf(sIn, e4, I0);
            const float lw = lwp + patch_loglik<R, false>(geom, v[0], v[1], v[4]);
#pragma unroll
            for (int c = 0; c < 5; ++c)
                dst[(size_t)c * N + i] = v[c];
            dst[5 * (size_t)N + i] = lw;
            acc.add_cur(lw, v);
            if (carry)
                acc.add_prev(lwp);
            else
                acc.add_prev_zero();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            acc.shfl_merge(o);
        if (lane == 0) {
            Partial q;
            q.m = acc.m;
            q.s0 = acc.s0;
            q.s2 = acc.s2;
            for (int c = 0; c < 5; ++c)
                q.s[c] = acc.s[c];
            q.mp = acc.mp;
            q.sp = acc.sp;
            a.part[u] = q;
        }
    }
}

// one warp per filter: FP64 combination of its units' partials
__global__ void batch_finalize_kernel(const Partial *__restrict__ part, const int32_t *__restrict__ fu_off, int32_t F,
                                      FilterSummary *__restrict__ fs, const BatchCursor *__restrict__ cur)
{
    const int32_t f = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= F)
        return;
    const int32_t u0 = fu_off[f], u1 = fu_off[f + 1];
    float m = -INFINITY, mp = -INFINITY;
    for (int32_t u = u0 + lane; u < u1; u += 32) {
        m = fmaxf(m, part[u].m);
        mp = fmaxf(mp, part[u].mp);
    }
    m = warp_max(m);
    mp = warp_max(mp);
    double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int32_t u = u0 + lane; u < u1; u += 32) {
        const Partial q = part[u];
        if (q.m > -INFINITY) {
            const double sc = (double)expf(q.m - m);
            t[0] += q.s0 * sc;
            for (int c = 0; c < 5; ++c)
                t[1 + c] += q.s[c] * sc;
            t[6] += q.s2 * sc * sc;
        }
        if (q.mp > -INFINITY)
            t[7] += q.sp * (double)expf(q.mp - mp);
    }
    for (int c = 0; c < 8; ++c)
        t[c] = warp_sum_d(t[c]);
    if (lane == 0) {
        FilterSummary s;
        for (int c = 0; c < 5; ++c)
            s.mean[c] = t[1 + c] / t[0];
        s.ess = t[0] * t[0] / t[6];
        s.log_evidence = ((double)m + log(t[0])) - ((double)mp + log(t[7]));
        s.M = m;
        s.degenerate = (t[0] > 0.0) ? 0 : 1;
        fs[f] = s;
        if (cur->est)
            cur->est[(int64_t)cur->t * F + f] = s;
    }
}

// Systematic resampling of every filter (Alg. 1) on 64-bit fixed point,
// the same tickets as a single filter with filter id f, in three balanced
// passes over tiles of at most TILE particles:
//   1. tile totals of the fixed-point weights (one block per tile);
//   2. per filter (one warp): exclusive prefix over its tiles, total Q_f,
//      ticket offset u_f and each tile's first ticket;
//   3. one block per tile: its cumulative weights and the parents of its
//      tickets.  A filter with no usable weight keeps its particles.
__global__ void __launch_bounds__(TILE_THREADS) batch_tile_totals(const float *st0, const float *st1, int64_t Ntot,
                                                                  const FilterParams *__restrict__ fp,
                                                                  const FilterSummary *__restrict__ fs,
                                                                  const BatchCursor *__restrict__ cur,
                                                                  const int32_t *__restrict__ tile_f,
                                                                  const int64_t *__restrict__ tile_lo,
                                                                  const int32_t *__restrict__ tile_n,
                                                                  uint64_t *__restrict__ tQ)
{
    __shared__ uint64_t red[33];
    const float *__restrict__ lw = (cur->cur ? st0 : st1) + 5 * Ntot;
    const int32_t t = blockIdx.x, f = tile_f[t];
    if (fs[f].ess >= fp[f].ess_thr)
        return;  // N_eff test: this filter keeps its particles
    const float Mf = fs[f].M;
    const int s = scale_bits(fp[f].n);
    const int n = tile_n[t];
    const float *__restrict__ w = lw + tile_lo[t];
    // all loads first (independent, in flight together), then the quantiser
    float v[TILE_ITEMS];
#pragma unroll
    for (int k = 0; k < TILE_ITEMS; ++k) {
        const int i = threadIdx.x + k * TILE_THREADS;
        v[k] = (i < n) ? __ldg(w + i) : -INFINITY;
    }
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < TILE_ITEMS; k += 2) {
        uint64_t a, b;
        quantise2(v[k], v[k + 1], Mf, s, a, b);
        acc += a + b;
    }
    uint64_t total;
    block_excl_scan_u64(acc, red, &total);
    if (threadIdx.x == 0)
        tQ[t] = total;
}

__global__ void batch_tile_scan(const FilterParams *__restrict__ fp, const FilterSummary *__restrict__ fs,
                                const BatchCursor *__restrict__ cur, const int32_t *__restrict__ ft_off, int32_t F,
                                const uint64_t *__restrict__ tQ, uint64_t *__restrict__ tC, int64_t *__restrict__ tT,
                                uint64_t *__restrict__ fQu, int32_t *__restrict__ fkeep, int32_t *__restrict__ flags)
{
    const int32_t f = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= F)
        return;
    const int32_t t0 = ft_off[f], t1 = ft_off[f + 1];
    const FilterParams P = fp[f];
    if (fs[f].ess >= P.ess_thr) {  // N_eff test: keep the particles, carry the weights
        if (lane == 0) {
            fQu[4 * f] = 0ull;
            fkeep[f] = 1;
        }
        return;
    }
    uint64_t carry = 0;
    for (int32_t base = t0; base < t1; base += 32) {
        const int32_t t = base + lane;
        const uint64_t v = (t < t1) ? tQ[t] : 0ull;
        const uint64_t incl = warp_incl_scan_u64(v);
        if (t < t1)
            tC[t] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    const uint64_t Q = carry;
    const uint64_t u = (Q == 0ull) ? 0ull : ticket_offset(P.seed, P.fid, (uint32_t)cur->k, PURPOSE_RESAMPLE, 0u, Q);
    if (lane == 0) {
        fQu[4 * f] = Q;
        fQu[4 * f + 1] = u;
        fQu[4 * f + 2] = Q / (uint64_t)P.n;
        fQu[4 * f + 3] = Q % (uint64_t)P.n;
        fkeep[f] = (Q == 0ull) ? 1 : 0;  // no usable weight: kept as well
        if (Q == 0ull)
            atomicOr(flags, FLAG_DEGENERATE);
    }
    if (Q == 0ull) {
        for (int32_t t = t0 + lane; t < t1; t += 32)
            tT[t] = 0;
        return;
    }
    const TicketGrid tg = ticket_grid(Q, u, Q / (uint64_t)P.n, (uint32_t)(Q % (uint64_t)P.n), P.ndiv);
    for (int32_t t = t0 + lane; t < t1; t += 32)
        tT[t] = tickets_below_grid(tC[t], tg);
}

__global__ void __launch_bounds__(TILE_THREADS) batch_fill(const float *st0, const float *st1, int64_t Ntot,
                                                           const FilterParams *__restrict__ fp,
                                                           const FilterSummary *__restrict__ fs,
                                                           const BatchCursor *__restrict__ cur,
                                                           const int32_t *__restrict__ tile_f,
                                                           const int64_t *__restrict__ tile_lo,
                                                           const int32_t *__restrict__ tile_n,
                                                           const int32_t *__restrict__ ft_off,
                                                           const uint64_t *__restrict__ tC,
                                                           const int64_t *__restrict__ tT,
                                                           const uint64_t *__restrict__ fQu, int32_t *__restrict__ anc,
                                                           int32_t *flags)
{
    extern __shared__ uint64_t fill_smem[];  // FILL_SMEM_BYTES
    uint64_t *C = fill_smem;
    uint16_t *stage = reinterpret_cast<uint16_t *>(fill_smem + TILE_SMEM_U64);
    __shared__ uint64_t red[33];
    const float *__restrict__ lw = (cur->cur ? st0 : st1) + 5 * Ntot;
    const int32_t t = blockIdx.x, f = tile_f[t];
    const FilterParams P = fp[f];
    const int64_t lo = tile_lo[t];
    const int n = tile_n[t];
    const uint64_t Q = fQu[4 * f], u = fQu[4 * f + 1];
    if (Q == 0ull) {  // kept by the N_eff test, or no usable weight: identity ancestry
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            anc[lo + i] = (int32_t)(lo + i);
        return;
    }
    const int32_t tl = ft_off[f + 1] - 1;
    const int64_t j_lo = tT[t];
    const int64_t j_hi = (t < tl) ? tT[t + 1] : P.n;
    uint64_t q[TILE_ITEMS];
    tile_weights(lw, lo, n, fs[f].M, scale_bits(P.n), C, q);
    tile_scan(q, C, red);
    const TicketGrid tg = ticket_grid(Q, u, fQu[4 * f + 2], (uint32_t)fQu[4 * f + 3], P.ndiv);
    ticket_parents_contig(C, n, tC[t], tg, j_lo, j_hi, stage, anc + P.off, (int32_t)lo,
                          (P.n < Ntot - P.off) ? P.n : Ntot - P.off, flags);
}

// ------------------------------------------------------------------ host side
template <typename T>
cudaError_t dmalloc(T **p, size_t n)
{
    *p = nullptr;
    return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
}

cudaError_t build_units(ppf_batch *b, int32_t unit)
{
    std::vector<int32_t> uf, un, fo(b->F + 1);
    std::vector<int64_t> ul;
    for (int32_t f = 0; f < b->F; ++f) {
        fo[f] = (int32_t)uf.size();
        for (int64_t s = 0; s < b->n[f]; s += unit) {
            uf.push_back(f);
            ul.push_back(b->off[f] + s);
            un.push_back((int32_t)((b->n[f] - s) < unit ? (b->n[f] - s) : unit));
        }
    }
    fo[b->F] = (int32_t)uf.size();
    if (b->unit_f) {
        cudaFree(b->unit_f);
        cudaFree(b->unit_lo);
        cudaFree(b->unit_n);
        cudaFree(b->upart);
    }
    b->U = (int32_t)uf.size();
    cudaError_t e;
    if ((e = dmalloc(&b->unit_f, b->U)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->unit_lo, b->U)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->unit_n, b->U)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->upart, b->U)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->unit_f, uf.data(), sizeof(int32_t) * b->U, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->unit_lo, ul.data(), sizeof(int64_t) * b->U, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->unit_n, un.data(), sizeof(int32_t) * b->U, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->fu_off, fo.data(), sizeof(int32_t) * (b->F + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    b->unit = unit;
    return cudaSuccess;
}

cudaError_t build_tiles(ppf_batch *b)
{
    std::vector<int32_t> tf, tn, fo(b->F + 1);
    std::vector<int64_t> tl;
    for (int32_t f = 0; f < b->F; ++f) {
        fo[f] = (int32_t)tf.size();
        for (int64_t s = 0; s < b->n[f]; s += TILE) {
            tf.push_back(f);
            tl.push_back(b->off[f] + s);
            tn.push_back((int32_t)((b->n[f] - s) < TILE ? (b->n[f] - s) : TILE));
        }
    }
    fo[b->F] = (int32_t)tf.size();
    b->T = (int32_t)tf.size();
    cudaError_t e;
    if ((e = dmalloc(&b->tile_f, b->T)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->tile_lo, b->T)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->tile_n, b->T)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->ft_off, b->F + 1)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->tQ, b->T)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->tC, b->T)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->tT, b->T + 1)) != cudaSuccess) return e;
    if ((e = dmalloc(&b->fQu, 4 * (size_t)b->F)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->tile_f, tf.data(), sizeof(int32_t) * b->T, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->tile_lo, tl.data(), sizeof(int64_t) * b->T, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->tile_n, tn.data(), sizeof(int32_t) * b->T, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    return cudaMemcpy(b->ft_off, fo.data(), sizeof(int32_t) * (b->F + 1), cudaMemcpyHostToDevice);
}

template <int R>
void launch_batch_step_r(const BatchStepArgs &a, int grid, int block, cudaStream_t s)
{
    batch_step_kernel<R><<<grid, block, 0, s>>>(a);
}

cudaError_t launch_batch_step(ppf_batch *b, bool commit)
{
    BatchStepArgs a;
    a.Ntot = b->Ntot;
    a.W = b->W;
    a.H = b->H;
    a.Wp = b->Wp;
    a.Hp = b->Hp;
    a.pad = b->pad;
    a.cur = b->cursor;
    a.fp = b->fp;
    a.unit_f = b->unit_f;
    a.unit_lo = b->unit_lo;
    a.unit_n = b->unit_n;
    a.U = b->U;
    a.st0 = b->state[0];
    a.st1 = b->state[1];
    a.anc = b->anc;
    a.fkeep = b->fkeep;
    a.Zp = b->Zp;
    a.flags = b->flags;
    a.part = b->upart;
    int grid = b->num_sms * b->bps;
    if (grid > b->U)
        grid = b->U;
    switch (b->r) {
    case 0: launch_batch_step_r<0>(a, grid, b->block, b->stream); break;
    case 1: launch_batch_step_r<1>(a, grid, b->block, b->stream); break;
    case 2: launch_batch_step_r<2>(a, grid, b->block, b->stream); break;
    case 3: launch_batch_step_r<3>(a, grid, b->block, b->stream); break;
    case 4: launch_batch_step_r<4>(a, grid, b->block, b->stream); break;
    case 5: launch_batch_step_r<5>(a, grid, b->block, b->stream); break;
    case 6: launch_batch_step_r<6>(a, grid, b->block, b->stream); break;
    case 7: launch_batch_step_r<7>(a, grid, b->block, b->stream); break;
    default: launch_batch_step_r<8>(a, grid, b->block, b->stream); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !commit)
        return e;
    const int fgrid = (b->F * 32 + 255) / 256;
    batch_finalize_kernel<<<fgrid, 256, 0, b->stream>>>(b->upart, b->fu_off, b->F, b->fsum, b->cursor);
    b->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_batch_prepare(ppf_batch *b)
{
    const int64_t rows = (int64_t)b->F * b->Hp;  // one warp per row, 8 warps per block
    const int grid = (int)((rows + 7) / 8 < 8192 ? (rows + 7) / 8 : 8192);
    switch (b->dtype) {
    case PPF_BF16:
        batch_prepare_kernel<__nv_bfloat16><<<grid, 256, 0, b->stream>>>(b->cursor, b->Zp, b->F, b->W, b->H, b->Wp,
                                                                         b->Hp, b->pad, b->fp);
        break;
    case PPF_F16:
        batch_prepare_kernel<__half><<<grid, 256, 0, b->stream>>>(b->cursor, b->Zp, b->F, b->W, b->H, b->Wp, b->Hp,
                                                                  b->pad, b->fp);
        break;
    default:
        batch_prepare_kernel<float><<<grid, 256, 0, b->stream>>>(b->cursor, b->Zp, b->F, b->W, b->H, b->Wp, b->Hp,
                                                                 b->pad, b->fp);
    }
    b->launches += 1;
    return cudaGetLastError();
}

cudaError_t set_cursor(ppf_batch *b, const void *frames, FilterSummary *est, int32_t k, int32_t t)
{
    batch_set_cursor<<<1, 1, 0, b->stream>>>(b->cursor, (const char *)frames, (int64_t)(b->frame_bytes * b->F), est,
                                             k, t, b->cur, b->first ? 1 : 0);
    b->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_batch_resample(ppf_batch *b)
{
    batch_tile_totals<<<b->T, TILE_THREADS, 0, b->stream>>>(b->state[0], b->state[1], b->Ntot, b->fp, b->fsum,
                                                            b->cursor, b->tile_f, b->tile_lo, b->tile_n, b->tQ);
    batch_tile_scan<<<(b->F * 32 + 255) / 256, 256, 0, b->stream>>>(b->fp, b->fsum, b->cursor, b->ft_off, b->F,
                                                                      b->tQ, b->tC, b->tT, b->fQu, b->fkeep,
                                                                      b->flags);
    batch_fill<<<b->T, TILE_THREADS, FILL_SMEM_BYTES, b->stream>>>(b->state[0], b->state[1], b->Ntot, b->fp, b->fsum, b->cursor,
                                                     b->tile_f, b->tile_lo, b->tile_n, b->ft_off, b->tC, b->tT, b->fQu,
                                                     b->anc, b->flags);
    b->launches += 3;
    return cudaGetLastError();
}

// one frame iteration of a sequence: advance, prepare, step, finalise, resample
cudaError_t launch_iteration(ppf_batch *b)
{
    batch_advance<<<1, 1, 0, b->stream>>>(b->cursor);
    b->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_batch_prepare(b);
    if (e == cudaSuccess)
        e = launch_batch_step(b, true);
    if (e == cudaSuccess)
        e = launch_batch_resample(b);
    return e;
}

void drop_graph(ppf_batch *b)
{
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

void free_batch(ppf_batch *b)
{
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    if (b->gstream)
        cudaStreamDestroy(b->gstream);
    void *p[] = {b->fp, b->state[0], b->state[1], b->anc, b->Zp, b->unit_f, b->unit_lo, b->unit_n, b->fu_off,
                 b->upart, b->fsum, b->flags, b->fkeep, b->fsum_run, b->cursor, b->tile_f, b->tile_lo, b->tile_n,
                 b->ft_off,
                 b->tQ, b->tC, b->tT, b->fQu};
    for (void *q : p)
        if (q)
            cudaFree(q);
    if (b->fsum_host)
        cudaFreeHost(b->fsum_host);
}

}  // namespace
}  // namespace ppf

using namespace ppf;

#define BCK(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            snprintf(b->err, sizeof(b->err), "%s: %s", #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? PPF_ENOMEM : PPF_ECUDA;       \
        }                                                                          \
    } while (0)

extern "C" {

ppf_status ppf_batch_create(const ppf_model *models, const int64_t *n, int32_t F, void *cuda_stream, ppf_batch **out)
{
    if (!models || !n || !out || F < 1)
        return PPF_EINVAL;
    const ppf_model &m0 = models[0];
    int64_t Ntot = 0;
    for (int32_t f = 0; f < F; ++f) {
        const ppf_model &m = models[f];
        if (m.width != m0.width || m.height != m0.height || m.patch_radius != m0.patch_radius ||
            m.frame_dtype != m0.frame_dtype || m.likelihood != 0)  // batches use eq. 4 at the particle
            return PPF_EINVAL;
        if (!(m.psf_sigma > 0.0f) || !(m.sigma_xi > 0.0f) || !(m.sigma_m >= 0.0f) || !(m.sigma_v >= 0.0f) ||
            !(m.sigma_I >= 0.0f) || !(m.v0_max >= 0.0f))
            return PPF_EINVAL;
        if (n[f] < 1)
            return PPF_EINVAL;
        Ntot += n[f];
    }
    if (Ntot > 2147483647LL || m0.width < 1 || m0.height < 1 || m0.patch_radius < 0 || m0.patch_radius > MAX_RADIUS)
        return PPF_EINVAL;
    if (m0.frame_dtype != PPF_F32 && m0.frame_dtype != PPF_BF16 && m0.frame_dtype != PPF_F16)
        return PPF_EINVAL;
    ppf_batch *b = new (std::nothrow) ppf_batch();
    if (!b)
        return PPF_ENOMEM;
    b->F = F;
    b->Ntot = Ntot;
    b->W = m0.width;
    b->H = m0.height;
    b->r = m0.patch_radius;
    b->pad = 2 * b->r;
    b->Wp = b->W + 2 * b->pad + 1;  // pixel pairs per row: one zero column past the padded frame
    b->Hp = b->H + 2 * b->pad;
    b->dtype = m0.frame_dtype;
    b->frame_bytes = (size_t)b->W * b->H * (b->dtype == PPF_F32 ? 4 : 2);
    b->stream = (cudaStream_t)cuda_stream;
    b->models.assign(models, models + F);
    b->n.assign(n, n + F);
    b->off.resize(F);
    int64_t o = 0;
    for (int32_t f = 0; f < F; ++f) {
        b->off[f] = o;
        o += n[f];
    }
    b->block = 256;
    b->bps = 4;
    b->first = true;
    auto fail = [&](ppf_status st) {
        free_batch(b);
        delete b;
        return st;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(PPF_ECUDA);
    std::vector<FilterParams> hp(F);
    std::vector<float> v0A(2 * (size_t)F);
    for (int32_t f = 0; f < F; ++f) {
        const ppf_model &m = models[f];
        FilterParams &P = hp[f];
        P.off = b->off[f];
        P.n = n[f];
        P.ndiv = make_divisor((uint32_t)n[f]);
        P.ess_thr = INFINITY;
        P.seed = m.seed;
        P.fid = m.filter_id;
        P.inv2s2 = 1.0f / (2.0f * m.psf_sigma * m.psf_sigma);
        P.inv_sxi2 = 1.0f / (m.sigma_xi * m.sigma_xi);
        P.sm = m.sigma_m;
        P.sv = m.sigma_v;
        P.sI = m.sigma_I;
        P.bg = m.background;
        for (int k = 0; k < MAX_RADIUS; ++k)
            P.Kc[k] = (float)exp(-(2.0 * k + 1.0) * (double)P.inv2s2);
        v0A[2 * f] = m.v0_max;
        v0A[2 * f + 1] = m.amplitude;
    }
    float *dv0A = nullptr;
    if (dmalloc(&b->fp, F) != cudaSuccess || dmalloc(&b->state[0], 6 * Ntot) != cudaSuccess ||
        dmalloc(&b->state[1], 6 * Ntot) != cudaSuccess || dmalloc(&b->anc, Ntot) != cudaSuccess ||
        dmalloc(&b->Zp, 2 * (size_t)F * b->Wp * b->Hp) != cudaSuccess || dmalloc(&b->fu_off, F + 1) != cudaSuccess ||
        dmalloc(&b->fsum, F) != cudaSuccess || dmalloc(&b->flags, 1) != cudaSuccess ||
        dmalloc(&b->fkeep, F) != cudaSuccess ||
        dmalloc(&b->cursor, 1) != cudaSuccess ||
        cudaMallocHost((void **)&b->fsum_host, sizeof(FilterSummary) * F) != cudaSuccess ||
        dmalloc(&dv0A, 2 * (size_t)F) != cudaSuccess)
        return (dv0A ? cudaFree(dv0A) : cudaSuccess), fail(PPF_ENOMEM);
    if (cudaMemcpy(b->fp, hp.data(), sizeof(FilterParams) * F, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dv0A, v0A.data(), sizeof(float) * 2 * F, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->flags, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(b->fkeep, 0, sizeof(int32_t) * F) != cudaSuccess || build_units(b, 1024) != cudaSuccess ||
        build_tiles(b) != cudaSuccess ||
        cudaFuncSetAttribute(batch_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FILL_SMEM_BYTES) !=
            cudaSuccess) {
        cudaFree(dv0A);
        return fail(PPF_ECUDA);
    }
    b->hp = hp;
    batch_init_kernel<<<4 * b->num_sms, 256, 0, b->stream>>>(b->state[0], Ntot, b->fp, b->unit_f, b->unit_lo,
                                                               b->unit_n, b->U, (float)b->W, (float)b->H, dv0A);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    cudaFree(dv0A);
    if (e != cudaSuccess)
        return fail(PPF_ECUDA);
    *out = b;
    return PPF_OK;
}

void ppf_batch_destroy(ppf_batch *b)
{
    if (!b)
        return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

ppf_status ppf_batch_step(ppf_batch *b, const void *frames_dev, int32_t k)
{
    const ppf::NvtxRange nvtx_range("ppf_batch_step");
    if (!b || !frames_dev || k < 1)
        return PPF_EINVAL;
    if (b->weighted)
        return PPF_ESTATE;  // every batched step follows a resample (or the prior)
    BCK(set_cursor(b, frames_dev, nullptr, k, 0));
    BCK(launch_batch_prepare(b));
    BCK(launch_batch_step(b, true));
    b->cur ^= 1;
    b->first = false;
    b->weighted = true;
    b->last_k = k;
    return PPF_OK;
}

ppf_status ppf_batch_resample(ppf_batch *b, int32_t k)
{
    const ppf::NvtxRange nvtx_range("ppf_batch_resample");
    if (!b)
        return PPF_EINVAL;
    if (!b->weighted)
        return PPF_ESTATE;
    if (k != b->last_k)
        return PPF_EINVAL;  // the cursor still holds the last step's frame
    BCK(launch_batch_resample(b));
    b->weighted = false;
    return PPF_OK;
}

ppf_status ppf_batch_run(ppf_batch *b, const void *frames_dev, int32_t k0, int32_t K, int32_t use_graph,
                         ppf_filter_estimate_t *est_host)
{
    const ppf::NvtxRange nvtx_range("ppf_batch_run");
    if (!b || !frames_dev || k0 < 1 || K < 1)
        return PPF_EINVAL;
    if (b->weighted)
        return PPF_ESTATE;
    if (est_host && b->fsum_run_cap < (int64_t)K * b->F) {
        if (b->fsum_run)
            cudaFree(b->fsum_run);
        b->fsum_run = nullptr;
        BCK(cudaMalloc((void **)&b->fsum_run, sizeof(FilterSummary) * (size_t)K * b->F));
        b->fsum_run_cap = (int64_t)K * b->F;
    }
    cudaStream_t user = b->stream;
    if (use_graph && user == nullptr) {  // the legacy stream cannot be captured
        if (!b->gstream)
            BCK(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
        BCK(cudaStreamSynchronize(nullptr));
        b->stream = b->gstream;
    }
    ppf_status st = PPF_OK;
    cudaError_t e = set_cursor(b, frames_dev, est_host ? b->fsum_run : nullptr, k0 - 1, -1);
    if (e == cudaSuccess && use_graph && !b->gexec) {
        // capture one iteration; every replay advances the cursor to the next frame
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int64_t launches = b->launches;
            cudaError_t ec = launch_iteration(b);
            b->launches = launches;
            e = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess)
                e = ec;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->gexec, g, 0);
        if (g)
            cudaGraphDestroy(g);
    }
    for (int32_t t = 0; t < K && e == cudaSuccess; ++t) {
        if (use_graph) {
            e = cudaGraphLaunch(b->gexec, b->stream);
            b->launches += 7;
        } else {
            e = launch_iteration(b);
        }
    }
    if (e == cudaSuccess && est_host)
        e = cudaMemcpyAsync(est_host, b->fsum_run, sizeof(FilterSummary) * (size_t)K * b->F, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        snprintf(b->err, sizeof(b->err), "batch run: %s", cudaGetErrorString(e));
        st = PPF_ECUDA;
    }
    b->stream = user;
    if (st == PPF_OK) {
        b->cur ^= (K & 1);
        b->first = false;
        b->last_k = k0 + K - 1;
    }
    return st;
}

ppf_status ppf_batch_estimates(ppf_batch *b, ppf_filter_estimate_t *out_host)
{
    if (!b || !out_host)
        return PPF_EINVAL;
    BCK(cudaMemcpyAsync(b->fsum_host, b->fsum, sizeof(FilterSummary) * b->F, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    memcpy(out_host, b->fsum_host, sizeof(FilterSummary) * b->F);
    int32_t fl = 0;
    BCK(cudaMemcpy(&fl, b->flags, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (fl) {
        BCK(cudaMemset(b->flags, 0, sizeof(int32_t)));
        if (fl & FLAG_INTERNAL) {
            snprintf(b->err, sizeof(b->err), "device flags 0x%x: an index check of the debug build failed", fl);
            return PPF_EINVAL;
        }
        return PPF_EDEGENERATE;
    }
    return PPF_OK;
}

ppf_status ppf_batch_get_particles(ppf_batch *b, float *state_dev, int32_t *anc_dev)
{
    if (!b)
        return PPF_EINVAL;
    if (state_dev)
        BCK(cudaMemcpyAsync(state_dev, b->state[b->cur], sizeof(float) * 6 * b->Ntot, cudaMemcpyDeviceToDevice,
                            b->stream));
    if (anc_dev)
        BCK(cudaMemcpyAsync(anc_dev, b->anc, sizeof(int32_t) * b->Ntot, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return PPF_OK;
}

ppf_status ppf_batch_autotune(ppf_batch *b, const void *frames_dev, int32_t k, int32_t *config_out)
{
    if (!b || !frames_dev || k < 1)
        return PPF_EINVAL;
    if (b->weighted)
        return PPF_ESTATE;
    drop_graph(b);  // the launch shape is baked into a captured graph
    BCK(set_cursor(b, frames_dev, nullptr, k, 0));
    BCK(launch_batch_prepare(b));
    const int32_t units[] = {512, 1024, 2048, 4096};
    const int32_t blocks[] = {128, 256, 512};
    const int32_t bpss[] = {2, 4, 8};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    // each candidate: one untimed launch, then the best of 3 timings of 3 launches
    auto time_cfg = [&](int32_t un, int32_t bl, int32_t bp, float *out) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (un != b->unit)
            e = build_units(b, un);
        b->block = bl;
        b->bps = bp;
        if (e == cudaSuccess)
            e = launch_batch_step(b, false);
        float best_ms = 1e30f;
        for (int trial = 0; trial < 3 && e == cudaSuccess; ++trial) {
            e = cudaEventRecord(e0, b->stream);
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
                e = launch_batch_step(b, false);
            if (e == cudaSuccess)
                e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, e0, e1);
            best_ms = ms < best_ms ? ms : best_ms;
        }
        *out = best_ms;
        return e;
    };
    float base_ms;
    const int32_t du = 1024, db = 256, dp = 4;  // the default shape
    BCK(time_cfg(du, db, dp, &base_ms));
    float best = base_ms;
    int32_t bu = du, bb = db, bs = dp;
    for (int32_t un : units)
        for (int32_t bl : blocks)
            for (int32_t bp : bpss) {
                float ms;
                BCK(time_cfg(un, bl, bp, &ms));
                if (ms < 0.98f * best) {  // a change must win by 2 %
                    best = ms;
                    bu = un;
                    bb = bl;
                    bs = bp;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(build_units(b, bu));
    b->block = bb;
    b->bps = bs;
    if (config_out) {
        config_out[0] = bu;
        config_out[1] = bb;
        config_out[2] = bs;
    }
    return PPF_OK;
}

ppf_status ppf_batch_set_ess_threshold(ppf_batch *b, double fraction)
{
    if (!b || fraction != fraction || fraction < 0.0)
        return PPF_EINVAL;
    for (int32_t f = 0; f < b->F; ++f)
        b->hp[f].ess_thr = (fraction == INFINITY) ? INFINITY : fraction * (double)b->n[f];
    BCK(cudaStreamSynchronize(b->stream));  // no kernel of the batch reads the parameters meanwhile
    BCK(cudaMemcpy(b->fp, b->hp.data(), sizeof(FilterParams) * b->F, cudaMemcpyHostToDevice));
    return PPF_OK;
}

const char *ppf_batch_last_error(const ppf_batch *b)
{
    return b ? b->err : "";
}

}  // extern "C"
