// ppf_tiles.cuh -- block-level building blocks of the fixed-point resampling
// (Alg. 1 resampling step): tile staging, tile scans, and the parents of a
// range of systematic tickets.  Shared by the single-filter, RNA and batched
// resampling kernels.
#pragma once

#include <cstdint>

#include "ppf_device.cuh"
#include "ppf_internal.h"

namespace ppf {

// Shared-memory layout of one tile: the float32 weights are staged with one
// pad word per 32 (thread t then reads its 16 consecutive weights without bank
// conflicts) and the u64 inclusive sums with one pad per 16 (conflict-free for
// the per-thread writes); both live in the same buffer, one after the other.
__device__ __forceinline__ int padf(int i) { return i + (i >> 5); }
__device__ __forceinline__ int padc(int i) { return i + (i >> 4); }
constexpr int TILE_SMEM_U64 = TILE + TILE / 16;  // >= (TILE + TILE/32) / 2 floats

// Quantised weights of particles [lo, lo + n): coalesced loads into smem, then
// thread t takes items [16t, 16t + 16).  q = 0 beyond n.  Every caller runs
// TILE_THREADS threads: each thread issues all of its TILE / TILE_THREADS
// loads before its first shared store, so that they are in flight together
// (a load-store loop waits one memory latency per element).
constexpr int TILE_LOADS = TILE / TILE_THREADS;  // weights a thread loads per tile

// The loads of tile_weights on their own: thread t gets elements
// t + k TILE_THREADS of [lo, lo + n) (-inf beyond n), all in flight together.
__device__ __forceinline__ void tile_load(const float *__restrict__ lw, int64_t lo, int n, float (&v)[TILE_LOADS])
{
#pragma unroll
    for (int k = 0; k < TILE_LOADS; ++k) {
        const int e = (int)threadIdx.x + k * TILE_THREADS;
        v[k] = (e < n) ? __ldg(lw + lo + e) : -INFINITY;
    }
}

// The rest of tile_weights: the loaded weights through shared memory to the
// per-thread layout, quantised against M.
__device__ __forceinline__ void tile_quantise(const float (&v)[TILE_LOADS], float M, int s, uint64_t *buf,
                                              uint64_t q[TILE_ITEMS])
{
    float *f = reinterpret_cast<float *>(buf);
#pragma unroll
    for (int k = 0; k < TILE_LOADS; ++k)
        f[padf((int)threadIdx.x + k * TILE_THREADS)] = v[k];
    __syncthreads();
    const int base = threadIdx.x * TILE_ITEMS;
#pragma unroll
    for (int k = 0; k < TILE_ITEMS; k += 2)
        quantise2(f[padf(base + k)], f[padf(base + k + 1)], M, s, q[k], q[k + 1]);
    __syncthreads();
}

__device__ __forceinline__ void tile_weights(const float *__restrict__ lw, int64_t lo, int n, float M, int s,
                                             uint64_t *buf, uint64_t q[TILE_ITEMS])
{
    float *f = reinterpret_cast<float *>(buf);
    float v[TILE_LOADS];
    tile_load(lw, lo, n, v);
#pragma unroll
    for (int k = 0; k < TILE_LOADS; ++k)
        f[padf((int)threadIdx.x + k * TILE_THREADS)] = v[k];
    __syncthreads();
    const int base = threadIdx.x * TILE_ITEMS;
#pragma unroll
    for (int k = 0; k < TILE_ITEMS; k += 2)
        quantise2(f[padf(base + k)], f[padf(base + k + 1)], M, s, q[k], q[k + 1]);
    __syncthreads();
}

// Inclusive scan of a tile's weights into C (padded with padc).  Returns the total.
__device__ __forceinline__ uint64_t tile_scan(const uint64_t q[TILE_ITEMS], uint64_t *C, uint64_t *red)
{
    uint64_t loc[TILE_ITEMS];
    uint64_t run = 0;
#pragma unroll
    for (int k = 0; k < TILE_ITEMS; ++k) {
        run += q[k];
        loc[k] = run;
    }
    uint64_t total;
    const uint64_t pre = block_excl_scan_u64(run, red, &total);
    const int base = threadIdx.x * TILE_ITEMS;
#pragma unroll
    for (int k = 0; k < TILE_ITEMS; ++k)
        C[padc(base + k)] = pre + loc[k];
    __syncthreads();
    return total;
}

// floor(x / d) for a fixed divisor d >= 1 and any x < 2^64, from the
// precomputed m = floor((2^64 - 1) / d): the product estimate floor(x m / 2^64)
// lies within 2 below the quotient and never above it.
struct Divisor {
    uint64_t m;
    uint32_t d;
};

__host__ __device__ inline Divisor make_divisor(uint32_t d)
{
    Divisor v;
    v.m = ~0ull / d;
    v.d = d;
    return v;
}

__device__ __forceinline__ uint64_t div_by(uint64_t x, Divisor v, uint32_t *rem)
{
    uint64_t q = __umul64hi(x, v.m);
    uint64_t r = x - q * v.d;
    while (r >= v.d) {
        ++q;
        r -= v.d;
    }
    *rem = (uint32_t)r;
    return q;
}

// The ticket grid of one systematic draw: nt tickets at (u + jQ)/nt of the
// cumulative fixed-point weight, Q = qN nt + qR.
struct TicketGrid {
    uint64_t Q, u, qN;
    uint32_t qR;
    Divisor nt;
};

__device__ __forceinline__ TicketGrid ticket_grid(uint64_t Q, uint64_t u, uint64_t qN, uint32_t qR, Divisor nt)
{
    TicketGrid g;
    g.Q = Q;
    g.u = u;
    g.qN = qN;
    g.qR = qR;
    g.nt = nt;
    return g;
}

// The threshold of ticket j, thr_j = floor((u + jQ)/nt) = j qN + floor((u + j qR)/nt):
// exact in 64-bit arithmetic (j < nt < 2^31 and u < Q <= 2^63, so
// u + j qR < 2^64).
__device__ __forceinline__ uint64_t ticket_threshold(int64_t j, const TicketGrid &tg)
{
    uint32_t r;
    return (uint64_t)j * tg.qN + div_by(tg.u + (uint64_t)j * tg.qR, tg.nt, &r);
}

// Number of tickets below cumulative weight c, #{j in [0, nt) : u + jQ < nt c}
// = #{j : thr_j < c} (thr_j < c iff (u + jQ)/nt < c for integer c): a float
// estimate c nt / Q, corrected once by the float estimate of the distance
// from c to the estimate's exact threshold, then moved to the exact boundary
// by comparing thresholds (they do not decrease with j).  No 128-bit or FP64
// arithmetic.
__device__ __forceinline__ int64_t tickets_below_grid(uint64_t c, const TicketGrid &tg)
{
    const int64_t n = tg.nt.d;
    const float rstep = (float)n / (float)tg.Q;
    int64_t j = (int64_t)((float)c * rstep);
    j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
    const int64_t d = (int64_t)(c - ticket_threshold(j, tg));
    j += (int64_t)floorf((float)d * rstep);
    j = j < 0 ? 0 : (j > n ? n : j);
    while (j > 0 && ticket_threshold(j - 1, tg) >= c)
        --j;
    while (j < n && ticket_threshold(j, tg) < c)
        ++j;
    return j;
}

// Parents of the tickets [j_lo, j_hi) of one run of particles with inclusive
// cumulative weights C[0..n) (local; the run starts at cumulative weight c0,
// n <= TILE).  Ticket j sits at (u + jQ)/nt; its parent is the first i with
// c0 + C[i] > thr_j = floor((u + jQ)/nt) = j qN + floor((u + j qR)/nt), and the
// thresholds step as thr_{j+1} = thr_j + qN + [rem_j + qR >= nt]
// (rem_j = (u + jQ) mod nt).
//
// The parents are a merge of two sorted sequences: particle i comes before
// ticket j iff C[i] <= thr_j - c0, and a ticket's parent is the particle that
// follows it.  The merged sequence (n + L elements, L = j_hi - j_lo) is cut
// into equal pieces, one per thread (merge path): a binary search along the
// thread's cross diagonal finds where its piece starts, then the thread walks
// its piece, advancing either the particle or the ticket at every step.  Every
// thread does the same number of steps whatever the weights.
// emit(j, i) receives every (ticket, parent), a thread's tickets in
// increasing order.  L <= STAGE_TICKETS (so the ticket offsets within the run
// and the merge positions fit 32 bits).  Called by every thread of the block;
// contains barriers.
template <typename Emit>
__device__ __forceinline__ void ticket_parents(const uint64_t *C, int n, uint64_t c0, const TicketGrid &tg,
                                               int64_t j_lo, int L, Emit emit)
{
    __shared__ uint64_t s_thr;
    __shared__ uint32_t s_rem;
    const uint32_t nt = tg.nt.d;
    const uint64_t qN = tg.qN;
    const uint32_t qR = tg.qR;
    __syncthreads();
    if (threadIdx.x == 0) {
        // threshold and remainder of ticket j_lo (j_lo < nt < 2^31, so
        // u + j_lo qR < 2^63 + 2^62)
        uint32_t r0;
        s_thr = (uint64_t)j_lo * qN + div_by(tg.u + (uint64_t)j_lo * qR, tg.nt, &r0);
        s_rem = r0;
    }
    __syncthreads();
    const int D = n + L;
    const int K = (D + (int)blockDim.x - 1) / (int)blockDim.x;
    const int d0 = (int)threadIdx.x * K;
    if (L <= 0 || d0 >= D)
        return;
    // the run's first ticket has thr >= c0 (it is not below the run)
    const uint64_t lt0 = s_thr - c0;
    const uint32_t rem0 = s_rem;
    const float frem0 = (float)rem0, fqR = (float)qR, rnt = 1.0f / (float)nt;
    // thr_{j_lo + b} - c0 and rem_{j_lo + b}: with v = rem0 + b qR the step
    // past lt0 is b qN + floor(v / nt); the quotient is at most b + 1 <= 2^14,
    // so its float estimate is off by at most one (and converts as a 32-bit
    // integer: a 64-bit conversion runs on the FP64 pipe)
    auto lt_at = [&](int b, uint32_t *rem) -> uint64_t {
        const int64_t v = (int64_t)rem0 + (int64_t)b * qR;
        int64_t q = (int32_t)(fmaf((float)b, fqR, frem0) * rnt);
        int64_t r = v - q * (int64_t)nt;
        while (r < 0) {
            --q;
            r += nt;
        }
        while (r >= (int64_t)nt) {
            ++q;
            r -= nt;
        }
        *rem = (uint32_t)r;
        return lt0 + (uint64_t)b * qN + (uint64_t)q;
    };
    // particles among the first d0 merged elements: the first a in
    // [max(0, d0 - L), min(d0, n)] with C[a] > lt(d0 - a - 1)
    int lo = d0 > L ? d0 - L : 0, hi = d0 < n ? d0 : n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        uint32_t rm;
        if (C[padc(mid)] <= lt_at(d0 - mid - 1, &rm))
            lo = mid + 1;
        else
            hi = mid;
    }
    int i = lo;
    int b = d0 - lo;
    if (b >= L)
        return;
    uint32_t r;
    uint64_t lt = lt_at(b, &r);
    const int steps = (D - d0 < K) ? D - d0 : K;
    // every ticket has lt < C[n-1], so i stays below n while tickets remain.
    // Each step either advances the particle or emits the ticket and moves to
    // the next threshold; both updates are formed and selected, so the lanes
    // of a warp do not diverge (r + qR < 2 nt < 2^32).
    for (int s = 0; s < steps; ++s) {
        const bool adv = C[padc(i)] <= lt;
        if (!adv)
            emit(j_lo + b, i);
        const uint32_t rn = r + qR;
        const bool cy = rn >= nt;
        const uint64_t ltn = lt + qN + (cy ? 1u : 0u);
        i += adv ? 1 : 0;
        b += adv ? 0 : 1;
        lt = adv ? lt : ltn;
        r = adv ? r : (cy ? rn - nt : rn);
        if (b >= L)
            break;
    }
}

// Shared memory of the fill kernels: the tile's cumulative weights, then the
// staged parents (local indices) of up to STAGE_TICKETS tickets.
constexpr int STAGE_TICKETS = ITEM_TICKETS;
constexpr size_t FILL_SMEM_BYTES = sizeof(uint64_t) * TILE_SMEM_U64 + sizeof(uint16_t) * STAGE_TICKETS;

// ticket_parents in chunks of STAGE_TICKETS tickets: the parents are staged in
// shared memory and handed to store(j, i) in ticket order, thread k taking
// tickets k, k + blockDim, ... of the chunk (coalesced global writes).
template <typename Store>
__device__ __forceinline__ void ticket_parents_staged(const uint64_t *C, int n, uint64_t c0, const TicketGrid &tg,
                                                      int64_t j_lo, int64_t j_hi, uint16_t *stage, Store store)
{
    for (int64_t c = j_lo; c < j_hi; c += STAGE_TICKETS) {
        const int64_t ce = (j_hi - c < STAGE_TICKETS) ? j_hi : c + STAGE_TICKETS;
        ticket_parents(C, n, c0, tg, c, (int)(ce - c), [&](int64_t j, int i) { stage[j - c] = (uint16_t)i; });
        __syncthreads();
        const int m = (int)(ce - c);
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            store(c + k, (int)stage[k]);
        __syncthreads();
    }
}

// Writes o[k] = base + st[k] for k < m, called by every thread of the block:
// up to three single stores reach a 16-byte boundary of o, then four tickets
// per thread and iteration as int4.  The debug build checks every parent
// against [0, n).
__device__ __forceinline__ void store_staged(int32_t *__restrict__ o, const uint16_t *st, int m, int32_t base,
                                             int n, const int32_t *flags)
{
    const int head = (int)((4u - ((uint32_t)(reinterpret_cast<uintptr_t>(o) >> 2) & 3u)) & 3u);
    const int h = head < m ? head : m;
    const int m4 = (m - h) >> 2;
    const int t0 = h + 4 * m4;
    const int k = threadIdx.x;
    if (k < h && PPF_DCHECK(st[k] < n, flags, FLAG_INTERNAL))
        o[k] = base + st[k];
    int4 *o4 = reinterpret_cast<int4 *>(o + h);
    for (int q = k; q < m4; q += blockDim.x) {
        const int e = h + 4 * q;
        const int32_t p0 = st[e], p1 = st[e + 1], p2 = st[e + 2], p3 = st[e + 3];
        if (PPF_DCHECK(p0 < n && p1 < n && p2 < n && p3 < n, flags, FLAG_INTERNAL))
            o4[q] = make_int4(base + p0, base + p1, base + p2, base + p3);
    }
    if (k < m - t0 && PPF_DCHECK(st[t0 + k] < n, flags, FLAG_INTERNAL))
        o[t0 + k] = base + st[t0 + k];
}

// ticket_parents_staged for the common contiguous output out[j] = base + i,
// each staged chunk written by store_staged.  The debug build checks every
// ticket's slot against [0, j_max).
__device__ __forceinline__ void ticket_parents_contig(const uint64_t *C, int n, uint64_t c0, const TicketGrid &tg,
                                                      int64_t j_lo, int64_t j_hi, uint16_t *stage,
                                                      int32_t *__restrict__ out, int32_t base, int64_t j_max,
                                                      const int32_t *flags)
{
    for (int64_t c = j_lo; c < j_hi; c += STAGE_TICKETS) {
        const int64_t ce = (j_hi - c < STAGE_TICKETS) ? j_hi : c + STAGE_TICKETS;
        const int m = (int)(ce - c);
        ticket_parents(C, n, c0, tg, c, m, [&](int64_t j, int i) { stage[j - c] = (uint16_t)i; });
        __syncthreads();
        if (PPF_DCHECK(c >= 0 && ce <= j_max, flags, FLAG_INTERNAL))
            store_staged(out + c, stage, m, base, n, flags);
        __syncthreads();
    }
}

}  // namespace ppf
