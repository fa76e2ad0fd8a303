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
// thread t takes items [16t, 16t + 16).  q = 0 beyond n.
__device__ __forceinline__ void tile_weights(const float *__restrict__ lw, int64_t lo, int n, float M, int s,
                                             uint64_t *buf, uint64_t q[TILE_ITEMS])
{
    float *f = reinterpret_cast<float *>(buf);
    for (int e = threadIdx.x; e < TILE; e += blockDim.x)
        f[padf(e)] = (e < n) ? __ldg(lw + lo + e) : -INFINITY;
    __syncthreads();
    const int base = threadIdx.x * TILE_ITEMS;
#pragma unroll
    for (int k = 0; k < TILE_ITEMS; ++k)
        q[k] = quantise(f[padf(base + k)], M, s);
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

// floor(X / d) for X < 2^96 whose quotient fits 64 bits, d < 2^32, by long
// division in 32-bit limbs; *rem = X mod d.
__device__ __forceinline__ uint64_t div_u96(u128 X, uint32_t d, uint32_t *rem)
{
    const uint64_t l2 = (uint64_t)(X >> 64), l1 = (uint64_t)(uint32_t)(X >> 32), l0 = (uint64_t)(uint32_t)X;
    uint64_t r = l2 % d;
    uint64_t cur = (r << 32) | l1;
    const uint64_t q1 = cur / d;
    r = cur % d;
    cur = (r << 32) | l0;
    const uint64_t q0 = cur / d;
    *rem = (uint32_t)(cur % d);
    return (q1 << 32) + q0;
}

// floor(v / d), v mod d for v < 2^52, d < 2^32: float estimate, exact fix-up
__device__ __forceinline__ uint64_t div_small(uint64_t v, uint32_t d, float rd, uint32_t *rem)
{
    uint64_t q = (uint64_t)((float)v * rd);
    int64_t r = (int64_t)v - (int64_t)(q * d);
    while (r < 0) {
        --q;
        r += d;
    }
    while (r >= (int64_t)d) {
        ++q;
        r -= d;
    }
    *rem = (uint32_t)r;
    return q;
}

// Parents of the tickets [j_lo, j_hi) of one run of particles with inclusive
// cumulative weights C[0..n) (local; the run starts at cumulative weight c0,
// n <= TILE).  Ticket j sits at (u + jQ)/nt; its parent is the first i with
// c0 + C[i] > thr_j = floor((u + jQ)/nt).  One exact 96/32 division gives thr
// at j_lo; with Q = qN nt + qR, ticket j_lo + o has
// thr = thr(j_lo) + o qN + floor((rem(j_lo) + o qR) / nt).  Thread t takes
// tickets j_lo + t, j_lo + t + blockDim, ... (coalesced writes) and finds each
// parent with a fixed 12-step branch-free binary search (no divergence, no
// barriers between tickets).  emit(j, i) receives every (ticket, parent).
// Called by every thread of the block.
template <typename Emit>
__device__ __forceinline__ void ticket_parents(const uint64_t *C, int n, uint64_t c0, uint64_t u, uint64_t Q,
                                               uint32_t nt, int64_t j_lo, int64_t j_hi, Emit emit)
{
    __shared__ uint64_t s_thr;
    __shared__ uint32_t s_rem;
    const uint64_t qN = Q / nt;
    const uint32_t qR = (uint32_t)(Q % nt);
    const float rnt = 1.0f / (float)nt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t r0;
        s_thr = div_u96((u128)u + (u128)(uint64_t)j_lo * (u128)Q, nt, &r0);
        s_rem = r0;
    }
    __syncthreads();
    const uint64_t thr0 = s_thr;
    const uint64_t rem0 = s_rem;
    for (int64_t j = j_lo + threadIdx.x; j < j_hi; j += blockDim.x) {
        const uint64_t o = (uint64_t)(j - j_lo);
        uint32_t r;
        const uint64_t thr = thr0 + o * qN + div_small(rem0 + o * qR, nt, rnt, &r);
        const uint64_t lt = thr - c0;
        // number of C[i] <= lt over i < TILE (C[i] for i >= n is never reached:
        // every ticket of this run has lt < C[n-1])
        int pos = 0;
#pragma unroll
        for (int step = TILE / 2; step > 0; step >>= 1) {
            const int k = pos + step - 1;
            if (k < n && C[padc(k)] <= lt)
                pos += step;
        }
        emit(j, pos);
    }
}

}  // namespace ppf
