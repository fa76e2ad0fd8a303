// ppf_device.cuh -- device-side building blocks of the SIR step (sm_103a).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), keyed by the model seed, counter
// (index, frame, filter, purpose << 8 | block).  Prior uniforms are odd
// multiples of 2^-24 from 32-bit words; the propagation noise takes six 21-bit
// fields of one block as odd multiples of 2^-22 (all exact in float32);
// normals by the Box-Muller transform.
//
// Resampling weights (Alg. 1 resampling step) are 64-bit fixed point:
// q = floor(2^(s + t)), t = (lw - M) log2(e), computed by one fixed float32
// operation sequence (round-to-nearest, no contraction) so that the integer
// result is fully determined by lw and M.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ppf {

typedef unsigned __int128 u128;

// Debug builds (-DPPF_DEBUG) check the index of every scattered store of the
// resampling kernels and the window of every patch read before the access:
// a failed check ors `bit` into *flags (the internal-error flag, which
// ppf_estimate reports as PPF_EINVAL) and skips the access, so a broken
// invariant shows up as an error status instead of a memory fault.  Release
// builds compile the checks away.
#ifdef PPF_DEBUG
__device__ __forceinline__ bool debug_check(bool ok, const int32_t *flags, int32_t bit)
{
    if (!ok && flags)
        atomicOr(const_cast<int32_t *>(flags), bit);
    return ok;
}
#define PPF_DCHECK(cond, flags, bit) ::ppf::debug_check((cond), (flags), (bit))
#else
#define PPF_DCHECK(cond, flags, bit) true
#endif

// Programmatic dependent launch: pdl_wait() blocks until the previous kernel
// of the stream has completed and its writes are visible (a no-op for a
// kernel launched without the attribute); pdl_trigger() lets the next kernel,
// if launched with the attribute, be scheduled before this one completes.
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

enum : uint32_t { PURPOSE_INIT = 0, PURPOSE_PROP = 1, PURPOSE_RESAMPLE = 2, PURPOSE_GROUP = 3, PURPOSE_RING = 4 };

// One Philox4x32-10 block: ten rounds of two 32x32->64 multiplications of
// counter words 0 and 2, the high halves xor-ed with the other counter words
// and the key, the key advanced by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The ten round keys of one Philox key (the key advanced by the Weyl
// increments), computed once on the host so that a kernel reads them from its
// parameters instead of recomputing them for every block it draws.
struct PhiloxKeys {
    uint32_t k[10][2];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys r;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        r.k[round][0] = k0;
        r.k[round][1] = k1;
    }
    return r;
}

// philox() with precomputed round keys (the same block)
__device__ __forceinline__ uint4 philox_rk(uint4 c, const PhiloxKeys &rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk.k[round][0], lo1, hi0 ^ c.w ^ rk.k[round][1], lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t index, uint32_t frame, uint32_t filter,
                                      uint32_t purpose, uint32_t block)
{
    return philox(make_uint4(index, frame, filter, (purpose << 8) | block), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

// odd multiple of 2^-24 in (0, 1); the integer is < 2^24, so this is exact
__device__ __forceinline__ float u01(uint32_t r)
{
    return __uint2float_rn(2u * (r >> 9) + 1u) * 0x1p-24f;
}

// odd multiple of 2^-22 in (0, 1) from a 21-bit field; exact in float32
__device__ __forceinline__ float u21(uint32_t f)
{
    return __uint2float_rn(2u * f + 1u) * 0x1p-22f;
}

// The six 21-bit fields of one Philox block (word 0 least significant):
// field k holds bits [21k, 21k + 21) of the 128-bit block.
__device__ __forceinline__ void prop_fields(uint4 r, uint32_t f[6])
{
    const uint64_t lo = (uint64_t)r.x | ((uint64_t)r.y << 32);
    const uint64_t hi = (uint64_t)r.z | ((uint64_t)r.w << 32);
    const uint64_t m = 0x1FFFFFull;
    f[0] = (uint32_t)(lo & m);
    f[1] = (uint32_t)((lo >> 21) & m);
    f[2] = (uint32_t)((lo >> 42) & m);
    f[3] = (uint32_t)(((lo >> 63) | (hi << 1)) & m);
    f[4] = (uint32_t)((hi >> 20) & m);
    f[5] = (uint32_t)((hi >> 41) & m);
}

// Box-Muller: rho = sqrt(-2 ln u1) (accurate log: u1 -> 1 needs it), angle
// 2 pi u2 = theta + pi with theta in (-pi, pi) for the hardware sine/cosine.
__device__ __forceinline__ void box_muller(float u1, float u2, float &z0, float &z1)
{
    const float rho = sqrtf(-2.0f * logf(u1));
    float s, c;
    __sincosf(__fmaf_rn(6.28318530717958647692f, u2, -3.14159265358979323846f), &s, &c);
    z0 = -rho * c;
    z1 = -rho * s;
}

// ceil(log2 n) complement: s = 63 - ceil(log2 n), so that n * 2^s <= 2^63
__host__ __device__ inline int scale_bits(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n)
        ++c;
    return 63 - c;
}

// 2^f for f in [0, 1): Taylor polynomial of e^(f ln 2) to degree 9, the
// coefficients (ln 2)^n / n! rounded to float32, evaluated by Horner's rule
// with fused multiply-adds.
__device__ __forceinline__ float exp2_frac(float f)
{
    float p = 0x1.b5253ep-24f;
    p = __fmaf_rn(p, f, 0x1.62c022p-20f);
    p = __fmaf_rn(p, f, 0x1.ffcbfcp-17f);
    p = __fmaf_rn(p, f, 0x1.430912p-13f);
    p = __fmaf_rn(p, f, 0x1.5d87fep-10f);
    p = __fmaf_rn(p, f, 0x1.3b2ab6p-7f);
    p = __fmaf_rn(p, f, 0x1.c6b08ep-5f);
    p = __fmaf_rn(p, f, 0x1.ebfbep-3f);
    p = __fmaf_rn(p, f, 0x1.62e43p-1f);
    p = __fmaf_rn(p, f, 1.0f);
    return p;
}

// The integer part of the quantiser: q = floor(p 2^(s + kf)) for t > -64.
__device__ __forceinline__ uint64_t quantise_tail(float t, float kf, float p, int s)
{
    const int e = s + (int)kf;
    // p lies in [1, 2]: P = p 2^23 is its mantissa with the implicit bit,
    // doubled when p = 2.  q = floor(P 2^(e - 23)) without branches:
    // X = P 2^39 < 2^64, q = X / 2^(62 - e); e = 63 only for p = 1 (t = 0),
    // and q = 0 for e < -1.
    const uint32_t pb = __float_as_uint(p);
    const uint64_t X = ((uint64_t)((pb & 0x7FFFFFu) | 0x800000u) << (((pb >> 23) - 127u) & 1u)) << 39;
    const int sh = 62 - e;
    const uint64_t q = (sh < 0) ? (X << 1) : (X >> (sh < 63 ? sh : 63));
    return (t > -64.0f && e >= -1) ? q : 0ull;  // t <= -64 or NaN: zero weight
}

__device__ __forceinline__ uint64_t quantise(float lw, float M, int s)
{
    const float d = __fsub_rn(lw, M);
    const float t = __fmul_rn(d, 0x1.715476p+0f);
    const float kf = fmaxf(floorf(t), -64.0f);  // the clamp only affects results that are 0 anyway
    const float f = __fsub_rn(t, kf);
    return quantise_tail(t, kf, exp2_frac(f), s);
}

// exp2_frac of two values at once: the same Horner steps as packed two-lane
// FMAs, each lane rounding as the scalar form.
__device__ __forceinline__ float2 exp2_frac2(float2 f)
{
    auto c = [](float v) { return make_float2(v, v); };
    float2 p = c(0x1.b5253ep-24f);
    p = __ffma2_rn(p, f, c(0x1.62c022p-20f));
    p = __ffma2_rn(p, f, c(0x1.ffcbfcp-17f));
    p = __ffma2_rn(p, f, c(0x1.430912p-13f));
    p = __ffma2_rn(p, f, c(0x1.5d87fep-10f));
    p = __ffma2_rn(p, f, c(0x1.3b2ab6p-7f));
    p = __ffma2_rn(p, f, c(0x1.c6b08ep-5f));
    p = __ffma2_rn(p, f, c(0x1.ebfbep-3f));
    p = __ffma2_rn(p, f, c(0x1.62e43p-1f));
    p = __ffma2_rn(p, f, c(1.0f));
    return p;
}

// quantise of two weights: the float32 steps as packed two-lane operations
// (a - M as a + (-M), exact in IEEE arithmetic), so both results equal the
// scalar quantise bit for bit.
__device__ __forceinline__ void quantise2(float a, float b, float M, int s, uint64_t &qa, uint64_t &qb)
{
    const float2 d = __fadd2_rn(make_float2(a, b), make_float2(-M, -M));
    const float2 t = __fmul2_rn(d, make_float2(0x1.715476p+0f, 0x1.715476p+0f));
    const float2 kf = make_float2(fmaxf(floorf(t.x), -64.0f), fmaxf(floorf(t.y), -64.0f));
    const float2 f = __fadd2_rn(t, make_float2(-kf.x, -kf.y));
    const float2 p = exp2_frac2(f);
    qa = quantise_tail(t.x, kf.x, p.x, s);
    qb = quantise_tail(t.y, kf.y, p.y, s);
}

// Number of systematic tickets below cumulative weight c (the per-group
// draws of RNA and two-stage RPA; the global draw uses tickets_below_grid):
// #{j in [0, n) : u + j Q < n c} = clamp(ceil((n c - u) / Q), 0, n).
// Exact integer result: the quotient (at most n < 2^31) is estimated twice
// with a float reciprocal of Q (the second time on the remainder) and then
// corrected with 128-bit arithmetic.
__device__ __forceinline__ float u128_to_float(u128 v)
{
    return (float)(uint64_t)(v >> 64) * 18446744073709551616.0f + (float)(uint64_t)v;
}

__device__ __forceinline__ int64_t tickets_below(uint64_t c, int64_t n, uint64_t u, uint64_t Q)
{
    typedef __int128 s128;
    const u128 nc = (u128)c * (u128)(uint64_t)n;
    if (nc <= (u128)u)
        return 0;
    const u128 num = nc - (u128)u;
    if (num > (u128)Q * (u128)(uint64_t)n)
        return n;
    const float rq = 1.0f / (float)Q;
    int64_t q = (int64_t)(u128_to_float(num) * rq);
    s128 r = (s128)num - (s128)q * (s128)Q;
    const float rf = (r < 0) ? -u128_to_float((u128)(-r)) : u128_to_float((u128)r);
    const int64_t dq = (int64_t)floorf(rf * rq);
    q += dq;
    r -= (s128)dq * (s128)Q;
    while (r < 0) {
        --q;
        r += (s128)Q;
    }
    while (r >= (s128)Q) {
        ++q;
        r -= (s128)Q;
    }
    if (r != 0)
        ++q;
    return q > n ? n : q;
}

// u = floor(r64 * Q / 2^64): a uniform ticket offset in [0, Q)
__device__ __forceinline__ uint64_t ticket_offset(uint64_t seed, uint32_t filter, uint32_t frame,
                                                  uint32_t purpose, uint32_t index, uint64_t Q)
{
    const uint4 r = draw(seed, index, frame, filter, purpose, 0);
    const uint64_t r64 = ((uint64_t)r.y << 32) | (uint64_t)r.x;
    return __umul64hi(r64, Q);
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += t;
    }
    return v;
}

// exclusive scan over the block (blockDim.x a multiple of 32, <= 1024);
// smem: 33 u64 (32 warp prefixes and the block total).  Returns the
// exclusive prefix; *total gets the block sum.
__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t v, uint64_t *smem, uint64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint64_t incl = warp_incl_scan_u64(v);
    __syncthreads();
    if (lane == 31)
        smem[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < nw ? smem[lane] : 0ull;
        const uint64_t wi = warp_incl_scan_u64(w);
        smem[lane] = wi - w;
        if (lane == 31)
            smem[32] = wi;
    }
    __syncthreads();
    const uint64_t res = smem[warp] + incl - v;
    *total = smem[32];
    return res;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace ppf
