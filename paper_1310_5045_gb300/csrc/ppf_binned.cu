// ppf_binned.cu -- the binned likelihood path: Sec. 6.3's input-space
// decomposition on one GPU.  When a step's particles are spread over the
// frame (the prior draw, a weak signal), the direct path's patch reads touch
// a separate cache line per lane and the step becomes bound by L2 traffic.
// The binned path instead:
//   1. propagates every slot, writes its bin and counts the bin sizes (the
//      step kernel's bin_propagate; a bin is an image tile of T x T patch
//      anchors, plus one bin for particles that need no patch sum);
//   2. scatters each particle's record (x, y, I0) into its bin: each block
//      turns the bin sizes into bin starts, takes chunks of slots, ranks them
//      by bin in shared memory and reserves one range per bin with one
//      atomic, so a bin's records from one chunk are written contiguously;
//      the slot keeps its record's place; the last block cuts the bins into
//      work items;
//   3. runs the likelihood over work items of one bin: the tile's window
//      (the tile plus the patch halo) is copied into shared memory by the
//      tensor-memory accelerator (cp.async.bulk.tensor, completion on an
//      mbarrier), the next item's window copied while this one is summed,
//      every patch read comes from shared memory, and l is written in bin
//      order;
//   4. sums in the direct path's slot order (the step kernel's phase 1),
//      fetching each slot's l from its record's place.
// A particle's likelihood has the same bits on both paths (the same PSF
// samples and the same patch_rows arithmetic), and the sums are taken in
// the same order, so the two paths give the same results bit for bit, and
// the order of the records inside a bin does not matter.  The step's
// finaliser picks the path of the next step from the spread of its warps.
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>

#include "ppf_device.cuh"
#include "ppf_internal.h"
#include "ppf_kernels.cuh"

namespace ppf {

constexpr int BIN_ITEM = 4096;        // records per likelihood work item
constexpr int BIN_SORT_PER_THREAD = BIN_ITEM / 256;
constexpr int BIN_MAX_BOX = 128;      // window edge T + 2R (a tensor copy box is at most 256 floats wide)

// ---------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// a 2D tile of the prepared frame into shared memory; completion is counted
// on the mbarrier in bytes (x is the float column, a multiple of 4 here)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Waits for the phase of the given parity to complete.  Bounded: gives up
// after about a second of clock cycles (or 2^26 polls) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (clock64() - t0 > (1ll << 31))
            break;
    }
    return false;
}

// ---------------------------------------------------------- the scatter
// Each block first turns the bin sizes into their exclusive prefix (each
// bin's first record).  It then takes chunks of BIN_CHUNK consecutive slots,
// each thread 16 consecutive slots read as 16-byte vectors.  A chunk is
// ranked by bin in shared memory and staged there in bin order; one global
// atomic per nonempty bin reserves the chunk's range inside the bin (its
// cursor), and the staged records are then copied out so that consecutive
// threads write consecutive records of a run.  Each slot's key entry receives
// its record's place (read by the sums of phase 1).  The last block to finish
// cuts every bin into work items of at most BIN_ITEM records for the
// likelihood.
constexpr int BIN_PER_THREAD = 16;
constexpr int BIN_CHUNK = 256 * BIN_PER_THREAD;

__global__ void __launch_bounds__(256) bin_scatter_kernel(const float *__restrict__ st, int64_t N, int nbins,
                                                          uint32_t *__restrict__ key,
                                                          const uint32_t *__restrict__ size,
                                                          uint32_t *__restrict__ cursor, float4 *__restrict__ rec,
                                                          int32_t *__restrict__ items, int items_max,
                                                          DevSummary *sum)
{
    pdl_wait();  // launched as a dependent of the step kernel
    pdl_trigger();
    if (__ldcg(&sum->bin_this) == 0)
        return;
    int32_t *flags = &sum->flags;
    // [BIN_CHUNK] staged records, [BIN_CHUNK] their bins, then per bin: count,
    // local start, global start, bin start
    extern __shared__ float4 stage[];
    uint16_t *sbin = reinterpret_cast<uint16_t *>(stage + BIN_CHUNK);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(sbin + BIN_CHUNK);
    uint32_t *lstart = cnt + nbins, *gstart = lstart + nbins, *bstart = gstart + nbins;
    __shared__ uint64_t red[33];
    {   // bin starts: exclusive prefix of the sizes
        const int per = (nbins + blockDim.x - 1) / blockDim.x, t0 = threadIdx.x * per;
        uint64_t sm = 0;
        for (int t = t0; t < t0 + per && t < nbins; ++t)
            sm += __ldcg(size + t);
        uint64_t tot;
        uint64_t run = block_excl_scan_u64(sm, red, &tot);
        for (int t = t0; t < t0 + per && t < nbins; ++t) {
            bstart[t] = (uint32_t)run;
            run += __ldcg(size + t);
        }
        __syncthreads();
    }
    const uint32_t n = (uint32_t)N;
    const bool vec_ok = (N & 3) == 0;  // 16-byte vectors need 16-byte aligned planes
    for (uint32_t lo = blockIdx.x * (uint32_t)BIN_CHUNK; lo < n; lo += gridDim.x * (uint32_t)BIN_CHUNK) {
        for (int t = threadIdx.x; t < nbins; t += blockDim.x)
            cnt[t] = 0u;
        const uint32_t i0 = lo + threadIdx.x * BIN_PER_THREAD;
        const bool full = vec_ok && i0 + BIN_PER_THREAD <= n;
        uint32_t k[BIN_PER_THREAD], r[BIN_PER_THREAD];
        if (full) {
#pragma unroll
            for (int q = 0; q < BIN_PER_THREAD / 4; ++q) {
                const uint4 kk = __ldg(reinterpret_cast<const uint4 *>(key + i0) + q);
                k[4 * q] = kk.x; k[4 * q + 1] = kk.y; k[4 * q + 2] = kk.z; k[4 * q + 3] = kk.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < BIN_PER_THREAD; ++e)
                k[e] = i0 + e < n ? __ldg(key + i0 + e) : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < BIN_PER_THREAD; ++e)
            r[e] = (i0 + e < n) ? atomicAdd(&cnt[k[e]], 1u) : 0u;
        __syncthreads();
        {   // local starts (exclusive prefix of the counts) and the global reservations
            const int per = (nbins + blockDim.x - 1) / blockDim.x, t0 = threadIdx.x * per;
            uint64_t sm = 0;
            for (int t = t0; t < t0 + per && t < nbins; ++t)
                sm += cnt[t];
            uint64_t tot;
            uint64_t run = block_excl_scan_u64(sm, red, &tot);
            for (int t = t0; t < t0 + per && t < nbins; ++t) {
                const uint32_t c = cnt[t];
                lstart[t] = (uint32_t)run;
                gstart[t] = c ? bstart[t] + atomicAdd(cursor + t, c) : 0u;
                run += c;
            }
        }
        __syncthreads();
        // stage the records in bin order (the state read now, as 16-byte vectors)
#pragma unroll
        for (int q = 0; q < BIN_PER_THREAD / 4; ++q) {
            float4 xx, yy, zz;
            if (full) {
                xx = __ldg(reinterpret_cast<const float4 *>(st + i0) + q);
                yy = __ldg(reinterpret_cast<const float4 *>(st + N + i0) + q);
                zz = __ldg(reinterpret_cast<const float4 *>(st + 4 * N + i0) + q);
            } else {
                auto at = [&](const float *p, int e) { return i0 + e < n ? __ldg(p + i0 + e) : 0.0f; };
                xx = make_float4(at(st, 4 * q), at(st, 4 * q + 1), at(st, 4 * q + 2), at(st, 4 * q + 3));
                yy = make_float4(at(st + N, 4 * q), at(st + N, 4 * q + 1), at(st + N, 4 * q + 2), at(st + N, 4 * q + 3));
                zz = make_float4(at(st + 4 * N, 4 * q), at(st + 4 * N, 4 * q + 1), at(st + 4 * N, 4 * q + 2),
                                 at(st + 4 * N, 4 * q + 3));
            }
            const float xs[4] = {xx.x, xx.y, xx.z, xx.w}, ys[4] = {yy.x, yy.y, yy.z, yy.w};
            const float zs[4] = {zz.x, zz.y, zz.z, zz.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = 4 * q + c;
                if (i0 + e < n) {
                    const uint32_t j = lstart[k[e]] + r[e];
                    stage[j] = make_float4(xs[c], ys[c], zs[c], 0.0f);
                    sbin[j] = (uint16_t)k[e];
                    k[e] = gstart[k[e]] + r[e];  // the record's place, for the slot's key entry
                }
            }
        }
        if (full) {
#pragma unroll
            for (int q = 0; q < BIN_PER_THREAD / 4; ++q)
                reinterpret_cast<uint4 *>(key + i0)[q] = make_uint4(k[4 * q], k[4 * q + 1], k[4 * q + 2], k[4 * q + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < BIN_PER_THREAD; ++e)
                if (i0 + e < n)
                    key[i0 + e] = k[e];
        }
        __syncthreads();
        // copy out: consecutive threads, consecutive records of a bin's run
        const uint32_t m = (n - lo < (uint32_t)BIN_CHUNK) ? n - lo : (uint32_t)BIN_CHUNK;
        for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) {
            const uint32_t t = sbin[j];
            const uint32_t pos = gstart[t] + (j - lstart[t]);
            if (PPF_DCHECK(pos < n, flags, FLAG_INTERNAL))
                rec[pos] = stage[j];
        }
        __syncthreads();
    }
    // the last block: the likelihood's work items (no block waits for it)
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&sum->bin_blocks_done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    uint32_t *sio = reinterpret_cast<uint32_t *>(stage);  // [nbins + 1] item prefix (the stage is free now)
    {
        const int per = (nbins + blockDim.x - 1) / blockDim.x, t0 = threadIdx.x * per;
        uint64_t sm = 0;
        for (int t = t0; t < t0 + per && t < nbins; ++t)
            sm += (__ldcg(size + t) + BIN_ITEM - 1) / BIN_ITEM;
        uint64_t iall;
        uint64_t run = block_excl_scan_u64(sm, red, &iall);
        for (int t = t0; t < t0 + per && t < nbins; ++t) {
            sio[t] = (uint32_t)run;
            run += (__ldcg(size + t) + BIN_ITEM - 1) / BIN_ITEM;
        }
        if (threadIdx.x == 0) {
            sio[nbins] = (uint32_t)iall;
            sum->n_bin_items = (int32_t)iall;
            sum->bin_blocks_done = 0u;
        }
    }
    __syncthreads();
    const uint32_t ni = sio[nbins];
    for (uint32_t j = threadIdx.x; j < ni; j += blockDim.x) {
        int lo = 0, hi = nbins;  // sio[lo] <= j < sio[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sio[mid] <= j)
                lo = mid;
            else
                hi = mid;
        }
        const uint32_t s0 = (j - sio[lo]) * (uint32_t)BIN_ITEM;
        const uint32_t sz = __ldcg(size + lo);
        if (PPF_DCHECK(j < (uint32_t)items_max && s0 < sz, flags, FLAG_INTERNAL)) {
            items[j] = lo;
            items[items_max + j] = (int32_t)(bstart[lo] + s0);
            items[2 * items_max + j] = (int32_t)((sz - s0) < (uint32_t)BIN_ITEM ? (sz - s0) : BIN_ITEM);
        }
    }
}

// ------------------------------------------------------- the likelihood
struct BinLikArgs {
    int64_t N;
    int W, H, T, nx, nbins, box;   // box = T + 2R: window edge in pairs and rows
    int items_max;
    int win_stride;                // bytes between the two windows (a multiple of 128)
    float inv2s2, inv_sxi2;
    float Kc[MAX_RADIUS];
    const float4 *__restrict__ rec;
    const int32_t *__restrict__ items;
    float *__restrict__ l;         // l of every record, in bin order
    DevSummary *sum;
};

template <int R>
__global__ void __launch_bounds__(256) bin_loglik_kernel(const __grid_constant__ CUtensorMap tmap, BinLikArgs a)
{
    pdl_wait();  // launched as a dependent of the scatter
    pdl_trigger();
    DevSummary *sum = a.sum;
    if (__ldcg(&sum->bin_this) == 0)
        return;
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int failed;
    const int n_items = __ldcg(&sum->n_bin_items);
    // the windows start on a 128-byte boundary (the launch adds 128 bytes of
    // slack); then the item's records sorted by anchor and the anchor counts
    const uint32_t base = smem_u32(bsm), pad = ((base + 127u) & ~127u) - base;
    unsigned char *wbase = bsm + pad;
    float4 *srt = reinterpret_cast<float4 *>(wbase + 2 * a.win_stride);
    uint32_t *hist = reinterpret_cast<uint32_t *>(srt + BIN_ITEM);
    __shared__ uint64_t red[33];
    const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
    const uint32_t win0 = base + pad, win1 = win0 + (uint32_t)a.win_stride;
    const uint32_t box_bytes = (uint32_t)(a.box * a.box * 8);
    if (threadIdx.x == 0) {
        mbar_init(bar0);
        mbar_init(bar1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    __syncthreads();
    const int32_t *ibin = a.items, *istart = a.items + a.items_max, *icount = a.items + 2 * a.items_max;
    const int special = a.nbins - 1;
    auto issue = [&](int j, int buf) {  // thread 0: the window of item j into buffer buf
        const int t = __ldg(ibin + j);
        if (t == special)
            return;
        const int tx = t % a.nx, ty = t / a.nx;
        const uint32_t bar = buf ? bar1 : bar0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, box_bytes);
        tma_load_2d(buf ? win1 : win0, &tmap, 2 * tx * a.T, ty * a.T, bar);
    };
    const PatchGeom geom{nullptr, a.W, a.H, 0, 0, a.inv2s2, a.inv_sxi2, a.Kc, 0, &sum->flags};
    const float4 *__restrict__ rec = a.rec;
    // Thread 0 issues every window copy; all threads wait on its barrier.  A
    // wait that times out stops the block's work (the flag reports it), and
    // thread 0 then waits once more, bounded, for the copies it left in
    // flight before the block's shared memory is released.
    // bit b of phase: the parity of buffer b's next copy; bit b of pend: a
    // copy into buffer b issued and not yet waited for
    uint32_t phase = 0u, pend = 0u;
    int k = 0;
    if ((int)blockIdx.x < n_items) {
        if (threadIdx.x == 0)
            issue(blockIdx.x, 0);
        pend |= (__ldg(ibin + blockIdx.x) != special) ? 1u : 0u;
    }
    for (int j = blockIdx.x; j < n_items; j += gridDim.x, ++k) {
        const int buf = k & 1;
        const int jn = j + (int)gridDim.x;
        if (jn < n_items) {  // the next item's window, copied while this one is summed
            if (threadIdx.x == 0)
                issue(jn, buf ^ 1);
            if (__ldg(ibin + jn) != special)
                pend |= 1u << (buf ^ 1);
        }
        const int t = __ldg(ibin + j);
        const int s0 = __ldg(istart + j), cntj = __ldg(icount + j);
        if (t != special) {
            if (mbar_wait(buf ? bar1 : bar0, (phase >> buf) & 1u)) {
                phase ^= 1u << buf;
                pend &= ~(1u << buf);
            } else {
                atomicOr(&sum->flags, FLAG_TIMEOUT);
                failed = 1;
            }
            __syncthreads();
            if (failed)
                break;
        }
        const float2 *win = reinterpret_cast<const float2 *>(wbase + (buf ? a.win_stride : 0));
        const int tx = t % a.nx, ty = t / a.nx;
        constexpr int P = 2 * R + 1;
        if (t == special) {  // no patch sums: l = -inf (non-finite) or 0 (no pixel in the image)
            for (int r = s0 + threadIdx.x; r < s0 + cntj; r += blockDim.x) {
                const float4 q = rec[r];
                int cx, cy;
                float gx[P], gy[P], C, l;
                patch_setup<R>(geom, q.x, q.y, q.z, cx, cy, gx, gy, C, &l);
                a.l[r] = l;
            }
        } else {
            // Sort the item's records by patch anchor (a counting sort over the
            // T x T anchors of the tile), so that the lanes of a warp hold
            // neighbouring anchors and their window reads share shared-memory
            // words instead of colliding in the banks.
            for (int u = threadIdx.x; u < a.T * a.T; u += blockDim.x)
                hist[u] = 0u;
            __syncthreads();
            uint32_t an[BIN_SORT_PER_THREAD], rk[BIN_SORT_PER_THREAD];
#pragma unroll
            for (int e = 0; e < BIN_SORT_PER_THREAD; ++e) {
                const int r = threadIdx.x + e * (int)blockDim.x;
                const float2 xy = r < cntj ? *reinterpret_cast<const float2 *>(rec + s0 + r) : make_float2(0.0f, 0.0f);
                const int lu = (int)floorf(xy.x + 0.5f) + R - tx * a.T;
                const int lv = (int)floorf(xy.y + 0.5f) + R - ty * a.T;
                const bool ok = r < cntj && PPF_DCHECK(lu >= 0 && lu < a.T && lv >= 0 && lv < a.T, &sum->flags,
                                                       FLAG_INTERNAL);
                an[e] = ok ? (uint32_t)(lv * a.T + lu) : 0xFFFFFFFFu;
                rk[e] = ok ? atomicAdd(&hist[an[e]], 1u) : 0u;
            }
            __syncthreads();
            // exclusive prefix of the T x T counts (at most 4096: 16 per thread)
            {
                const int na = a.T * a.T, per = (na + blockDim.x - 1) / blockDim.x, u0 = threadIdx.x * per;
                uint64_t sm = 0;
                for (int u = u0; u < u0 + per && u < na; ++u)
                    sm += hist[u];
                uint64_t tot;
                uint64_t run = block_excl_scan_u64(sm, red, &tot);
                for (int u = u0; u < u0 + per && u < na; ++u) {
                    const uint32_t c = hist[u];
                    hist[u] = (uint32_t)run;
                    run += c;
                }
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < BIN_SORT_PER_THREAD; ++e)
                if (an[e] != 0xFFFFFFFFu) {  // the record again (from L2), to its sorted place
                    const int r = threadIdx.x + e * (int)blockDim.x;
                    const float4 q = rec[s0 + r];
                    srt[hist[an[e]] + rk[e]] = make_float4(q.x, q.y, q.z, __uint_as_float((uint32_t)r));
                }
            __syncthreads();
            for (int j = threadIdx.x; j < cntj; j += blockDim.x) {
                const float4 v = srt[j];  // (x, y, I0, the record's place in the item)
                int cx, cy;
                float gx[P], gy[P], C, l;
                if (patch_setup<R>(geom, v.x, v.y, v.z, cx, cy, gx, gy, C, &l)) {
                    const int lu = cx + R - tx * a.T, lv = cy + R - ty * a.T;
                    const float Bs = patch_rows<R, true, true>(win + lv * a.box + lu, a.box, gx, gy);
                    l = v.z * fmaf(-0.5f * v.z, C, Bs) * a.inv_sxi2;
                }
                a.l[s0 + __float_as_uint(v.w)] = l;
            }
        }
        __syncthreads();  // this window is free for the copy two items on
    }
    if (failed && threadIdx.x == 0) {
        if (pend & 1u)
            mbar_wait(bar0, phase & 1u);
        if (pend & 2u)
            mbar_wait(bar1, (phase >> 1) & 1u);
    }
}

// ------------------------------------------------------------ host side
namespace {

int win_stride_bytes(int box)
{
    const int b = box * box * 8;
    return (b + 127) / 128 * 128;
}

size_t scatter_smem(int nbins)
{
    // staged records, their bins, and four words per bin
    return sizeof(float4) * BIN_CHUNK + sizeof(uint16_t) * BIN_CHUNK + 4 * sizeof(uint32_t) * (size_t)nbins;
}

size_t loglik_smem(int box, int T)
{
    // two windows, the alignment slack, the sorted records, the anchor counts
    return 2 * (size_t)win_stride_bytes(box) + 128 + sizeof(float4) * BIN_ITEM + sizeof(uint32_t) * T * T;
}

// The dynamic shared memory limit of a kernel is raised to the device's
// opt-in maximum less the kernel's static shared memory (a limit, not a
// reservation): contexts with other window sizes then never lower it under
// one another.
template <typename K>
cudaError_t raise_smem_limit(K kernel, size_t need)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess)
        return e;
    const int lim = optin - (int)fa.sharedSizeBytes;
    if ((int64_t)need > lim)
        return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <int R>
cudaError_t loglik_attr(size_t smem, int *per_sm)
{
    cudaError_t e = raise_smem_limit(bin_loglik_kernel<R>, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, bin_loglik_kernel<R>, 256, smem);
    return e;
}

cudaError_t loglik_setup(int R, size_t smem, int *per_sm)
{
    switch (R) {
    case 0: return loglik_attr<0>(smem, per_sm);
    case 1: return loglik_attr<1>(smem, per_sm);
    case 2: return loglik_attr<2>(smem, per_sm);
    case 3: return loglik_attr<3>(smem, per_sm);
    case 4: return loglik_attr<4>(smem, per_sm);
    case 5: return loglik_attr<5>(smem, per_sm);
    case 6: return loglik_attr<6>(smem, per_sm);
    case 7: return loglik_attr<7>(smem, per_sm);
    default: return loglik_attr<8>(smem, per_sm);
    }
}

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

cudaError_t bin_setup(ppf_ctx *c)
{
    const int R = c->m.patch_radius;
    if (c->m.likelihood != 0)
        return cudaSuccess;  // pcSIR: one lookup per particle, no patch to stage
    int T = 32;
    auto bins = [&](int t) { return (int64_t)((c->m.width + 2 * R + t - 1) / t) * ((c->m.height + 2 * R + t - 1) / t) + 1; };
    while (bins(T) > BIN_MAX_BINS && T + 2 * R <= BIN_MAX_BOX / 2)
        T *= 2;
    if (bins(T) > BIN_MAX_BINS || T + 2 * R > BIN_MAX_BOX)
        return cudaSuccess;  // frames this large keep the direct path
    c->bin_T = T;
    c->bin_nx = (c->m.width + 2 * R + T - 1) / T;
    c->bin_nbins = (int32_t)bins(T);
    c->bin_items_max = c->bin_nbins + (int32_t)((c->N + BIN_ITEM - 1) / BIN_ITEM);
    const int box = T + 2 * R;
    const size_t smem = loglik_smem(box, T);
    int per_sm = 0;
    cudaError_t e = loglik_setup(R, smem, &per_sm);
    if (e != cudaSuccess)
        return e;
    c->bin_grid = c->num_sms * (per_sm > 0 ? (per_sm < 4 ? per_sm : 4) : 1);
    e = raise_smem_limit(bin_scatter_kernel, scatter_smem(c->bin_nbins));
    if (e != cudaSuccess)
        return e;
    if ((e = dalloc(&c->bin_key, (size_t)c->N)) != cudaSuccess ||
        (e = dalloc(&c->bin_l, (size_t)c->N)) != cudaSuccess ||
        (e = dalloc(&c->bin_tot, 2 * ((size_t)c->bin_nbins + 1))) != cudaSuccess ||
        (e = dalloc(&c->bin_item, 3 * (size_t)c->bin_items_max)) != cudaSuccess ||
        (e = dalloc(&c->bin_rec, (size_t)c->N)) != cudaSuccess)
        return e;
    // the prepared frame as a 2D float tensor (2 Wp floats per row, Hp rows);
    // a window is 2 box floats by box rows, copied with zero fill outside
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return e != cudaSuccess ? e : cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * c->Wp, (cuuint64_t)c->Hp};
    const cuuint64_t strides[1] = {(cuuint64_t)2 * c->Wp * sizeof(float)};
    const cuuint32_t boxd[2] = {(cuuint32_t)(2 * box), (cuuint32_t)box};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<EncodeTiled>(fn)(
        &c->bin_tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->Zp, dims, strides, boxd, estr,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return bin_set_next(c, 1);  // the prior draw is spread over the frame
}

cudaError_t bin_set_next(ppf_ctx *c, int binned)
{
    if (!c->bin_key)
        return cudaSuccess;
    const int32_t v = binned ? 1 : 0;
    cudaError_t e = cudaMemcpyAsync((char *)c->sum + offsetof(DevSummary, bin_next), &v, sizeof(v),
                                    cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(c->stream) : e;
}

template <int R>
static void launch_loglik_r(const CUtensorMap &tm, const BinLikArgs &a, int grid, size_t smem, cudaStream_t s)
{
    launch_pdl(bin_loglik_kernel<R>, grid, 256, smem, s, tm, a);
}

cudaError_t launch_binned(ppf_ctx *c)
{
    const int R = c->m.patch_radius;
    const int nb = c->bin_nbins;
    float *dst = c->state[c->cur ^ 1];
    const int64_t chunks = (c->N + BIN_CHUNK - 1) / BIN_CHUNK;
    const int gscat = (int)(chunks < 4 * (int64_t)c->num_sms ? chunks : 4 * (int64_t)c->num_sms);
    launch_pdl(bin_scatter_kernel, gscat, 256, scatter_smem(nb), c->stream, (const float *)dst, c->N, nb, c->bin_key,
               (const uint32_t *)c->bin_tot, c->bin_tot + nb + 1, c->bin_rec, c->bin_item, c->bin_items_max, c->sum);
    BinLikArgs a;
    memset(&a, 0, sizeof(a));
    a.N = c->N;
    a.W = c->m.width;
    a.H = c->m.height;
    a.T = c->bin_T;
    a.nx = c->bin_nx;
    a.nbins = nb;
    a.box = c->bin_T + 2 * R;
    a.items_max = c->bin_items_max;
    a.win_stride = win_stride_bytes(a.box);
    a.inv2s2 = 1.0f / (2.0f * c->m.psf_sigma * c->m.psf_sigma);
    a.inv_sxi2 = 1.0f / (c->m.sigma_xi * c->m.sigma_xi);
    for (int q = 0; q < MAX_RADIUS; ++q)
        a.Kc[q] = (float)exp(-(2.0 * q + 1.0) * (double)a.inv2s2);
    a.rec = c->bin_rec;
    a.items = c->bin_item;
    a.l = c->bin_l;
    a.sum = c->sum;
    const size_t smem = loglik_smem(a.box, a.T);
    switch (R) {
    case 0: launch_loglik_r<0>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    case 1: launch_loglik_r<1>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    case 2: launch_loglik_r<2>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    case 3: launch_loglik_r<3>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    case 4: launch_loglik_r<4>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    case 5: launch_loglik_r<5>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    case 6: launch_loglik_r<6>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    case 7: launch_loglik_r<7>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    default: launch_loglik_r<8>(c->bin_tmap, a, c->bin_grid, smem, c->stream); break;
    }
    c->launches += 2;
    return cudaGetLastError();
}

}  // namespace ppf
