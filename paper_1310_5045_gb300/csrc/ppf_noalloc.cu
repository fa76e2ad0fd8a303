// ppf_noalloc.cu -- systematic resampling with no device allocation.
//
// Some callers cannot call cudaMalloc: a serving or real-time loop that
// pre-plans every byte of device memory (cudaMalloc may block and
// synchronise the device, stalling other streams), or a host whose device
// memory is owned by another runtime's allocator and must not be bypassed.
// For them, ppf_systematic_resample_noalloc runs the library's systematic
// resampling kernels with all their scratch in one file-scope device array
// of fixed size, so the call allocates nothing.
//
// The array lives as long as the library is loaded, on every device that
// loads it.  All calls share it and it keeps the last call's contents: every
// call first clears what must start at zero, and calls whose work overlaps on
// the GPU (two streams, two host threads) race on it and must be serialised
// by the caller.
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "ppf_device.cuh"
#include "ppf_internal.h"
#include "ppf_tiles.cuh"

namespace ppf {

// kernels of ppf_resample.cu used unchanged
__global__ void __launch_bounds__(TILE_THREADS, 5) tile_totals_kernel(const float *__restrict__ lw, int64_t N,
                                                                      const DevSummary *__restrict__ sum,
                                                                      double ess_thr, uint64_t *__restrict__ Qt);
__global__ void __launch_bounds__(1024) tile_scan_kernel(int64_t N, int32_t T, const uint64_t *__restrict__ Qt, uint64_t *__restrict__ Ct,
                                 int64_t *__restrict__ Tt, int32_t *__restrict__ item_off,
                                 int32_t *__restrict__ item_tile, DevSummary *sum, double ess_thr, uint64_t seed,
                                 uint32_t fid, uint32_t frame, const int64_t *__restrict__ goff, int32_t G, int rpa,
                                 const uint64_t *__restrict__ Cbl, int64_t *__restrict__ Tg, int32_t smem_tiles,
                                 Divisor ndiv, int prefix_only, int2 *__restrict__ extra);
__global__ void __launch_bounds__(TILE_THREADS) fill_kernel(const float *__restrict__ lw, int64_t N, int32_t T, Divisor ndiv,
                            const DevSummary *__restrict__ sum, const uint64_t *__restrict__ Ct,
                            const int64_t *__restrict__ Tt, const int32_t *__restrict__ item_off,
                            const int32_t *__restrict__ item_tile, int32_t *__restrict__ out);

namespace {

constexpr int64_t NOALLOC_MAX_N = (int64_t)1 << 24;               // particles per call
constexpr int32_t NOALLOC_MAX_T = (int32_t)(NOALLOC_MAX_N / TILE);  // 4096 tiles

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_SUM = 0;
constexpr size_t OFF_MAX = align256(OFF_SUM + sizeof(DevSummary));   // ordered max of lw + block counter
constexpr size_t OFF_QT = align256(OFF_MAX + 2 * sizeof(uint32_t));
constexpr size_t OFF_CT = align256(OFF_QT + sizeof(uint64_t) * NOALLOC_MAX_T);
constexpr size_t OFF_TT = align256(OFF_CT + sizeof(uint64_t) * (NOALLOC_MAX_T + 1));
constexpr size_t OFF_IT = align256(OFF_TT + sizeof(int64_t) * (NOALLOC_MAX_T + 1));
constexpr size_t SCRATCH_BYTES = align256(OFF_IT + sizeof(int32_t) * (NOALLOC_MAX_T + 1));  // ~113 KB

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// order-preserving map of a float to an unsigned key (NaN never used)
__device__ __forceinline__ uint32_t float_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// clears what every call needs at zero: the summary and the max / counter words
__global__ void noalloc_clear_kernel(unsigned char *scratch)
{
    DevSummary *sum = reinterpret_cast<DevSummary *>(scratch + OFF_SUM);
    uint32_t *mx = reinterpret_cast<uint32_t *>(scratch + OFF_MAX);
    if (threadIdx.x == 0) {
        memset(sum, 0, sizeof(DevSummary));
        mx[0] = float_key(-INFINITY);
        mx[1] = 0u;
    }
}

// M = max lw (NaN ignored); the last block to finish stores it in the summary
__global__ void noalloc_max_kernel(const float *__restrict__ lw, int64_t n, unsigned char *scratch)
{
    DevSummary *sum = reinterpret_cast<DevSummary *>(scratch + OFF_SUM);
    uint32_t *mx = reinterpret_cast<uint32_t *>(scratch + OFF_MAX);
    float m = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, __ldg(lw + i));  // fmaxf drops NaN
    m = warp_max(m);
    __shared__ float sm[32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0)
        sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            b = fmaxf(b, sm[w]);
        atomicMax(&mx[0], float_key(b));
        __threadfence();
        last = (atomicAdd(&mx[1], 1u) == gridDim.x - 1);
        if (last) {
            __threadfence();
            sum->M = key_float(atomicAdd(&mx[0], 0u));
        }
    }
}

// all weights zero or NaN: the ancestry is the identity
__global__ void noalloc_identity_if_degenerate(int32_t *__restrict__ anc, int64_t n, const unsigned char *scratch)
{
    const DevSummary *sum = reinterpret_cast<const DevSummary *>(scratch + OFF_SUM);
    if (!sum->degenerate)
        return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        anc[i] = (int32_t)i;
}

// The unique id of the calling thread's current CUDA context (cuCtxGetId,
// reached through the runtime's driver entry points, so the library does
// not link the driver library).  0 when it cannot be had.
unsigned long long current_context_id()
{
    typedef CUresult (*GetCurrent)(CUcontext *);
    typedef CUresult (*GetId)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f);
            get_id = reinterpret_cast<GetId>(g);
        }
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_scratch, looked up with the device current: once per
// device and CUDA context.  A reset device (cudaDeviceReset) gets a new
// context, and with it a new lookup and the fill kernel's attribute set again.
std::mutex g_mu;
unsigned char *g_addr[128] = {};
unsigned long long g_ctx[128] = {};

unsigned char *scratch_address(int dev, cudaError_t *err)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev < 0 || dev >= 128) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    // (no context current yet on this thread: id 0, and the lookup below
    // makes the device's primary context current)
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_scratch);
        if (*err != cudaSuccess)
            return nullptr;
        // the fill kernel's dynamic shared memory size (an attribute, no allocation)
        *err = resample_kernel_attributes();
        if (*err != cudaSuccess)
            return nullptr;
        g_addr[dev] = static_cast<unsigned char *>(p);
        g_ctx[dev] = current_context_id();
    }
    *err = cudaSuccess;
    return g_addr[dev];
}

}  // namespace
}  // namespace ppf

extern "C" ppf_status ppf_systematic_resample_noalloc(const float *lw_dev, int64_t n, uint64_t seed,
                                                      uint32_t filter_id, int32_t frame, int32_t *anc_dev,
                                                      void *cuda_stream)
{
    using namespace ppf;
    if (!lw_dev || !anc_dev || n < 1 || n > NOALLOC_MAX_N || frame < 0)
        return PPF_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return PPF_ECUDA;
    cudaError_t e;
    unsigned char *s = scratch_address(dev, &e);
    if (!s)
        return PPF_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DevSummary *sum = reinterpret_cast<DevSummary *>(s + OFF_SUM);
    uint64_t *Qt = reinterpret_cast<uint64_t *>(s + OFF_QT);
    uint64_t *Ct = reinterpret_cast<uint64_t *>(s + OFF_CT);
    int64_t *Tt = reinterpret_cast<int64_t *>(s + OFF_TT);
    int32_t *item_off = reinterpret_cast<int32_t *>(s + OFF_IT);
    const int32_t T = (int32_t)((n + TILE - 1) / TILE);
    noalloc_clear_kernel<<<1, 32, 0, st>>>(s);
    const int gmax = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    noalloc_max_kernel<<<gmax, 256, 0, st>>>(lw_dev, n, s);
    // (every call resamples: the N_eff threshold is +inf)
    tile_totals_kernel<<<T, TILE_THREADS, 0, st>>>(lw_dev, n, sum, INFINITY, Qt);
    // (no item-to-tile map: the fill blocks find their tile by binary search)
    // (T <= 4096 tiles: the scan's tile values, 32 KB, fit the default shared memory)
    tile_scan_kernel<<<1, 1024, sizeof(uint64_t) * (T + 1), st>>>(n, T, Qt, Ct, Tt, item_off, nullptr, sum, INFINITY,
                                                                  seed, filter_id, (uint32_t)frame, nullptr, 0, 0,
                                                                  nullptr, nullptr, T, make_divisor((uint32_t)n), 0,
                                                                  nullptr);
    const int max_items = T + (int)((n + ITEM_TICKETS - 1) / ITEM_TICKETS);
    fill_kernel<<<max_items, TILE_THREADS, FILL_SMEM_BYTES, st>>>(lw_dev, n, T, make_divisor((uint32_t)n), sum, Ct,
                                                                  Tt, item_off, nullptr, anc_dev);
    noalloc_identity_if_degenerate<<<gmax, 256, 0, st>>>(anc_dev, n, s);
    return cudaGetLastError() == cudaSuccess ? PPF_OK : PPF_ECUDA;
}
