// ppf_probe.cu -- measurement hook: the FP32 FMA throughput of the current
// device, the denominator of the likelihood's ALU roofline.  Every thread runs
// eight independent FMA chains (or four packed two-lane chains), so the FMA
// pipes stay busy without waiting on a chain's latency; the grid fills every
// SM several times over.  No part of the filter uses it.
#include <cuda_runtime.h>

#include <cstdint>

#include "ppf.h"

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 16;

template <bool kPacked>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(float *out, int iters, float a, float b)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        x[j] = 1e-6f * (float)(t & 1023) + (float)j;
    if constexpr (kPacked) {
        float2 v[4], av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            v[j] = make_float2(x[2 * j], x[2 * j + 1]);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    v[j] = __ffma2_rn(v[j], av, bv);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            x[2 * j] = v[j].x;
            x[2 * j + 1] = v[j].y;
        }
    } else {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    x[j] = fmaf(x[j], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        s += x[j];
    out[t] = s;  // keeps the chains live
}

}  // namespace

extern "C" ppf_status ppf_fp32_peak(int32_t packed, int32_t repeats, double *tflops_out, double *ms_out)
{
    if (!tflops_out || repeats < 1 || repeats > 100)
        return PPF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PPF_ECUDA;
    const int blocks = sms * 8;  // 2048 threads per SM, eight times over in blocks of 256
    const int iters = 256;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ppf_status st = PPF_OK;
    double best = 0.0;
    if (cudaMalloc((void **)&out, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess)
        return PPF_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = PPF_ECUDA;
    } else {
        // FMAs per launch: 8 lanes of chains x unroll x iterations per thread
        const double flops = 2.0 * 8.0 * kUnroll * (double)iters * (double)blocks * kThreads;
        for (int r = 0; r <= repeats && st == PPF_OK; ++r) {  // launch 0 warms up
            cudaEventRecord(e0, 0);
            if (packed)
                fma_chain_kernel<true><<<blocks, kThreads>>>(out, iters, 0.999999f, 1e-6f);
            else
                fma_chain_kernel<false><<<blocks, kThreads>>>(out, iters, 0.999999f, 1e-6f);
            cudaEventRecord(e1, 0);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                st = PPF_ECUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms > 0.0f) {
                const double tf = flops / (ms * 1e-3) / 1e12;
                if (tf > best) {
                    best = tf;
                    if (ms_out)
                        *ms_out = ms;
                }
            }
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(out);
    *tflops_out = best;
    return st;
}
