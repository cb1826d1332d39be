// rime_peaks.cu -- measured issue rates of the arithmetic pipes the roofline
// fractions are quoted against: FP32 FMA (scalar and packed pairs), FP64 FMA
// and the SFU's exp2. Each kernel keeps eight independent chains per thread
// in registers over enough warps to fill every SM, so that the rate is the
// pipe's and not the chains' latency.
#include "rime_internal.cuh"
#include "rime_fused_common.cuh"

#include <algorithm>

namespace rime {
namespace peaks {

constexpr int THREADS = 256, CHAINS = 8, UNROLL = 16;

template <int KIND>
__global__ void __launch_bounds__(THREADS) k_pipe(float *out, int iters, float m, float c) {
    float acc = 0.f;
    if (KIND == RIME_PIPE_FFMA) {
        float a[CHAINS];
#pragma unroll
        for (int j = 0; j < CHAINS; j++) a[j] = threadIdx.x * 1e-3f + j;
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int u = 0; u < UNROLL; u++)
#pragma unroll
                for (int j = 0; j < CHAINS; j++) a[j] = fmaf(a[j], m, c);
#pragma unroll
        for (int j = 0; j < CHAINS; j++) acc += a[j];
    } else if (KIND == RIME_PIPE_FFMA2) {
        float2 a[CHAINS];
#pragma unroll
        for (int j = 0; j < CHAINS; j++) a[j] = make_float2(threadIdx.x * 1e-3f + j, j - threadIdx.x * 1e-3f);
        const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int u = 0; u < UNROLL; u++)
#pragma unroll
                for (int j = 0; j < CHAINS; j++) a[j] = __ffma2_rn(a[j], m2, c2);
#pragma unroll
        for (int j = 0; j < CHAINS; j++) acc += a[j].x + a[j].y;
    } else if (KIND == RIME_PIPE_DFMA) {
        double a[CHAINS];
#pragma unroll
        for (int j = 0; j < CHAINS; j++) a[j] = threadIdx.x * 1e-3 + j;
        const double md = m, cd = c;
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int u = 0; u < UNROLL; u++)
#pragma unroll
                for (int j = 0; j < CHAINS; j++) a[j] = fma(a[j], md, cd);
#pragma unroll
        for (int j = 0; j < CHAINS; j++) acc += (float)a[j];
    } else {
        float a[CHAINS];
#pragma unroll
        for (int j = 0; j < CHAINS; j++) a[j] = -1e-3f * (threadIdx.x + j);
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int u = 0; u < UNROLL; u++)
#pragma unroll
                for (int j = 0; j < CHAINS; j++) a[j] = ex2_approx(a[j]) - c;
#pragma unroll
        for (int j = 0; j < CHAINS; j++) acc += a[j];
    }
    if (acc == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;   // keeps the chains alive
}

template <int KIND>
static cudaError_t time_pipe(int nsm, float *d, double *rate) {
    const int blocks = nsm * 8;   // 64 warps per SM at most resident; 8 blocks of 8 warps
    int iters = 64;
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    float ms = 0.f;
    // grow the work until a launch takes at least 20 ms
    for (int round = 0; round < 20 && e == cudaSuccess; round++) {
        k_pipe<KIND><<<blocks, THREADS>>>(d, iters, 0.999f, 1e-3f);
        e = cudaEventRecord(a);
        if (e != cudaSuccess) break;
        k_pipe<KIND><<<blocks, THREADS>>>(d, iters, 0.999f, 1e-3f);
        e = cudaEventRecord(b);
        if (e != cudaSuccess) break;
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) break;
        e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess || ms >= 20.f) break;
        iters *= 2;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    const double lanes_per_op = KIND == RIME_PIPE_FFMA2 ? 2.0 : 1.0;
    const double ops = (double)blocks * THREADS * iters * UNROLL * CHAINS * lanes_per_op;
    *rate = ops / (ms * 1e-3);
    return cudaSuccess;
}

}  // namespace peaks
}  // namespace rime

extern "C" rime_status rime_pipe_rate(int32_t pipe, double *ops_per_s) {
    using namespace rime;
    if (!ops_per_s || pipe < RIME_PIPE_FFMA || pipe > RIME_PIPE_EX2) {
        set_global_error("rime_pipe_rate: unknown pipe or NULL output");
        return RIME_E_INVALID;
    }
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    float *d = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&d, (size_t)nsm * 8 * peaks::THREADS * sizeof(float));
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RIME_E_OOM : RIME_E_CUDA;
    }
    switch (pipe) {
        case RIME_PIPE_FFMA: e = peaks::time_pipe<RIME_PIPE_FFMA>(nsm, d, ops_per_s); break;
        case RIME_PIPE_FFMA2: e = peaks::time_pipe<RIME_PIPE_FFMA2>(nsm, d, ops_per_s); break;
        case RIME_PIPE_DFMA: e = peaks::time_pipe<RIME_PIPE_DFMA>(nsm, d, ops_per_s); break;
        default: e = peaks::time_pipe<RIME_PIPE_EX2>(nsm, d, ops_per_s); break;
    }
    cudaFree(d);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return RIME_E_CUDA;
    }
    return RIME_OK;
}
