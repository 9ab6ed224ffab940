// cm_probe.cu -- measured arithmetic throughput (roofline denominators).
//
// The sweep kernels are bound by FP32 and MUFU instruction issue, not by
// memory, so their roofline needs the GPU's arithmetic rates.  Two fixed-work
// kernels measure them: eight independent dependency chains per thread (one
// FFMA, or one rsqrtf, per step) on 8 CTAs of 256 threads per SM, timed with
// CUDA events after a warm-up launch.  rsqrtf is the instruction the sweep
// kernels use; with -ftz=true it is one MUFU operation.
#include <cuda_runtime.h>

#include "../../include/cm.h"

namespace cm {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 8;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) probe_fma_kernel(int iters, float a, float b,
                                                                  float* sink) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = 1e-3f * threadIdx.x + (float)i;
#pragma unroll 16
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
    if (s == -1.0f) sink[0] = s;   // never true: keeps the chains live
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_rsqrt_kernel(int iters, float* sink) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = 1.5f + 1e-3f * threadIdx.x + (float)i;
    // x -> x^(-1/2) -> x^(1/4) ...: every value stays near 1
#pragma unroll 16
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = rsqrtf(x[i]);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
    if (s == -1.0f) sink[0] = s;
}

// Operations per second of one probe kernel (the second of two launches).
template <class Launch>
static cudaError_t probe_rate(Launch launch, double ops, cudaStream_t st, double* rate) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch();   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) *rate = ops / (1e-3 * (double)ms);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace cm

extern "C" int cm_probe_alu(int device, double* fma_per_s, double* rsqrt_per_s, void* stream) {
    if (!fma_per_s || !rsqrt_per_s || device < 0) return CM_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return CM_ERR_CUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        nsm < 1)
        return CM_ERR_CUDA;
    float* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return CM_ERR_OOM;
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 grid(nsm * cm::PROBE_CTAS_PER_SM), block(cm::PROBE_THREADS);
    const double threads = (double)grid.x * block.x;
    const int fma_iters = 1 << 17, rsqrt_iters = 1 << 14;
    cudaError_t e = cm::probe_rate(
        [&] {
            cm::probe_fma_kernel<<<grid, block, 0, st>>>(fma_iters, 0.999f, 1e-3f, sink);
            return cudaGetLastError();
        },
        threads * fma_iters * cm::PROBE_CHAINS, st, fma_per_s);
    if (e == cudaSuccess)
        e = cm::probe_rate(
            [&] {
                cm::probe_rsqrt_kernel<<<grid, block, 0, st>>>(rsqrt_iters, sink);
                return cudaGetLastError();
            },
            threads * rsqrt_iters * cm::PROBE_CHAINS, st, rsqrt_per_s);
    cudaFree(sink);
    return e == cudaSuccess ? CM_OK : CM_ERR_CUDA;
}
