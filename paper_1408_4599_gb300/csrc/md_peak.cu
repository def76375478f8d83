// md_peak.cu -- md_fp32_peak: the measured FP32 FMA throughput of the GPU,
// the denominator of the force kernel's FP32 roofline beside the unit-count
// figure (SMs x 128 FP32 lanes x 2 FLOP x clock).
//
// Every thread runs eight independent FMA chains (enough independent work
// to cover the FMA latency at full occupancy), as scalar fma.rn.f32 or as
// the paired fma.rn.f32x2 of sm_100-class GPUs (two FMAs per instruction on
// a register pair).  The chains converge to a fixed point (x <- a x + b with
// |a| < 1), so no value overflows or becomes subnormal; a store that never
// happens in practice keeps the compiler from removing the chains.
#include <cuda_runtime.h>

#include "../../include/md.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_UNROLL = 16;  // FMA rounds per loop iteration

template <bool PAIRED>
__global__ void __launch_bounds__(PK_THREADS) k_fma_peak(float *sink, int iters, float a, float b)
{
    const float s = (float)(threadIdx.x + blockIdx.x) * 1.0e-3f;
    float t = 0.f;
    if constexpr (PAIRED) {
        float2 x[4];
#pragma unroll
        for (int k = 0; k < 4; k++) x[k] = make_float2(s + (float)k, s - (float)k);
        const float2 A = make_float2(a, a), B = make_float2(b, b);
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < PK_UNROLL; u++)
#pragma unroll
                for (int k = 0; k < 4; k++) x[k] = __ffma2_rn(x[k], A, B);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) t += x[k].x + x[k].y;
    } else {
        float x[8];
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = s + (float)k;
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < PK_UNROLL; u++)
#pragma unroll
                for (int k = 0; k < 8; k++) x[k] = fmaf(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) t += x[k];
    }
    if (t == -1.0f) sink[blockIdx.x * PK_THREADS + threadIdx.x] = t;  // never true: chains stay positive
}

}  // namespace

extern "C" md_status md_fp32_peak(int32_t paired, double *out, void *cuda_stream)
{
    if (!out || (paired != 0 && paired != 1)) return MD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MD_ERR_CUDA;
    const void *fn = paired ? (const void *)k_fma_peak<true> : (const void *)k_fma_peak<false>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PK_THREADS, 0) != cudaSuccess || per_sm < 1)
        return MD_ERR_CUDA;
    const int blocks = sms * per_sm;
    float *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * (size_t)blocks * PK_THREADS) != cudaSuccess) return MD_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    md_status rc = MD_OK;
    // ~5 ms per launch at the nominal rate
    int iters = 4096;
    float a = 0.99999f, b = 0.5f;
    float best = 1e30f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MD_ERR_CUDA;
    } else {
        for (int rep = 0; rep < 4 && rc == MD_OK; rep++) {  // the first launch is a warm-up
            void *args[] = {&sink, &iters, &a, &b};
            if (cudaEventRecord(e0, st) != cudaSuccess ||
                cudaLaunchKernel(fn, dim3(blocks), dim3(PK_THREADS), args, 0, st) != cudaSuccess ||
                cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = MD_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = MD_ERR_CUDA;
            if (rep > 0 && ms < best) best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != MD_OK) return rc;
    const double fmas = 8.0 * PK_UNROLL * (double)iters * (double)blocks * PK_THREADS;
    out[0] = 2.0 * fmas / (best * 1e-3);
    out[1] = best;
    return MD_OK;
}
