// Floating-point issue-rate probe: the peak the roofline of the pair
// kernels divides by.  Every thread runs NCH independent chains of fused
// multiply-adds (enough independent work to hide the pipeline latency), so
// the launch is bound by the FMA units alone; flops = 2 x FMAs.  Three
// forms: scalar FP32, packed FP32 (two lanes per instruction, the form the
// density pass uses) and FP64.
#include <cuda_runtime.h>

#include "pta.h"

namespace {

constexpr int NCH = 16;
constexpr int PEAK_TPB = 256;

__global__ void __launch_bounds__(PEAK_TPB) k_fma_f32(long long iters, float a, float b,
                                                      float *out) {
    float x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    if (s == 1234.5678f) out[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(PEAK_TPB) k_fma_f32x2(long long iters, float a, float b,
                                                        float *out) {
    float2 x[NCH / 2];
#pragma unroll
    for (int c = 0; c < NCH / 2; ++c)
        x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)(threadIdx.x - c) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCH / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NCH / 2; ++c) s += x[c].x + x[c].y;
    if (s == 1234.5678f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_TPB) k_fma_f64(long long iters, double a, double b,
                                                      float *out) {
    double x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    if (s == 1234.5678) out[blockIdx.x] = (float)s;
}

}  // namespace

extern "C" int pta_measure_fma_rate(int kind, int64_t iters, void *stream, double *flops,
                                    double *ms) {
    if (kind < 0 || kind > 2 || iters < 1 || !flops || !ms) return PTA_EINVAL;
    int dev = 0, nsm = 0, per_sm = 0;
    const void *fn = kind == 0 ? (const void *)k_fma_f32
                               : (kind == 1 ? (const void *)k_fma_f32x2 : (const void *)k_fma_f64);
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PEAK_TPB, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return PTA_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // exactly one wave of resident blocks: every SM full, no tail
    const int blocks = nsm * per_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return PTA_ECUDA;
    }
    cudaEventRecord(e0, st);
    if (kind == 0)
        k_fma_f32<<<blocks, PEAK_TPB, 0, st>>>(iters, 0.999999f, 1e-7f, nullptr);
    else if (kind == 1)
        k_fma_f32x2<<<blocks, PEAK_TPB, 0, st>>>(iters, 0.999999f, 1e-7f, nullptr);
    else
        k_fma_f64<<<blocks, PEAK_TPB, 0, st>>>(iters, 0.999999, 1e-7, nullptr);
    cudaEventRecord(e1, st);
    float t = 0.f;
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return PTA_ECUDA;
    *flops = 2.0 * (double)blocks * PEAK_TPB * (double)iters * NCH;
    *ms = t;
    return PTA_OK;
}
