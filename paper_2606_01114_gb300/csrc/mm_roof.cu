// Measured arithmetic roofs for the paths that are bound by an ALU rather
// than by HBM: the native FP64 demag passes (GB300's FP64 units) and the
// float-float passes (the FP32 pipes).
//
// Each kernel runs kChains independent FMA chains per thread over a grid of
// 8 blocks per SM, so the pipe, not the FMA latency, sets the rate; the
// chain results are written out so that nothing is folded away.  Kinds:
//   MM_ROOF_FP64    fma.rn.f64                 (2 flops per instruction)
//   MM_ROOF_FP32    fma.rn.f32                 (2 flops per instruction)
//   MM_ROOF_FP32X2  fma.rn.f32x2 on lane pairs (4 flops per instruction)
// mm_alu_peak allocates its output buffer and events per call: it is an
// instrumentation call, not part of the hot path.
#include "mm_internal.cuh"

namespace mm {
namespace {

constexpr int kChains = 8;
constexpr int kRoofThreads = 256;

__global__ void __launch_bounds__(kRoofThreads) k_roof_fp64(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kRoofThreads) k_roof_fp32(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long x, unsigned long long a,
                                                       unsigned long long b) {
    unsigned long long r;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

__global__ void __launch_bounds__(kRoofThreads) k_roof_fp32x2(float* out, int iters, float a, float b) {
    unsigned long long x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = pack2(1e-3f * (threadIdx.x + c), 2e-3f * (threadIdx.x + c));
    const unsigned long long a2 = pack2(a, a), b2 = pack2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma_f32x2(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += __uint_as_float((unsigned)x[c]) + __uint_as_float((unsigned)(x[c] >> 32));
    out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" int mm_alu_peak(int kind, double* flops_per_s, void* stream) {
    if (!flops_per_s) return fail(nullptr, MM_ERR_INVALID_ARG, "mm_alu_peak: flops_per_s is NULL");
    if (kind != MM_ROOF_FP64 && kind != MM_ROOF_FP32 && kind != MM_ROOF_FP32X2)
        return fail(nullptr, MM_ERR_INVALID_ARG, "mm_alu_peak: bad kind %d", kind);
    cudaStream_t st = (cudaStream_t)stream;
    int caller_dev = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&caller_dev);
    dev = caller_dev;
    if (e == cudaSuccess && st) e = cudaStreamGetDevice(st, &dev);
    if (e == cudaSuccess && dev != caller_dev) e = cudaSetDevice(dev);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, MM_ERR_CUDA, "mm_alu_peak: %s", cudaGetErrorString(e));
    }
    const int blocks = 8 * sms;
    // about 10 ms per launch at the nominal rates
    const int iters = kind == MM_ROOF_FP64 ? 4096 : 65536;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best_ms = 0.f;
    e = cudaMalloc(&out, (size_t)blocks * kRoofThreads * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up, the best of the rest counts
        e = cudaEventRecord(e0, st);
        if (kind == MM_ROOF_FP64)
            k_roof_fp64<<<blocks, kRoofThreads, 0, st>>>((double*)out, iters, 0.999999, 1e-7);
        else if (kind == MM_ROOF_FP32)
            k_roof_fp32<<<blocks, kRoofThreads, 0, st>>>((float*)out, iters, 0.9999f, 1e-4f);
        else
            k_roof_fp32x2<<<blocks, kRoofThreads, 0, st>>>((float*)out, iters, 0.9999f, 1e-4f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (dev != caller_dev) cudaSetDevice(caller_dev);
    if (e != cudaSuccess || !(best_ms > 0.f)) {
        cudaGetLastError();
        return fail(nullptr, MM_ERR_CUDA, "mm_alu_peak: %s", cudaGetErrorString(e));
    }
    const double flops_per_fma = kind == MM_ROOF_FP32X2 ? 4.0 : 2.0;
    const double fmas = (double)blocks * kRoofThreads * kChains * (double)iters;
    *flops_per_s = fmas * flops_per_fma / (best_ms * 1e-3);
    return MM_OK;
}
