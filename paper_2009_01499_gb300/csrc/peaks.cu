// peaks.cu -- throughput of the GPU's FMA pipes, measured with dependent-free FMA loops:
// the denominators of the benchmark's ALU rooflines (FP64 for the FP64 form's kernels,
// FP32 for the mixed form's inner cycle).  Not part of the solver.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace iga2l {
namespace {

constexpr int kPeakIters = 4096;
constexpr int kPeakChains = 8;   // independent accumulators per thread

__global__ void k_peak_f64(double *out, double a, double b)
{
    double x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = threadIdx.x * 1e-9 + c;
    for (int i = 0; i < kPeakIters; ++i)
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    if (s == 1.2345) out[0] = s;   // never true for these inputs; keeps the loop alive
}

__global__ void k_peak_f32(float *out, float a, float b)
{
    float x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = threadIdx.x * 1e-7f + c;
    for (int i = 0; i < kPeakIters; ++i)
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    if (s == 1.2345f) out[0] = s;
}

__global__ void k_peak_f32x2(float *out, float a, float b)
{
    float2 x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = make_float2(threadIdx.x * 1e-7f + c, c + 0.5f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < kPeakIters; ++i)
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c].x + x[c].y;
    if (s == 1.2345f) out[0] = s;
}

}  // namespace
}  // namespace iga2l

extern "C" int iga2l_fma_peak(int kind, double *gflops, void *stream)
{
    using namespace iga2l;
    if (!gflops || kind < 0 || kind > 2) {
        set_last_error("fma_peak: kind must be 0 (FP64), 1 (FP32) or 2 (packed FP32 pairs)");
        return IGA2L_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    void *buf = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, 16);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 1e30f;
    const int threads = 256, blocks = nsm * 8;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (kind == 0) k_peak_f64<<<blocks, threads, 0, st>>>(static_cast<double *>(buf), 0.999999, 1e-9);
        else if (kind == 1) k_peak_f32<<<blocks, threads, 0, st>>>(static_cast<float *>(buf), 0.9999f, 1e-7f);
        else k_peak_f32x2<<<blocks, threads, 0, st>>>(static_cast<float *>(buf), 0.9999f, 1e-7f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;   // first run warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) {
        set_last_error(std::string("fma_peak: ") + cudaGetErrorString(e));
        return IGA2L_ERR_CUDA;
    }
    const double lanes = kind == 2 ? 2.0 : 1.0;
    const double flops = 2.0 * lanes * kPeakIters * kPeakChains * (double)threads * blocks;
    *gflops = flops / (best_ms * 1e-3) / 1e9;
    return IGA2L_OK;
}
