// FP32 FMA throughput microbenchmark (the measured counterpart of the derived
// FP32 peak used for the shift-and-add roofline: SMs x 128 lanes x 2 flop x
// clock).  Every thread runs 8 independent FMA chains (scalar FFMA or packed
// FFMA2) for `iters` iterations on register operands; the result is stored
// so the chains are live.  Timed with CUDA events on the caller's stream.
#include <algorithm>

#include "ppm_internal.cuh"

namespace ppm {
namespace {

constexpr int kChains = 8;

template <bool PAIRED>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float seed, float *out)
{
    const float a = 1.0f + 1e-7f * (float)threadIdx.x, b = 1e-7f * seed;
    if (PAIRED) {
        float2 v[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = make_float2(seed + c, seed - c);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], a2, b2);
        }
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
        if (s == 1.2345f) out[blockIdx.x] = s;  // keeps the chains live
    } else {
        float v[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = seed + c;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
        }
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += v[c];
        if (s == 1.2345f) out[blockIdx.x] = s;
    }
}

}  // namespace
}  // namespace ppm

using namespace ppm;

extern "C" ppm_status ppm_fp32_peak(int device, int paired, void *stream, double *tflops)
{
    if (!tflops || (paired != 0 && paired != 1)) return PPM_EINVAL;
    *tflops = 0.0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return PPM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    ppm_status s = PPM_OK;
    int sms = 0;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&out, 4096 * sizeof(float)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        s = PPM_ECUDA;
    } else {
        const int blocks = std::min(sms * 8, 4096), iters = 1 << 14;
        auto launch = [&]() {
            if (paired) k_fma_peak<true><<<blocks, 256, 0, st>>>(iters, 0.5f, out);
            else k_fma_peak<false><<<blocks, 256, 0, st>>>(iters, 0.5f, out);
        };
        launch();  // warm-up
        cudaEventRecord(e0, st);
        const int reps = 5;
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, st);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess) {
            s = PPM_ECUDA;
        } else {
            const double fma = (double)reps * blocks * 256.0 * iters * kChains * (paired ? 2 : 1);
            *tflops = 2.0 * fma / (ms * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (prev >= 0) cudaSetDevice(prev);
    return s;
}
