// Throughput of the ALU pipes the path's rooflines divide by, measured on the device at hand:
// FP32 fused multiply-add (the expansions, the FP32-core near field), the special-function
// unit's base-2 logarithm (the tree-code's log |z - z_c| terms) and FP64 fused multiply-add
// (the FP64 path, the monopole and constant terms).  Each kernel keeps every SM full of
// warps that run independent dependency chains of the one instruction, so the pipe and not
// the chain latency sets the rate.  The paper has no counterpart: this is measurement
// support for the rooflines.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/pp.h"

namespace {

constexpr int kChains = 8;     // independent chains per thread
constexpr int kThreads = 256;  // threads per CTA
constexpr int kCtasPerSm = 8;  // 2048 threads per SM

// a <- a * m + b on kChains chains; m, b come from the host so nothing folds at compile time.
__global__ void __launch_bounds__(kThreads) k_peak_fma32(int iters, float m, float b, float* sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = float(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0f) sink[blockIdx.x * kThreads + threadIdx.x] = s;  // never taken; keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_peak_fma64(int iters, double m, double b, double* sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = double(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

// x <- lg2(x) + b: with b = 2 the chain sits at its fixed point x = 4.  The add runs on the
// FMA pipe, which is eight times wider than the special-function unit, so lg2 sets the rate.
__global__ void __launch_bounds__(kThreads) k_peak_lg2(int iters, float b, float* sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 4.0f + float(threadIdx.x + c) * 1e-6f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                float y;
                asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
                a[c] = y + b;
            }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int pp_measure_alu_peaks(double* out, int reps, void* stream) {
    if (!out || reps < 1 || reps > 1000) return PP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return PP_ERR_CUDA;
    const int grid = nsm * kCtasPerSm;
    // about 1-3 ms per launch at the expected rates: long enough that launch overhead is noise
    const int it32 = 2048, it64 = 64, itlg = 512;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return PP_ERR_CUDA;
    }
    int status = PP_OK;
    double best[3] = {1e30, 1e30, 1e30};
    for (int r = 0; r < reps + 1 && status == PP_OK; ++r) {  // the first round is a warm-up
        for (int k = 0; k < 3 && status == PP_OK; ++k) {
            if (cudaEventRecord(e0, st) != cudaSuccess) status = PP_ERR_CUDA;
            if (k == 0)
                k_peak_fma32<<<grid, kThreads, 0, st>>>(it32, 0.999999f, 1e-6f, nullptr);
            else if (k == 1)
                k_peak_lg2<<<grid, kThreads, 0, st>>>(itlg, 2.0f, nullptr);
            else
                k_peak_fma64<<<grid, kThreads, 0, st>>>(it64, 0.999999, 1e-6, nullptr);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess) {
                status = PP_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) status = PP_ERR_CUDA;
            if (r > 0) best[k] = std::min(best[k], double(ms));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != PP_OK) {
        cudaGetLastError();
        return status;
    }
    const double threads = double(grid) * kThreads;
    const double fma32 = threads * it32 * 8.0 * kChains, lg2 = threads * itlg * 4.0 * kChains,
                 fma64 = threads * it64 * 8.0 * kChains;
    out[0] = 2.0 * fma32 / (best[0] * 1e-3) / 1e12;  // FP32 TFLOP/s (2 per FMA)
    out[1] = lg2 / (best[1] * 1e-3) / 1e9;           // lg2 results, 1e9 per second
    out[2] = 2.0 * fma64 / (best[2] * 1e-3) / 1e12;  // FP64 TFLOP/s
    out[3] = best[0];
    out[4] = best[1];
    out[5] = best[2];
    out[6] = double(nsm);
    return PP_OK;
}
