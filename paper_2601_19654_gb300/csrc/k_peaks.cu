// Measured ALU peaks of the device the kernels run on: FP32 FMA, FP64 FMA
// and MUFU reciprocal square root throughput, for the rooflines of the
// kick (FP32 pipe; FP64 pipe in the FP64 form) and of the encounter
// integrator (FP64 pipe).  Each kernel runs CH independent chains a thread
// over a fixed trip count on 8 blocks of 256 threads an SM, so the pipes,
// not the dependences, set the rate; the result is kept behind a test the
// compiler cannot resolve, so no work is removed.
#include "opal_internal.cuh"
#include "../../include/opal_testing.h"

namespace opal {

constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(256) k_peak_ffma(float* out, int iters, float a, float b) {
    float r[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) r[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kPeakChains; c++) r[c] = fmaf(r[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) s += r[c];
    if (s == 12345.0f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(double* out, int iters, double a, double b) {
    double r[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) r[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kPeakChains; c++) r[c] = fma(r[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) s += r[c];
    if (s == 12345.0) out[0] = s;
}

// one MUFU rsqrt and one FADD a step of each chain
__global__ void __launch_bounds__(256) k_peak_mufu(float* out, int iters) {
    float r[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) r[c] = 1.0f + threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kPeakChains; c++) {
            float y;
            asm volatile("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(r[c]));
            r[c] = y + 1.0f;
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) s += r[c];
    if (s == 12345.0f) out[0] = s;
}

}  // namespace opal

using namespace opal;

extern "C" opal_status opal_probe_alu_peaks(double out[3]) {
    if (!out) return OPAL_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OPAL_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return OPAL_ECUDA;
    void* buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) return OPAL_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const dim3 grid((unsigned)(nsm * 8)), block(256);
    const double threads = (double)grid.x * block.x;
    // each measurement: one launch to warm up, then one timed
    auto timed = [&](auto launch) -> double {
        launch();
        cudaEventRecord(e0, 0);
        launch();
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const int it32 = 20000, it64 = 2000, itmu = 20000;
    const double ms32 = timed([&] { k_peak_ffma<<<grid, block>>>((float*)buf, it32, 1.0001f, 0.5f); });
    const double ms64 = timed([&] { k_peak_dfma<<<grid, block>>>((double*)buf, it64, 1.0001, 0.5); });
    const double msmu = timed([&] { k_peak_mufu<<<grid, block>>>((float*)buf, itmu); });
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess || ms32 <= 0 || ms64 <= 0 || msmu <= 0) return OPAL_ECUDA;
    out[0] = 2.0 * threads * it32 * kPeakChains / (ms32 * 1e-3) / 1e12;   // FP32 TFLOP/s (FMA = 2)
    out[1] = 2.0 * threads * it64 * kPeakChains / (ms64 * 1e-3) / 1e12;   // FP64 TFLOP/s
    out[2] = threads * itmu * kPeakChains / (msmu * 1e-3) / 1e12;         // MUFU rsqrt, Tops/s
    return OPAL_OK;
}
