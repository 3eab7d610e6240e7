// Diagnostic: the FP32 CUDA-core peak of the current device, measured (fdas_measure_fp32_peak).
//
// The FP32 convolution is bound by FP32 arithmetic issue, so its roofline needs the rate at which
// this GPU retires FFMAs, at the clocks and power state it actually runs. The kernel keeps every
// FP32 lane busy with independent dependent-FFMA chains: 8 chains per thread hide the FMA latency,
// and 1024 threads per SM (8 warps per scheduler) fill the issue slots. Each FFMA counts 2 flop.
#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;
constexpr int kChains = 8;
constexpr int kUnroll = 64;  // FFMAs per chain per loop iteration

// x <- x * a + b along 8 chains for `iters` iterations. a and b are kernel parameters close to 1 and
// 0, so the values stay finite and the compiler cannot fold the chains; one store of their sum,
// behind a flag that is never set, keeps the work live.
__global__ void __launch_bounds__(kPeakThreads)
    fdas_ffma_peak(int iters, float a, float b, int write, float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (write) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t measure_fp32_peak(float ms, double *tflops, float *elapsed_ms) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = sms * kPeakCtasPerSm;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    // Two short launches size the loop for the requested duration (the second one corrects for the
    // launch overhead in the first); the second also brings the clocks up; then the timed launch.
    int iters = 64;
    float t = 0.0f;
    for (int pass = 0; pass < 4 && e == cudaSuccess; ++pass) {
        if (pass == 1 || pass == 2) {
            // At most 1000x per step and 2^21 iterations in all (about 4 s on a GB300), whatever
            // the first timings say.
            double scale = t > 0.0f ? ms / t : 1000.0;
            scale = scale < 1000.0 ? scale : 1000.0;
            const double want = iters * scale;
            iters = want > 1.0 ? (want < 2097152.0 ? (int)want : 2097152) : 1;
        }
        e = cudaEventRecord(a, 0);
        if (e == cudaSuccess) {
            fdas_ffma_peak<<<grid, kPeakThreads>>>(iters, 1.0000001f, 1e-7f, 0, nullptr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    const double ffma = (double)grid * kPeakThreads * (double)iters * kUnroll * kChains;
    *tflops = 2.0 * ffma / (t * 1e-3) / 1e12;
    *elapsed_ms = t;
    return cudaSuccess;
}

}  // namespace fdas
