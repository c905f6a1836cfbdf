// Measured arithmetic peaks of this GPU (no counterpart in the paper: these are
// the denominators of the roofline of the kernels that run on the FP32 and FP64
// pipes, the Jacobi SVD above all).
//
// Each kernel keeps every thread busy on independent chains of fused
// multiply-adds held in registers (no memory traffic in the loop), with enough
// chains per thread and warps per SM that the pipe, not the FMA latency, is the
// limit.  Three forms are timed: scalar FP32 (fma.rn.f32), packed FP32
// (fma.rn.f32x2: two lanes of FP32 arithmetic per instruction, the form the
// Jacobi rotations use) and FP64 (fma.rn.f64).  The result is the flop rate of
// one launch over CUDA events on the caller's stream, 2 flops per FMA lane.
#include <cstdint>

#include "ptebd_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_peak_f32(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long pk(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__global__ void __launch_bounds__(kThreads) k_peak_f32x2(float* out, int iters, float a, float b) {
    unsigned long long x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = pk((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x - k) * 1e-3f);
    const unsigned long long av = pk(a, a), bv = pk(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
        s += lo + hi;
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f64(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int ptebd_alu_peak(int32_t kind, int32_t iters, void* scratch, size_t scratch_bytes, void* stream,
                              double* tflops, double* ms) {
    if (kind < 0 || kind > 2 || iters < 1 || !scratch || !tflops) return PTEBD_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PTEBD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PTEBD_ERR_CUDA;
    // 8 blocks of 256 threads per SM: 64 warps, 16 per scheduler
    const int blocks = 8 * sms;
    const size_t need = (size_t)blocks * kThreads * sizeof(double);
    if (scratch_bytes < need) return PTEBD_ERR_MEMORY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto launch = [&](int it) {
        if (kind == 0)
            k_peak_f32<<<blocks, kThreads, 0, s>>>(static_cast<float*>(scratch), it, 0.999f, 1e-4f);
        else if (kind == 1)
            k_peak_f32x2<<<blocks, kThreads, 0, s>>>(static_cast<float*>(scratch), it, 0.999f, 1e-4f);
        else
            k_peak_f64<<<blocks, kThreads, 0, s>>>(static_cast<double*>(scratch), it, 0.999, 1e-4);
        return cudaGetLastError();
    };
    if (launch(1) != cudaSuccess) return PTEBD_ERR_CUDA;  // warm-up (module load, clocks)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PTEBD_ERR_CUDA;
    int rc = PTEBD_OK;
    float t = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess || launch(iters) != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        rc = PTEBD_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double lanes_per_fma = kind == 1 ? 2.0 : 1.0;
    const double flops = 2.0 * lanes_per_fma * (double)blocks * kThreads * (double)iters * kUnroll * kChains;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return PTEBD_OK;
}
