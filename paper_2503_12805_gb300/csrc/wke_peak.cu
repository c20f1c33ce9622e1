// Arithmetic-throughput probes: the FP32 and FP64 fused multiply-add rates of
// the current device, measured with register-resident FMA chains.  These give
// the ALU roofs the collision kernels are reported against; they are a
// measurement service of the library (the paper has no counterpart).
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "wke_internal.h"

namespace {

constexpr int kChains = 8;          // independent chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pk(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

// FP32, packed: every instruction is two multiply-adds (4 flops).
__global__ void __launch_bounds__(kThreads) k_fma32x2(float *out, int iters, float a, float b) {
    unsigned long long x[kChains];
    const float s = 1e-7f * (float)threadIdx.x;
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = pk(s + (float)i, s - (float)i);
    const unsigned long long A = pk(a, a), B = pk(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma2(x[i], A, B);
    }
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float2 v = upk(x[i]);
        acc += v.x + v.y;
    }
    if (acc == -1.2345f) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;   // keeps the chains live
}

// FP32, scalar: every instruction is one multiply-add (2 flops).
__global__ void __launch_bounds__(kThreads) k_fma32(float *out, int iters, float a, float b) {
    float x[2 * kChains];
    const float s = 1e-7f * (float)threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) x[i] = s + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 2 * kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 2 * kChains; ++i) acc += x[i];
    if (acc == -1.2345f) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_fma64(double *out, int iters, double a, double b) {
    double x[kChains];
    const double s = 1e-9 * (double)threadIdx.x;
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = s + (double)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i];
    if (acc == -1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

int cuda_fail(cudaError_t e, const char *what) {
    return wke::fail(WKE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" int wke_alu_peak(int precision, int reps, double *tflops, double *best_ms) {
    if (!tflops || (precision != WKE_FP32 && precision != WKE_FP64) || reps < 1 || reps > 1000)
        return wke::fail(WKE_ERR_INVALID, "wke_alu_peak: precision must be WKE_FP32 or WKE_FP64, reps in [1, 1000]");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "wke_alu_peak: device query");
    const int blocks = sms * kBlocksPerSm;
    void *out = nullptr;
    if ((e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(double))) != cudaSuccess) {
        cudaGetLastError();
        return wke::fail(WKE_ERR_OOM, "wke_alu_peak: scratch allocation failed");
    }
    cudaStream_t s = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    double best = 0.0, best_t = 0.0;
    int rc = WKE_OK;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
        rc = cuda_fail(e, "wke_alu_peak: stream/event creation");
    }
    // variant 0: packed FP32 (4 flops per instruction), 1: scalar FP32, 2: FP64
    const int first = precision == WKE_FP32 ? 0 : 2, last = precision == WKE_FP32 ? 1 : 2;
    for (int v = first; v <= last && rc == WKE_OK; ++v) {
        const int iters = v == 2 ? 2048 : 32768;
        const double flops = (double)blocks * kThreads * iters * kChains * (v == 2 ? 2.0 : 4.0);
        for (int r = -1; r < reps && rc == WKE_OK; ++r) {   // r = -1: warm-up
            cudaEventRecord(t0, s);
            if (v == 0) k_fma32x2<<<blocks, kThreads, 0, s>>>(static_cast<float *>(out), iters, 0.999f, 1e-3f);
            else if (v == 1) k_fma32<<<blocks, kThreads, 0, s>>>(static_cast<float *>(out), iters, 0.999f, 1e-3f);
            else k_fma64<<<blocks, kThreads, 0, s>>>(static_cast<double *>(out), iters, 0.999, 1e-3);
            cudaEventRecord(t1, s);
            if ((e = cudaEventSynchronize(t1)) != cudaSuccess) {
                rc = cuda_fail(e, "wke_alu_peak: probe kernel");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, t0, t1);
            if (r >= 0 && ms > 0.0f && flops / (ms * 1e-3) / 1e12 > best) {
                best = flops / (ms * 1e-3) / 1e12;
                best_t = ms;
            }
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    if (rc != WKE_OK) return rc;
    *tflops = best;
    if (best_ms) *best_ms = best_t;
    return WKE_OK;
}
