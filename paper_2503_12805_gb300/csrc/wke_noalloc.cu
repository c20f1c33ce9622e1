// Mass, momentum and energy of a grid without any memory allocation.
//
// wke_moments works through a plan, and creating a plan allocates device
// memory.  Some callers cannot do that where they need these sums: code
// that runs inside a memory budget owned by another allocator (a framework
// pool, a fixed arena), or code that must not allocate while a CUDA stream
// capture is open.  wke_moments_noalloc serves them: it takes only the grid
// and an output slot from the caller and keeps its per-block partial sums in
// a fixed array compiled into the library's device image, so no call to
// cudaMalloc, cudaFree or any allocating routine is made.
//
// The array is shared by every call in the process on a given device and
// keeps whatever the last call left there; each call overwrites the slots it
// reads before reading them.  Calls whose kernels overlap on the GPU (on
// different streams without ordering) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "wke_internal.h"

namespace {

constexpr int kMaxBlocks = 1024;          // partial-sum slots per moment
constexpr int kMaxMoments = 5;            // d + 2 with d <= 3
constexpr int kThreads = 256;
constexpr int kPointsPerBlock = 4096;     // each block sums this many points
constexpr long long kMaxPoints = (long long)kMaxBlocks * kPointsPerBlock;
constexpr int kMaxDevices = 64;

// 40 KiB of partial sums; held by every GPU that loads the library until the
// process exits.
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks * kMaxMoments];

std::mutex g_addr_mutex;
double *g_addr[kMaxDevices] = {nullptr};

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_moments_partials_static(const T *__restrict__ g, int d, int N, double L, long long nd, double *__restrict__ part) {
    const double h = 2.0 * L / N;
    double acc[kMaxMoments] = {0, 0, 0, 0, 0};
    const long long lo = (long long)blockIdx.x * kPointsPerBlock;
    const long long hi = lo + kPointsPerBlock < nd ? lo + kPointsPerBlock : nd;
    for (long long i = lo + threadIdx.x; i < hi; i += kThreads) {
        const double v = (double)g[i];
        long long rest = i;
        double k2 = 0.0;
        double kk[3] = {0, 0, 0};
        for (int a = d - 1; a >= 0; --a) {
            const double ka = -L + (double)(rest % N) * h;
            rest /= N;
            kk[a] = ka;
            k2 += ka * ka;
        }
        acc[0] += v;
        for (int a = 0; a < d; ++a) acc[1 + a] += kk[a] * v;
        acc[d + 1] += k2 * v;
    }
    __shared__ double red[kMaxMoments][kThreads];
    for (int k = 0; k < d + 2; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < d + 2; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < d + 2; ++k) part[blockIdx.x * (d + 2) + k] = red[k][0];
}

__global__ void k_moments_reduce_static(const double *__restrict__ part, int nblocks, int K, double hd,
                                        double *__restrict__ out) {
    const int k = threadIdx.x;
    if (k < K) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[b * K + k];
        out[k] = hd * s;
    }
}

// Device address of the partial-sum array on the current device.  Outside a
// stream capture it is resolved on every call (a device reset reloads the
// library's device image, which may move the array); inside a capture the
// address resolved by the last call outside one is used.
int scratch_address(cudaStream_t s, double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return wke::fail(WKE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return wke::fail(WKE_ERR_UNSUPPORTED, "device ordinal above 63");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess)
        return wke::fail(WKE_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cs == cudaStreamCaptureStatusNone || !g_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess || !ptr)
            return wke::fail(WKE_ERR_CUDA, std::string("cudaGetSymbolAddress of the moment scratch: ") +
                                               cudaGetErrorString(e));
        g_addr[dev] = static_cast<double *>(ptr);
    }
    *out = g_addr[dev];
    return WKE_OK;
}

}  // namespace

extern "C" int wke_moments_noalloc(int d, int N, double L, int precision, const void *g_dev, double *out_dev,
                                   void *stream) {
    if (!g_dev || !out_dev) return wke::fail(WKE_ERR_INVALID, "g and out must be non-NULL");
    if (d != 2 && d != 3) return wke::fail(WKE_ERR_INVALID, "d must be 2 or 3");
    if (N < 1 || !(L > 0.0) || !std::isfinite(L)) return wke::fail(WKE_ERR_INVALID, "need N >= 1 and L > 0");
    if (precision != WKE_FP64 && precision != WKE_FP32)
        return wke::fail(WKE_ERR_INVALID, "precision must be WKE_FP64 or WKE_FP32");
    long long nd = 1;
    for (int a = 0; a < d; ++a) {
        nd *= N;
        if (nd > kMaxPoints) break;
    }
    if (nd > kMaxPoints)
        return wke::fail(WKE_ERR_INVALID, "grid has more than " + std::to_string(kMaxPoints) +
                                              " points, the most the fixed moment scratch can reduce");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *part = nullptr;
    int rc = scratch_address(s, &part);
    if (rc) return rc;
    const int nblocks = (int)((nd + kPointsPerBlock - 1) / kPointsPerBlock);
    if (precision == WKE_FP64)
        k_moments_partials_static<double><<<nblocks, kThreads, 0, s>>>(static_cast<const double *>(g_dev), d, N, L,
                                                                        nd, part);
    else
        k_moments_partials_static<float><<<nblocks, kThreads, 0, s>>>(static_cast<const float *>(g_dev), d, N, L,
                                                                       nd, part);
    const double h = 2.0 * L / N;
    const double hd = d == 2 ? h * h : h * h * h;
    k_moments_reduce_static<<<1, 32, 0, s>>>(part, nblocks, d + 2, hd, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wke::fail(WKE_ERR_CUDA, std::string("moment launch: ") + cudaGetErrorString(e));
    return WKE_OK;
}
