// FMA-rate microbenchmark (no counterpart in the paper): the FP32 and FP64
// fused multiply-add issue rates of the device, measured with chains of
// independent FMAs in every thread of a grid that fills every SM.  The mixed
// and FP64 steps are bound by these pipes rather than by HBM, so their
// rooflines are stated against these rates beside the derived peaks.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tlsph.h"

namespace {

constexpr int CHAINS = 8;      // independent accumulators per thread (covers the FMA latency)
constexpr int INNER = 64;      // FMAs per chain per outer iteration

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T *sink, int write)
{
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < INNER; ++k)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (write) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename T>
int run(int iters, double *fma_per_s)
{
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_chains<T>, 256, 0);
    if (e != cudaSuccess || sms <= 0 || per <= 0) return TLSPH_ERR_CUDA;
    const int grid = sms * per;
    T *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TLSPH_ERR_CUDA;
    if (cudaMalloc(&sink, (size_t)grid * 256 * sizeof(T)) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        // (T)0.999 and (T)1e-3 keep the chains finite for any iteration count
        k_fma_chains<T><<<grid, 256, 0, st>>>(iters / 4 + 1, (T)0.999, (T)1e-3, sink, 1);   // warm-up
        cudaEventRecord(e0, st);
        k_fma_chains<T><<<grid, 256, 0, st>>>(iters, (T)0.999, (T)1e-3, sink, 1);
        cudaEventRecord(e1, st);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0) {
            const double fmas = (double)grid * 256 * (double)iters * INNER * CHAINS;
            *fma_per_s = fmas / (ms * 1e-3);
            rc = TLSPH_OK;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    return rc;
}

}  // namespace

extern "C" int tlsph_fma_peak(int fp64, int iters, double *fma_per_s)
{
    if (!fma_per_s || iters <= 0 || iters > (1 << 20)) return TLSPH_ERR_ARG;
    *fma_per_s = 0.0;
    return fp64 ? run<double>(iters, fma_per_s) : run<float>(iters, fma_per_s);
}
