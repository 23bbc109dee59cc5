// fresco_smem_peak: measured throughput of the two shared-memory operations that bound the
// spread (32-bit integer atomic adds) and the kernel-derivative interpolation (32-bit loads) on
// the current device, for the roofline denominators of the benchmark.
//
// Each of 8 blocks per SM (256 threads, 32 KB of shared memory each) issues a fixed number of
// operations in which the 32 lanes of a warp always address 32 distinct banks (lane-consecutive
// words), the best case of the pipe: one wavefront per warp instruction. The kernel is launched
// a few times untimed, then timed with CUDA events on the caller's stream; the rate is operations
// (lanes) per second.
#include <cuda_runtime.h>

#include <cstdint>

#include "fresco.h"

namespace {

constexpr int kWords = 8192;     // 32 KB of shared memory per block
constexpr int kIters = 256;      // loop trips per thread
constexpr int kPerIter = 32;     // operations per trip

__global__ void __launch_bounds__(256) k_probe_atomics(int *sink) {
    __shared__ int s[kWords];
    for (int i = threadIdx.x; i < kWords; i += blockDim.x) s[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *base = s + warp * 1024 + lane;
#pragma unroll 1
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kPerIter; ++k) atomicAdd(base + k * 32, it + k);
    }
    __syncthreads();
    if (s[threadIdx.x] == 0x7fffffff) sink[blockIdx.x] = 1;   // never true; keeps the adds
}

__global__ void __launch_bounds__(256) k_probe_loads(int *sink) {
    __shared__ float s[kWords];
    for (int i = threadIdx.x; i < kWords; i += blockDim.x) s[i] = (float)(i & 7);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const volatile float *base = s + warp * 1024 + lane;
    float acc = 0.f;
#pragma unroll 1
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kPerIter; ++k) acc += base[k * 32];
    }
    if (acc == -1.f) sink[blockIdx.x] = 1;   // never true; keeps the loads
}

}  // namespace

extern "C" fresco_status fresco_smem_peak(int op, void *d_sink, void *stream,
                                          double *ops_per_s) {
    if ((op != FRESCO_SMEM_ATOMIC_ADD && op != FRESCO_SMEM_LOAD) || !d_sink || !ops_per_s)
        return FRESCO_ERR_ARG;
    cudaGetLastError();
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FRESCO_ERR_CUDA;
    const int blocks = sms * 8;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *sink = static_cast<int *>(d_sink);
    auto launch = [&]() {
        if (op == FRESCO_SMEM_ATOMIC_ADD) k_probe_atomics<<<blocks, 256, 0, s>>>(sink);
        else k_probe_loads<<<blocks, 256, 0, s>>>(sink);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FRESCO_ERR_CUDA;
    }
    for (int i = 0; i < 3; ++i) launch();
    const int reps = 10;
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i) launch();
    cudaEventRecord(e1, s);
    float ms = 0.f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                    cudaGetLastError() == cudaSuccess && ms > 0.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return FRESCO_ERR_CUDA;
    const double ops = (double)reps * blocks * 256.0 * kIters * kPerIter;
    *ops_per_s = ops / (ms * 1e-3);
    return FRESCO_OK;
}
