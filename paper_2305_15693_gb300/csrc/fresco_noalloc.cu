// fresco_loss_noalloc: the structure-factor loss sum_q W_q (S_q - S0_q)^2 over caller-provided
// device arrays, computed without allocating any memory.
//
// It sums like the plan's loss reduction (per-block FP64 partial sums, then a fixed-order second
// stage). A plan keeps its partial sums in memory it allocated at plan time; this entry point
// keeps them instead in one file-scope device array, g_loss_partials, that the library image
// brings with it (512 KiB, held by every GPU on which the library's module is loaded, until the
// process exits).
//
// CUDA loads a library's modules lazily by default (CUDA_MODULE_LOADING=LAZY): the module holding
// the array, and with it the array's device memory, is loaded on a device by the first
// cudaGetSymbolAddress made with that device current, that is, by the first call of this entry
// point there. Callers under a fixed memory budget make one warm-up call per device at start-up.
//
// The array's name, used in host code, is only a host-side stand-in for the device symbol, never
// a device address. Every call looks the device address up with cudaGetSymbolAddress while the
// caller's device is current (no allocation once the module is loaded), checks the result, and
// passes the pointer to the kernels; nothing is cached, so a context that was torn down and
// created again (cudaDeviceReset) gets the address of its own copy.
#include <cuda_runtime.h>

#include <cstdint>

#include "fresco.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                                  // rows per thread
constexpr int64_t kRowsPerBlock = (int64_t)kThreads * kItems;
constexpr int kMaxPartials = 65536;                         // 65536 doubles = 512 KiB

static __device__ __align__(256) double g_loss_partials[kMaxPartials];

// Block b sums W (S - S0)^2 over rows [b * kRowsPerBlock, (b + 1) * kRowsPerBlock) in FP64 and
// writes partial[b]. Every partial that the final stage reads is written first, in the same call.
template <typename TS>
__global__ void __launch_bounds__(kThreads) k_loss_partials(const TS *__restrict__ S,
                                                            const double *__restrict__ S0,
                                                            const double *__restrict__ W,
                                                            int64_t n, double *__restrict__ partial) {
    __shared__ double wsum[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kRowsPerBlock;
    double acc = 0.0;
#pragma unroll 4
    for (int i = 0; i < kItems; ++i) {
        const int64_t q = base + (int64_t)i * kThreads + threadIdx.x;
        if (q < n) {
            const double d = (double)S[q] - S0[q];
            acc += W[q] * d * d;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) b += wsum[w];
        partial[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(512) k_loss_final(const double *__restrict__ partial, int nb,
                                                    double *__restrict__ loss) {
    __shared__ double sm[512];
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += 512) v += partial[i];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 256; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sm[0];
}

// Device address of g_loss_partials on the current device (loading the module on the first use
// per context).
fresco_status scratch_on_current_device(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_loss_partials);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return FRESCO_ERR_CUDA;
    }
    *out = static_cast<double *>(p);
    return FRESCO_OK;
}

}  // namespace

extern "C" fresco_status fresco_loss_noalloc(int precision, int64_t n_k, const void *d_S,
                                             const double *d_S0, const double *d_W,
                                             double *d_loss, void *stream) {
    if (precision != FRESCO_F32 && precision != FRESCO_F64) return FRESCO_ERR_ARG;
    if (n_k < 1 || !d_S || !d_S0 || !d_W || !d_loss) return FRESCO_ERR_ARG;
    const int64_t nb = (n_k + kRowsPerBlock - 1) / kRowsPerBlock;
    if (nb > kMaxPartials) return FRESCO_ERR_UNSUPPORTED;   // n_k above FRESCO_LOSS_NOALLOC_MAX_ROWS
    cudaGetLastError();   // a pending launch error of earlier, unrelated work is not this call's
    double *partial = nullptr;
    fresco_status st = scratch_on_current_device(&partial);
    if (st != FRESCO_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == FRESCO_F32)
        k_loss_partials<float><<<(unsigned)nb, kThreads, 0, s>>>(
            static_cast<const float *>(d_S), d_S0, d_W, n_k, partial);
    else
        k_loss_partials<double><<<(unsigned)nb, kThreads, 0, s>>>(
            static_cast<const double *>(d_S), d_S0, d_W, n_k, partial);
    k_loss_final<<<1, 512, 0, s>>>(partial, (int)nb, d_loss);
    return cudaGetLastError() == cudaSuccess ? FRESCO_OK : FRESCO_ERR_CUDA;
}
