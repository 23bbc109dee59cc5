// Weights on a uniform grid with constraints at arbitrary real frequencies (UwNU, Methods
// "Analytical gradients"): S at the constraints by one type-2 NUFFT of the weights, the weight
// gradient by one type-1 NUFFT of the constraint coefficients.
//
// Pixel m (0 <= m_a < M_a) carries a real weight c_m; constraint q sits at the real frequency
// nu_q (cycles per grid length). With the pixel index centred, mt = m - floor(M / 2), and the
// target x_q = -nu_q / M (per axis, taken modulo 1),
//   rho~(nu_q) = sum_m c_m exp(-2 pi i nu_q . mt / M) = sum_m c_m exp(+2 pi i mt . x_q),
// which differs from the uncentred rho by a phase only, so S = |rho|^2 / rho0 is unchanged, and
//   dL/dc_m = Re sum_q C_q exp(+2 pi i nu_q . mt / M) - (4 c_m / rho0) sum_q W S (S - S0),
//   C_q = 4 W_q (S_q - S0_q) rho~_q / rho0,
// where the phase of rho~ cancels against the centred exponent. The transforms:
//   type 2: U[k] = c_mt / Psi(mt) at k = mt mod n_f, U <- inverse FFT(U), rho~_q = sum_l U[l]
//           psi(n_f x_q - l) over the w^d cells of the kernel's support;
//   type 1: U[l] = sum_q C_q psi(n_f x_q - l), U <- forward FFT(U), G(mt) = U[mt mod n_f] / Psi(mt).
// Psi is the kernel's Fourier transform at integer frequencies (fresco_kernel_ft). The
// constraints are few next to the pixels, so both NUFFT passes run one thread per constraint
// straight on the fine grid in global memory (float atomics for the spread) and evaluate the
// exponential-of-semicircle kernel directly.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fresco.h"
#include "fresco_kernels.cuh"

using namespace fresco;

namespace fresco {
FRESCO_EXTERN_WIDTH_OPS(float)
FRESCO_EXTERN_WIDTH_OPS(double)
extern template struct Launch<float>;
extern template struct Launch<double>;
}  // namespace fresco

namespace {

constexpr double kPiU = 3.141592653589793238462643383279502884;
constexpr int kUBlocks = 1024;

// The plan's rules for the fine grid and the kernel (the same error estimate of the
// exponential-of-semicircle kernel as fresco_plan): w = ceil(ln(1/eps) / (pi sqrt(1 - 1/sigma))),
// beta = 0.976 pi (1 - 1/(2 sigma)) w, n_f the smallest even 2-3-5-7-smooth size >= sigma M, 2w.
int uwnu_width(double eps, double sigma) {
    const double w = std::ceil(std::log(1.0 / eps) / (kPiU * std::sqrt(1.0 - 1.0 / sigma)));
    return (int)std::max(w, (double)kMinWidth);
}
double uwnu_beta(int w, double sigma) { return 0.976 * kPiU * (1.0 - 0.5 / sigma) * w; }
int64_t uwnu_smooth_even(int64_t n) {
    for (n = std::max<int64_t>(n, 2);; ++n) {
        if (n & 1) continue;
        int64_t r = n;
        for (int p : {2, 3, 5, 7})
            while (r % p == 0) r /= p;
        if (r == 1) return n;
    }
}

template <typename T>
using CxT = typename std::conditional<sizeof(T) == 4, float2, double2>::type;

__device__ __forceinline__ int wrap_index(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// psi(x1 + k), k = 0..W-1, psi(u) = exp(beta (sqrt(1 - (2u/W)^2) - 1)) for |u| < W/2, and the
// first cell of the support relative to the point's cell
template <typename T, int W>
__device__ __forceinline__ int kernel_row(T frac, T beta, T (&wt)[W]) {
    T x1;
    const int c0 = support_start<T, W>(frac, x1);
    const T s = T(2) / T(W);
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const T z = (x1 + T(k)) * s;
        const T q = T(1) - z * z;
        wt[k] = q > T(0) ? exp(beta * (sqrt(q) - T(1))) : T(0);
    }
    return c0;
}

__device__ __forceinline__ double ublock_sum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double b = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += ws[w];
    return b;
}

template <typename T>
__global__ void __launch_bounds__(256) k_un_sumsq(const T *__restrict__ c, int64_t n,
                                                  double *__restrict__ part) {
    DotAcc<T> acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc.add(c[i], c[i]);
    const double b = ublock_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// out[k] = sum of part[k * nb .. (k + 1) * nb), k < n_out, in a fixed order
__global__ void __launch_bounds__(256) k_un_sum(const double *__restrict__ part, int nb, int n_out,
                                                double *__restrict__ out) {
    for (int k = 0; k < n_out; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[(int64_t)k * nb + i];
        const double s = ublock_sum(v);
        if (threadIdx.x == 0) out[k] = s;
        __syncthreads();
    }
}

struct UGrid {
    int dim;
    int M[3];    // pixels per axis (1 beyond dim)
    int nf[3];   // fine grid per axis (1 beyond dim)
};

// pixel m -> centred index mt and fine-grid position; returns 1 / Psi(mt)
template <typename T>
__device__ __forceinline__ T pixel_site(const UGrid &g, int64_t m, const T *__restrict__ ip0,
                                        const T *__restrict__ ip1, const T *__restrict__ ip2,
                                        int64_t &fine) {
    const int m0 = (int)(m % g.M[0]);
    const int m1 = (int)((m / g.M[0]) % g.M[1]);
    const int m2 = (int)(m / ((int64_t)g.M[0] * g.M[1]));
    const int t0 = m0 - g.M[0] / 2, t1 = m1 - g.M[1] / 2, t2 = m2 - g.M[2] / 2;
    const int f0 = t0 < 0 ? t0 + g.nf[0] : t0;
    const int f1 = t1 < 0 ? t1 + g.nf[1] : t1;
    const int f2 = t2 < 0 ? t2 + g.nf[2] : t2;
    fine = ((int64_t)f2 * g.nf[1] + f1) * g.nf[0] + f0;
    T ip = ip0[t0 < 0 ? -t0 : t0] * ip1[t1 < 0 ? -t1 : t1];
    if (g.dim == 3) ip *= ip2[t2 < 0 ? -t2 : t2];
    return ip;
}

// type 2, step 1: U[mt mod n_f] = c_m / Psi(mt) (the rest of U was zeroed)
template <typename T>
__global__ void __launch_bounds__(256) k_un_fill(UGrid g, int64_t cells, const T *__restrict__ c,
                                                 const T *__restrict__ ip0,
                                                 const T *__restrict__ ip1,
                                                 const T *__restrict__ ip2, CxT<T> *__restrict__ U) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < cells;
         m += (int64_t)gridDim.x * blockDim.x) {
        int64_t f;
        const T ip = pixel_site<T>(g, m, ip0, ip1, ip2, f);
        U[f] = CxT<T>{c[m] * ip, T(0)};
    }
}

// type 2, step 3, and the loss: rho~_q by interpolation, S_q, the loss and F partials, and the
// type-1 strengths C_q = 4 W (S - S0) rho~ / rho0
// dq (optional, point plans with constraints at real wavevectors): a per-constraint factor that
// multiplies the interpolated sum before S is formed (the deconvolution of the points' own
// spreading kernel); then C_q = 4 W (S - S0) dq rho_q / norm. norm = scal[0] (rho0, or N).
template <typename T, int W, int D>
__global__ void __launch_bounds__(256) k_un_interp(UGrid g, int64_t n_k,
                                                   const int *__restrict__ tcell,
                                                   const T *__restrict__ tfrac, T beta,
                                                   const CxT<T> *__restrict__ U,
                                                   const T *__restrict__ s0,
                                                   const T *__restrict__ wq,
                                                   const double *__restrict__ scal,
                                                   const T *__restrict__ dq,
                                                   CxT<T> *__restrict__ coef, T *__restrict__ S_out,
                                                   double *__restrict__ part) {
    const double rho0 = scal[0];
    const T inv_rho0 = (T)(1.0 / rho0);
    double lsum = 0.0, fsum = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_k;
         q += (int64_t)gridDim.x * blockDim.x) {
        T wt[D][W];
        int st[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) st[a] = tcell[q * D + a] + kernel_row<T, W>(tfrac[q * D + a], beta, wt[a]);
        T re = T(0), im = T(0);
        if constexpr (D == 2) {
            for (int k1 = 0; k1 < W; ++k1) {
                const int64_t row = (int64_t)wrap_index(st[1] + k1, g.nf[1]) * g.nf[0];
                T rr = T(0), ri = T(0);
#pragma unroll
                for (int k0 = 0; k0 < W; ++k0) {
                    const CxT<T> v = U[row + wrap_index(st[0] + k0, g.nf[0])];
                    rr = fma(wt[0][k0], v.x, rr);
                    ri = fma(wt[0][k0], v.y, ri);
                }
                re = fma(wt[1][k1], rr, re);
                im = fma(wt[1][k1], ri, im);
            }
        } else {
            for (int k2 = 0; k2 < W; ++k2) {
                const int64_t pl = (int64_t)wrap_index(st[2] + k2, g.nf[2]) * g.nf[1];
                T pr = T(0), pm = T(0);
                for (int k1 = 0; k1 < W; ++k1) {
                    const int64_t row = (pl + wrap_index(st[1] + k1, g.nf[1])) * g.nf[0];
                    T rr = T(0), ri = T(0);
#pragma unroll
                    for (int k0 = 0; k0 < W; ++k0) {
                        const CxT<T> v = U[row + wrap_index(st[0] + k0, g.nf[0])];
                        rr = fma(wt[0][k0], v.x, rr);
                        ri = fma(wt[0][k0], v.y, ri);
                    }
                    pr = fma(wt[1][k1], rr, pr);
                    pm = fma(wt[1][k1], ri, pm);
                }
                re = fma(wt[2][k2], pr, re);
                im = fma(wt[2][k2], pm, im);
            }
        }
        T dk = T(1);
        if (dq) {
            dk = dq[q];
            re *= dk;
            im *= dk;
        }
        const T S = (re * re + im * im) * inv_rho0;
        const double d = (double)S - (double)s0[q];
        const double w = (double)wq[q];
        lsum = fma(w * d, d, lsum);
        fsum = fma(w * (double)S, d, fsum);
        const T h = (T)(4.0 * w * d / rho0) * dk;
        coef[q] = CxT<T>{h * re, h * im};
        S_out[q] = S;
    }
    const double bl = ublock_sum(lsum);
    const double bf = ublock_sum(fsum);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bl;
        part[gridDim.x + blockIdx.x] = bf;
    }
}

// type 1, step 1: U[l] += C_q psi(n_f x_q - l) over the support of every constraint
template <typename T, int W, int D>
__global__ void __launch_bounds__(256) k_un_spread(UGrid g, int64_t n_k,
                                                   const int *__restrict__ tcell,
                                                   const T *__restrict__ tfrac, T beta,
                                                   const CxT<T> *__restrict__ coef,
                                                   CxT<T> *__restrict__ U) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_k;
         q += (int64_t)gridDim.x * blockDim.x) {
        T wt[D][W];
        int st[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) st[a] = tcell[q * D + a] + kernel_row<T, W>(tfrac[q * D + a], beta, wt[a]);
        const CxT<T> cq = coef[q];
        const int n2 = D == 3 ? W : 1;
        for (int k2 = 0; k2 < n2; ++k2) {
            const int64_t pl = D == 3 ? (int64_t)wrap_index(st[2] + k2, g.nf[2]) * g.nf[1] : 0;
            const T w2 = D == 3 ? wt[D - 1][k2] : T(1);
            for (int k1 = 0; k1 < W; ++k1) {
                const int64_t row = (pl + wrap_index(st[1] + k1, g.nf[1])) * g.nf[0];
                const T w12 = w2 * wt[1][k1];
#pragma unroll
                for (int k0 = 0; k0 < W; ++k0) {
                    const T w = w12 * wt[0][k0];
                    T *cell = reinterpret_cast<T *>(U + row + wrap_index(st[0] + k0, g.nf[0]));
                    atomicAdd(cell, w * cq.x);
                    atomicAdd(cell + 1, w * cq.y);
                }
            }
        }
    }
}

// type 1, step 3, and the weight gradient: grad_m = Re U[mt mod n_f] / Psi(mt) - (4 F / rho0) c_m
template <typename T>
__global__ void __launch_bounds__(256) k_un_grad(UGrid g, int64_t cells, const T *__restrict__ c,
                                                 const T *__restrict__ ip0,
                                                 const T *__restrict__ ip1,
                                                 const T *__restrict__ ip2,
                                                 const CxT<T> *__restrict__ U,
                                                 const double *__restrict__ scal,
                                                 T *__restrict__ grad) {
    const T coef = (T)(4.0 * scal[2] / scal[0]);
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < cells;
         m += (int64_t)gridDim.x * blockDim.x) {
        int64_t f;
        const T ip = pixel_site<T>(g, m, ip0, ip1, ip2, f);
        grad[m] = U[f].x * ip - coef * c[m];
    }
}

template <typename T, int W>
cudaError_t launch_un_interp(const UGrid &g, int64_t n_k, const int *tcell, const T *tfrac,
                             T beta, const void *U, const T *s0, const T *wq, const double *scal,
                             const T *dq, void *coef, T *S, double *part, int nb, cudaStream_t s) {
    if (g.dim == 2)
        k_un_interp<T, W, 2><<<nb, 256, 0, s>>>(g, n_k, tcell, tfrac, beta, (const CxT<T> *)U,
                                                s0, wq, scal, dq, (CxT<T> *)coef, S, part);
    else
        k_un_interp<T, W, 3><<<nb, 256, 0, s>>>(g, n_k, tcell, tfrac, beta, (const CxT<T> *)U,
                                                s0, wq, scal, dq, (CxT<T> *)coef, S, part);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t launch_un_spread(const UGrid &g, int64_t n_k, const int *tcell, const T *tfrac,
                             T beta, const void *coef, void *U, int nb, cudaStream_t s) {
    if (g.dim == 2)
        k_un_spread<T, W, 2><<<nb, 256, 0, s>>>(g, n_k, tcell, tfrac, beta,
                                                (const CxT<T> *)coef, (CxT<T> *)U);
    else
        k_un_spread<T, W, 3><<<nb, 256, 0, s>>>(g, n_k, tcell, tfrac, beta,
                                                (const CxT<T> *)coef, (CxT<T> *)U);
    return cudaGetLastError();
}

template <typename T>
cudaError_t un_interp(int width, const UGrid &g, int64_t n_k, const int *tcell, const T *tfrac,
                      T beta, const void *U, const T *s0, const T *wq, const double *scal,
                      const T *dq, void *coef, T *S, double *part, int nb, cudaStream_t s) {
    FRESCO_WIDTH_SWITCH(width, return (launch_un_interp<T, WW>(g, n_k, tcell, tfrac, beta, U, s0,
                                                               wq, scal, dq, coef, S, part, nb,
                                                               s)));
}

template <typename T>
cudaError_t un_spread(int width, const UGrid &g, int64_t n_k, const int *tcell, const T *tfrac,
                      T beta, const void *coef, void *U, int nb, cudaStream_t s) {
    FRESCO_WIDTH_SWITCH(width, return (launch_un_spread<T, WW>(g, n_k, tcell, tfrac, beta, coef,
                                                               U, nb, s)));
}

fresco_status un_status(cudaError_t e) {
    if (e == cudaSuccess) return FRESCO_OK;
    if (e == cudaErrorMemoryAllocation) return FRESCO_ERR_OOM;
    return FRESCO_ERR_CUDA;
}

#define UN_CUDA(call)                                   \
    do {                                                \
        const cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return un_status(e_);    \
    } while (0)
#define UN_CUFFT(call)                                  \
    do {                                                \
        if ((call) != CUFFT_SUCCESS) return FRESCO_ERR_CUFFT; \
    } while (0)

}  // namespace

struct fresco_uwnu_s {
    UGrid g{};
    int precision = FRESCO_F32, width = 0;
    double beta = 0.0;
    int64_t cells = 0, fine = 0, n_k = 0;
    int nb = 1;   // blocks of the per-constraint kernels
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    void *ip[3] = {nullptr, nullptr, nullptr};   // 1 / Psi_a(nu), nu = 0..M_a/2
    int *tcell = nullptr;                        // [n_k][dim] fine cell of each target
    void *tfrac = nullptr;                       // [n_k][dim] position inside it, [0, 1)
    void *s0 = nullptr, *wq = nullptr, *S = nullptr, *coef = nullptr, *U = nullptr;
    double *part = nullptr, *scal = nullptr;     // scal: rho0, loss, F sum
    cufftHandle fft = 0;
    bool have_fft = false;
    bool evaluated = false;
};

namespace {

bool un_alloc(fresco_uwnu_s *u, void **p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    u->allocs.push_back(*p);
    return true;
}

void un_free(fresco_uwnu_s *u) {
    if (!u) return;
    if (u->stream) cudaStreamSynchronize(u->stream);
    else cudaDeviceSynchronize();
    if (u->have_fft) cufftDestroy(u->fft);
    for (void *p : u->allocs) cudaFree(p);
    delete u;
}

template <typename T>
fresco_status un_build(fresco_uwnu_s *u, const double *nu, const double *S0, const double *W) {
    using C2 = CxT<T>;
    const UGrid &g = u->g;
    const int dim = g.dim;
    const int64_t nk = u->n_k;
    bool ok = un_alloc(u, (void **)&u->tcell, sizeof(int) * (size_t)(nk * dim)) &&
              un_alloc(u, &u->tfrac, sizeof(T) * (size_t)(nk * dim)) &&
              un_alloc(u, &u->s0, sizeof(T) * (size_t)nk) &&
              un_alloc(u, &u->wq, sizeof(T) * (size_t)nk) &&
              un_alloc(u, &u->S, sizeof(T) * (size_t)nk) &&
              un_alloc(u, &u->coef, sizeof(C2) * (size_t)nk) &&
              un_alloc(u, &u->U, sizeof(C2) * (size_t)u->fine) &&
              un_alloc(u, (void **)&u->part, sizeof(double) * 2 * kUBlocks) &&
              un_alloc(u, (void **)&u->scal, sizeof(double) * 4);
    for (int a = 0; a < 3 && ok; ++a)
        ok = un_alloc(u, &u->ip[a], sizeof(T) * (size_t)(g.M[a] / 2 + 1));
    if (!ok) return FRESCO_ERR_OOM;
    for (int a = 0; a < 3; ++a) {   // deconvolution tables (axes beyond dim: the single entry 1)
        const int64_t n_nu = g.M[a] / 2 + 1;
        std::vector<double> psi((size_t)n_nu, 1.0);
        if (a < dim) {
            const fresco_status st = fresco_kernel_ft(u->width, u->beta, g.nf[a], n_nu, psi.data());
            if (st) return st;
        }
        std::vector<T> ipt((size_t)n_nu);
        for (int64_t i = 0; i < n_nu; ++i) ipt[(size_t)i] = (T)(1.0 / psi[(size_t)i]);
        UN_CUDA(cudaMemcpy(u->ip[a], ipt.data(), sizeof(T) * ipt.size(), cudaMemcpyHostToDevice));
    }
    {   // targets x = -nu / M (modulo 1) on the fine grid: cell and fraction, from FP64
        std::vector<int> cell((size_t)(nk * dim));
        std::vector<T> frac((size_t)(nk * dim)), s0((size_t)nk), w((size_t)nk);
        for (int64_t q = 0; q < nk; ++q) {
            for (int a = 0; a < dim; ++a) {
                const double x = -nu[q * dim + a] / (double)g.M[a];
                const double t = (x - std::floor(x)) * (double)g.nf[a];
                double c = std::floor(t);
                double f = t - c;
                int64_t ci = (int64_t)c % g.nf[a];
                if (ci < 0) ci += g.nf[a];
                cell[(size_t)(q * dim + a)] = (int)ci;
                frac[(size_t)(q * dim + a)] = (T)f;
            }
            s0[(size_t)q] = (T)S0[q];
            w[(size_t)q] = (T)W[q];
        }
        UN_CUDA(cudaMemcpy(u->tcell, cell.data(), sizeof(int) * cell.size(), cudaMemcpyHostToDevice));
        UN_CUDA(cudaMemcpy(u->tfrac, frac.data(), sizeof(T) * frac.size(), cudaMemcpyHostToDevice));
        UN_CUDA(cudaMemcpy(u->s0, s0.data(), sizeof(T) * s0.size(), cudaMemcpyHostToDevice));
        UN_CUDA(cudaMemcpy(u->wq, w.data(), sizeof(T) * w.size(), cudaMemcpyHostToDevice));
    }
    const cufftType type = sizeof(T) == 4 ? CUFFT_C2C : CUFFT_Z2Z;
    if (dim == 2) UN_CUFFT(cufftPlan2d(&u->fft, g.nf[1], g.nf[0], type));
    else UN_CUFFT(cufftPlan3d(&u->fft, g.nf[2], g.nf[1], g.nf[0], type));
    u->have_fft = true;
    UN_CUFFT(cufftSetStream(u->fft, u->stream));
    UN_CUDA(cudaDeviceSynchronize());
    return FRESCO_OK;
}

template <typename T>
fresco_status un_fft(fresco_uwnu_s *u, int dir) {
    if (sizeof(T) == 4)
        UN_CUFFT(cufftExecC2C(u->fft, (cufftComplex *)u->U, (cufftComplex *)u->U, dir));
    else
        UN_CUFFT(cufftExecZ2Z(u->fft, (cufftDoubleComplex *)u->U, (cufftDoubleComplex *)u->U, dir));
    return FRESCO_OK;
}

template <typename T>
fresco_status un_eval(fresco_uwnu_s *u, const T *c, double *loss, T *grad) {
    using C2 = CxT<T>;
    const UGrid &g = u->g;
    cudaStream_t s = u->stream;
    const unsigned pb = (unsigned)std::min<int64_t>((u->cells + 255) / 256, 152 * 16);
    const T *ip0 = (const T *)u->ip[0], *ip1 = (const T *)u->ip[1], *ip2 = (const T *)u->ip[2];
    const T beta = (T)u->beta;
    // rho0 = sum c^2
    k_un_sumsq<T><<<kUBlocks, 256, 0, s>>>(c, u->cells, u->part);
    k_un_sum<<<1, 256, 0, s>>>(u->part, kUBlocks, 1, u->scal);
    // type 2: rho~ at the constraints, with S, the loss and the type-1 strengths
    UN_CUDA(cudaMemsetAsync(u->U, 0, sizeof(C2) * (size_t)u->fine, s));
    k_un_fill<T><<<pb, 256, 0, s>>>(g, u->cells, c, ip0, ip1, ip2, (C2 *)u->U);
    fresco_status st = un_fft<T>(u, CUFFT_INVERSE);
    if (st) return st;
    UN_CUDA(un_interp<T>(u->width, g, u->n_k, u->tcell, (const T *)u->tfrac, beta, u->U,
                         (const T *)u->s0, (const T *)u->wq, u->scal, (const T *)nullptr, u->coef,
                         (T *)u->S, u->part, u->nb, s));
    k_un_sum<<<1, 256, 0, s>>>(u->part, u->nb, 2, u->scal + 1);
    UN_CUDA(cudaMemcpyAsync(loss, u->scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    u->evaluated = true;
    if (!grad) return un_status(cudaGetLastError());
    // type 1: the strengths back onto the pixels, then the weight gradient
    UN_CUDA(cudaMemsetAsync(u->U, 0, sizeof(C2) * (size_t)u->fine, s));
    UN_CUDA(un_spread<T>(u->width, g, u->n_k, u->tcell, (const T *)u->tfrac, beta, u->coef, u->U,
                         u->nb, s));
    st = un_fft<T>(u, CUFFT_FORWARD);
    if (st) return st;
    k_un_grad<T><<<pb, 256, 0, s>>>(g, u->cells, c, ip0, ip1, ip2, (const C2 *)u->U, u->scal,
                                    grad);
    return un_status(cudaGetLastError());
}

}  // namespace

extern "C" {

fresco_status fresco_uwnu_plan(fresco_uwnu_t *out, int dim, const int64_t *grid, int64_t n_k,
                               const double *nu, const double *S0, const double *W,
                               const fresco_opts *opts, void *stream) {
    if (!out) return FRESCO_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !grid || !nu || !S0 || !W || n_k < 1 || n_k > (1ll << 30))
        return FRESCO_ERR_ARG;
    fresco_opts o;
    fresco_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != FRESCO_F32 && o.precision != FRESCO_F64) return FRESCO_ERR_ARG;
    const double sigma = o.upsample == 0.0 ? 2.0 : o.upsample;
    if (!(sigma >= 1.25 && sigma <= 3.0)) return FRESCO_ERR_ARG;
    const double tol = o.tol == 0.0 ? (o.precision == FRESCO_F64 ? 1e-12 : 1e-6) : o.tol;
    if (!(tol > 0.0 && tol < 1.0)) return FRESCO_ERR_ARG;
    const int w = uwnu_width(tol, sigma);
    if (w > kMaxWidth) return FRESCO_ERR_UNSUPPORTED;
    UGrid g{};
    g.dim = dim;
    double fine = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.M[a] = 1;
        g.nf[a] = 1;
    }
    for (int a = 0; a < dim; ++a) {
        if (grid[a] < 2 || grid[a] > (1 << 20)) return FRESCO_ERR_ARG;
        g.M[a] = (int)grid[a];
        const int64_t need = std::max<int64_t>((int64_t)std::ceil(sigma * (double)grid[a]), 2 * w);
        const int64_t nf = uwnu_smooth_even(need);
        if (nf > (1 << 26)) return FRESCO_ERR_UNSUPPORTED;
        g.nf[a] = (int)nf;
        fine *= (double)nf;
    }
    if (fine > 4.0e9) return FRESCO_ERR_UNSUPPORTED;
    for (int64_t q = 0; q < n_k * dim; ++q)
        if (!std::isfinite(nu[q]) || std::fabs(nu[q]) > 1e9) return FRESCO_ERR_ARG;
    for (int64_t q = 0; q < n_k; ++q)
        if (!std::isfinite(S0[q]) || !std::isfinite(W[q]) || W[q] < 0.0) return FRESCO_ERR_ARG;
    fresco_uwnu_s *u = new (std::nothrow) fresco_uwnu_s();
    if (!u) return FRESCO_ERR_OOM;
    u->g = g;
    u->precision = o.precision;
    u->width = w;
    u->beta = uwnu_beta(w, sigma);
    u->cells = (int64_t)g.M[0] * g.M[1] * g.M[2];
    u->fine = (int64_t)fine;
    u->n_k = n_k;
    u->nb = (int)std::max<int64_t>(1, std::min<int64_t>((n_k + 255) / 256, kUBlocks));
    u->stream = (cudaStream_t)stream;
    const fresco_status st = o.precision == FRESCO_F64 ? un_build<double>(u, nu, S0, W)
                                                       : un_build<float>(u, nu, S0, W);
    if (st) {
        un_free(u);
        return st;
    }
    *out = u;
    return FRESCO_OK;
}

fresco_status fresco_uwnu_loss_grad(fresco_uwnu_t u, const void *d_c, double *d_loss,
                                    void *d_grad) {
    if (!u || !d_c || !d_loss) return FRESCO_ERR_ARG;
    if (u->precision == FRESCO_F64)
        return un_eval<double>(u, (const double *)d_c, d_loss, (double *)d_grad);
    return un_eval<float>(u, (const float *)d_c, d_loss, (float *)d_grad);
}

fresco_status fresco_uwnu_get_S(fresco_uwnu_t u, void *d_S) {
    if (!u || !d_S || !u->evaluated) return FRESCO_ERR_ARG;
    const size_t es = u->precision == FRESCO_F64 ? 8 : 4;
    return un_status(cudaMemcpyAsync(d_S, u->S, es * (size_t)u->n_k, cudaMemcpyDeviceToDevice,
                                     u->stream));
}

fresco_status fresco_uwnu_get_info(fresco_uwnu_t u, int *width, double *beta, int *n_fine) {
    if (!u) return FRESCO_ERR_ARG;
    if (width) *width = u->width;
    if (beta) *beta = u->beta;
    if (n_fine)
        for (int a = 0; a < 3; ++a) n_fine[a] = u->g.nf[a];
    return FRESCO_OK;
}

fresco_status fresco_uwnu_destroy(fresco_uwnu_t u) {
    un_free(u);
    return FRESCO_OK;
}

}  // extern "C"

// =============================================================================================
// Points at free positions with constraints at real wavevectors (NUwNU, Methods "Analytical
// gradients"): rho(k_q) = sum_j exp(-i k_q . r_j) for points r_j in [-L_a / 2, L_a / 2] (no
// periodicity) and wavevectors k_q anywhere, S_q = |rho_q|^2 / N, L = sum_q W_q (S_q - S0_q)^2,
// dL/dr_j = Re sum_q (4 i k_q W_q (S_q - S0_q) rho_q / N) exp(+i k_q . r_j).
//
// The type-3 transform is a spread followed by a type-2 transform. With a grid spacing h_a =
// pi / (sigma K_a) (K_a = max_q |k_q,a|) the points spread with the ES kernel psi onto a periodic
// grid of n1_a > L_a / h_a + w + 2 cells, cell c at position l h (l = c, or c - n1 past the middle,
// so the windows never meet across the seam), give b_l = sum_j psi(l - r_j / h), and by Poisson
// summation sum_l b_l exp(-i theta l) = Psi(theta) rho(k) at theta_a = k_a h_a (|theta_a| <= pi /
// sigma, where the kernel's aliases are below the tolerance): rho_q = [sum_l b_l exp(-i theta_q
// l)] / Psi(theta_q). The bracket is the type-2 sum of the weights-on-a-grid plan above, at nu_q =
// theta_q n1 / (2 pi) cycles per grid length; Psi(theta) = prod_a integral psi(u) cos(theta_a u)
// du, tabulated per constraint at plan time. The gradient is the chain rule through the same
// steps: G_l = Re sum_q C_q exp(+i theta_q l), C_q = 4 W_q (S_q - S0_q) rho_q / (N Psi(theta_q)),
// is the type-1 sum of that plan, and dL/dr_j,a = sum_l G_l d b_l / d r_j,a, the derivative of the
// points' spreading kernel: the kernel-derivative interpolation at the points with scale -2 / h_a.
// =============================================================================================

namespace {

// grid cell c of the points' grid (n1 per axis) -> centred index l, its cell on the fine grid of
// the type-2 transform (n2 per axis), and 1 / Psi2(l)
template <typename T>
__device__ __forceinline__ T grid_site(const UGrid &g, int64_t c, const T *__restrict__ ip0,
                                       const T *__restrict__ ip1, const T *__restrict__ ip2,
                                       int64_t &fine) {
    int l[3], f[3];
    const int64_t cc[3] = {c % g.M[0], (c / g.M[0]) % g.M[1], c / ((int64_t)g.M[0] * g.M[1])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        l[a] = (int)cc[a] < g.M[a] / 2 ? (int)cc[a] : (int)cc[a] - g.M[a];
        f[a] = l[a] < 0 ? l[a] + g.nf[a] : l[a];
    }
    fine = ((int64_t)f[2] * g.nf[1] + f[1]) * g.nf[0] + f[0];
    T ip = ip0[l[0] < 0 ? -l[0] : l[0]] * ip1[l[1] < 0 ? -l[1] : l[1]];
    if (g.dim == 3) ip *= ip2[l[2] < 0 ? -l[2] : l[2]];
    return ip;
}

// type 2, step 1: U[l mod n2] = b_c / Psi2(l)
template <typename T>
__global__ void __launch_bounds__(256) k_nu_fill(UGrid g, int64_t cells, const T *__restrict__ b,
                                                 const T *__restrict__ ip0,
                                                 const T *__restrict__ ip1,
                                                 const T *__restrict__ ip2, CxT<T> *__restrict__ U) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t f;
        const T ip = grid_site<T>(g, c, ip0, ip1, ip2, f);
        U[f] = CxT<T>{b[c] * ip, T(0)};
    }
}

// type 1, step 3: G_c = Re U[l mod n2] / Psi2(l) on the points' grid
template <typename T>
__global__ void __launch_bounds__(256) k_nu_field(UGrid g, int64_t cells,
                                                  const T *__restrict__ ip0,
                                                  const T *__restrict__ ip1,
                                                  const T *__restrict__ ip2,
                                                  const CxT<T> *__restrict__ U, T *__restrict__ G) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t f;
        const T ip = grid_site<T>(g, c, ip0, ip1, ip2, f);
        G[c] = U[f].x * ip;
    }
}

// flags (bit 2 of err) a point outside [-half_a, half_a] on some axis
template <typename T>
__global__ void __launch_bounds__(256) k_nu_bounds(const T *__restrict__ pts, int64_t n, int dim,
                                                   double hx, double hy, double hz,
                                                   int *__restrict__ err) {
    const double half[3] = {hx, hy, hz};
    bool out = false;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < dim; ++a) {
            const double r = (double)pts[j * dim + a];
            out |= r < -half[a] || r > half[a];   // NaN passes here: k_count flags it
        }
    if (out) atomicOr(err, 2);
}

}  // namespace

struct fresco_nuwnu_s {
    fresco_uwnu_s *c = nullptr;   // the constraint side: grid <-> wavevectors (type 2 / type 1)
    fresco::PointSide ps;         // the point side: the points spread onto the n1 grid
    int dim = 0, precision = FRESCO_F32;
    double box[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    int64_t n_points = 0, cells = 0;
    void *dq = nullptr;           // [n_k] 1 / Psi1(theta_q)
    cudaStream_t stream = nullptr;
    int64_t launches = 0;
};

namespace {

void nu_free(fresco_nuwnu_s *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    if (p->c) un_free(p->c);
    fresco::point_side_free(p->ps);
    if (p->dq) cudaFree(p->dq);
    delete p;
}

template <typename T>
fresco_status nu_build(fresco_nuwnu_s *p, const double *kvec, const double *S0, const double *W,
                       int64_t n_k) {
    fresco_uwnu_s *u = p->c;
    const int dim = p->dim;
    // constraint side: nu_q = k_q h n1 / (2 pi)
    std::vector<double> nu((size_t)(n_k * dim));
    std::vector<double> theta((size_t)n_k);
    std::vector<double> psi((size_t)n_k);
    std::vector<T> dq((size_t)n_k, T(1));
    for (int a = 0; a < dim; ++a) {
        for (int64_t q = 0; q < n_k; ++q) {
            theta[(size_t)q] = kvec[q * dim + a] * p->h[a];
            nu[(size_t)(q * dim + a)] = theta[(size_t)q] * (double)u->g.M[a] / (2.0 * kPiU);
        }
        fresco::kernel_ft_at(u->width, u->beta, theta.data(), n_k, psi.data());
        for (int64_t q = 0; q < n_k; ++q) dq[(size_t)q] = (T)((double)dq[(size_t)q] / psi[(size_t)q]);
    }
    fresco_status st = un_build<T>(u, nu.data(), S0, W);
    if (st) return st;
    if (cudaMalloc(&p->dq, sizeof(T) * (size_t)n_k) != cudaSuccess) {
        cudaGetLastError();
        p->dq = nullptr;
        return FRESCO_ERR_OOM;
    }
    UN_CUDA(cudaMemcpy(p->dq, dq.data(), sizeof(T) * (size_t)n_k, cudaMemcpyHostToDevice));
    const double norm = (double)p->n_points;   // S = |rho|^2 / N
    UN_CUDA(cudaMemcpy(u->scal, &norm, sizeof(double), cudaMemcpyHostToDevice));
    // point side: the n1 grid over the periodic box n1 h
    int n1[3] = {1, 1, 1};
    double pbox[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
        n1[a] = u->g.M[a];
        pbox[a] = (double)n1[a] * p->h[a];
    }
    st = fresco::point_side_build(p->ps, dim, n1, pbox, p->n_points, u->width, u->beta,
                                  p->precision, p->stream);
    if (st) return st;
    UN_CUDA(cudaDeviceSynchronize());
    return FRESCO_OK;
}

template <typename T>
fresco_status nu_eval(fresco_nuwnu_s *p, const T *pts, double *loss, T *grad) {
    using C2 = CxT<T>;
    fresco_uwnu_s *u = p->c;
    const UGrid &g = u->g;
    cudaStream_t s = p->stream;
    const unsigned pb = (unsigned)std::min<int64_t>((p->cells + 255) / 256, 152 * 16);
    const T *ip0 = (const T *)u->ip[0], *ip1 = (const T *)u->ip[1], *ip2 = (const T *)u->ip[2];
    // the grid keeps spare cells beyond the box, so half a cell of slack (FP32 coordinates of
    // points on a face may round just outside it) changes nothing
    k_nu_bounds<T><<<(unsigned)std::min<int64_t>((p->n_points + 255) / 256, 152 * 8), 256, 0, s>>>(
        pts, p->n_points, p->dim, 0.5 * (p->box[0] + p->h[0]), 0.5 * (p->box[1] + p->h[1]),
        0.5 * (p->box[2] + p->h[2]), p->ps.err);
    fresco_status st = fresco::point_side_spread<T>(p->ps, pts, s, &p->launches);
    if (st) return st;
    // type 2 of the spread grid at the wavevectors, S, the loss and the type-1 strengths
    UN_CUDA(cudaMemsetAsync(u->U, 0, sizeof(C2) * (size_t)u->fine, s));
    k_nu_fill<T><<<pb, 256, 0, s>>>(g, p->cells, (const T *)p->ps.grid, ip0, ip1, ip2, (C2 *)u->U);
    st = un_fft<T>(u, CUFFT_INVERSE);
    if (st) return st;
    UN_CUDA(un_interp<T>(u->width, g, u->n_k, u->tcell, (const T *)u->tfrac, (T)u->beta, u->U,
                         (const T *)u->s0, (const T *)u->wq, u->scal, (const T *)p->dq, u->coef,
                         (T *)u->S, u->part, u->nb, s));
    k_un_sum<<<1, 256, 0, s>>>(u->part, u->nb, 1, u->scal + 1);
    UN_CUDA(cudaMemcpyAsync(loss, u->scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    p->launches += 4;
    u->evaluated = true;
    if (!grad) return un_status(cudaGetLastError());
    // type 1 of the strengths onto the grid, then the kernel-derivative interpolation
    UN_CUDA(cudaMemsetAsync(u->U, 0, sizeof(C2) * (size_t)u->fine, s));
    UN_CUDA(un_spread<T>(u->width, g, u->n_k, u->tcell, (const T *)u->tfrac, (T)u->beta, u->coef,
                         u->U, u->nb, s));
    st = un_fft<T>(u, CUFFT_FORWARD);
    if (st) return st;
    k_nu_field<T><<<pb, 256, 0, s>>>(g, p->cells, ip0, ip1, ip2, (const C2 *)u->U, (T *)p->ps.grid);
    const double dscale[3] = {-2.0 / p->h[0], -2.0 / p->h[1], -2.0 / p->h[2]};
    const EsPoly<T> &ep = *reinterpret_cast<const EsPoly<T> *>(
        sizeof(T) == 4 ? (const void *)&p->ps.p32 : (const void *)&p->ps.p64);
    UN_CUDA(Launch<T>::interp_kd(p->ps.g, ep, p->ps.sorted, p->ps.perm, p->ps.tr,
                                 (const T *)p->ps.grid, nullptr, dscale, grad, s));
    p->launches += 3;
    return un_status(cudaGetLastError());
}

}  // namespace

extern "C" {

fresco_status fresco_nuwnu_plan(fresco_nuwnu_t *out, int dim, const double *box,
                                int64_t n_points, int64_t n_k, const double *kvec,
                                const double *S0, const double *W, const fresco_opts *opts,
                                void *stream) {
    if (!out) return FRESCO_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !box || !kvec || !S0 || !W || n_k < 1 || n_k > (1ll << 30) ||
        n_points < 1 || n_points > 2147483647LL)
        return FRESCO_ERR_ARG;
    fresco_opts o;
    fresco_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != FRESCO_F32 && o.precision != FRESCO_F64) return FRESCO_ERR_ARG;
    const double sigma = o.upsample == 0.0 ? 2.0 : o.upsample;
    if (!(sigma >= 1.25 && sigma <= 3.0)) return FRESCO_ERR_ARG;
    const double tol = o.tol == 0.0 ? (o.precision == FRESCO_F64 ? 1e-12 : 1e-6) : o.tol;
    if (!(tol > 0.0 && tol < 1.0)) return FRESCO_ERR_ARG;
    const int w = uwnu_width(tol, sigma);
    if (w > kMaxWidth) return FRESCO_ERR_UNSUPPORTED;
    for (int a = 0; a < dim; ++a)
        if (!(box[a] > 0.0) || !std::isfinite(box[a])) return FRESCO_ERR_ARG;
    for (int64_t q = 0; q < n_k * dim; ++q)
        if (!std::isfinite(kvec[q])) return FRESCO_ERR_ARG;
    for (int64_t q = 0; q < n_k; ++q)
        if (!std::isfinite(S0[q]) || !std::isfinite(W[q]) || W[q] < 0.0) return FRESCO_ERR_ARG;
    fresco_nuwnu_s *p = new (std::nothrow) fresco_nuwnu_s();
    if (!p) return FRESCO_ERR_OOM;
    p->dim = dim;
    p->precision = o.precision;
    p->n_points = n_points;
    p->stream = (cudaStream_t)stream;
    UGrid g{};
    g.dim = dim;
    double fine = 1.0, cells = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.M[a] = 1;
        g.nf[a] = 1;
    }
    for (int a = 0; a < dim; ++a) {
        p->box[a] = box[a];
        double kmax = 0.0;
        for (int64_t q = 0; q < n_k; ++q) kmax = std::max(kmax, std::fabs(kvec[q * dim + a]));
        kmax = std::max(kmax, kPiU / box[a]);   // at least one cycle per box: any spacing works
        p->h[a] = kPiU / (sigma * kmax);
        // the points span box / h cells; their windows w more; two cells to spare at the seam
        const double need = std::ceil(box[a] / p->h[a]) + w + 2;
        if (need > (double)(1 << 24)) {
            delete p;
            return FRESCO_ERR_UNSUPPORTED;
        }
        const int64_t n1 = uwnu_smooth_even(std::max<int64_t>((int64_t)need, 2 * w));
        const int64_t n2 = uwnu_smooth_even(std::max<int64_t>((int64_t)std::ceil(sigma * (double)n1), 2 * w));
        if (n1 > 255 * 65535 || n2 > (1 << 26)) {
            delete p;
            return FRESCO_ERR_UNSUPPORTED;
        }
        g.M[a] = (int)n1;
        g.nf[a] = (int)n2;
        fine *= (double)n2;
        cells *= (double)n1;
    }
    if (fine > 4.0e9 || cells > 4.0e9) {
        delete p;
        return FRESCO_ERR_UNSUPPORTED;
    }
    fresco_uwnu_s *u = new (std::nothrow) fresco_uwnu_s();
    if (!u) {
        delete p;
        return FRESCO_ERR_OOM;
    }
    p->c = u;
    u->g = g;
    u->precision = o.precision;
    u->width = w;
    u->beta = uwnu_beta(w, sigma);
    u->cells = (int64_t)cells;
    u->fine = (int64_t)fine;
    u->n_k = n_k;
    u->nb = (int)std::max<int64_t>(1, std::min<int64_t>((n_k + 255) / 256, kUBlocks));
    u->stream = p->stream;
    p->cells = (int64_t)cells;
    const fresco_status st = o.precision == FRESCO_F64 ? nu_build<double>(p, kvec, S0, W, n_k)
                                                       : nu_build<float>(p, kvec, S0, W, n_k);
    if (st) {
        nu_free(p);
        return st;
    }
    *out = p;
    return FRESCO_OK;
}

fresco_status fresco_nuwnu_loss_grad(fresco_nuwnu_t p, const void *d_points, double *d_loss,
                                     void *d_grad) {
    if (!p || !d_points || !d_loss) return FRESCO_ERR_ARG;
    cudaGetLastError();
    if (p->precision == FRESCO_F64)
        return nu_eval<double>(p, (const double *)d_points, d_loss, (double *)d_grad);
    return nu_eval<float>(p, (const float *)d_points, d_loss, (float *)d_grad);
}

fresco_status fresco_nuwnu_get_S(fresco_nuwnu_t p, void *d_S) {
    if (!p) return FRESCO_ERR_ARG;
    return fresco_uwnu_get_S(p->c, d_S);
}

fresco_status fresco_nuwnu_status_check(fresco_nuwnu_t p) {
    if (!p) return FRESCO_ERR_ARG;
    UN_CUDA(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    int err = 0;
    UN_CUDA(cudaMemcpy(&err, p->ps.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        const int zero = 0;
        UN_CUDA(cudaMemcpy(p->ps.err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return (err & 1) ? FRESCO_ERR_NONFINITE : FRESCO_ERR_BOUNDS;
    }
    return un_status(cudaGetLastError());
}

fresco_status fresco_nuwnu_get_info(fresco_nuwnu_t p, int *width, int *n_grid, int *n_fine,
                                    int64_t *launches) {
    if (!p) return FRESCO_ERR_ARG;
    if (width) *width = p->c->width;
    for (int a = 0; a < 3; ++a) {
        if (n_grid) n_grid[a] = p->c->g.M[a];
        if (n_fine) n_fine[a] = p->c->g.nf[a];
    }
    if (launches) *launches = p->launches;
    return FRESCO_OK;
}

fresco_status fresco_nuwnu_destroy(fresco_nuwnu_t p) {
    nu_free(p);
    return FRESCO_OK;
}

}  // extern "C"
