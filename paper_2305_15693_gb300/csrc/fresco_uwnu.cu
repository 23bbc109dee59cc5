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
// Psi is the kernel's Fourier transform at integer frequencies (fresco_kernel_ft).
//
// The constraints' positions are fixed for the plan's life, so the plan orders them once, on the
// host, by the tile of the fine grid that holds their cell, and lists for every tile the
// constraints whose kernel support meets it. The type-2 interpolation then runs over the
// constraints in that order (in 2D a block stages its tile's window of U in shared memory), and
// the type-1 spread runs one block per tile: the block adds its list's contributions into the
// tile in shared memory, in fixed point, and stores every cell of the tile once, so U needs
// neither global atomics nor zeroing and the result repeats bitwise. Within a tile (or a list)
// the host deals the constraints over the shared-memory banks their first cells fall in, so the
// lanes of a warp meet distinct banks. Both evaluate the kernel with the plan's piecewise
// polynomials (es_weights).
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fresco.h"
#include "fresco_kernels.cuh"
#include "fresco_uwnu_tiles.h"

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
constexpr int kUWinBlocks = 16384;

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

constexpr int kUTileCells = 1024;   // T[0] T[1] T[2] at most (UTiles, fresco_uwnu_tiles.h)

// the weight of support cell k of one axis out of the unrolled row (k known only at run time)
template <typename T, int W>
__device__ __forceinline__ T pick_weight(const T (&w)[W], int k) {
    T r = w[0];
#pragma unroll
    for (int i = 1; i < W; ++i)
        if (i == k) r = w[i];
    return r;
}

// type 2, step 3, and the loss, over the constraints in tile order (slot q; perm[q] is the
// caller's index): rho~_q by interpolation, S_q, the loss and F partials, and the type-1
// strengths C_q = 4 W (S - S0) rho~ / rho0, which stay in tile order for the spread.
// dq (optional, point plans with constraints at real wavevectors): a per-constraint factor that
// multiplies the interpolated sum before S is formed (the deconvolution of the points' own
// spreading kernel); then C_q = 4 W (S - S0) dq rho_q / norm. norm = scal[0] (rho0, or N).
template <typename T, int W, int D>
__global__ void __launch_bounds__(256) k_un_interp(UGrid g, EsPoly<T> ep, int64_t n_k,
                                                   const int *__restrict__ tcell,
                                                   const T *__restrict__ tfrac,
                                                   const CxT<T> *__restrict__ U,
                                                   const T *__restrict__ s0,
                                                   const T *__restrict__ wq,
                                                   const double *__restrict__ scal,
                                                   const T *__restrict__ dq,
                                                   const int *__restrict__ perm,
                                                   CxT<T> *__restrict__ coef, T *__restrict__ S_out,
                                                   double *__restrict__ part) {
    const T inv_rho0 = (T)(1.0 / scal[0]);
    DotAcc<T> lacc, facc;   // the loss and F partial sums (no FP64 pipe in the FP32 loop)
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_k;
         q += (int64_t)gridDim.x * blockDim.x) {
        T wt[D][W];
        int st[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T x1;
            st[a] = tcell[q * D + a] + support_start<T, W>(tfrac[q * D + a], x1);
            es_weights<T, W>(ep, x1, wt[a]);
        }
        T re = T(0), im = T(0);
        const int n2 = D == 3 ? W : 1;
        for (int k2 = 0; k2 < n2; ++k2) {
            const int64_t pl = D == 3 ? (int64_t)wrap_index(st[2] + k2, g.nf[2]) * g.nf[1] : 0;
            T pr = T(0), pm = T(0);
#pragma unroll
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
            const T w2 = D == 3 ? pick_weight<T, W>(wt[D - 1], k2) : T(1);
            re = fma(w2, pr, re);
            im = fma(w2, pm, im);
        }
        T dk = T(1);
        if (dq) {
            dk = dq[q];
            re *= dk;
            im *= dk;
        }
        const T S = (re * re + im * im) * inv_rho0;
        const T d = S - s0[q];
        const T wd = wq[q] * d;
        lacc.add(wd, d);
        facc.add(wq[q] * S, d);
        const T h = T(4) * wd * inv_rho0 * dk;
        coef[q] = CxT<T>{h * re, h * im};
        S_out[perm[q]] = S;
    }
    const double bl = ublock_sum(lacc.value());
    const double bf = ublock_sum(facc.value());
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bl;
        part[gridDim.x + blockIdx.x] = bf;
    }
}

constexpr int kUWinEdge = 48;   // the 2D window edge: tile edge (at most 32) + w (at most 16)

// Blocks per multiprocessor the window interpolation asks for: FP32 at widths 4 to 7 fits in 32
// registers a thread without spilling, so eight blocks (all 64 warps) stay resident.
template <typename T, int W>
constexpr int kWinMinBlocks = sizeof(T) == 4 && W >= 4 && W <= 7 ? 8 : 1;

// The same in 2D from shared memory: a block takes the constraints of one home tile at a time
// (slots hoff[t] .. hoff[t + 1]), stages the window of U their supports cover (the tile and
// floor(w / 2) cells before it, w - floor(w / 2) after, wrapped) as real and imaginary planes,
// and sums each support there.
template <typename T, int W>
__global__ void __launch_bounds__(256, kWinMinBlocks<T, W>)
    k_un_interp_win(UGrid g, UTiles tl, EsPoly<T> ep, int64_t n_tiles,
                    const int64_t *__restrict__ hoff, const int *__restrict__ tcell,
                    const T *__restrict__ tfrac, const CxT<T> *__restrict__ U,
                    const T *__restrict__ s0, const T *__restrict__ wq,
                    const double *__restrict__ scal, const T *__restrict__ dq,
                    const int *__restrict__ perm, CxT<T> *__restrict__ coef,
                    T *__restrict__ S_out, double *__restrict__ part) {
    constexpr int kWin = kUWinEdge * kUWinEdge;
    __shared__ T sw[2 * kWin];   // real parts, then imaginary parts at + kWin
    const T inv_rho0 = (T)(1.0 / scal[0]);
    DotAcc<T> lacc, facc;   // the loss and F partial sums (no FP64 pipe in the FP32 loop)
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t q0 = hoff[t], q1 = hoff[t + 1];
        if (q0 == q1) continue;
        const int tx = (int)(t % tl.nt[0]), ty = (int)(t / tl.nt[0]);
        const int ws0 = tx * tl.T[0] - W / 2, ws1 = ty * tl.T[1] - W / 2;
        const int wl0 = min(tl.T[0], g.nf[0] - tx * tl.T[0]) + W;
        const int wl1 = min(tl.T[1], g.nf[1] - ty * tl.T[1]) + W;
        __syncthreads();   // the previous tile's sums are done with the window
        for (int i = threadIdx.x; i < wl0 * wl1; i += blockDim.x) {
            const int y = i / wl0, x = i - y * wl0;
            const CxT<T> v = U[(int64_t)wrap_index(ws1 + y, g.nf[1]) * g.nf[0] +
                               wrap_index(ws0 + x, g.nf[0])];
            sw[i] = v.x;
            sw[kWin + i] = v.y;
        }
        __syncthreads();
        for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            T wx[W], wy[W], x1;
            const int x0 = tcell[q * 2] + support_start<T, W>(tfrac[q * 2], x1) - ws0;
            es_weights<T, W>(ep, x1, wx);
            const int y0 = tcell[q * 2 + 1] + support_start<T, W>(tfrac[q * 2 + 1], x1) - ws1;
            es_weights<T, W>(ep, x1, wy);
            const T *row = sw + y0 * wl0 + x0;
            T re = T(0), im = T(0);
#pragma unroll
            for (int k1 = 0; k1 < W; ++k1) {
                T rr = T(0), ri = T(0);
#pragma unroll
                for (int k0 = 0; k0 < W; ++k0) {
                    rr = fma(wx[k0], row[k0], rr);
                    ri = fma(wx[k0], row[kWin + k0], ri);
                }
                re = fma(wy[k1], rr, re);
                im = fma(wy[k1], ri, im);
                row += wl0;
            }
            T dk = T(1);
            if (dq) {
                dk = dq[q];
                re *= dk;
                im *= dk;
            }
            const T S = (re * re + im * im) * inv_rho0;
            const T d = S - s0[q];
            const T wd = wq[q] * d;
            lacc.add(wd, d);
            facc.add(wq[q] * S, d);
            const T h = T(4) * wd * inv_rho0 * dk;
            coef[q] = CxT<T>{h * re, h * im};
            S_out[perm[q]] = S;
        }
    }
    const double bl = ublock_sum(lacc.value());
    const double bf = ublock_sum(facc.value());
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bl;
        part[gridDim.x + blockIdx.x] = bf;
    }
}

// Fixed-point cells of the spread: 32-bit integers for FP32 plans, 64-bit for FP64. A tile's
// strengths are scaled by 2^s, s the largest exponent that keeps its largest possible cell sum,
// (the most supports that cover one of its cells) x (its largest strength component), below
// 2^kBits; every term is rounded to an integer and the integer adds need no rounding order, so
// the spread repeats bitwise. The quantum is 2^-kBits of that bound (about 2^-24 of the largest
// strength for a few dozen covering supports in FP32), finer than the rounding of a float sum
// of as many terms.
template <typename T>
struct SpreadFixed;
template <>
struct SpreadFixed<float> {
    using I = int;
    static constexpr int kBits = 30;
    static __device__ __forceinline__ I to_fixed(float v) { return __float2int_rn(v); }
    static __device__ __forceinline__ void add(I *p, I v) { atomicAdd(p, v); }
    static __device__ __forceinline__ float from_fixed(I v, int s) { return ldexpf((float)v, -s); }
};
template <>
struct SpreadFixed<double> {
    using I = long long;
    static constexpr int kBits = 62;
    static __device__ __forceinline__ I to_fixed(double v) { return __double2ll_rn(v); }
    static __device__ __forceinline__ void add(I *p, I v) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
    }
    static __device__ __forceinline__ double from_fixed(I v, int s) { return ldexp((double)v, -s); }
};

// type 1, step 1: one block per tile of U. The block adds C_q psi(n_f x_q - l) of every
// constraint on the tile's list (slots ent[toff[t] .. toff[t + 1]), in bank order) into the
// tile's cells in shared memory, clipped to the tile, in fixed point (SpreadFixed; kcov[t]: the
// most supports that cover one cell of the tile), then stores all of the tile's cells. Every
// cell of U belongs to one tile, so U is written in full, zeros included.
template <typename T, int W, int D>
__global__ void __launch_bounds__(256) k_un_spread(UGrid g, UTiles tl, EsPoly<T> ep,
                                                   int64_t n_tiles,
                                                   const int64_t *__restrict__ toff,
                                                   const int *__restrict__ ent,
                                                   const int *__restrict__ kcov,
                                                   const int *__restrict__ tcell,
                                                   const T *__restrict__ tfrac,
                                                   const CxT<T> *__restrict__ coef,
                                                   CxT<T> *__restrict__ U) {
    using F = SpreadFixed<T>;
    using I = typename F::I;
    __shared__ I sh[2 * kUTileCells];   // real parts, then imaginary parts at + kUTileCells
    __shared__ T s_max[8];
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int tx = (int)(t % tl.nt[0]);
        const int ty = (int)((t / tl.nt[0]) % tl.nt[1]);
        const int tz = (int)(t / ((int64_t)tl.nt[0] * tl.nt[1]));
        const int o[3] = {tx * tl.T[0], ty * tl.T[1], tz * tl.T[2]};
        const int len[3] = {min(tl.T[0], g.nf[0] - o[0]), min(tl.T[1], g.nf[1] - o[1]),
                            min(tl.T[2], g.nf[2] - o[2])};
        const int cells = len[0] * len[1] * len[2];
        const int64_t e0 = toff[t], e1 = toff[t + 1];
        // the tile's largest strength component, and its scale
        T m = T(0);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const CxT<T> c = coef[ent[e]];
            m = fmax(m, fmax(fabs(c.x), fabs(c.y)));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            sh[i] = 0;
            sh[kUTileCells + i] = 0;
        }
        __syncthreads();
        m = s_max[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_max[w]);
        int sc = 0;
        if (m > T(0)) {
            int ex;
            frexp((double)kcov[t] * (double)m, &ex);   // kcov m < 2^ex
            sc = F::kBits - ex;
        }
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int64_t q = ent[e];
            T wt[D][W];
            int lo[3] = {0, 0, 0}, k0[3] = {0, 0, 0}, k1[3] = {1, 1, 1};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                T x1;
                // first support cell relative to the tile, at the one shift that meets it
                int d = tcell[q * D + a] + support_start<T, W>(tfrac[q * D + a], x1) - o[a];
                if (d >= len[a]) d -= g.nf[a];
                else if (d + W <= 0) d += g.nf[a];
                lo[a] = d;
                k0[a] = max(0, -d);
                k1[a] = min(W, len[a] - d);
                es_weights<T, W>(ep, x1, wt[a]);
            }
            const CxT<T> c = coef[q];
            const T csr = ldexp(c.x, sc), csi = ldexp(c.y, sc);
            for (int k2 = k0[2]; k2 < k1[2]; ++k2) {
                const T w2 = D == 3 ? pick_weight<T, W>(wt[D - 1], k2) : T(1);
                for (int k1y = k0[1]; k1y < k1[1]; ++k1y) {
                    const T wy = w2 * pick_weight<T, W>(wt[1], k1y);
                    const T cr = wy * csr, ci = wy * csi;
                    const int row = ((lo[2] + k2) * len[1] + lo[1] + k1y) * len[0] + lo[0];
#pragma unroll
                    for (int k = 0; k < W; ++k)
                        if (k >= k0[0] && k < k1[0]) {
                            F::add(sh + row + k, F::to_fixed(wt[0][k] * cr));
                            F::add(sh + kUTileCells + row + k, F::to_fixed(wt[0][k] * ci));
                        }
                }
            }
        }
        __syncthreads();
        const int64_t sx = g.nf[0], sxy = (int64_t)g.nf[0] * g.nf[1];
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            const int x = i % len[0];
            const int r = i / len[0];
            const int y = r % len[1];
            const int z = r / len[1];
            U[(int64_t)(o[2] + z) * sxy + (int64_t)(o[1] + y) * sx + o[0] + x] =
                CxT<T>{F::from_fixed(sh[i], sc), F::from_fixed(sh[kUTileCells + i], sc)};
        }
        __syncthreads();
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
    UTiles tl{};
    int precision = FRESCO_F32, width = 0;
    double beta = 0.0;
    int64_t cells = 0, fine = 0, n_k = 0, n_tiles = 0, n_ent = 0;
    int nb = 1;   // blocks of the per-constraint kernels
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    EsPoly<float> p32{};
    EsPoly<double> p64{};
    void *ip[3] = {nullptr, nullptr, nullptr};   // 1 / Psi_a(nu), nu = 0..M_a/2
    // the constraints in tile order (slot q): caller's index, fine cell and position inside it
    int *perm = nullptr;                         // [n_k]
    int *tcell = nullptr;                        // [n_k][dim]
    void *tfrac = nullptr;                       // [n_k][dim], [0, 1)
    void *s0 = nullptr, *wq = nullptr, *dq = nullptr;   // [n_k] in tile order (dq: point plans)
    void *S = nullptr;                           // [n_k] in the caller's order
    void *coef = nullptr, *U = nullptr;          // strengths in tile order; the fine grid
    int64_t *hoff = nullptr;                     // [n_tiles + 1] slots of each home tile
    int64_t *toff = nullptr;                     // [n_tiles + 1] list offsets of the tiles
    int *ent = nullptr;                          // [n_ent] constraint slots, tile by tile
    int *kcov = nullptr;                         // [n_tiles] most supports covering one cell
    double *part = nullptr, *scal = nullptr;     // scal: rho0 (or N), loss, F sum
    cufftHandle fft = 0;
    bool have_fft = false;
    bool evaluated = false;
    int64_t launches = 0;
    fresco::StageProfile prof;
};

// Stages of the per-stage timing (fresco_uwnu_profile, fresco_nuwnu_profile)
enum {
    UST_POINT_SPREAD = 0,   // point plans: bounds check, binning and spreading of the points
    UST_TYPE2 = 1,          // rho0, the weights (or the points' grid) onto U, inverse FFT
    UST_INTERP = 2,         // interpolation at the constraints, S, loss, strengths
    UST_SPREAD = 3,         // the strengths onto the tiles of U
    UST_TYPE1 = 4,          // forward FFT and the weight gradient (or the points' field)
    UST_POINT_INTERP = 5,   // point plans: kernel-derivative interpolation at the points
    UST_COUNT = 6
};
static_assert((int)UST_COUNT <= (int)fresco::ST_COUNT, "the stage timers hold every stage");

namespace {

template <typename T, int W>
cudaError_t launch_un_interp(const fresco_uwnu_s *u, const EsPoly<T> &ep, cudaStream_t s) {
    const auto *U = (const CxT<T> *)u->U;
    if (u->g.dim == 2)
        k_un_interp_win<T, W><<<u->nb, 256, 0, s>>>(
            u->g, u->tl, ep, u->n_tiles, u->hoff, u->tcell, (const T *)u->tfrac, U,
            (const T *)u->s0, (const T *)u->wq, u->scal, (const T *)u->dq, u->perm,
            (CxT<T> *)u->coef, (T *)u->S, u->part);
    else
        k_un_interp<T, W, 3><<<u->nb, 256, 0, s>>>(
            u->g, ep, u->n_k, u->tcell, (const T *)u->tfrac, U, (const T *)u->s0,
            (const T *)u->wq, u->scal, (const T *)u->dq, u->perm, (CxT<T> *)u->coef, (T *)u->S,
            u->part);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t launch_un_spread(const fresco_uwnu_s *u, const EsPoly<T> &ep, cudaStream_t s) {
    const unsigned nb = (unsigned)std::min<int64_t>(u->n_tiles, 152 * 64);
    if (u->g.dim == 2)
        k_un_spread<T, W, 2><<<nb, 256, 0, s>>>(u->g, u->tl, ep, u->n_tiles, u->toff, u->ent,
                                                u->kcov, u->tcell, (const T *)u->tfrac,
                                                (const CxT<T> *)u->coef, (CxT<T> *)u->U);
    else
        k_un_spread<T, W, 3><<<nb, 256, 0, s>>>(u->g, u->tl, ep, u->n_tiles, u->toff, u->ent,
                                                u->kcov, u->tcell, (const T *)u->tfrac,
                                                (const CxT<T> *)u->coef, (CxT<T> *)u->U);
    return cudaGetLastError();
}

template <typename T>
const EsPoly<T> &un_poly(const fresco_uwnu_s *u) {
    return *reinterpret_cast<const EsPoly<T> *>(sizeof(T) == 4 ? (const void *)&u->p32
                                                                : (const void *)&u->p64);
}

// rho~ at the constraints with S, the loss partials and the strengths (one launch)
template <typename T>
cudaError_t un_interp(const fresco_uwnu_s *u, cudaStream_t s) {
    const EsPoly<T> &ep = un_poly<T>(u);
    FRESCO_WIDTH_SWITCH(u->width, return (launch_un_interp<T, WW>(u, ep, s)));
}

// the strengths onto every tile of U (one launch)
template <typename T>
cudaError_t un_spread(const fresco_uwnu_s *u, cudaStream_t s) {
    const EsPoly<T> &ep = un_poly<T>(u);
    FRESCO_WIDTH_SWITCH(u->width, return (launch_un_spread<T, WW>(u, ep, s)));
}

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
    u->prof.release();
    if (u->have_fft) cufftDestroy(u->fft);
    for (void *p : u->allocs) cudaFree(p);
    delete u;
}

// Builds the constraint side of a plan: the deconvolution tables, the kernel polynomials, the
// constraints' fine cells and positions (from FP64), their tile order and the tiles' lists, and
// the FFT plan. dq (point plans; may be null): a factor per constraint in the caller's order.
template <typename T>
fresco_status un_build(fresco_uwnu_s *u, const double *nu, const double *S0, const double *W,
                       const double *dq) {
    using C2 = CxT<T>;
    const UGrid &g = u->g;
    const int dim = g.dim;
    const int64_t nk = u->n_k;
    const int w = u->width;
    u->tl = utiles_for(dim, g.nf);
    const UTiles &tl = u->tl;
    u->n_tiles = (int64_t)tl.nt[0] * tl.nt[1] * tl.nt[2];
    if (dim == 2)   // the window interpolation: a block per home tile (up to kUWinBlocks)
        u->nb = (int)std::max<int64_t>(1, std::min<int64_t>(u->n_tiles, kUWinBlocks));
    fresco::es_poly_table(w, u->beta, u->p32);
    fresco::es_poly_table(w, u->beta, u->p64);

    // fine cell and fraction of every target x = -nu / M (modulo 1), in the caller's order
    std::vector<int> cell((size_t)(nk * dim));
    std::vector<double> frac((size_t)(nk * dim));
    for (int64_t q = 0; q < nk; ++q)
        for (int a = 0; a < dim; ++a) {
            const double x = -nu[q * dim + a] / (double)g.M[a];
            const double t = (x - std::floor(x)) * (double)g.nf[a];
            const double c = std::floor(t);
            int64_t ci = (int64_t)c % g.nf[a];
            if (ci < 0) ci += g.nf[a];
            cell[(size_t)(q * dim + a)] = (int)ci;
            frac[(size_t)(q * dim + a)] = t - c;
        }
    // tile order, the tiles' lists and their cover counts (fresco_uwnu_tiles.h)
    UTilePlan tp;
    if (!build_utile_plan<T>(dim, g.nf, w, tl, cell.data(), frac.data(), nk, tp))
        return FRESCO_ERR_UNSUPPORTED;
    u->n_ent = tp.n_ent;
    const std::vector<int> &perm = tp.perm;
    const std::vector<int64_t> &hoff = tp.hoff, &toff = tp.toff;
    const std::vector<int> &ent = tp.ent, &kcov = tp.kcov;
    std::vector<int> scell((size_t)(nk * dim));
    std::vector<T> sfrac((size_t)(nk * dim)), s0((size_t)nk), wq((size_t)nk), sdq;
    if (dq) sdq.resize((size_t)nk);
    for (int64_t i = 0; i < nk; ++i) {
        const int64_t q = perm[(size_t)i];
        for (int a = 0; a < dim; ++a) {
            scell[(size_t)(i * dim + a)] = cell[(size_t)(q * dim + a)];
            sfrac[(size_t)(i * dim + a)] = (T)frac[(size_t)(q * dim + a)];
        }
        s0[(size_t)i] = (T)S0[q];
        wq[(size_t)i] = (T)W[q];
        if (dq) sdq[(size_t)i] = (T)dq[q];
    }

    bool ok = un_alloc(u, (void **)&u->perm, sizeof(int) * (size_t)nk) &&
              un_alloc(u, (void **)&u->tcell, sizeof(int) * (size_t)(nk * dim)) &&
              un_alloc(u, &u->tfrac, sizeof(T) * (size_t)(nk * dim)) &&
              un_alloc(u, &u->s0, sizeof(T) * (size_t)nk) &&
              un_alloc(u, &u->wq, sizeof(T) * (size_t)nk) &&
              (!dq || un_alloc(u, &u->dq, sizeof(T) * (size_t)nk)) &&
              un_alloc(u, &u->S, sizeof(T) * (size_t)nk) &&
              un_alloc(u, &u->coef, sizeof(C2) * (size_t)nk) &&
              un_alloc(u, &u->U, sizeof(C2) * (size_t)u->fine) &&
              un_alloc(u, (void **)&u->hoff, sizeof(int64_t) * hoff.size()) &&
              un_alloc(u, (void **)&u->toff, sizeof(int64_t) * toff.size()) &&
              un_alloc(u, (void **)&u->ent, sizeof(int) * ent.size()) &&
              un_alloc(u, (void **)&u->kcov, sizeof(int) * kcov.size()) &&
              un_alloc(u, (void **)&u->part, sizeof(double) * 2 * std::max(kUBlocks, u->nb)) &&
              un_alloc(u, (void **)&u->scal, sizeof(double) * 4);
    for (int a = 0; a < 3 && ok; ++a)
        ok = un_alloc(u, &u->ip[a], sizeof(T) * (size_t)(g.M[a] / 2 + 1));
    if (!ok) return FRESCO_ERR_OOM;
    for (int a = 0; a < 3; ++a) {   // deconvolution tables (axes beyond dim: the single entry 1)
        const int64_t n_nu = g.M[a] / 2 + 1;
        std::vector<double> psi((size_t)n_nu, 1.0);
        if (a < dim) {
            const fresco_status st = fresco_kernel_ft(w, u->beta, g.nf[a], n_nu, psi.data());
            if (st) return st;
        }
        std::vector<T> ipt((size_t)n_nu);
        for (int64_t i = 0; i < n_nu; ++i) ipt[(size_t)i] = (T)(1.0 / psi[(size_t)i]);
        UN_CUDA(cudaMemcpy(u->ip[a], ipt.data(), sizeof(T) * ipt.size(), cudaMemcpyHostToDevice));
    }
    UN_CUDA(cudaMemcpy(u->perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->tcell, scell.data(), sizeof(int) * scell.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->tfrac, sfrac.data(), sizeof(T) * sfrac.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->s0, s0.data(), sizeof(T) * s0.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->wq, wq.data(), sizeof(T) * wq.size(), cudaMemcpyHostToDevice));
    if (dq) UN_CUDA(cudaMemcpy(u->dq, sdq.data(), sizeof(T) * sdq.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->hoff, hoff.data(), sizeof(int64_t) * hoff.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->toff, toff.data(), sizeof(int64_t) * toff.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->ent, ent.data(), sizeof(int) * ent.size(), cudaMemcpyHostToDevice));
    UN_CUDA(cudaMemcpy(u->kcov, kcov.data(), sizeof(int) * kcov.size(), cudaMemcpyHostToDevice));
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
    {   // rho0 = sum c^2; type 2: the weights over Psi onto U, inverse FFT
        fresco::StageScope sc(u->prof, s, UST_TYPE2);
        k_un_sumsq<T><<<kUBlocks, 256, 0, s>>>(c, u->cells, u->part);
        k_un_sum<<<1, 256, 0, s>>>(u->part, kUBlocks, 1, u->scal);
        UN_CUDA(cudaMemsetAsync(u->U, 0, sizeof(C2) * (size_t)u->fine, s));
        k_un_fill<T><<<pb, 256, 0, s>>>(g, u->cells, c, ip0, ip1, ip2, (C2 *)u->U);
        const fresco_status st = un_fft<T>(u, CUFFT_INVERSE);
        if (st) return st;
    }
    {   // rho~ at the constraints, with S, the loss and the type-1 strengths
        fresco::StageScope sc(u->prof, s, UST_INTERP);
        UN_CUDA(un_interp<T>(u, s));
        k_un_sum<<<1, 256, 0, s>>>(u->part, u->nb, 2, u->scal + 1);
        UN_CUDA(cudaMemcpyAsync(loss, u->scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    u->launches += 5;
    u->evaluated = true;
    if (!grad) return un_status(cudaGetLastError());
    {   // type 1: the strengths onto U
        fresco::StageScope sc(u->prof, s, UST_SPREAD);
        UN_CUDA(un_spread<T>(u, s));
    }
    {   // forward FFT, then the weight gradient
        fresco::StageScope sc(u->prof, s, UST_TYPE1);
        const fresco_status st = un_fft<T>(u, CUFFT_FORWARD);
        if (st) return st;
        k_un_grad<T><<<pb, 256, 0, s>>>(g, u->cells, c, ip0, ip1, ip2, (const C2 *)u->U, u->scal,
                                        grad);
    }
    u->launches += 2;
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
    const fresco_status st = o.precision == FRESCO_F64 ? un_build<double>(u, nu, S0, W, nullptr)
                                                       : un_build<float>(u, nu, S0, W, nullptr);
    if (st) {
        un_free(u);
        return st;
    }
    *out = u;
    return FRESCO_OK;
}

fresco_status fresco_uwnu_loss_grad(fresco_uwnu_t u, const void *d_c, double *d_loss,
                                    void *d_grad) {
    fresco::clear_pending_error();
    if (!u || !d_c || !d_loss) return FRESCO_ERR_ARG;
    if (u->precision == FRESCO_F64)
        return un_eval<double>(u, (const double *)d_c, d_loss, (double *)d_grad);
    return un_eval<float>(u, (const float *)d_c, d_loss, (float *)d_grad);
}

fresco_status fresco_uwnu_get_S(fresco_uwnu_t u, void *d_S) {
    fresco::clear_pending_error();
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

fresco_status fresco_uwnu_profile(fresco_uwnu_t u, int enable) {
    if (!u) return FRESCO_ERR_ARG;
    u->prof.on = enable != 0;
    return FRESCO_OK;
}

fresco_status fresco_uwnu_profile_read(fresco_uwnu_t u, double *ms, int64_t *counts) {
    if (!u || !ms) return FRESCO_ERR_ARG;
    UN_CUDA(u->stream ? cudaStreamSynchronize(u->stream) : cudaDeviceSynchronize());
    double all_ms[fresco::ST_COUNT];
    int64_t all_counts[fresco::ST_COUNT];
    u->prof.read(all_ms, all_counts);
    for (int i = 0; i < UST_COUNT; ++i) {
        ms[i] = all_ms[i];
        if (counts) counts[i] = all_counts[i];
    }
    return FRESCO_OK;
}

int64_t fresco_uwnu_launch_count(fresco_uwnu_t u) { return u ? u->launches : 0; }

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
    std::vector<double> dq((size_t)n_k, 1.0);   // 1 / Psi1(theta_q)
    for (int a = 0; a < dim; ++a) {
        for (int64_t q = 0; q < n_k; ++q) {
            theta[(size_t)q] = kvec[q * dim + a] * p->h[a];
            nu[(size_t)(q * dim + a)] = theta[(size_t)q] * (double)u->g.M[a] / (2.0 * kPiU);
        }
        fresco::kernel_ft_at(u->width, u->beta, theta.data(), n_k, psi.data());
        for (int64_t q = 0; q < n_k; ++q) dq[(size_t)q] /= psi[(size_t)q];
    }
    fresco_status st = un_build<T>(u, nu.data(), S0, W, dq.data());
    if (st) return st;
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
    fresco_status st;
    {   // the points onto their grid; the grid keeps spare cells beyond the box, so half a cell
        // of slack (FP32 coordinates of points on a face may round just outside it) changes nothing
        fresco::StageScope sc(u->prof, s, UST_POINT_SPREAD);
        k_nu_bounds<T><<<(unsigned)std::min<int64_t>((p->n_points + 255) / 256, 152 * 8), 256, 0,
                         s>>>(pts, p->n_points, p->dim, 0.5 * (p->box[0] + p->h[0]),
                              0.5 * (p->box[1] + p->h[1]), 0.5 * (p->box[2] + p->h[2]),
                              p->ps.err);
        st = fresco::point_side_spread<T>(p->ps, pts, s, &p->launches);
        if (st) return st;
    }
    {   // type 2 of the spread grid: onto U, inverse FFT
        fresco::StageScope sc(u->prof, s, UST_TYPE2);
        UN_CUDA(cudaMemsetAsync(u->U, 0, sizeof(C2) * (size_t)u->fine, s));
        k_nu_fill<T><<<pb, 256, 0, s>>>(g, p->cells, (const T *)p->ps.grid, ip0, ip1, ip2,
                                        (C2 *)u->U);
        st = un_fft<T>(u, CUFFT_INVERSE);
        if (st) return st;
    }
    {   // at the wavevectors: S, the loss and the type-1 strengths
        fresco::StageScope sc(u->prof, s, UST_INTERP);
        UN_CUDA(un_interp<T>(u, s));
        k_un_sum<<<1, 256, 0, s>>>(u->part, u->nb, 1, u->scal + 1);
        UN_CUDA(cudaMemcpyAsync(loss, u->scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    p->launches += 4;
    u->evaluated = true;
    if (!grad) return un_status(cudaGetLastError());
    {   // type 1 of the strengths onto U
        fresco::StageScope sc(u->prof, s, UST_SPREAD);
        UN_CUDA(un_spread<T>(u, s));
    }
    {   // forward FFT, the field on the points' grid
        fresco::StageScope sc(u->prof, s, UST_TYPE1);
        st = un_fft<T>(u, CUFFT_FORWARD);
        if (st) return st;
        k_nu_field<T><<<pb, 256, 0, s>>>(g, p->cells, ip0, ip1, ip2, (const C2 *)u->U,
                                         (T *)p->ps.grid);
    }
    {   // the kernel-derivative interpolation at the points
        fresco::StageScope sc(u->prof, s, UST_POINT_INTERP);
        const double dscale[3] = {-2.0 / p->h[0], -2.0 / p->h[1], -2.0 / p->h[2]};
        const EsPoly<T> &ep = *reinterpret_cast<const EsPoly<T> *>(
            sizeof(T) == 4 ? (const void *)&p->ps.p32 : (const void *)&p->ps.p64);
        UN_CUDA(Launch<T>::interp_kd(p->ps.g, ep, p->ps.sorted, p->ps.perm, p->ps.tr,
                                     (const T *)p->ps.grid, nullptr, dscale, grad, s));
    }
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
    fresco::clear_pending_error();
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

fresco_status fresco_nuwnu_profile(fresco_nuwnu_t p, int enable) {
    if (!p) return FRESCO_ERR_ARG;
    return fresco_uwnu_profile(p->c, enable);
}

fresco_status fresco_nuwnu_profile_read(fresco_nuwnu_t p, double *ms, int64_t *counts) {
    if (!p) return FRESCO_ERR_ARG;
    return fresco_uwnu_profile_read(p->c, ms, counts);
}

}  // extern "C"
