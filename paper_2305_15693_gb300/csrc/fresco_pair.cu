// Repulsive pair term of the hybrid loss (Eq. 6): E = sum_{m<n} U(|r_m - r_n|), minimum image in
// the periodic box, U(r) = (eps / alpha)(1 - r / sigma)^alpha for r < sigma (alpha = 2.5 is the
// Hertzian potential of Eq. 6, alpha = 2 the harmonic soft sphere), evaluated with a cell list:
// cells at least sigma wide, points counting-sorted by cell, each point scanning its own and the
// neighbouring cells (a finite-ranged potential keeps the cost O(N), as the text after Eq. 6 notes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "fresco.h"
#include "fresco_internal.h"

namespace {

constexpr int kPairBlocks = 2048;

struct PairGeom {
    int dim;
    int nc[3];          // cells per axis
    int nd[3];          // distinct neighbour offsets per axis: 1 (nc = 1), 2 (nc = 2) or 3
    double box[3];
    int64_t n;
    double sigma, eps, alpha;
};

template <typename T>
__device__ __forceinline__ T wrap_coord(T r, T L) {
    T x = r - L * floor(r / L);
    if (x >= L) x -= L;
    if (x < T(0)) x = T(0);
    return x;
}

template <typename T, int D>
__device__ __forceinline__ int cell_of(const T (&x)[3], const PairGeom &g, int (&c)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c[a] = 0;
        if (a < D) {
            int v = (int)(x[a] * (T)g.nc[a] / (T)g.box[a]);
            c[a] = v < 0 ? 0 : (v >= g.nc[a] ? g.nc[a] - 1 : v);
        }
    }
    return c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_cell_bin(PairGeom g, const T *__restrict__ pts,
                                                  int *__restrict__ cnt, int *__restrict__ key,
                                                  int *__restrict__ slot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.n; j += stride) {
        T x[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = wrap_coord<T>(pts[j * D + a], (T)g.box[a]);
        int c[3];
        const int lin = cell_of<T, D>(x, g, c);
        key[j] = lin;
        slot[j] = atomicAdd(&cnt[lin], 1);
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_cell_scatter(PairGeom g, const T *__restrict__ pts,
                                                      const int *__restrict__ key,
                                                      const int *__restrict__ slot,
                                                      const int *__restrict__ off,
                                                      T *__restrict__ sorted,
                                                      int *__restrict__ perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.n; j += stride) {
        const int64_t pos = (int64_t)off[key[j]] + slot[j];
#pragma unroll
        for (int a = 0; a < D; ++a) sorted[pos * D + a] = wrap_coord<T>(pts[j * D + a], (T)g.box[a]);
        perm[pos] = (int)j;
    }
}

// one thread per (sorted) point: scan its cell and the neighbouring ones; every pair is seen
// from both ends, so each end books half of the pair energy and its own force
template <typename T, int D>
__global__ void __launch_bounds__(256) k_pair(PairGeom g, const T *__restrict__ sorted,
                                              const int *__restrict__ perm,
                                              const int *__restrict__ off, int accumulate,
                                              T *__restrict__ grad, double *__restrict__ partial) {
    __shared__ double ws[8];
    double e = 0.0;
    const T sig = (T)g.sigma, inv_sig = T(1) / sig, sig2 = sig * sig;
    const T eps = (T)g.eps, alpha = (T)g.alpha;
    const bool harmonic = g.alpha == 2.0, hertz = g.alpha == 2.5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
        T x[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = sorted[i * D + a];
        int c[3];
        cell_of<T, D>(x, g, c);
        T f[3] = {T(0), T(0), T(0)};
        const int zl = D == 3 ? g.nd[2] : 1;
        for (int oz = 0; oz < zl; ++oz)
            for (int oy = 0; oy < g.nd[1]; ++oy)
                for (int ox = 0; ox < g.nd[0]; ++ox) {
                    const int o[3] = {ox, oy, oz};
                    int cc[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (a >= D) { cc[a] = 0; continue; }
                        // offsets -1, 0, +1 (only the distinct ones when nc < 3)
                        int d = g.nd[a] == 1 ? 0 : (g.nd[a] == 2 ? o[a] : o[a] - 1);
                        int v = c[a] + d;
                        v += v < 0 ? g.nc[a] : (v >= g.nc[a] ? -g.nc[a] : 0);
                        cc[a] = v;
                    }
                    const int lin = cc[0] + g.nc[0] * (cc[1] + g.nc[1] * cc[2]);
                    const int q0 = off[lin], q1 = off[lin + 1];
                    for (int q = q0; q < q1; ++q) {
                        if (q == i) continue;
                        T dx[3] = {T(0), T(0), T(0)};
                        T r2 = T(0);
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            T v = x[a] - sorted[(int64_t)q * D + a];
                            const T L = (T)g.box[a];
                            v -= L * rint(v / L);
                            dx[a] = v;
                            r2 = fma(v, v, r2);
                        }
                        if (r2 >= sig2 || r2 <= T(0)) continue;
                        const T r = sqrt(r2);
                        const T u = T(1) - r * inv_sig;
                        T up;   // u^(alpha - 1)
                        if (harmonic) up = u;
                        else if (hertz) up = u * sqrt(u);
                        else up = pow(u, alpha - T(1));
                        e += 0.5 * (double)(eps / alpha * up * u);
                        const T coef = -eps * inv_sig * up / r;
#pragma unroll
                        for (int a = 0; a < D; ++a) f[a] = fma(coef, dx[a], f[a]);
                    }
                }
        const int64_t j = perm[i];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (accumulate) grad[j * D + a] += f[a];
            else grad[j * D + a] = f[a];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) k_pair_final(const double *__restrict__ partial, int nb,
                                                    int accumulate, double *__restrict__ energy) {
    __shared__ double sm[256];
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) v += partial[i];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *energy = accumulate ? *energy + sm[0] : sm[0];
}

}  // namespace

struct fresco_pair_s {
    PairGeom g{};
    int precision = FRESCO_F32;
    size_t es = 4;
    cudaStream_t stream = nullptr;
    int64_t ncell = 0;
    int *cnt = nullptr, *off = nullptr, *bsum = nullptr, *key = nullptr, *slot = nullptr;
    int *perm = nullptr;
    void *sorted = nullptr;
    double *partial = nullptr;
    int n_blocks = 0;
};

namespace {

void pair_free(fresco_pair_s *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    void *b[] = {p->cnt, p->off, p->bsum, p->key, p->slot, p->perm, p->sorted, p->partial};
    for (void *x : b)
        if (x) cudaFree(x);
    delete p;
}

template <typename T>
fresco_status pair_eval(fresco_pair_s *p, const void *pts, double *energy, void *grad,
                        int accumulate) {
    const PairGeom &g = p->g;
    cudaStream_t s = p->stream;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + 255) / 256, 152 * 16));
    if (cudaMemsetAsync(p->cnt, 0, sizeof(int) * (size_t)p->ncell, s) != cudaSuccess)
        return FRESCO_ERR_CUDA;
    if (g.dim == 2)
        k_cell_bin<T, 2><<<grid, 256, 0, s>>>(g, (const T *)pts, p->cnt, p->key, p->slot);
    else
        k_cell_bin<T, 3><<<grid, 256, 0, s>>>(g, (const T *)pts, p->cnt, p->key, p->slot);
    int nl = 0;
    if (fresco::Launch<float>::scan(p->cnt, p->off, p->bsum, p->ncell, s, &nl) != cudaSuccess)
        return FRESCO_ERR_CUDA;
    if (g.dim == 2) {
        k_cell_scatter<T, 2><<<grid, 256, 0, s>>>(g, (const T *)pts, p->key, p->slot, p->off,
                                                  (T *)p->sorted, p->perm);
        k_pair<T, 2><<<p->n_blocks, 256, 0, s>>>(g, (const T *)p->sorted, p->perm, p->off,
                                                 accumulate, (T *)grad, p->partial);
    } else {
        k_cell_scatter<T, 3><<<grid, 256, 0, s>>>(g, (const T *)pts, p->key, p->slot, p->off,
                                                  (T *)p->sorted, p->perm);
        k_pair<T, 3><<<p->n_blocks, 256, 0, s>>>(g, (const T *)p->sorted, p->perm, p->off,
                                                 accumulate, (T *)grad, p->partial);
    }
    k_pair_final<<<1, 256, 0, s>>>(p->partial, p->n_blocks, accumulate, energy);
    return cudaGetLastError() == cudaSuccess ? FRESCO_OK : FRESCO_ERR_CUDA;
}

}  // namespace

extern "C" {

fresco_status fresco_pair_plan(fresco_pair_t *out, int dim, const double *box, int64_t n_points,
                               double sigma, double eps, double alpha, int precision,
                               void *stream) {
    if (!out) return FRESCO_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !box || n_points < 1 || n_points > 2147483647LL ||
        !(sigma > 0.0) || !(eps >= 0.0) || !(alpha > 1.0) || !std::isfinite(alpha) ||
        (precision != FRESCO_F32 && precision != FRESCO_F64))
        return FRESCO_ERR_ARG;
    PairGeom g{};
    g.dim = dim;
    g.n = n_points;
    g.sigma = sigma;
    g.eps = eps;
    g.alpha = alpha;
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < dim) {
            if (!(box[a] > 0.0) || !std::isfinite(box[a])) return FRESCO_ERR_ARG;
            if (!(sigma < 0.5 * box[a])) return FRESCO_ERR_UNSUPPORTED;   // minimum image
            double nc = std::floor(box[a] / sigma);
            if (nc > 4096.0) nc = 4096.0;
            g.nc[a] = (int)nc;
            g.nd[a] = g.nc[a] >= 3 ? 3 : g.nc[a];
            g.box[a] = box[a];
        } else {
            g.nc[a] = 1;
            g.nd[a] = 1;
            g.box[a] = 1.0;
        }
        ncell *= g.nc[a];
    }
    if (ncell >= 2147483647LL) return FRESCO_ERR_UNSUPPORTED;
    fresco_pair_s *p = new (std::nothrow) fresco_pair_s();
    if (!p) return FRESCO_ERR_OOM;
    p->g = g;
    p->precision = precision;
    p->es = precision == FRESCO_F64 ? 8 : 4;
    p->stream = (cudaStream_t)stream;
    p->ncell = ncell;
    p->n_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n_points + 255) / 256, kPairBlocks));
    auto A = [](void **q, size_t b) {
        if (cudaMalloc(q, b) != cudaSuccess) {
            cudaGetLastError();
            *q = nullptr;
            return false;
        }
        return true;
    };
    const size_t N = (size_t)n_points;
    bool ok = A((void **)&p->cnt, sizeof(int) * ncell) &&
              A((void **)&p->off, sizeof(int) * (ncell + 1)) &&
              A((void **)&p->bsum, sizeof(int) * ((ncell + 1023) / 1024 + 1)) &&
              A((void **)&p->key, sizeof(int) * N) && A((void **)&p->slot, sizeof(int) * N) &&
              A((void **)&p->perm, sizeof(int) * N) && A(&p->sorted, p->es * N * dim) &&
              A((void **)&p->partial, sizeof(double) * p->n_blocks);
    if (!ok) {
        pair_free(p);
        return FRESCO_ERR_OOM;
    }
    *out = p;
    return FRESCO_OK;
}

fresco_status fresco_pair_energy_grad(fresco_pair_t p, const void *d_points, double *d_energy,
                                      void *d_grad, int accumulate) {
    fresco::clear_pending_error();
    if (!p || !d_points || !d_energy || !d_grad) return FRESCO_ERR_ARG;
    if (p->precision == FRESCO_F64) return pair_eval<double>(p, d_points, d_energy, d_grad, accumulate);
    return pair_eval<float>(p, d_points, d_energy, d_grad, accumulate);
}

fresco_status fresco_pair_set_stream(fresco_pair_t p, void *stream) {
    if (!p) return FRESCO_ERR_ARG;
    p->stream = (cudaStream_t)stream;
    return FRESCO_OK;
}

fresco_status fresco_pair_destroy(fresco_pair_t p) {
    pair_free(p);
    return FRESCO_OK;
}

}  // extern "C"
