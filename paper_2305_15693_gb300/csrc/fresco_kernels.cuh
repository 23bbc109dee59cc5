// CUDA kernels of libfresco for sm_103a, templated on the working precision T (float / double).
//
// Data layouts (axis 0 = x is contiguous everywhere):
//   points      [N][D] caller order, type T.
//   sorted      one record per point in sub-bin order, words of type U (uint32 for float, uint64
//               for double): word a holds the cell of the point relative to its tile origin in
//               the top 8 bits and the fractional position inside that cell, frac * 2^FB, in the
//               low FB bits (FB = 24 / 56). Float records are 16 bytes {u0, u1, u2 or 0, caller
//               index}; double records are 2 (2D) or 4 (3D) words.
//   perm        [N] sorted position -> caller index (double plans only).
//   off         [n_tiles + 1] first sorted position of each tile.
//   grid        real fine grid [nf2][nf1][nf0].
//   spec        forward half spectrum after the x pass [nf2][nf1][nf0/2 + 1], complex T.
//   specT       its columns x = 0..kx, transposed: [kx + 1][nf2][nf1] ("plane" = nf2 * nf1),
//               transformed over (z, y) in place: specT[n_x][n_z][n_y] is the forward spectrum.
//   hc          transposed compact backward spectrum [2 kx + 2][nf2][nf1]: column c holds
//               n_x = c - kx - 1.
//   g           complex gradient grid [nf2][nf1][nf0]: re = d/dr_x, im = d/dr_y (pipeline 0),
//               re = d/dr_z (pipeline 1, 3D only).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include "fresco_internal.h"

namespace fresco {

template <typename T> struct PT;
template <> struct PT<float> {
    using C = float2;
    using U = uint32_t;
    static constexpr int FB = 24;
};
template <> struct PT<double> {
    using C = double2;
    using U = uint64_t;
    static constexpr int FB = 56;
};

// ---------------------------------------------------------------------------------------------
// Fine-grid coordinate t = r * n_f / L of one coordinate, split into a cell index in [0, n_f)
// and a fraction in [0, 1). The product uses the two-term scale s_hi + s_lo and an fma residual,
// so the fraction is accurate to the working precision even when t is large (for n_f = 25000
// in float a plain product would carry ~1e-3 cells of error).
template <typename T>
__device__ __forceinline__ bool fine_coord(T r, T s_hi, T s_lo, int nf, int &cell, T &frac) {
    bool ok = isfinite(r);
    if (!ok) r = T(0);
    T p = r * s_hi;
    T e = fma(r, s_hi, -p);
    T lo = fma(r, s_lo, e);
    T c = floor(p);
    T f = (p - c) + lo;
    if (f < T(0)) { c -= T(1); f += T(1); }
    if (f >= T(1)) { c += T(1); f -= T(1); }
    frac = f;
    if (c >= T(0) && c < T(nf)) {   // a point inside the box: no wrap (the common case)
        cell = (int)c;
        return ok;
    }
    long long ci = (long long)c;
    ci %= nf;
    if (ci < 0) ci += nf;
    cell = (int)ci;
    return ok;
}

template <typename T>
__device__ __forceinline__ typename PT<T>::U pack_coord(int rel, T frac) {
    using U = typename PT<T>::U;
    const T scale = T((U)1 << PT<T>::FB);
    return ((U)rel << PT<T>::FB) | (U)(frac * scale);
}

template <typename T>
__device__ __forceinline__ void unpack_coord(typename PT<T>::U u, int &rel, T &frac) {
    using U = typename PT<T>::U;
    rel = (int)(u >> PT<T>::FB);
    const U m = ((U)1 << PT<T>::FB) - 1;
    frac = T(u & m) * (T(1) / T((U)1 << PT<T>::FB));
}

// Sorted records. Float plans store one 16-byte record per point, {u0, u1, u2 (3D) or 0, caller
// index}, so the scatter costs one partial-sector write per point; double plans store D (2D) or
// 4 (3D) 64-bit words and keep the caller index in the separate perm array.
template <typename T, int D>
__device__ __forceinline__ void load_packed(const typename PT<T>::U *__restrict__ s, int64_t p,
                                            typename PT<T>::U (&u)[3]) {
    if constexpr (sizeof(T) == 4) {
        const uint4 v = reinterpret_cast<const uint4 *>(s)[p];
        u[0] = v.x; u[1] = v.y; u[2] = v.z;
    } else if constexpr (D == 2) {
        ulonglong2 v = reinterpret_cast<const ulonglong2 *>(s)[p];
        u[0] = v.x; u[1] = v.y; u[2] = 0;
    } else {
        ulonglong2 v0 = reinterpret_cast<const ulonglong2 *>(s)[2 * p];
        ulonglong2 v1 = reinterpret_cast<const ulonglong2 *>(s)[2 * p + 1];
        u[0] = v0.x; u[1] = v0.y; u[2] = v1.x;
    }
}

// as load_packed, plus the caller index of the point
template <typename T, int D>
__device__ __forceinline__ int load_record(const typename PT<T>::U *__restrict__ s,
                                           const int *__restrict__ perm, int64_t p,
                                           typename PT<T>::U (&u)[3]) {
    if constexpr (sizeof(T) == 4) {
        const uint4 v = reinterpret_cast<const uint4 *>(s)[p];
        u[0] = v.x; u[1] = v.y; u[2] = v.z;
        return (int)v.w;
    } else {
        load_packed<T, D>(s, p, u);
        return perm[p];
    }
}

template <typename T, int D>
__device__ __forceinline__ void store_record(typename PT<T>::U *__restrict__ s,
                                             int *__restrict__ perm, int64_t p,
                                             const typename PT<T>::U (&u)[3], int j) {
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<uint4 *>(s)[p] = make_uint4(u[0], u[1], D == 3 ? u[2] : 0u, (unsigned)j);
    } else if constexpr (D == 2) {
        reinterpret_cast<ulonglong2 *>(s)[p] = make_ulonglong2(u[0], u[1]);
        perm[p] = j;
    } else {
        reinterpret_cast<ulonglong2 *>(s)[2 * p] = make_ulonglong2(u[0], u[1]);
        reinterpret_cast<ulonglong2 *>(s)[2 * p + 1] = make_ulonglong2(u[2], 0ull);
        perm[p] = j;
    }
}

// words of type U per sorted record
template <typename T, int D>
__host__ __device__ constexpr int record_words() {
    return sizeof(T) == 4 ? 4 : (D == 3 ? 4 : 2);
}

// ES kernel weights psi(x1 + k), k = 0..W-1, from the plan's piecewise polynomials in
// tau = 2 (x1 + W/2) - 1 in [-1, 1); coefficients come from the kernel parameter bank.
// psi is even, so the polynomial of interval W-1-k is that of interval k at -tau. With
// p_k(tau) = E_k(s) + tau O_k(s), s = tau^2 (E_k, O_k: the even and odd coefficients of p_k),
// the pair is w[k] = E_k + tau O_k and w[W-1-k] = E_k - tau O_k: one Horner pass in s per pair.
// The middle interval of an odd width is symmetric about tau = 0 (odd part zero to the fit's
// rounding) and takes E only.
template <typename T, int W>
__device__ __forceinline__ void es_weights(const EsPoly<T> &ep, T x1, T (&w)[W]) {
    constexpr int P = PolyDeg<T>::value;
    constexpr int PE = P & ~1, PO = (P & 1) ? P : P - 1;   // highest even / odd power
    const T tau = T(2) * x1 + T(W - 1);
    const T s = tau * tau;
#pragma unroll
    for (int k = 0; k < (W + 1) / 2; ++k) {
        T e = ep.c[k][PE];
#pragma unroll
        for (int j = PE - 2; j >= 0; j -= 2) e = fma(e, s, ep.c[k][j]);
        if (2 * k + 1 == W) {
            w[k] = e;
        } else {
            T o = ep.c[k][PO];
#pragma unroll
            for (int j = PO - 2; j >= 1; j -= 2) o = fma(o, s, ep.c[k][j]);
            w[k] = fma(tau, o, e);
            w[W - 1 - k] = fma(-tau, o, e);
        }
    }
}

// The weights and their derivatives d psi(x1 + k) / d tau; d psi / d x1 = 2 d psi / d tau.
// In the even/odd form above, d/dtau (E + tau O) = 2 tau E'(s) + (O(s) + 2 s O'(s)) and
// d/dtau (E - tau O) = 2 tau E'(s) - (O(s) + 2 s O'(s)) (Horner for each value and its
// s-derivative together).
template <typename T, int W>
__device__ __forceinline__ void es_weights_d(const EsPoly<T> &ep, T x1, T (&w)[W], T (&dw)[W]) {
    constexpr int P = PolyDeg<T>::value;
    constexpr int PE = P & ~1, PO = (P & 1) ? P : P - 1;
    const T tau = T(2) * x1 + T(W - 1);
    const T s = tau * tau, s2 = s + s, tau2 = tau + tau;
#pragma unroll
    for (int k = 0; k < (W + 1) / 2; ++k) {
        T e = ep.c[k][PE], de = T(0);
#pragma unroll
        for (int j = PE - 2; j >= 0; j -= 2) {
            de = fma(de, s, e);
            e = fma(e, s, ep.c[k][j]);
        }
        const T a = tau2 * de;
        if (2 * k + 1 == W) {
            w[k] = e;
            dw[k] = a;
        } else {
            T o = ep.c[k][PO], dO = T(0);
#pragma unroll
            for (int j = PO - 2; j >= 1; j -= 2) {
                dO = fma(dO, s, o);
                o = fma(o, s, ep.c[k][j]);
            }
            const T b = fma(s2, dO, o);
            w[k] = fma(tau, o, e);
            w[W - 1 - k] = fma(-tau, o, e);
            dw[k] = a + b;
            dw[W - 1 - k] = a - b;
        }
    }
}

// Start of the kernel support (first cell) relative to the cell holding the point, and the
// offset x1 = start - t in [-W/2, -W/2 + 1).
template <typename T, int W>
__device__ __forceinline__ int support_start(T frac, T &x1) {
    T c = ceil(frac - T(0.5) * T(W));
    x1 = c - frac;
    return (int)c;
}

// ---------------------------------------------------------------------------------------------
// Sub-bin part of a tile-relative cell along one axis: 0 for the low border strip (cells whose
// kernel support can reach the previous tile), 2 for the high border strip (support can reach
// the next tile), 1 otherwise; always 1 when the axis's tiles are narrower than w.
__device__ __forceinline__ int strip_part(int rel, int wd, int w, int strips) {
    if (!strips) return 1;
    if (rel < w / 2) return 0;
    if (rel >= wd - (w + 1) / 2) return 2;
    return 1;
}

// K1b: exclusive prefix sum of the tile counts, in three passes over blocks of 1024. With a guard
// (not null) the passes do nothing unless *guard != 0.
static __global__ void __launch_bounds__(1024) k_scan_blocks(const int *__restrict__ cnt,
                                                      int *__restrict__ off,
                                                      int *__restrict__ bsum, int64_t n,
                                                      const int *__restrict__ guard) {
    if (guard && !*guard) return;
    __shared__ int warp_tot[32];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    int v = (i < n) ? cnt[i] : 0;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    int incl = x + (wid > 0 ? warp_tot[wid - 1] : 0);
    if (i < n) off[i] = incl - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

static __global__ void __launch_bounds__(1024) k_scan_sums(int *__restrict__ bsum, int64_t nb,
                                                    int *__restrict__ off_end,
                                                    const int *__restrict__ guard) {
    if (guard && !*guard) return;
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        int v = (i < nb) ? bsum[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        int incl = x + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (i < nb) bsum[i] = carry + incl - v;  // exclusive
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *off_end = carry;
}

static __global__ void __launch_bounds__(1024) k_scan_add(int *__restrict__ off,
                                                   const int *__restrict__ bsum, int64_t n,
                                                   int *__restrict__ cur,
                                                   const int *__restrict__ guard) {
    if (guard && !*guard) return;
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) {
        const int v = off[i] + bsum[blockIdx.x];
        off[i] = v;
        if (cur) cur[i] = v;
    }
}

// Largest i with first[i] <= v (first is ascending, first[0] = 0).
__device__ __forceinline__ int find_segment(const int64_t *__restrict__ first, int n, int64_t v) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched K1a / K1c: the points of all instances, packed in instance order; each point finds its
// instance by binary search over the first-point offsets and bins with that instance's geometry
// into the instance's own range of sub-bins.
template <typename T, int D>
__device__ __forceinline__ int bin_point(const Geom &g, const T *__restrict__ p, bool &ok) {
    int t[3] = {0, 0, 0}, part[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int cell;
        T frac;
        ok &= fine_coord<T>(p[a], (T)g.s_hi[a], (T)g.s_lo[a], g.nf[a], cell, frac);
        t[a] = tile_of_cell(cell, g.tq[a], g.tr[a], g.tinv[a]);
        const int st = tile_start(t[a], g.tq[a], g.tr[a]);
        const int wd = tile_start(t[a] + 1, g.tq[a], g.tr[a]) - st;
        part[a] = strip_part(cell - st, wd, g.width, g.strips[a]);
    }
    const int lin = t[0] + g.nb[0] * (t[1] + g.nb[1] * t[2]);
    return lin * g.sub + (part[0] + 3 * part[1] + 9 * part[2]);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_bin_b(const BInst *__restrict__ inst,
                                               const int64_t *__restrict__ pt_first, int n_inst,
                                               int64_t n_points, const T *__restrict__ pts,
                                               int *__restrict__ cnt, int *__restrict__ key,
                                               int *__restrict__ slot, int *__restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool ok = true;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_points; j += stride) {
        const int i = find_segment(pt_first, n_inst, j);
        const BInst &I = inst[i];
        const int bin = (int)I.bo + bin_point<T, D>(I.g, pts + j * D, ok);
        key[j] = bin;
        slot[j] = atomicAdd(&cnt[bin], 1);
    }
    if (!ok) atomicOr(err, 1);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_scatter_b(const BInst *__restrict__ inst,
                                                   const int64_t *__restrict__ pt_first,
                                                   int n_inst, int64_t n_points,
                                                   const T *__restrict__ pts,
                                                   const int *__restrict__ key,
                                                   const int *__restrict__ slot,
                                                   const int *__restrict__ off,
                                                   typename PT<T>::U *__restrict__ sorted,
                                                   int *__restrict__ perm) {
    using U = typename PT<T>::U;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_points; j += stride) {
        const int i = find_segment(pt_first, n_inst, j);
        const Geom &g = inst[i].g;
        const int bin = key[j];
        const int64_t pos = (int64_t)off[bin] + slot[j];
        const int lin = (bin - (int)inst[i].bo) / g.sub;
        const int tc[3] = {lin % g.nb[0], (lin / g.nb[0]) % g.nb[1], lin / (g.nb[0] * g.nb[1])};
        U u[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int cell;
            T frac;
            fine_coord<T>(pts[j * D + a], (T)g.s_hi[a], (T)g.s_lo[a], g.nf[a], cell, frac);
            u[a] = pack_coord<T>(cell - tile_start(tc[a], g.tq[a], g.tr[a]), frac);
        }
        store_record<T, D>(sorted, perm, pos, u, (int)j);
    }
}

// ---------------------------------------------------------------------------------------------
// K2: type-1 spreading. One block owns one tile of the fine grid: it accumulates, in shared
// memory, the kernel contributions of every point (from its own tile and the 3^D neighbouring
// tiles, periodic images included) that land inside the tile, then writes the tile to the grid
// with plain coalesced stores. Every cell is written exactly once per call: no zero fill of the
// grid and no global atomics.
//
// The block first scans the neighbouring tiles' point lists and compacts the points that reach
// it into a shared list (support start and kernel offsets, already decoded), so the expensive
// weight/accumulate loop runs with full warps.
//
// Float plans accumulate in 32-bit fixed point (shared-memory integer atomics are several times
// faster than float ones on this part): each contribution is rounded to a multiple of 2^-s with
// s chosen per tile from the number P of points that reach the tile, so that P * 2^s < 2^31 and
// no sum can overflow (every weight is at most 1); s is capped at 21 (resolution 4.8e-7). Integer
// sums are order independent, so the float result is bitwise reproducible. A tile reached by more
// points than the shared list holds falls back to float atomics straight from the point lists.
// Double plans always use double atomics.
template <typename T, int W, int D>
__device__ __forceinline__ void spread_point(const EsPoly<T> &ep, int i0x, int i0y, int i0z,
                                             T x1x, T x1y, T x1z, int wdx, int wdy, int wdz,
                                             int sx, int sxy, T *ftile, int *itile, bool fixed,
                                             float fscale) {
    const int i0[3] = {i0x, i0y, i0z};
    const int wd[3] = {wdx, wdy, wdz};
    T wx[W], wy[W];
    es_weights<T, W>(ep, x1x, wx);
    es_weights<T, W>(ep, x1y, wy);
    if constexpr (sizeof(T) == 4 && D == 2) {
        // footprint entirely inside the tile (most points): no per-cell bounds checks
        if (fixed && i0x >= 0 && i0x + W <= wdx && i0y >= 0 && i0y + W <= wdy) {
            int *base = itile + i0y * sx + i0x;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float wys = wy[b] * fscale;
#pragma unroll
                for (int a = 0; a < W; ++a)
                    atomicAdd(base + b * sx + a,
                              __float_as_int(fmaf(wys, wx[a], 12582912.0f)) - 0x4B400000);
            }
            return;
        }
    }
    if constexpr (D == 2) {
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const int yy = i0[1] + b;
            if ((unsigned)yy >= (unsigned)wd[1]) continue;
            if constexpr (sizeof(T) == 4) {
                if (fixed) {
                    int *row = itile + yy * sx;
                    const float wys = wy[b] * fscale;
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        const int xx = i0[0] + a;
                        const int qv = __float_as_int(fmaf(wys, wx[a], 12582912.0f)) - 0x4B400000;
                        if ((unsigned)xx < (unsigned)wd[0] && qv != 0) atomicAdd(row + xx, qv);
                    }
                    continue;
                }
            }
            T *row = ftile + yy * sx;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                const int xx = i0[0] + a;
                if ((unsigned)xx < (unsigned)wd[0]) atomicAdd(row + xx, wy[b] * wx[a]);
            }
        }
    } else {
        T wz[W];
        es_weights<T, W>(ep, x1z, wz);
#pragma unroll 1
        for (int c = 0; c < W; ++c) {
            const int zz = i0[2] + c;
            if ((unsigned)zz >= (unsigned)wd[2]) continue;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const int yy = i0[1] + b;
                if ((unsigned)yy >= (unsigned)wd[1]) continue;
                const T wzy = wz[c] * wy[b];
                if constexpr (sizeof(T) == 4) {
                    if (fixed) {
                        int *row = itile + zz * sxy + yy * sx;
                        const float wzys = wzy * fscale;
#pragma unroll
                        for (int a = 0; a < W; ++a) {
                            const int xx = i0[0] + a;
                            const int qv =
                                __float_as_int(fmaf(wzys, wx[a], 12582912.0f)) - 0x4B400000;
                            if ((unsigned)xx < (unsigned)wd[0] && qv != 0)
                                atomicAdd(row + xx, qv);
                        }
                        continue;
                    }
                }
                T *row = ftile + zz * sxy + yy * sx;
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const int xx = i0[0] + a;
                    if ((unsigned)xx < (unsigned)wd[0]) atomicAdd(row + xx, wzy * wx[a]);
                }
            }
        }
    }
}

// The compacted points of a tile are held in (dynamic) shared memory after the tile itself;
// the list has g.list_cap entries, sized at plan time from the expected points per tile.

__host__ __device__ inline size_t spread_tile_bytes(const Geom &g, size_t esize) {
    size_t cells = (size_t)g.tmax[0] * g.tmax[1] * (g.dim == 3 ? g.tmax[2] : 1);
    size_t b = cells * (esize > 4 ? esize : 4);
    return (b + 15) & ~(size_t)15;
}

template <typename T, int W, int D>
__device__ __forceinline__ void spread_tile(const Geom &g, const EsPoly<T> &ep,
                                            const typename PT<T>::U *__restrict__ sorted,
                                            const int *__restrict__ off, T *__restrict__ grid,
                                            const int64_t t) {
    using U = typename PT<T>::U;
    constexpr int NNB = (D == 3) ? 27 : 9;     // neighbouring tiles, this one included
    constexpr int S = (D == 3) ? 27 : 9;       // sub-bins per tile
    constexpr int MAXR = NNB * S;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    __shared__ int nb_org[NNB][3], nb_tile[NNB];
    __shared__ int r_p0[MAXR], r_start[MAXR + 1], r_q[MAXR];
    __shared__ int s_nr, s_hits, s_edge;
    const int kSpreadList = g.list_cap;
    T *ftile = reinterpret_cast<T *>(sm_raw);
    int *itile = reinterpret_cast<int *>(sm_raw);
    // compacted list: support starts (packed 3 x 10 bits) and kernel offsets per axis
    const size_t tb = spread_tile_bytes(g, sizeof(T));
    T *l_x1 = reinterpret_cast<T *>(sm_raw + tb);                       // [D][kSpreadList]
    int *l_i0 = reinterpret_cast<int *>(sm_raw + tb + sizeof(T) * D * kSpreadList);

    const int tc[3] = {(int)(t % g.nb[0]), (int)((t / g.nb[0]) % g.nb[1]),
                       (int)(t / ((int64_t)g.nb[0] * g.nb[1]))};
    int s[3], wd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            s[a] = tile_start(tc[a], g.tq[a], g.tr[a]);
            wd[a] = tile_start(tc[a] + 1, g.tq[a], g.tr[a]) - s[a];
        } else {
            s[a] = 0;
            wd[a] = 1;
        }
    }
    if (threadIdx.x < NNB) {
        const int q = threadIdx.x;
        const int dd[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
        int nt[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a < D) {
                int b = tc[a] + dd[a], shift = 0;
                if (b < 0) { b += g.nb[a]; shift = -g.nf[a]; }
                else if (b >= g.nb[a]) { b -= g.nb[a]; shift = g.nf[a]; }
                nt[a] = b;
                nb_org[q][a] = tile_start(b, g.tq[a], g.tr[a]) + shift - s[a];
            } else {
                nt[a] = 0;
                nb_org[q][a] = 0;
            }
        }
        nb_tile[q] = nt[0] + g.nb[0] * (nt[1] + g.nb[1] * nt[2]);
    }
    if (threadIdx.x == 0) {
        s_nr = 0;
        s_hits = 0;
        s_edge = 0;
    }
    __syncthreads();

    // 1. candidate ranges: every sub-bin of this tile, and of each neighbour only the border
    //    strips that face this tile
    for (int e = threadIdx.x; e < MAXR; e += blockDim.x) {
        const int q = e / S, sb = e % S;
        const int dd[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
        const int pp[3] = {sb % 3, (sb / 3) % 3, sb / 9};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (g.strips[a]) ok = ok && (dd[a] == 0 || (dd[a] < 0 ? pp[a] == 2 : pp[a] == 0));
        if (ok) {
            const int64_t bin = (int64_t)nb_tile[q] * S + sb;
            const int p0 = off[bin], p1 = off[bin + 1];
            if (p1 > p0) {
                const int r = atomicAdd(&s_nr, 1);
                r_p0[r] = p0;
                r_start[r] = p1 - p0;
                r_q[r] = q;
            }
        }
    }
    __syncthreads();
    const int nr = s_nr;
    if (threadIdx.x < 32) {   // lengths -> exclusive starts, total in r_start[nr]
        int carry = 0;
        for (int base = 0; base < nr; base += 32) {
            const int i = base + threadIdx.x;
            const int v = i < nr ? r_start[i] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if ((int)threadIdx.x >= o) x += y;
            }
            if (i < nr) r_start[i] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (threadIdx.x == 0) r_start[nr] = carry;
    }
    __syncthreads();
    const int total = r_start[nr];

    // candidate e -> (range, point); ranges are few (<= 25 in 2D), binary search over starts
    auto candidate = [&](int e, int &q) -> int {
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (r_start[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        q = r_q[lo];
        return r_p0[lo] + (e - r_start[lo]);
    };

    // 2. compact the candidates that reach this tile (support starts are >= -W and < the tile
    //    width; the packed form stores i0 + W in 10 bits per axis, tile edges are <= 255).
    //    Points whose whole support lies inside the tile go to the front of the list, the others
    //    to the back, so warps run the unchecked and the checked accumulate separately.
    const int lane = threadIdx.x & 31;
    for (int eb = 0; eb < total; eb += blockDim.x) {
        const int e = eb + threadIdx.x;
        bool hit = e < total, inner = true;
        int i0[3] = {0, 0, 0};
        T x1[3] = {T(0), T(0), T(0)};
        if (hit) {
            int q;
            const int p = candidate(e, q);
            U u[3];
            load_packed<T, D>(sorted, p, u);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                int rel;
                T f;
                unpack_coord<T>(u[a], rel, f);
                i0[a] = nb_org[q][a] + rel + support_start<T, W>(f, x1[a]);
                hit = hit && (i0[a] < wd[a]) && (i0[a] + W > 0);
                inner = inner && (i0[a] >= 0) && (i0[a] + W <= wd[a]);
            }
        }
        const unsigned mi = __ballot_sync(0xffffffffu, hit && inner);
        const unsigned me = __ballot_sync(0xffffffffu, hit && !inner);
        int bi = 0, be = 0;
        if (lane == 0) {
            if (mi) bi = atomicAdd(&s_hits, __popc(mi));
            if (me) be = atomicAdd(&s_edge, __popc(me));
        }
        bi = __shfl_sync(0xffffffffu, bi, 0);
        be = __shfl_sync(0xffffffffu, be, 0);
        if (hit) {
            const unsigned lt = (1u << lane) - 1u;
            const int slot = inner ? bi + __popc(mi & lt) : kSpreadList - 1 - (be + __popc(me & lt));
            if (slot >= 0 && slot < kSpreadList) {
                l_i0[slot] = (i0[0] + W) | ((i0[1] + W) << 10) | ((i0[2] + W) << 20);
#pragma unroll
                for (int a = 0; a < D; ++a) l_x1[a * kSpreadList + slot] = x1[a];
            }
        }
    }
    const int sx = wd[0], sxy = wd[0] * wd[1], cells = sxy * wd[2];
    __syncthreads();
    const int n_inner = s_hits, n_edge = s_edge;
    const int hits = n_inner + n_edge;
    const bool listed = hits <= kSpreadList;
    bool fixed = false;
    int sc = 0;
    if constexpr (sizeof(T) == 4) {
        fixed = listed;
        sc = fixed ? min(21, __clz(max(hits, 1)) - 1) : 0;
        for (int i = threadIdx.x; i < cells; i += blockDim.x) itile[i] = 0;
    } else {
        for (int i = threadIdx.x; i < cells; i += blockDim.x) ftile[i] = T(0);
    }
    __syncthreads();
    const float fscale = __int_as_float((127 + sc) << 23);   // 2^sc

    if (listed) {
        // 3. accumulate the compacted points with full warps: interior entries [0, n_inner),
        //    edge entries [kSpreadList - n_edge, kSpreadList)
        for (int k = threadIdx.x; k < hits; k += blockDim.x) {
            const int h = k < n_inner ? k : kSpreadList - hits + k;
            const int pk = l_i0[h];
            const T x1x = l_x1[h], x1y = l_x1[kSpreadList + h];
            const T x1z = D == 3 ? l_x1[(D - 1) * kSpreadList + h] : T(0);
            spread_point<T, W, D>(ep, (pk & 1023) - W, ((pk >> 10) & 1023) - W,
                                  ((pk >> 20) & 1023) - W, x1x, x1y, x1z, wd[0], wd[1], wd[2],
                                  sx, sxy, ftile, itile, fixed, fscale);
        }
    } else {
        // 3'. crowded tile: float atomics straight from the candidate ranges
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int q;
            const int p = candidate(e, q);
            U u[3];
            load_packed<T, D>(sorted, p, u);
            int i0[3] = {0, 0, 0};
            T x1[3] = {T(0), T(0), T(0)};
            bool hit = true;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                int rel;
                T f;
                unpack_coord<T>(u[a], rel, f);
                i0[a] = nb_org[q][a] + rel + support_start<T, W>(f, x1[a]);
                hit = hit && (i0[a] < wd[a]) && (i0[a] + W > 0);
            }
            if (hit)
                spread_point<T, W, D>(ep, i0[0], i0[1], i0[2], x1[0], x1[1], x1[2], wd[0], wd[1],
                                      wd[2], sx, sxy, ftile, itile, false, fscale);
        }
    }
    __syncthreads();
    const float finv = __int_as_float((127 - sc) << 23);     // 2^-sc
    const int nrows = wd[1] * wd[2];
    for (int row = threadIdx.x >> 5; row < nrows; row += blockDim.x >> 5) {
        const int z = D == 3 ? row / wd[1] : 0, y = D == 3 ? row - z * wd[1] : row;
        T *dst = grid + ((int64_t)(s[2] + z) * g.nf[1] + (s[1] + y)) * g.nf[0] + s[0];
        const int i0 = row * sx;
        for (int x = lane; x < sx; x += 32) {
            T v;
            if constexpr (sizeof(T) == 4) v = fixed ? (float)itile[i0 + x] * finv : ftile[i0 + x];
            else v = ftile[i0 + x];
            dst[x] = v;
        }
    }
}

// Batched spread: a persistent grid walks the tiles of every instance of the ensemble.
template <typename T, int W, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_spread_b(
    const BInst *__restrict__ inst, const int64_t *__restrict__ tile_first, int n_inst,
    int64_t n_tiles, EsPoly<T> ep, const typename PT<T>::U *__restrict__ sorted,
    const int *__restrict__ off, T *__restrict__ grid) {
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int i = find_segment(tile_first, n_inst, t);
        const BInst &I = inst[i];
        spread_tile<T, W, D>(I.g, ep, sorted, off + I.bo, grid + I.go, t - tile_first[i]);
        __syncthreads();
    }
}

}  // namespace fresco

#include "fresco_tiles.cuh"

namespace fresco {

// ---------------------------------------------------------------------------------------------
// K4: deconvolve and crop to the mask, S, the loss partial sums and the gradient coefficients.
// For each half-space representative n (n_x >= 0), with ip = 1 / Psi(n):
//   rho = F(n) ip, S = |rho|^2 / N, loss += W' (S - S0')^2 (to FP64 accuracy),
//   E = 4 W' (S - S0') / N, a_d = i k_d E rho (Eq. 4 coefficient, both members of the +-n pair),
//   H[n] = (a_x + i a_y) ip / 2 and H[-n] = (conj a_x + i conj a_y) ip / 2 (pipeline 0),
//   H1[n] = a_z ip / 2, H1[-n] = conj(a_z) ip / 2 (pipeline 1, 3D).
// The inverse FFT of H then gives d/dr_x + i d/dr_y on the grid (before interpolation).
template <typename T, int D>
__device__ __forceinline__ double mask_range(const MaskGeom &m, const int *__restrict__ rep_n,
                                             const T *__restrict__ rep_s0,
                                             const T *__restrict__ rep_w,
                                             const typename PT<T>::C *__restrict__ spec,
                                             const T *__restrict__ ip0, const T *__restrict__ ip1,
                                             const T *__restrict__ ip2,
                                             typename PT<T>::C *__restrict__ hc0,
                                             typename PT<T>::C *__restrict__ hc1, int64_t e0,
                                             int64_t stride) {
    using C = typename PT<T>::C;
    double lsum = 0.0;          // FP64 plans
    float ah = 0.f, al = 0.f;   // FP32 plans: the thread's sum as an unevaluated float pair
    const T inv_n = (T)m.inv_n;
    for (int64_t e = e0; e < m.n_rep; e += stride) {
        const int nx = rep_n[e * D + 0];
        const int ny = rep_n[e * D + 1];
        const int nz = (D == 3) ? rep_n[e * D + 2] : 0;
        const int ry = ny < 0 ? ny + m.nf[1] : ny;
        const int rz = nz < 0 ? nz + m.nf[2] : nz;
        const int64_t row = (int64_t)rz * m.nf[1] + ry;
        const C F = spec[(int64_t)nx * m.plane + row];
        T ip = ip0[nx] * ip1[ny < 0 ? -ny : ny];
        if (D == 3) ip *= ip2[nz < 0 ? -nz : nz];
        const T re = F.x * ip, im = F.y * ip;
        const T S = (re * re + im * im) * inv_n;
        const T wgt = rep_w[e];
        T dt;
        if constexpr (sizeof(T) == 4) {
            // W (S - S0)^2 by error-free transformations: S - S0 exactly as dh + dl, its square
            // and the product with W to about 46 bits, added to the thread's pair; the loss
            // keeps FP64-level accuracy while the narrow FP64 pipe sees one conversion per
            // thread instead of several operations per representative
            float dh, dl;
            two_sum(S, -rep_s0[e], dh, dl);
            const float p = dh * dh;
            const float pl = fmaf(2.f * dh, dl, fmaf(dh, dh, -p));
            const float th = wgt * p;
            const float tl = fmaf(wgt, pl, fmaf(wgt, p, -th));
            float sh, se;
            two_sum(ah, th, sh, se);
            ah = sh;
            al += se + tl;
            dt = dh;
        } else {
            const double d = S - rep_s0[e];
            lsum = fma(wgt * d, d, lsum);
            dt = d;
        }
        const T E = T(4) * wgt * dt * inv_n;
        const T h = T(0.5) * ip * E;
        const T er = re * h, ei = im * h;
        const int my = ny > 0 ? m.nf[1] - ny : -ny;
        const int mz = nz > 0 ? m.nf[2] - nz : -nz;
        const int64_t rowm = (int64_t)mz * m.nf[1] + my;
        if (m.kderiv) {
            // the scalar half spectrum E / Psi at n (and, on the n_x = 0 column, its conjugate at
            // -n, which the real inverse transform along x reads there)
            hc0[(int64_t)nx * m.plane + row] = C{er, ei};
            if (nx == 0) hc0[rowm] = C{er, -ei};
            continue;
        }
        const T kx = (T)(m.kscale[0] * nx), ky = (T)(m.kscale[1] * ny);
        const int64_t cp = (int64_t)(nx + m.kx + 1) * m.plane + row;
        const int64_t cm = (int64_t)(-nx + m.kx + 1) * m.plane + rowm;
        hc0[cp] = C{-er * ky - ei * kx, er * kx - ei * ky};
        hc0[cm] = C{er * ky - ei * kx, -er * kx - ei * ky};
        if (D == 3) {
            const T kz = (T)(m.kscale[2] * nz);
            hc1[cp] = C{-kz * ei, kz * er};
            hc1[cm] = C{-kz * ei, -kz * er};
        }
    }
    if constexpr (sizeof(T) == 4) lsum = (double)ah + (double)al;
    return lsum;
}

// block reduction of FP64 partials (fixed order: deterministic); result in thread 0
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double wsum[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    double b = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += wsum[w];
    return b;
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_mask(MaskGeom m, const int *__restrict__ rep_n,
                                              const T *__restrict__ rep_s0,
                                              const T *__restrict__ rep_w,
                                              const typename PT<T>::C *__restrict__ spec,
                                              const T *__restrict__ ip0, const T *__restrict__ ip1,
                                              const T *__restrict__ ip2,
                                              typename PT<T>::C *__restrict__ hc0,
                                              typename PT<T>::C *__restrict__ hc1,
                                              double *__restrict__ partial) {
    const double lsum = mask_range<T, D>(m, rep_n, rep_s0, rep_w, spec, ip0, ip1, ip2, hc0, hc1,
                                         (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                         (int64_t)gridDim.x * blockDim.x);
    const double b = block_sum(lsum);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// Batched mask: blocks [I.mb0, I.mb1) work on instance I only, so every partial belongs to one
// instance and the per-instance sums stay in a fixed order.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_mask_b(const BInst *__restrict__ inst,
                                                const int64_t *__restrict__ mblk_first, int n_inst,
                                                const int *__restrict__ rep_n,
                                                const T *__restrict__ rep_s0,
                                                const T *__restrict__ rep_w,
                                                const typename PT<T>::C *__restrict__ spec,
                                                const T *__restrict__ ip,
                                                typename PT<T>::C *__restrict__ hc0,
                                                typename PT<T>::C *__restrict__ hc1,
                                                double *__restrict__ partial) {
    const int i = find_segment(mblk_first, n_inst, blockIdx.x);
    const BInst &I = inst[i];
    const int64_t nb = mblk_first[i + 1] - mblk_first[i];
    const int64_t b = blockIdx.x - mblk_first[i];
    const double lsum = mask_range<T, D>(
        I.m, rep_n + I.reo * D, rep_s0 + I.reo, rep_w + I.reo, spec + I.ato, ip + I.ipo[0],
        ip + I.ipo[1], ip + I.ipo[2], hc0 + I.hco, D == 3 ? hc1 + I.hco : hc1,
        b * blockDim.x + threadIdx.x, nb * blockDim.x);
    const double s = block_sum(lsum);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// per-instance second stage: block i sums the partials of instance i in a fixed order
static __global__ void __launch_bounds__(256) k_finalize_b(const BInst *__restrict__ inst,
                                                           const int64_t *__restrict__ mblk_first,
                                                           const double *__restrict__ partial,
                                                           double *__restrict__ losses) {
    const int i = blockIdx.x;
    double v = 0.0;
    for (int64_t k = mblk_first[i] + threadIdx.x; k < mblk_first[i + 1]; k += blockDim.x)
        v += partial[k];
    const double s = block_sum(v);
    if (threadIdx.x == 0) losses[i] = s + inst[i].loss_const;
}

// K5: second-stage loss sum in a fixed order, plus the folding constant.
static __global__ void __launch_bounds__(512) k_finalize(const double *__restrict__ partial, int nb,
                                                  double loss_const, double *__restrict__ loss) {
    __shared__ double sm[512];
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += 512) v += partial[i];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 256; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sm[0] + loss_const;
}

// ---------------------------------------------------------------------------------------------
// K7: type-2 interpolation. One block per tile stages the tile plus a halo of the complex
// gradient grid(s) in shared memory, then every point of the tile sums its W^D kernel-weighted
// cells; the result, scaled by the incoming gradient, goes to the caller's order through perm.
template <typename T, int W, int D>
__device__ __forceinline__ void interp_tile(const Geom &g, const EsPoly<T> &ep,
                                            const typename PT<T>::U *__restrict__ sorted,
                                            const int *__restrict__ perm, const int p0,
                                            const int p1,
                                            const typename PT<T>::C *__restrict__ g0,
                                            const typename PT<T>::C *__restrict__ g1,
                                            const double *__restrict__ grad_out,
                                            T *__restrict__ grad, const int64_t t) {
    using U = typename PT<T>::U;
    using C = typename PT<T>::C;
    extern __shared__ __align__(128) unsigned char sm_raw[];

    const int tc[3] = {(int)(t % g.nb[0]), (int)((t / g.nb[0]) % g.nb[1]),
                       (int)(t / ((int64_t)g.nb[0] * g.nb[1]))};
    constexpr int HL = W / 2;  // halo before the tile; W - HL after it
    int s[3], rw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            s[a] = tile_start(tc[a], g.tq[a], g.tr[a]);
            rw[a] = tile_start(tc[a] + 1, g.tq[a], g.tr[a]) - s[a] + W;
        } else {
            s[a] = 0;
            rw[a] = 1;
        }
    }
    const int rxy = rw[0] * rw[1], cells = rxy * rw[2];
    C *sg0 = reinterpret_cast<C *>(sm_raw);
    T *sg1 = reinterpret_cast<T *>(sm_raw + sizeof(C) * (size_t)cells);
    {   // stage row by row; the staged region is narrower than the grid, so it wraps at most
        // once per axis
        const int lane = threadIdx.x & 31;
        const int nrows = rw[1] * rw[2];
        for (int row = threadIdx.x >> 5; row < nrows; row += blockDim.x >> 5) {
            const int z = D == 3 ? row / rw[1] : 0, y = D == 3 ? row - z * rw[1] : row;
            int gy = s[1] - HL + y, gz = (D == 3) ? s[2] - HL + z : 0;
            gy += gy < 0 ? g.nf[1] : (gy >= g.nf[1] ? -g.nf[1] : 0);
            if (D == 3) gz += gz < 0 ? g.nf[2] : (gz >= g.nf[2] ? -g.nf[2] : 0);
            const int64_t rbase = ((int64_t)gz * g.nf[1] + gy) * g.nf[0];
            for (int x = lane; x < rw[0]; x += 32) {
                int gx = s[0] - HL + x;
                gx += gx < 0 ? g.nf[0] : (gx >= g.nf[0] ? -g.nf[0] : 0);
                const int i = row * rw[0] + x;
                sg0[i] = g0[rbase + gx];
                if (D == 3) sg1[i] = g1[rbase + gx].x;
            }
        }
    }
    __syncthreads();

    const T scale = grad_out ? (T)(*grad_out) : T(1);
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        U u[3];
        const int64_t j = load_record<T, D>(sorted, perm, p, u);
        int i0[3] = {0, 0, 0};
        T x1[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int rel;
            T f;
            unpack_coord<T>(u[a], rel, f);
            i0[a] = rel + support_start<T, W>(f, x1[a]) + HL;
        }
        T wx[W], wy[W];
        es_weights<T, W>(ep, x1[0], wx);
        es_weights<T, W>(ep, x1[1], wy);
        T ax = T(0), ay = T(0), az = T(0);
        if constexpr (D == 2) {
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const C *row = sg0 + (i0[1] + b) * rw[0] + i0[0];
                T rx = T(0), ry = T(0);
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const C v = row[a];
                    rx = fma(wx[a], v.x, rx);
                    ry = fma(wx[a], v.y, ry);
                }
                ax = fma(wy[b], rx, ax);
                ay = fma(wy[b], ry, ay);
            }
            using T2 = typename PT<T>::C;
            reinterpret_cast<T2 *>(grad)[j] = T2{scale * ax, scale * ay};
        } else {
            T wz[W];
            es_weights<T, W>(ep, x1[2], wz);
#pragma unroll 1
            for (int c = 0; c < W; ++c) {
                T px = T(0), py = T(0), pz = T(0);
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const int base = (i0[2] + c) * rxy + (i0[1] + b) * rw[0] + i0[0];
                    T rx = T(0), ry = T(0), rz = T(0);
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        const C v = sg0[base + a];
                        rx = fma(wx[a], v.x, rx);
                        ry = fma(wx[a], v.y, ry);
                        rz = fma(wx[a], sg1[base + a], rz);
                    }
                    px = fma(wy[b], rx, px);
                    py = fma(wy[b], ry, py);
                    pz = fma(wy[b], rz, pz);
                }
                ax = fma(wz[c], px, ax);
                ay = fma(wz[c], py, ay);
                az = fma(wz[c], pz, az);
            }
            grad[j * 3 + 0] = scale * ax;
            grad[j * 3 + 1] = scale * ay;
            grad[j * 3 + 2] = scale * az;
        }
    }
}

// At most 6 resident blocks per SM (the tile and its halo in shared memory allow no more at the
// default tiles), so each thread may hold 40 registers: at the 32 that 8 blocks would impose the
// window loop spills (measured: kernel-derivative interpolation 6.10 -> 5.47 ms in 3D and
// 4.23 -> 4.13 ms in 2D at 1e8 points when the bound went from 8 to 6).
template <typename T, int W, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 2) k_interp(Geom g, EsPoly<T> ep,
                                                const typename PT<T>::U *__restrict__ sorted,
                                                const int *__restrict__ perm,
                                                const int2 *__restrict__ tr,
                                                const typename PT<T>::C *__restrict__ g0,
                                                const typename PT<T>::C *__restrict__ g1,
                                                const double *__restrict__ grad_out,
                                                T *__restrict__ grad) {
    const int2 r = tr[blockIdx.x];
    interp_tile<T, W, D>(g, ep, sorted, perm, r.x, r.y, g0, g1, grad_out, grad, blockIdx.x);
}

// Batched interpolation: a persistent grid walks the tiles of every instance.
template <typename T, int W, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 2) k_interp_b(
    const BInst *__restrict__ inst, const int64_t *__restrict__ tile_first, int n_inst,
    int64_t n_tiles, EsPoly<T> ep, const typename PT<T>::U *__restrict__ sorted,
    const int *__restrict__ perm, const int *__restrict__ off,
    const typename PT<T>::C *__restrict__ g0, const typename PT<T>::C *__restrict__ g1,
    const double *__restrict__ grad_out, T *__restrict__ grad) {
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int i = find_segment(tile_first, n_inst, t);
        const BInst &I = inst[i];
        const int64_t lt = t - tile_first[i];
        const int *o = off + I.bo;
        interp_tile<T, W, D>(I.g, ep, sorted, perm, o[lt * I.g.sub], o[(lt + 1) * I.g.sub],
                             g0 + I.ro, D == 3 ? g1 + I.ro : g1, grad_out, grad, lt);
        __syncthreads();
    }
}

// K7 in the kernel-derivative mode: the tile and halo of the real field h = F^-1[E / Psi] are
// staged in shared memory and each point takes the gradient of the interpolant,
//   dL/dr_a = -(2 n_f[a] / L[a]) sum_m h(m) (d psi / d tau along a) (psi along the other axes),
// scaled by the incoming gradient; dscale holds -2 n_f[a] / L[a].
template <typename T, int W, int D>
__device__ __forceinline__ void interp_window_kd(const EsPoly<T> &ep, const int (&i0)[3],
                                                 const T (&x1)[3], int64_t j, const T *sh, int rx,
                                                 int rxy, T dsx, T dsy, T dsz,
                                                 T *__restrict__ grad);

template <typename T, int W, int D>
__device__ __forceinline__ void interp_point_kd(const EsPoly<T> &ep,
                                                const typename PT<T>::U (&u)[3], int64_t j,
                                                const T *sh, int rx, int rxy, T dsx, T dsy, T dsz,
                                                T *__restrict__ grad) {
    int i0[3];
    T x1[3];
    window_of<T, W, D>(u, rx, rxy, i0, x1);
    interp_window_kd<T, W, D>(ep, i0, x1, j, sh, rx, rxy, dsx, dsy, dsz, grad);
}

// The window of one point (start i0 in the staged region, kernel offsets x1): the gradient of the
// interpolant, scaled per axis, written at the caller index j.
template <typename T, int W, int D>
__device__ __forceinline__ void interp_window_kd(const EsPoly<T> &ep, const int (&i0)[3],
                                                 const T (&x1)[3], int64_t j, const T *sh, int rx,
                                                 int rxy, T dsx, T dsy, T dsz,
                                                 T *__restrict__ grad) {
    T wx[W], dwx[W], wy[W], dwy[W];
    es_weights_d<T, W>(ep, x1[0], wx, dwx);
    es_weights_d<T, W>(ep, x1[1], wy, dwy);
    if constexpr (D == 2) {
        T gx = T(0), gy = T(0);
        if constexpr (sizeof(T) == 4) {
            const unsigned step = 4u * (unsigned)rx;
            unsigned row = smem_addr(sh) + 4u * (unsigned)(i0[1] * rx + i0[0]);
#pragma unroll
            for (int b = 0; b < W; ++b, row += step) {
                float r0 = 0.f, r1 = 0.f;
                dot_row_kd<W>(row, wx, dwx, r0, r1, std::make_integer_sequence<int, W>{});
                gx = fmaf(wy[b], r1, gx);
                gy = fmaf(dwy[b], r0, gy);
            }
        } else {
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const T *row = sh + (i0[1] + b) * rx + i0[0];
                T r0 = T(0), r1 = T(0);
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const T v = row[a];
                    r0 = fma(wx[a], v, r0);
                    r1 = fma(dwx[a], v, r1);
                }
                gx = fma(wy[b], r1, gx);
                gy = fma(dwy[b], r0, gy);
            }
        }
        using T2 = typename PT<T>::C;
        reinterpret_cast<T2 *>(grad)[j] = T2{dsx * gx, dsy * gy};
    } else {
        T wz[W], dwz[W];
        es_weights_d<T, W>(ep, x1[2], wz, dwz);
        T gx = T(0), gy = T(0), gz = T(0);
        if constexpr (sizeof(T) == 4) {
            const unsigned step = 4u * (unsigned)rx, pstep = 4u * (unsigned)rxy;
            unsigned plane = smem_addr(sh) + 4u * (unsigned)(i0[2] * rxy + i0[1] * rx + i0[0]);
#pragma unroll (W <= 8 ? W : 1)
            for (int c = 0; c < W; ++c, plane += pstep) {
                float px = 0.f, py = 0.f, pz = 0.f;
                unsigned row = plane;
#pragma unroll
                for (int b = 0; b < W; ++b, row += step) {
                    float r0 = 0.f, r1 = 0.f;
                    dot_row_kd<W>(row, wx, dwx, r0, r1, std::make_integer_sequence<int, W>{});
                    px = fmaf(wy[b], r1, px);
                    py = fmaf(dwy[b], r0, py);
                    pz = fmaf(wy[b], r0, pz);
                }
                gx = fmaf(wz[c], px, gx);
                gy = fmaf(wz[c], py, gy);
                gz = fmaf(dwz[c], pz, gz);
            }
        } else {
#pragma unroll 1
            for (int c = 0; c < W; ++c) {
                T px = T(0), py = T(0), pz = T(0);
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const T *row = sh + (i0[2] + c) * rxy + (i0[1] + b) * rx + i0[0];
                    T r0 = T(0), r1 = T(0);
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        const T v = row[a];
                        r0 = fma(wx[a], v, r0);
                        r1 = fma(dwx[a], v, r1);
                    }
                    px = fma(wy[b], r1, px);
                    py = fma(dwy[b], r0, py);
                    pz = fma(wy[b], r0, pz);
                }
                gx = fma(wz[c], px, gx);
                gy = fma(wz[c], py, gy);
                gz = fma(dwz[c], pz, gz);
            }
        }
        grad[j * 3 + 0] = dsx * gx;
        grad[j * 3 + 1] = dsy * gy;
        grad[j * 3 + 2] = dsz * gz;
    }
}

// bytes of the staged real field of a kernel-derivative interpolation tile (rounded up to 16)
// (a plan that stages by TMA boxes: the box of g.tbox elements, whose rows are up to 3 elements
// wider than the region)
__host__ __device__ inline size_t interp_kd_tile_bytes(const Geom &g, size_t esize) {
    const int w = g.width;
    size_t cells = g.tma ? (size_t)g.tbox[0] * g.tbox[1] * g.tbox[2]
                         : (size_t)(g.tmax[0] + w) * (g.tmax[1] + w) *
                               (g.dim == 3 ? (g.tmax[2] + w) : 1);
    return (cells * esize + 127) & ~(size_t)127;
}

// One element from global to shared memory without passing through registers (cp.async, 4 or 8
// bytes, cached in L1): the copies of a thread stay in flight until cp_async_wait_all().
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "n"(sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Tensor-memory-accelerator (TMA) tile loads completing on an mbarrier in shared memory.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    // make the initialised barrier visible to the asynchronous proxy that completes it
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// Polls phase `parity` of the barrier at most `tries` times (each poll may suspend the thread for
// a while); true once the phase has completed.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int tries) {
    for (int i = 0; i < tries; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// A box of the tensor map at element coordinates (x, y[, z]) (x a multiple of 4 floats: the box
// starts on a 16-byte boundary) into shared memory at dst (128-byte aligned).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_addr(bar))
        : "memory");
}
// Polls of a TMA tile load before the kernel gives up and latches FRESCO_ERR_TIMEOUT (bit 4 of
// the device error word): far beyond any real load (microseconds), tens of milliseconds.
constexpr int kTmaWaitTries = 1 << 16;

// How a kernel-derivative interpolation tile is staged in shared memory: with px == 0 the region
// is packed tightly (row pitch rw[0], plane rw[0] rw[1]); else rows have pitch px and planes pp
// elements, the region starting at column x0 % 4 of its row, and `map` (if not null) describes
// the field for TMA box loads of g.tbox elements at 16-byte aligned x. err: the plan's device
// error word (TMA timeouts).
struct InterpStage {
    int px, pp;
    const CUtensorMap *map;
    int *err;
};

// FP32 tiles of at most g.list_cap points run in the level-ordered bank-residue schedule of the
// spread (window loads of a warp hit distinct banks but where a run of 32 entries spans two
// levels); others one point per thread in sorted order. The tile and its halo are staged with
// asynchronous copies while the block builds the point list from the sorted records.
template <typename T, int W, int D>
__device__ __forceinline__ void interp_tile_kd(const Geom &g, const EsPoly<T> &ep,
                                               const typename PT<T>::U *__restrict__ sorted,
                                               const int *__restrict__ perm, const int p0,
                                               const int p1, const T *__restrict__ h, T dsx,
                                               T dsy, T dsz, T *__restrict__ grad,
                                               const int64_t t, const InterpStage st) {
    using U = typename PT<T>::U;
    extern __shared__ __align__(128) unsigned char sm_dyn[];
    __shared__ ResidueShared s_rl;
    __shared__ unsigned long long s_bar;
    // the dynamic buffer starts after the static shared state, 16-byte aligned; a TMA box needs a
    // 128-byte aligned destination, so the staged region starts at the next 128-byte boundary
    // (the launch requests 128 bytes more)
    unsigned char *sm_raw = sm_dyn + ((128u - (smem_addr(sm_dyn) & 127u)) & 127u);
    const int tc[3] = {(int)(t % g.nb[0]), (int)((t / g.nb[0]) % g.nb[1]),
                       (int)(t / ((int64_t)g.nb[0] * g.nb[1]))};
    constexpr int HL = W / 2;
    int s[3], rw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            s[a] = tile_start(tc[a], g.tq[a], g.tr[a]);
            rw[a] = tile_start(tc[a] + 1, g.tq[a], g.tr[a]) - s[a] + W;
        } else {
            s[a] = 0;
            rw[a] = 1;
        }
    }
    const int px = st.px ? st.px : rw[0], pp = st.px ? st.pp : rw[0] * rw[1];
    T *sh = reinterpret_cast<T *>(sm_raw);
    if (threadIdx.x < 32) s_rl.cnt[threadIdx.x] = 0;
    bool tma = false;
    {   // stage the tile and its halo. The staged region is narrower than the grid, so it wraps
        // at most once per axis. A region that does not wrap takes one TMA box load when the plan
        // has a tensor map (the box starts at the 16-byte boundary at or below the region's first
        // column), else one cell per thread and step without wrap tests; a wrapping region one
        // cell per thread and step with them (the cell's row and plane by multiply-high division).
        const FastDiv fx = tile_div<0, true>(g, rw[0] - W), fy = tile_div<1, true>(g, rw[1] - W);
        const int gx0 = s[0] - HL, gy0 = s[1] - HL, gz0 = D == 3 ? s[2] - HL : 0;
        const bool inside = gx0 >= 0 && gx0 + rw[0] <= g.nf[0] && gy0 >= 0 &&
                            gy0 + rw[1] <= g.nf[1] &&
                            (D < 3 || (gz0 >= 0 && gz0 + rw[2] <= g.nf[2]));
        const int64_t nx = g.nf[0], nxy = (int64_t)g.nf[0] * g.nf[1];
        const int cells = rw[0] * rw[1] * rw[2];
        tma = sizeof(T) == 4 && st.map != nullptr && inside;
        if (tma && ((smem_addr(sm_raw) & 127u) != 0 || ((gx0 & ~3) & 3) != 0)) {
            // (never taken: the destination is aligned above and the box's x is a multiple of
            // four) latch it and stage by copies instead of starting a misaligned TMA load
            if (threadIdx.x == 0 && st.err) atomicOr(st.err, 8);
            tma = false;
        }
        if (tma) {
            const int xa = gx0 & ~3;
            sh += gx0 - xa;
            if (threadIdx.x == 0) {
                mbar_init(&s_bar, 1);
                mbar_expect_tx(&s_bar, (unsigned)((size_t)g.tbox[0] * g.tbox[1] * g.tbox[2] *
                                                  sizeof(T)));
                if (D == 3) tma_load_3d(sm_raw, st.map, xa, gy0, gz0, &s_bar);
                else tma_load_2d(sm_raw, st.map, xa, gy0, &s_bar);
            }
        } else if (inside) {
            const T *src = h + gz0 * nxy + (int64_t)gy0 * nx + gx0;
            for (int i = threadIdx.x; i < cells; i += blockDim.x) {
                const int row = fx.div(i), x = i - row * rw[0];
                const int z = D == 3 ? fy.div(row) : 0, y = row - z * rw[1];
                cp_async_elem(sh + z * pp + y * px + x, src + z * nxy + (int64_t)y * nx + x);
            }
        } else {
            for (int i = threadIdx.x; i < cells; i += blockDim.x) {
                const int row = fx.div(i), x = i - row * rw[0];
                const int z = D == 3 ? fy.div(row) : 0, y = row - z * rw[1];
                int gx = gx0 + x, gy = gy0 + y, gz = gz0 + z;
                gx += gx < 0 ? g.nf[0] : (gx >= g.nf[0] ? -g.nf[0] : 0);
                gy += gy < 0 ? g.nf[1] : (gy >= g.nf[1] ? -g.nf[1] : 0);
                if (D == 3) gz += gz < 0 ? g.nf[2] : (gz >= g.nf[2] ? -g.nf[2] : 0);
                cp_async_elem(sh + z * pp + y * px + x, h + gz * nxy + (int64_t)gy * nx + gx);
            }
        }
    }
    __syncthreads();
    // the staged field is in place once the TMA load's barrier phase or this thread's copies have
    // completed (then the block barrier makes every thread's copies visible)
    auto staged = [&]() -> bool {
        if (tma) {
            if (mbar_wait(&s_bar, 0, kTmaWaitTries)) return true;
            if (threadIdx.x == 0 && st.err) atomicOr(st.err, 4);
            mbar_wait(&s_bar, 0, kTmaWaitTries);   // let a late load land before the block exits
            return false;
        }
        cp_async_wait_all();
        return true;
    };
    if (sizeof(T) == 4 && p1 - p0 <= g.list_cap) {
        // level-ordered entries: packed window start, D kernel offsets, caller index
        const int cap = g.list_cap;
        int *l_i0 = reinterpret_cast<int *>(sm_raw + interp_kd_tile_bytes(g, sizeof(T)));
        const int rxy = pp, rx = px;
        float *l_x1 = reinterpret_cast<float *>(l_i0 + cap);
        int *l_j = l_i0 + (1 + D) * cap;
        const int n = residue_lists<T, W, D>(
            sorted, p0, p1, rx, rxy, s_rl,
            [&](int slot, const int (&i0)[3], const T (&x1)[3], unsigned j) {
                l_i0[slot] = i0[0] | (i0[1] << 10) | (i0[2] << 20);
#pragma unroll
                for (int a = 0; a < D; ++a) l_x1[a * cap + slot] = (float)x1[a];
                l_j[slot] = (int)j;
            });
        const bool ok = staged();
        __syncthreads();
        if (!ok) return;
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const int pk = l_i0[q];
            const int i0[3] = {pk & 1023, (pk >> 10) & 1023, pk >> 20};
            T x1[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int a = 0; a < D; ++a) x1[a] = (T)l_x1[a * cap + q];
            interp_window_kd<T, W, D>(ep, i0, x1, (int64_t)l_j[q], sh, rx, rxy, dsx, dsy,
                                      dsz, grad);
        }
        return;
    }
    const bool ok = staged();
    __syncthreads();
    if (!ok) return;
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        U u[3];
        const int64_t j = load_record<T, D>(sorted, perm, p, u);
        interp_point_kd<T, W, D>(ep, u, j, sh, px, pp, dsx, dsy, dsz, grad);
    }
}

// FP32 tiles with their entry lists take 60-110 KB of shared memory, so at most three (2D) or
// two (3D) blocks are resident.
template <typename T, int W, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (D == 3 ? 2 : 3) : 2) k_interp_kd(
    Geom g, EsPoly<T> ep, const typename PT<T>::U *__restrict__ sorted,
    const int *__restrict__ perm, const int2 *__restrict__ tr, const T *__restrict__ h,
    const double *__restrict__ grad_out, T dsx, T dsy, T dsz, T *__restrict__ grad,
    const __grid_constant__ CUtensorMap map, int *__restrict__ err) {
    const T sc = grad_out ? (T)(*grad_out) : T(1);
    const int2 r = tr[blockIdx.x];
    InterpStage st{0, 0, nullptr, err};
    if (g.tma) st = InterpStage{g.tbox[0], g.tbox[0] * g.tbox[1], &map, err};
    interp_tile_kd<T, W, D>(g, ep, sorted, perm, r.x, r.y, h, sc * dsx, sc * dsy, sc * dsz, grad,
                            blockIdx.x, st);
}

// Batched kernel-derivative interpolation: a persistent grid walks the tiles of every instance;
// instance i's real field sits at h + I.go and its scale is -2 n_f / L per axis.
template <typename T, int W, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_interp_kd_b(
    const BInst *__restrict__ inst, const int64_t *__restrict__ tile_first, int n_inst,
    int64_t n_tiles, EsPoly<T> ep, const typename PT<T>::U *__restrict__ sorted,
    const int *__restrict__ perm, const int *__restrict__ off, const T *__restrict__ h,
    const double *__restrict__ grad_out, T *__restrict__ grad) {
    const double sc = grad_out ? *grad_out : 1.0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int i = find_segment(tile_first, n_inst, t);
        const BInst &I = inst[i];
        const Geom &g = I.g;
        const int64_t lt = t - tile_first[i];
        const int *o = off + I.bo;
        interp_tile_kd<T, W, D>(g, ep, sorted, perm, o[lt * g.sub], o[(lt + 1) * g.sub], h + I.go,
                                (T)(-2.0 * (g.s_hi[0] + g.s_lo[0]) * sc),
                                (T)(-2.0 * (g.s_hi[1] + g.s_lo[1]) * sc),
                                (T)(-2.0 * (g.s_hi[2] + g.s_lo[2]) * sc), grad,
                                t - tile_first[i], InterpStage{0, 0, nullptr, nullptr});
        __syncthreads();
    }
}

// rho and S for the mask rows as given to the plan (diagnostic output).
template <typename T, int D>
__global__ void k_rho_s(MaskGeom m, const int *__restrict__ mask_n, int64_t n_k,
                        const typename PT<T>::C *__restrict__ spec, const T *__restrict__ ip0,
                        const T *__restrict__ ip1, const T *__restrict__ ip2, T *__restrict__ rho,
                        T *__restrict__ S) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_k) return;
    int nx = mask_n[q * D + 0], ny = mask_n[q * D + 1], nz = (D == 3) ? mask_n[q * D + 2] : 0;
    T sgn = T(1);
    if (nx < 0) { nx = -nx; ny = -ny; nz = -nz; sgn = T(-1); }   // rho(-n) = conj rho(n)
    const int ry = ny < 0 ? ny + m.nf[1] : ny;
    const int rz = nz < 0 ? nz + m.nf[2] : nz;
    const auto F = spec[(int64_t)nx * m.plane + (int64_t)rz * m.nf[1] + ry];
    T ip = ip0[nx] * ip1[ny < 0 ? -ny : ny];
    if (D == 3) ip *= ip2[nz < 0 ? -nz : nz];
    const T re = F.x * ip, im = sgn * F.y * ip;
    if (rho) { rho[2 * q] = re; rho[2 * q + 1] = im; }
    if (S) S[q] = (re * re + im * im) * (T)m.inv_n;
}

// ---------------------------------------------------------------------------------------------
// Transposes around the (z,)y FFT pass, so that every cuFFT call is a batch of contiguous
// transforms (32 x 32 tiles through shared memory; coalesced on both sides).

// at[c][r] = a[r][c] for r < rows, c < ncols (a has row stride lda)
template <typename C>
__global__ void __launch_bounds__(256) k_cols_to_rows(const C *__restrict__ a, C *__restrict__ at,
                                                      int64_t rows, int64_t lda, int ncols,
                                                      int64_t a_stride, int64_t at_stride) {
    __shared__ C tile[32][33];
    a += blockIdx.z * a_stride;
    at += blockIdx.z * at_stride;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t r = r0 + k;
        const int c = c0 + threadIdx.x;
        if (r < rows && c < ncols) tile[k][threadIdx.x] = a[r * lda + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (c < ncols && r < rows) at[(int64_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

// r[row][x(c)] = bt[c][row] for c < 2 kx + 2, x(c) = c - kx - 1 taken modulo nf0
template <typename C>
__global__ void __launch_bounds__(256) k_rows_to_cols(const C *__restrict__ bt, C *__restrict__ r,
                                                      int64_t rows, int nf0, int kx,
                                                      int64_t bt_stride, int64_t r_stride) {
    __shared__ C tile[32][33];
    bt += blockIdx.z * bt_stride;
    r += blockIdx.z * r_stride;
    const int ncols = 2 * kx + 2;
    const int c0 = blockIdx.y * 32;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k;
        const int64_t row = r0 + threadIdx.x;
        if (c < ncols && row < rows) tile[k][threadIdx.x] = bt[(int64_t)c * rows + row];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t row = r0 + k;
        const int c = c0 + threadIdx.x;
        if (row < rows && c < ncols) {
            const int x = c <= kx ? nf0 - kx - 1 + c : c - kx - 1;
            r[row * nf0 + x] = tile[threadIdx.x][k];
        }
    }
}

// Kernel-derivative mode: the transformed columns [kx + 1][rows] back into the rows of the
// half spectrum [rows][half_row] (columns 0 .. kx; the others stay zero from plan time).
template <typename C>
__global__ void __launch_bounds__(256) k_rows_to_half(const C *__restrict__ bt, C *__restrict__ r,
                                                      int64_t rows, int64_t half_row, int ncols,
                                                      int64_t bt_stride, int64_t r_stride) {
    __shared__ C tile[32][33];
    bt += blockIdx.z * bt_stride;
    r += blockIdx.z * r_stride;
    const int c0 = blockIdx.y * 32;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k;
        const int64_t row = r0 + threadIdx.x;
        if (c < ncols && row < rows) tile[k][threadIdx.x] = bt[(int64_t)c * rows + row];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t row = r0 + k;
        const int c = c0 + threadIdx.x;
        if (row < rows && c < ncols) r[row * half_row + c] = tile[threadIdx.x][k];
    }
}

// A real row x of even length n_f = 2M is transformed as the complex row z[m] = x[2m] + i x[2m+1]
// of length M (Z = FFT_M z); its half spectrum is then
//   X[k] = E + tau_k O,  E = (Z[k] + conj Z[M-k]) / 2,  O = (Z[k] - conj Z[M-k]) / (2i),
//   X[M-k] = conj(E - tau_k O),  tau_k = exp(-2 pi i k / n_f),  indices of Z taken modulo M.
// One thread forms the pair (k, M-k) for 0 <= k <= M/2 from the same two values, so every Z is
// read once. The columns k <= kx are written transposed: xt[k][row], rows contiguous. z is
// [rows][M]; tw[k] = tau_k for k = 0..M/2. blockIdx.z selects one of a batch of such transforms
// (z and xt advanced by their strides).
template <typename C>
__global__ void __launch_bounds__(256) k_rfft_split_cols(const C *__restrict__ z, C *__restrict__ xt,
                                                         const C *__restrict__ tw, int64_t rows,
                                                         int M, int kx, int64_t z_stride,
                                                         int64_t xt_stride) {
    using R = decltype(C{}.x);
    __shared__ C ta[32][33];
    __shared__ C tb[32][33];
    z += blockIdx.z * z_stride;
    xt += blockIdx.z * xt_stride;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    const int half = M / 2;
    // nothing to write: every direct column beyond kx and every mirror column (M - k, for the
    // block's k) beyond kx as well
    if (k0 > kx && M - (k0 + 31) > kx) return;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i;
        const int k = k0 + threadIdx.x;
        if (r < rows && k <= half) {
            const int km = (k == 0) ? 0 : M - k;
            ta[i][threadIdx.x] = z[r * M + k];
            tb[i][threadIdx.x] = z[r * M + km];
        }
    }
    __syncthreads();
    const int64_t r = r0 + threadIdx.x;
    if (r >= rows) return;
    for (int t = threadIdx.y; t < 32; t += 8) {
        const int k = k0 + t;
        if (k > half) break;
        const C a = ta[threadIdx.x][t], b = tb[threadIdx.x][t];
        const C w = tw[k];
        // E = (a + conj b) / 2, O = -i (a - conj b) / 2
        const R ex = R(0.5) * (a.x + b.x), ey = R(0.5) * (a.y - b.y);
        const R ox = R(0.5) * (a.y + b.y), oy = R(-0.5) * (a.x - b.x);
        const R px = w.x * ox - w.y * oy, py = w.x * oy + w.y * ox;   // tau_k O
        if (k <= kx) {
            C v;
            v.x = ex + px;
            v.y = ey + py;
            xt[(int64_t)k * rows + r] = v;
        }
        const int km = M - k;
        if (km > half && km <= kx) {
            C v;
            v.x = ex - px;
            v.y = -(ey - py);
            xt[(int64_t)km * rows + r] = v;
        }
    }
}

// Inverse of the above for a Hermitian half spectrum X[k], k = 0..kx (zero beyond, and kx < M):
//   Z[k] = P + i Q,  P = X[k] + conj X[M-k],  Q = (X[k] - conj X[M-k]) conj(tau_k),
//   Z[M-k] = conj P + i conj Q,
// so that the inverse FFT_M of Z is x[2m] + i x[2m+1] with x[n] = sum_k X[k] e^{+2 pi i k n / n_f}
// (both halves of the Hermitian spectrum). xt is [kx+1][rows] (rows contiguous); z is
// [rows][M], every entry written. blockIdx.z selects one of a batch, as above.
template <typename C>
__global__ void __launch_bounds__(256) k_rfft_merge_rows(const C *__restrict__ xt, C *__restrict__ z,
                                                         const C *__restrict__ tw, int64_t rows,
                                                         int M, int kx, int64_t xt_stride,
                                                         int64_t z_stride) {
    using R = decltype(C{}.x);
    __shared__ C ta[32][33];
    __shared__ C tb[32][33];
    xt += blockIdx.z * xt_stride;
    z += blockIdx.z * z_stride;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    const int half = M / 2;
    for (int t = threadIdx.y; t < 32; t += 8) {
        const int k = k0 + t;
        const int64_t r = r0 + threadIdx.x;
        if (k <= half && r < rows) {
            const int km = M - k;   // M for k = 0: X[M] = 0 since kx < M
            C zero;
            zero.x = R(0);
            zero.y = R(0);
            ta[t][threadIdx.x] = k <= kx ? xt[(int64_t)k * rows + r] : zero;
            tb[t][threadIdx.x] = km <= kx ? xt[(int64_t)km * rows + r] : zero;
        }
    }
    __syncthreads();
    const int k = k0 + threadIdx.x;
    if (k > half) return;
    const C w = tw[k];
    const int km = M - k;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i;
        if (r >= rows) break;
        const C a = ta[threadIdx.x][i], b = tb[threadIdx.x][i];
        const R px = a.x + b.x, py = a.y - b.y;           // P = a + conj b
        const R dx = a.x - b.x, dy = a.y + b.y;           // a - conj b
        const R qx = dx * w.x + dy * w.y, qy = dy * w.x - dx * w.y;   // (a - conj b) conj(tau_k)
        C v;
        v.x = px - qy;
        v.y = py + qx;
        z[r * M + k] = v;
        if (km > half && km < M) {
            C u;   // conj P + i conj Q
            u.x = px + qy;
            u.y = -py + qx;
            z[r * M + km] = u;
        }
    }
}


// ---------------------------------------------------------------------------------------------
// Launchers

// Width-specialised launchers (one kernel instantiation per ES kernel width). Their definitions
// below are instantiated in the fresco_w_*.cu units, a few widths per unit so that the units
// compile in parallel; the units that instantiate Launch<T> see them through the extern
// declarations of FRESCO_EXTERN_WIDTH_OPS.
template <typename T, int W, int D>
struct WOps {
    static cudaError_t spread_own(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                  const int2 *tr, T *grid, T *ring, int64_t ring_slot,
                                  cudaStream_t s);
    static cudaError_t interp(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                              const int *perm, const int2 *tr, const void *g0, const void *g1,
                              const double *grad_out, T *grad, cudaStream_t s);
    static cudaError_t interp_kd(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                 const int *perm, const int2 *tr, const T *h,
                                 const double *grad_out, const double dscale[3], T *grad,
                                 cudaStream_t s, const CUtensorMap *map, int *err);
};

// the same for the (2D) ensemble kernels
template <typename T, int W>
struct WOpsB {
    static cudaError_t spread_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                const int *off, T *grid, cudaStream_t s);
    static cudaError_t interp_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                const int *perm, const int *off, const void *g0, const void *g1,
                                const double *grad_out, T *grad, cudaStream_t s);
    static cudaError_t interp_kd_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                   const int *perm, const int *off, const T *h,
                                   const double *grad_out, T *grad, cudaStream_t s);
};

#define FRESCO_WIDTHS_LO(M, ...) M(2, __VA_ARGS__) M(3, __VA_ARGS__) M(4, __VA_ARGS__) \
    M(5, __VA_ARGS__) M(6, __VA_ARGS__) M(7, __VA_ARGS__) M(8, __VA_ARGS__)
#define FRESCO_WIDTHS_HI(M, ...) M(9, __VA_ARGS__) M(10, __VA_ARGS__) M(11, __VA_ARGS__) \
    M(12, __VA_ARGS__) M(13, __VA_ARGS__) M(14, __VA_ARGS__) M(15, __VA_ARGS__) M(16, __VA_ARGS__)
#define FRESCO_EXTERN_WOPS(W, T, D) extern template struct WOps<T, W, D>;
#define FRESCO_EXTERN_WOPSB(W, T) extern template struct WOpsB<T, W>;
#define FRESCO_INST_WOPS(W, T, D) template struct WOps<T, W, D>;
#define FRESCO_INST_WOPSB(W, T) template struct WOpsB<T, W>;
#define FRESCO_EXTERN_WIDTH_OPS(T)                                                             \
    FRESCO_WIDTHS_LO(FRESCO_EXTERN_WOPS, T, 2) FRESCO_WIDTHS_HI(FRESCO_EXTERN_WOPS, T, 2)      \
    FRESCO_WIDTHS_LO(FRESCO_EXTERN_WOPS, T, 3) FRESCO_WIDTHS_HI(FRESCO_EXTERN_WOPS, T, 3)      \
    FRESCO_WIDTHS_LO(FRESCO_EXTERN_WOPSB, T) FRESCO_WIDTHS_HI(FRESCO_EXTERN_WOPSB, T)

inline int grid_for(int64_t n, int threads, int cap) {
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T>
cudaError_t Launch<T>::scan(const int *cnt, int *off, int *block_sums, int64_t n, cudaStream_t s,
                            int *launches, int *cur, const int *guard) {
    const int64_t nb = (n + 1023) / 1024;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, s>>>(cnt, off, block_sums, n, guard);
    k_scan_sums<<<1, 1024, 0, s>>>(block_sums, nb, off + n, guard);
    k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(off, block_sums, n, cur, guard);
    *launches += 3;
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::count(const Geom &g, const T *points, int *cnt, int *err, cudaStream_t s,
                             const int *guard) {
    const int grid = grid_for((g.n_points + 3) / 4, 256, 152 * 16);
    if (g.dim == 2) k_count<T, 2><<<grid, 256, 0, s>>>(g, points, cnt, err, guard);
    else k_count<T, 3><<<grid, 256, 0, s>>>(g, points, cnt, err, guard);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::place(const Geom &g, const T *points, int *cur, void *sorted, int *perm,
                             cudaStream_t s, const int *guard) {
    using U = typename PT<T>::U;
    const int grid = grid_for((g.n_points + 3) / 4, 256, 152 * 16);
    if (g.dim == 2) k_place<T, 2><<<grid, 256, 0, s>>>(g, points, cur, (U *)sorted, perm, guard);
    else k_place<T, 3><<<grid, 256, 0, s>>>(g, points, cur, (U *)sorted, perm, guard);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::place_direct(const Geom &g, const T *points, int64_t j0, int *tcur,
                                    void *sorted, int *perm, int *err, cudaStream_t s) {
    using U = typename PT<T>::U;
    constexpr int IL = kDirectPointsPerThread;
    const int grid = grid_for((g.n_points + IL - 1) / IL, 256, 152 * 16);
    if (g.dim == 2)
        k_place_direct<T, 2><<<grid, 256, 0, s>>>(g, points, j0, tcur, (U *)sorted, perm, err);
    else
        k_place_direct<T, 3><<<grid, 256, 0, s>>>(g, points, j0, tcur, (U *)sorted, perm, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::tile_ranges(const Geom &g, const int *tcur, const int *off, int2 *tr,
                                   cudaStream_t s) {
    k_tile_ranges<<<grid_for(g.n_tiles, 256, 152 * 16), 256, 0, s>>>(g, tcur, off, tr);
    return cudaGetLastError();
}

template <typename T>
int Launch<T>::spread_own_smem(const Geom &g) {
    // the extended region (3D columns: the plane buffer), then (FP32) the residue-grouped
    // entries: packed window start and D kernel offsets
    const size_t region = g.dim == 3 && g.zseg > 0 ? spread_col_tile_bytes(g, sizeof(T))
                                                   : spread_own_tile_bytes(g, sizeof(T));
    return (int)(region + (sizeof(T) == 4 ? (size_t)(1 + g.dim) * 4 * (size_t)g.list_cap : 0));
}

template <typename T>
int64_t Launch<T>::ring_slot(const Geom &g) {
    const int w = g.width;
    int64_t e = (int64_t)(g.tmax[0] + w) * (g.tmax[1] + w);
    int64_t i = (int64_t)g.tmax[0] * g.tmax[1];
    if (g.dim == 3) {
        e *= g.tmax[2] + w;
        i *= g.tmax[2];
    }
    return e - i;
}

template <typename T, int W, int D>
cudaError_t WOps<T, W, D>::spread_own(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                      const int2 *tr, T *grid, T *ring, int64_t ring_slot,
                                      cudaStream_t s) {
    using U = typename PT<T>::U;
    const int smem = Launch<T>::spread_own_smem(g);
    const unsigned nt = (unsigned)g.n_tiles;
    cudaError_t e;
    if (D == 3 && g.zseg > 0) {
        // z-columns: fold z (segment ends) first, then x, then y
        auto kern = k_spread_col<T, W>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        const unsigned nseg = (unsigned)((g.nb[2] + g.zseg - 1) / g.zseg);
        kern<<<(unsigned)(g.nb[0] * g.nb[1]) * nseg, 256, smem, s>>>(g, ep, (const U *)sorted,
                                                                     tr, grid, ring, ring_slot);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (g.tq[2] >= W) {
            k_halo_fold<T, W, D, 2, 3, 0><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        } else {
            k_halo_fold<T, W, D, 2, 1, 0><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
            k_halo_fold<T, W, D, 2, 2, 0><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        }
        if (g.tq[0] >= W) {
            k_halo_fold<T, W, D, 0, 3, 4><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        } else {
            k_halo_fold<T, W, D, 0, 1, 4><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
            k_halo_fold<T, W, D, 0, 2, 4><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        }
        if (g.tq[1] >= W) {
            k_halo_fold<T, W, D, 1, 3, 5><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        } else {
            k_halo_fold<T, W, D, 1, 1, 5><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
            k_halo_fold<T, W, D, 1, 2, 5><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        }
        return cudaGetLastError();
    }
    auto kern = k_spread_own<T, W, D>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<nt, 256, smem, s>>>(g, ep, (const U *)sorted, tr, grid, ring, ring_slot);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one launch per axis when every tile along it is at least W wide, else two (low, high)
    if (g.tq[0] >= W) {
        k_halo_fold<T, W, D, 0, 3, 0><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
    } else {
        k_halo_fold<T, W, D, 0, 1, 0><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        k_halo_fold<T, W, D, 0, 2, 0><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
    }
    if (g.tq[1] >= W) {
        k_halo_fold<T, W, D, 1, 3, 1><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
    } else {
        k_halo_fold<T, W, D, 1, 1, 1><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        k_halo_fold<T, W, D, 1, 2, 1><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
    }
    if constexpr (D == 3) {
        if (g.tq[2] >= W) {
            k_halo_fold<T, W, D, 2, 3, 3><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        } else {
            k_halo_fold<T, W, D, 2, 1, 3><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
            k_halo_fold<T, W, D, 2, 2, 3><<<nt, 256, 0, s>>>(g, ring, ring_slot, grid);
        }
    }
    return cudaGetLastError();
}

template <typename T>
int Launch<T>::spread_smem(const Geom &g) {
    const int D = g.dim;
    return (int)(spread_tile_bytes(g, sizeof(T)) +
                 (sizeof(T) * D + sizeof(int)) * (size_t)g.list_cap);
}

template <typename T>
int Launch<T>::interp_kd_smem(const Geom &g) {
    // up to 128 bytes to the first 128-byte boundary, the staged field, then (FP32) the level-
    // ordered entries: packed window start, D kernel offsets and the caller index
    return (int)(128 + interp_kd_tile_bytes(g, sizeof(T)) +
                 (sizeof(T) == 4 ? (size_t)(2 + g.dim) * 4 * (size_t)g.list_cap : 0));
}

template <typename T>
cudaError_t Launch<T>::rfft_split(const void *z, void *xt, const void *tw, int64_t rows, int M,
                                  int kx, cudaStream_t s, int batch, int64_t z_stride,
                                  int64_t xt_stride) {
    using C = typename PT<T>::C;
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)(M / 2 / 32 + 1), (unsigned)batch);
    k_rfft_split_cols<C><<<grid, dim3(32, 8), 0, s>>>((const C *)z, (C *)xt, (const C *)tw, rows,
                                                      M, kx, z_stride, xt_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::rfft_merge(const void *xt, void *z, const void *tw, int64_t rows, int M,
                                  int kx, cudaStream_t s, int batch, int64_t xt_stride,
                                  int64_t z_stride) {
    using C = typename PT<T>::C;
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)(M / 2 / 32 + 1), (unsigned)batch);
    k_rfft_merge_rows<C><<<grid, dim3(32, 8), 0, s>>>((const C *)xt, (C *)z, (const C *)tw, rows,
                                                      M, kx, xt_stride, z_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::rows_to_half(const void *bt, void *r, int64_t rows, int64_t half_row,
                                    int kx, cudaStream_t s, int batch, int64_t bt_stride,
                                    int64_t r_stride) {
    using C = typename PT<T>::C;
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((kx + 1 + 31) / 32), (unsigned)batch);
    k_rows_to_half<C><<<grid, dim3(32, 8), 0, s>>>((const C *)bt, (C *)r, rows, half_row, kx + 1,
                                                   bt_stride, r_stride);
    return cudaGetLastError();
}

template <typename T>
int Launch<T>::interp_smem(const Geom &g) {
    const int w = g.width;
    size_t cells = (size_t)(g.tmax[0] + w) * (g.tmax[1] + w) * (g.dim == 3 ? (g.tmax[2] + w) : 1);
    size_t per = sizeof(typename PT<T>::C) + (g.dim == 3 ? sizeof(T) : 0);
    return (int)(cells * per);
}

template <typename T, int W, int D>
cudaError_t WOps<T, W, D>::interp(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                  const int *perm, const int2 *tr, const void *g0, const void *g1,
                                  const double *grad_out, T *grad, cudaStream_t s) {
    using U = typename PT<T>::U;
    using C = typename PT<T>::C;
    const int smem = Launch<T>::interp_smem(g);
    auto kern = k_interp<T, W, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)g.n_tiles, 256, smem, s>>>(g, ep, (const U *)sorted, perm, tr,
                                                (const C *)g0, (const C *)g1, grad_out, grad);
    return cudaGetLastError();
}

template <typename T, int W, int D>
cudaError_t WOps<T, W, D>::interp_kd(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                     const int *perm, const int2 *tr, const T *h,
                                     const double *grad_out, const double dscale[3], T *grad,
                                     cudaStream_t s, const CUtensorMap *map, int *err) {
    using U = typename PT<T>::U;
    if (g.tma && !map) return cudaErrorInvalidValue;   // a TMA plan stages through its map
    const int smem = Launch<T>::interp_kd_smem(g);
    auto kern = k_interp_kd<T, W, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    CUtensorMap m{};
    if (map) m = *map;
    kern<<<(unsigned)g.n_tiles, 256, smem, s>>>(g, ep, (const U *)sorted, perm, tr, h, grad_out,
                                                (T)dscale[0], (T)dscale[1], (T)dscale[2], grad,
                                                m, err);
    return cudaGetLastError();
}

#define FRESCO_WIDTH_SWITCH(W_, CALL)                                                          \
    switch (W_) {                                                                              \
        case 2: { constexpr int WW = 2; CALL; }                                                \
        case 3: { constexpr int WW = 3; CALL; }                                                \
        case 4: { constexpr int WW = 4; CALL; }                                                \
        case 5: { constexpr int WW = 5; CALL; }                                                \
        case 6: { constexpr int WW = 6; CALL; }                                                \
        case 7: { constexpr int WW = 7; CALL; }                                                \
        case 8: { constexpr int WW = 8; CALL; }                                                \
        case 9: { constexpr int WW = 9; CALL; }                                                \
        case 10: { constexpr int WW = 10; CALL; }                                              \
        case 11: { constexpr int WW = 11; CALL; }                                              \
        case 12: { constexpr int WW = 12; CALL; }                                              \
        case 13: { constexpr int WW = 13; CALL; }                                              \
        case 14: { constexpr int WW = 14; CALL; }                                              \
        case 15: { constexpr int WW = 15; CALL; }                                              \
        case 16: { constexpr int WW = 16; CALL; }                                              \
        default: return cudaErrorInvalidValue;                                                 \
    }

template <typename T>
cudaError_t Launch<T>::spread_own(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                  const int2 *tr, T *grid, T *ring, int64_t ring_slot,
                                  cudaStream_t s, int *launches) {
    *launches += 1;   // (the column spread's folds: the same count, z first)
    for (int a = 0; a < g.dim; ++a) *launches += g.tq[a] >= g.width ? 1 : 2;
    if (g.dim == 2) {
        FRESCO_WIDTH_SWITCH(g.width, return (WOps<T, WW, 2>::spread_own(g, ep, sorted, tr, grid,
                                                                          ring, ring_slot, s)));
    } else {
        FRESCO_WIDTH_SWITCH(g.width, return (WOps<T, WW, 3>::spread_own(g, ep, sorted, tr, grid,
                                                                          ring, ring_slot, s)));
    }
}

template <typename T>
cudaError_t Launch<T>::interp(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                              const int *perm, const int2 *tr, const void *g0, const void *g1,
                              const double *grad_out, T *grad, cudaStream_t s) {
    if (g.dim == 2) {
        FRESCO_WIDTH_SWITCH(g.width, return (WOps<T, WW, 2>::interp(g, ep, sorted, perm, tr,
                                                                      g0, g1, grad_out, grad, s)));
    } else {
        FRESCO_WIDTH_SWITCH(g.width, return (WOps<T, WW, 3>::interp(g, ep, sorted, perm, tr,
                                                                      g0, g1, grad_out, grad, s)));
    }
}

template <typename T>
cudaError_t Launch<T>::interp_kd(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                 const int *perm, const int2 *tr, const T *h,
                                 const double *grad_out, const double dscale[3], T *grad,
                                 cudaStream_t s, const CUtensorMap *map, int *err) {
    if (g.dim == 2) {
        FRESCO_WIDTH_SWITCH(g.width, return (WOps<T, WW, 2>::interp_kd(
                                         g, ep, sorted, perm, tr, h, grad_out, dscale, grad, s,
                                         map, err)));
    } else {
        FRESCO_WIDTH_SWITCH(g.width, return (WOps<T, WW, 3>::interp_kd(
                                         g, ep, sorted, perm, tr, h, grad_out, dscale, grad, s,
                                         map, err)));
    }
}

template <typename T>
cudaError_t Launch<T>::mask(const MaskGeom &m, const int *rep_n, const T *rep_s0, const T *rep_w,
                            const void *spec, const T *ip0, const T *ip1, const T *ip2, void *hc0,
                            void *hc1, double *partial, int n_blocks, cudaStream_t s) {
    using C = typename PT<T>::C;
    if (m.dim == 2)
        k_mask<T, 2><<<n_blocks, 256, 0, s>>>(m, rep_n, rep_s0, rep_w, (const C *)spec, ip0, ip1,
                                               ip2, (C *)hc0, (C *)hc1, partial);
    else
        k_mask<T, 3><<<n_blocks, 256, 0, s>>>(m, rep_n, rep_s0, rep_w, (const C *)spec, ip0, ip1,
                                               ip2, (C *)hc0, (C *)hc1, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::finalize(const double *partial, int n_blocks, double loss_const,
                                double *loss, cudaStream_t s) {
    k_finalize<<<1, 512, 0, s>>>(partial, n_blocks, loss_const, loss);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::cols_to_rows(const void *a, void *at, int64_t rows, int64_t lda, int ncols,
                                    cudaStream_t s, int batch, int64_t a_stride,
                                    int64_t at_stride) {
    using C = typename PT<T>::C;
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((ncols + 31) / 32), (unsigned)batch);
    k_cols_to_rows<C><<<grid, dim3(32, 8), 0, s>>>((const C *)a, (C *)at, rows, lda, ncols,
                                                   a_stride, at_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::rows_to_cols(const void *bt, void *r, int64_t rows, int nf0, int kx,
                                    cudaStream_t s, int batch, int64_t bt_stride,
                                    int64_t r_stride) {
    using C = typename PT<T>::C;
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((2 * kx + 2 + 31) / 32), (unsigned)batch);
    k_rows_to_cols<C><<<grid, dim3(32, 8), 0, s>>>((const C *)bt, (C *)r, rows, nf0, kx,
                                                   bt_stride, r_stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::rho_s(const MaskGeom &m, const int *mask_n, int64_t n_k, const void *spec,
                             const T *ip0, const T *ip1, const T *ip2, T *rho, T *S,
                             cudaStream_t s) {
    using C = typename PT<T>::C;
    const unsigned grid = (unsigned)((n_k + 255) / 256);
    if (m.dim == 2)
        k_rho_s<T, 2><<<grid, 256, 0, s>>>(m, mask_n, n_k, (const C *)spec, ip0, ip1, ip2, rho, S);
    else
        k_rho_s<T, 3><<<grid, 256, 0, s>>>(m, mask_n, n_k, (const C *)spec, ip0, ip1, ip2, rho, S);
    return cudaGetLastError();
}

// ---- ensemble launchers ----------------------------------------------------------------------

inline Geom tiles_geom(const BTables &b) {
    Geom g{};
    g.dim = b.dim;
    g.width = b.width;
    g.list_cap = b.list_cap;
    for (int a = 0; a < 3; ++a) g.tmax[a] = b.tmax[a];
    return g;
}

template <typename T>
cudaError_t Launch<T>::bin_b(const BTables &b, const T *points, int *cnt, int *key, int *slot,
                             int *err, cudaStream_t s) {
    const int grid = grid_for(b.n_points, 256, 152 * 16);
    if (b.dim == 2)
        k_bin_b<T, 2><<<grid, 256, 0, s>>>(b.inst, b.pt_first, b.n_inst, b.n_points, points, cnt,
                                           key, slot, err);
    else
        k_bin_b<T, 3><<<grid, 256, 0, s>>>(b.inst, b.pt_first, b.n_inst, b.n_points, points, cnt,
                                           key, slot, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::scatter_b(const BTables &b, const T *points, const int *key,
                                 const int *slot, const int *off, void *sorted, int *perm,
                                 cudaStream_t s) {
    using U = typename PT<T>::U;
    const int grid = grid_for(b.n_points, 256, 152 * 16);
    if (b.dim == 2)
        k_scatter_b<T, 2><<<grid, 256, 0, s>>>(b.inst, b.pt_first, b.n_inst, b.n_points, points,
                                               key, slot, off, (U *)sorted, perm);
    else
        k_scatter_b<T, 3><<<grid, 256, 0, s>>>(b.inst, b.pt_first, b.n_inst, b.n_points, points,
                                               key, slot, off, (U *)sorted, perm);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t WOpsB<T, W>::spread_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                  const int *off, T *grid, cudaStream_t s) {
    constexpr int D = 2;
    using U = typename PT<T>::U;
    const int smem = Launch<T>::spread_smem(tiles_geom(b));
    auto kern = k_spread_b<T, W, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>(b.n_tiles, 152 * 8);
    kern<<<blocks, 256, smem, s>>>(b.inst, b.tile_first, b.n_inst, b.n_tiles, ep, (const U *)sorted,
                                   off, grid);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t WOpsB<T, W>::interp_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                  const int *perm, const int *off, const void *g0, const void *g1,
                                  const double *grad_out, T *grad, cudaStream_t s) {
    constexpr int D = 2;
    using U = typename PT<T>::U;
    using C = typename PT<T>::C;
    const int smem = Launch<T>::interp_smem(tiles_geom(b));
    auto kern = k_interp_b<T, W, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>(b.n_tiles, 152 * 8);
    kern<<<blocks, 256, smem, s>>>(b.inst, b.tile_first, b.n_inst, b.n_tiles, ep, (const U *)sorted,
                                   perm, off, (const C *)g0, (const C *)g1, grad_out, grad);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t WOpsB<T, W>::interp_kd_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                     const int *perm, const int *off, const T *h,
                                     const double *grad_out, T *grad, cudaStream_t s) {
    constexpr int D = 2;
    using U = typename PT<T>::U;
    const int smem = Launch<T>::interp_kd_smem(tiles_geom(b));
    auto kern = k_interp_kd_b<T, W, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>(b.n_tiles, 152 * 3);
    kern<<<blocks, 256, smem, s>>>(b.inst, b.tile_first, b.n_inst, b.n_tiles, ep, (const U *)sorted,
                                   perm, off, h, grad_out, grad);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::interp_kd_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                   const int *perm, const int *off, const T *h,
                                   const double *grad_out, T *grad, cudaStream_t s) {
    if (b.dim == 2) {
        FRESCO_WIDTH_SWITCH(b.width, return (WOpsB<T, WW>::interp_kd_b(b, ep, sorted, perm, off,
                                                                           h, grad_out, grad, s)));
    }
    return cudaErrorInvalidValue;   // ensembles are 2D
}

template <typename T>
cudaError_t Launch<T>::spread_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                const int *off, T *grid, cudaStream_t s) {
    if (b.dim == 2) {
        FRESCO_WIDTH_SWITCH(b.width, return (WOpsB<T, WW>::spread_b(b, ep, sorted, off, grid, s)));
    }
    return cudaErrorInvalidValue;   // ensembles are 2D
}

template <typename T>
cudaError_t Launch<T>::interp_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                const int *perm, const int *off, const void *g0, const void *g1,
                                const double *grad_out, T *grad, cudaStream_t s) {
    if (b.dim == 2) {
        FRESCO_WIDTH_SWITCH(b.width, return (WOpsB<T, WW>::interp_b(b, ep, sorted, perm, off,
                                                                        g0, g1, grad_out, grad, s)));
    }
    return cudaErrorInvalidValue;   // ensembles are 2D
}

template <typename T>
cudaError_t Launch<T>::mask_b(const BTables &b, const int *rep_n, const T *rep_s0, const T *rep_w,
                              const void *spec, const T *ip, void *hc0, void *hc1,
                              double *partial, cudaStream_t s) {
    using C = typename PT<T>::C;
    if (b.dim == 2)
        k_mask_b<T, 2><<<(unsigned)b.n_mblk, 256, 0, s>>>(b.inst, b.mblk_first, b.n_inst, rep_n,
                                                          rep_s0, rep_w, (const C *)spec, ip,
                                                          (C *)hc0, (C *)hc1, partial);
    else
        k_mask_b<T, 3><<<(unsigned)b.n_mblk, 256, 0, s>>>(b.inst, b.mblk_first, b.n_inst, rep_n,
                                                          rep_s0, rep_w, (const C *)spec, ip,
                                                          (C *)hc0, (C *)hc1, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::finalize_b(const BTables &b, const double *partial, double *losses,
                                  cudaStream_t s) {
    k_finalize_b<<<b.n_inst, 256, 0, s>>>(b.inst, b.mblk_first, partial, losses);
    return cudaGetLastError();
}

}  // namespace fresco
