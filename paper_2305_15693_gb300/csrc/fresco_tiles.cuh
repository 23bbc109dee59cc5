// Single-plan binning and type-1 spreading over tiles without border sub-bins.
//
// Binning (K1). A plan whose tiles can hold their expected points plus a wide margin in a fixed
// capacity Geom.tcap per tile places every point in one pass over the caller's points:
//   k_place_direct  computes each point's tile and record and takes its slot from the tile's
//                   cursor, pos = atomicAdd(&tcur[t], 1), at record t * tcap + pos;
// the tile's points are then records [t tcap, t tcap + tcur[t]). A point whose tile is full sets
// the overflow word tcur[n_tiles]; the compact form below then runs (its kernels do nothing
// unless the overflow word is set), so any input is binned correctly and uniform inputs pay for
// one pass only. The compact form, two passes with no per-point key or rank arrays:
//   k_count  counts the points of every bin (global atomics whose result is unused);
//   (exclusive scan of the counts into off[], and a copy of off[] into the cursor array cur[])
//   k_place  recomputes each point's bin and record and takes its sorted position from the
//            bin's cursor, pos = atomicAdd(&cur[bin], 1).
// In the compact form a tile owns Geom.sub consecutive bins, bin = tile * sub + (caller index mod
// sub): the points of a tile stay contiguous (off[t sub] .. off[(t + 1) sub]), and each cursor
// takes 1/sub of the tile's atomics, which keeps the returning atomics from queueing on few
// addresses. k_tile_ranges writes the record range of every tile, tr[t] = (first, end), from
// whichever form ran; the spread and interpolation kernels read only tr.
// The order of the points inside a tile depends on the order the atomics run in. Nothing
// downstream depends on it: the fixed-point spread sums integers (order independent), the
// interpolation writes each point's gradient through its caller index.
//
// Spreading (K2) with own points only: the block of tile t accumulates the full kernel windows of
// the points of tile t into the tile's extended region (the tile plus W/2 cells below and
// W - W/2 above on each axis, where a window of a point of the tile can reach) in shared memory,
// with no bounds checks. It writes the tile's own cells to the grid and the rest of the region
// (its ring) to a per-tile ring buffer; k_halo_fold then adds to every cell near a tile border the
// ring values that the neighbouring tiles' points put there, in a fixed order.
//
// Ring layout of one tile (extents E_a = w_a + W, HL = W/2): the extended region is walked plane
// by plane (z) and row by row (y); rows that lie outside the tile (in y or z) are stored whole
// (E_x cells), rows through the tile store only their W halo cells (HL below the tile in x, then
// W - HL above). ring_index maps an extended-region cell outside the tile to its position.
#pragma once

#include <utility>

namespace fresco {

template <int W, int D>
__host__ __device__ __forceinline__ int ring_index(int ex, int ey, int ez, int wx, int wy, int wz) {
    constexpr int HL = W / 2;
    const int Ex = wx + W, Ey = wy + W;
    const int full_plane = Ex * Ey;
    const int mid_plane = W * Ex + wy * W;
    int base = 0;
    bool mid = true;
    if (D == 3) {
        if (ez < HL) {
            base = ez * full_plane;
            mid = false;
        } else if (ez < HL + wz) {
            base = HL * full_plane + (ez - HL) * mid_plane;
        } else {
            base = HL * full_plane + wz * mid_plane + (ez - HL - wz) * full_plane;
            mid = false;
        }
    }
    if (!mid || ey < HL) return base + ey * Ex + ex;
    if (ey < HL + wy) return base + HL * Ex + (ey - HL) * W + (ex < HL ? ex : ex - wx);
    return base + HL * Ex + wy * W + (ey - HL - wy) * Ex + ex;
}

// ring cells of a tile of widths w (unused axes 1)
template <int W, int D>
__host__ __device__ inline int64_t ring_cells(int wx, int wy, int wz) {
    int64_t e = (int64_t)(wx + W) * (wy + W), i = (int64_t)wx * wy;
    if (D == 3) {
        e *= wz + W;
        i *= wz;
    }
    return e - i;
}

// tile of a point along every axis, its cell relative to the tile and the fraction
template <typename T, int D>
__device__ __forceinline__ int tile_cell(const Geom &g, const T (&r)[3], int (&rel)[3],
                                         T (&frac)[3], bool &ok) {
    int t[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int cell;
        ok &= fine_coord<T>(r[a], (T)g.s_hi[a], (T)g.s_lo[a], g.nf[a], cell, frac[a]);
        t[a] = tile_of_cell(cell, g.tq[a], g.tr[a], g.tinv[a]);
        rel[a] = cell - tile_start(t[a], g.tq[a], g.tr[a]);
    }
    return t[0] + g.nb[0] * (t[1] + g.nb[1] * t[2]);
}

// Whether some lane of the warp has the same bin as the lane before it: points that arrive in
// tile order (a solver that keeps them so) form runs, and the warp then combines its atomics per
// bin; points in random order almost never do, and skip the (costlier) matching.
__device__ __forceinline__ bool warp_has_runs(int bin, bool in) {
    const int prev = __shfl_up_sync(0xffffffffu, bin, 1);
    return __any_sync(0xffffffffu, in && (threadIdx.x & 31) > 0 && prev == bin);
}

// guard (k_count, k_place): when not null, the kernel does nothing unless *guard != 0
template <typename T, int D>
__global__ void __launch_bounds__(256) k_count(Geom g, const T *__restrict__ pts,
                                               int *__restrict__ cnt, int *__restrict__ err,
                                               const int *__restrict__ guard) {
    if (guard && !*guard) return;
    constexpr int IL = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * IL;
    bool ok = true;
    // the loop runs warp-uniformly (whole warps take part in the warp-level matching below)
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x * IL + (threadIdx.x & ~31u);
         w0 < g.n_points; w0 += stride) {
        const int64_t j0 = w0 + (threadIdx.x & 31);
        T r[IL][3];
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = j0 + (int64_t)k * blockDim.x;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                r[k][a] = (a < D && j < g.n_points) ? pts[j * D + a] : T(0);
        }
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = j0 + (int64_t)k * blockDim.x;
            int rel[3];
            T frac[3];
            const int t = tile_cell<T, D>(g, r[k], rel, frac, ok);
            const bool in = j < g.n_points;
            const int bin = in ? t * g.sub + (int)(j % g.sub) : -1;
            if (warp_has_runs(bin, in)) {
                // lanes that hit the same bin (points in tile order) add once together
                const unsigned grp = __match_any_sync(0xffffffffu, bin);
                if (in && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&cnt[bin], __popc(grp));
            } else if (in) {
                atomicAdd(&cnt[bin], 1);
            }
        }
    }
    if (!ok) atomicOr(err, 1);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_place(Geom g, const T *__restrict__ pts,
                                               int *__restrict__ cur,
                                               typename PT<T>::U *__restrict__ sorted,
                                               int *__restrict__ perm,
                                               const int *__restrict__ guard) {
    if (guard && !*guard) return;
    using U = typename PT<T>::U;
    constexpr int IL = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * IL;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x * IL + (threadIdx.x & ~31u);
         w0 < g.n_points; w0 += stride) {
        const int64_t j0 = w0 + (threadIdx.x & 31);
        T r[IL][3];
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = j0 + (int64_t)k * blockDim.x;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                r[k][a] = (a < D && j < g.n_points) ? pts[j * D + a] : T(0);
        }
        int pos[IL];
        U u[IL][3];
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = j0 + (int64_t)k * blockDim.x;
            int rel[3] = {0, 0, 0};
            T frac[3] = {T(0), T(0), T(0)};
            bool ok = true;
            const int t = tile_cell<T, D>(g, r[k], rel, frac, ok);
#pragma unroll
            for (int a = 0; a < 3; ++a) u[k][a] = a < D ? pack_coord<T>(rel[a], frac[a]) : U(0);
            const bool in = j < g.n_points;
            const int bin = in ? t * g.sub + (int)(j % g.sub) : -1;
            if (warp_has_runs(bin, in)) {
                // one cursor atomic per bin and warp; lanes take consecutive slots in lane order
                const unsigned grp = __match_any_sync(0xffffffffu, bin);
                const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
                int base = 0;
                if (in && lane == leader) base = atomicAdd(&cur[bin], __popc(grp));
                base = __shfl_sync(grp, base, leader);
                pos[k] = base + __popc(grp & ((1u << lane) - 1u));
            } else {
                pos[k] = in ? atomicAdd(&cur[bin], 1) : 0;
            }
        }
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = j0 + (int64_t)k * blockDim.x;
            if (j < g.n_points) store_record<T, D>(sorted, perm, pos[k], u[k], (int)j);
        }
    }
}

// One pass of the direct form: points j0 .. j0 + g.n_points - 1 of the caller's array (pts points
// at point j0), each to its tile's next slot. tcur[n_tiles] is the overflow word.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_place_direct(Geom g, const T *__restrict__ pts,
                                                      int64_t j0, int *__restrict__ tcur,
                                                      typename PT<T>::U *__restrict__ sorted,
                                                      int *__restrict__ perm,
                                                      int *__restrict__ err) {
    using U = typename PT<T>::U;
    constexpr int IL = kDirectPointsPerThread;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * IL;
    const int cap = g.tcap;
    bool ok = true, over = false;
    // the loop runs warp-uniformly (whole warps take part in the warp-level matching below)
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x * IL + (threadIdx.x & ~31u);
         w0 < g.n_points; w0 += stride) {
        const int64_t jl = w0 + (threadIdx.x & 31);
        T r[IL][3];
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = jl + (int64_t)k * blockDim.x;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                r[k][a] = (a < D && j < g.n_points) ? pts[j * D + a] : T(0);
        }
        int pos[IL], tile[IL];
        U u[IL][3];
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = jl + (int64_t)k * blockDim.x;
            int rel[3] = {0, 0, 0};
            T frac[3] = {T(0), T(0), T(0)};
            const int t = tile_cell<T, D>(g, r[k], rel, frac, ok);
#pragma unroll
            for (int a = 0; a < 3; ++a) u[k][a] = a < D ? pack_coord<T>(rel[a], frac[a]) : U(0);
            const bool in = j < g.n_points;
            tile[k] = in ? t : -1;
            if (warp_has_runs(tile[k], in)) {
                // one cursor atomic per tile and warp; lanes take consecutive slots in lane order
                const unsigned grp = __match_any_sync(0xffffffffu, tile[k]);
                const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
                int base = 0;
                if (in && lane == leader) base = atomicAdd(&tcur[t], __popc(grp));
                base = __shfl_sync(grp, base, leader);
                pos[k] = base + __popc(grp & ((1u << lane) - 1u));
            } else {
                pos[k] = in ? atomicAdd(&tcur[t], 1) : 0;
            }
        }
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            const int64_t j = jl + (int64_t)k * blockDim.x;
            if (j >= g.n_points) continue;
            if (pos[k] < cap)
                store_record<T, D>(sorted, perm, (int64_t)tile[k] * cap + pos[k], u[k],
                                   (int)(j0 + j));
            else
                over = true;
        }
    }
    if (!ok) atomicOr(err, 1);
    if (over) atomicOr(&tcur[g.n_tiles], 1);
}

// Record range of every tile: the direct form's (t tcap, t tcap + tcur[t]) unless its overflow
// word is set (or the plan has no direct form, tcur null), else the compact form's offsets.
static __global__ void __launch_bounds__(256) k_tile_ranges(Geom g, const int *__restrict__ tcur,
                                                            const int *__restrict__ off,
                                                            int2 *__restrict__ tr) {
    const bool direct = tcur && !tcur[g.n_tiles];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < g.n_tiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (direct) {
            const int b = (int)(t * g.tcap);
            tr[t] = make_int2(b, b + tcur[t]);
        } else {
            tr[t] = make_int2(off[t * g.sub], off[(t + 1) * g.sub]);
        }
    }
}

// Shared-memory accesses of the window loops, written as PTX on 32-bit shared-space addresses
// with the offset inside the window row as an immediate, so that each cell of a window costs one
// memory instruction (plus the arithmetic of its value) and no address arithmetic. They carry no
// memory clobber (that would make the compiler reload every value around each access); their
// order against the block's other shared-memory traffic comes from the __syncthreads() that
// separate the phases of the kernels (staging / accumulation / write-out).
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

template <int OFF>
__device__ __forceinline__ void red_add_shared(unsigned addr, int v) {
    asm volatile("red.shared.add.s32 [%0+%2], %1;" ::"r"(addr), "r"(v), "n"(OFF));
}

template <int OFF>
__device__ __forceinline__ float ld_shared_f32(unsigned addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
    return v;
}

// row[a] += round(ws * wx[a] * 2^s) for a < W (ws carries the scale), as fixed-point integers:
// adding 1.5 * 2^23 rounds the product to an integer held in the low mantissa bits.
template <int W, int... A>
__device__ __forceinline__ void red_row_fixed(unsigned row, float ws, const float (&wx)[W],
                                              std::integer_sequence<int, A...>) {
    (red_add_shared<4 * A>(row, __float_as_int(fmaf(ws, wx[A], 12582912.0f)) - 0x4B400000), ...);
}

template <int A, int W>
__device__ __forceinline__ void dot_cell_kd(unsigned row, const float (&wx)[W],
                                            const float (&dwx)[W], float &r0, float &r1) {
    const float v = ld_shared_f32<4 * A>(row);
    r0 = fmaf(wx[A], v, r0);
    r1 = fmaf(dwx[A], v, r1);
}

// (sum_a wx[a] row[a], sum_a dwx[a] row[a]) for a < W, one load per cell
template <int W, int... A>
__device__ __forceinline__ void dot_row_kd(unsigned row, const float (&wx)[W],
                                           const float (&dwx)[W], float &r0, float &r1,
                                           std::integer_sequence<int, A...>) {
    (dot_cell_kd<A, W>(row, wx, dwx, r0, r1), ...);
}

// Bytes of a tile's extended region in shared memory (rounded up to 16), before the index list.
__host__ __device__ inline size_t spread_own_tile_bytes(const Geom &g, size_t esize) {
    const int w = g.width;
    size_t cells = (size_t)(g.tmax[0] + w) * (g.tmax[1] + w) * (g.dim == 3 ? (g.tmax[2] + w) : 1);
    return (cells * (esize > 4 ? esize : 4) + 15) & ~(size_t)15;
}

// One point's full window into the extended region (i0: window start in extended-region
// coordinates, which keeps the whole window inside the region), no bounds checks.
template <typename T, int W, int D>
__device__ __forceinline__ void spread_point_own(const EsPoly<T> &ep, const int (&i0)[3],
                                                 const T (&x1)[3], int Ex, int Exy, T *ftile,
                                                 int *itile, bool fixed, float fscale) {
    T wx[W], wy[W];
    es_weights<T, W>(ep, x1[0], wx);
    es_weights<T, W>(ep, x1[1], wy);
    if constexpr (D == 2) {
        if constexpr (sizeof(T) == 4) {
            if (fixed) {
                const unsigned step = 4u * (unsigned)Ex;
                unsigned row = smem_addr(itile) + 4u * (unsigned)(i0[1] * Ex + i0[0]);
#pragma unroll
                for (int b = 0; b < W; ++b, row += step)
                    red_row_fixed<W>(row, wy[b] * fscale, wx, std::make_integer_sequence<int, W>{});
                return;
            }
        }
        T *base = ftile + i0[1] * Ex + i0[0];
#pragma unroll
        for (int b = 0; b < W; ++b)
#pragma unroll
            for (int a = 0; a < W; ++a) atomicAdd(base + b * Ex + a, wy[b] * wx[a]);
    } else {
        T wz[W];
        es_weights<T, W>(ep, x1[2], wz);
        const int o = (i0[2] * Exy) + i0[1] * Ex + i0[0];
        if constexpr (sizeof(T) == 4) {
            if (fixed) {
                const unsigned step = 4u * (unsigned)Ex, pstep = 4u * (unsigned)Exy;
                unsigned plane = smem_addr(itile) + 4u * (unsigned)o;
#pragma unroll (W <= 8 ? W : 1)
                for (int c = 0; c < W; ++c, plane += pstep) {
                    const float wzs = wz[c] * fscale;
                    unsigned row = plane;
#pragma unroll
                    for (int b = 0; b < W; ++b, row += step)
                        red_row_fixed<W>(row, wzs * wy[b], wx, std::make_integer_sequence<int, W>{});
                }
                return;
            }
        }
#pragma unroll 1
        for (int c = 0; c < W; ++c) {
            T *plane = ftile + o + c * Exy;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const T wzy = wz[c] * wy[b];
#pragma unroll
                for (int a = 0; a < W; ++a) atomicAdd(plane + b * Ex + a, wzy * wx[a]);
            }
        }
    }
}

// Extended-region extents (and tile start / widths) of tile t.
__device__ __forceinline__ void tile_extent(const Geom &g, int64_t t, int W, int (&s)[3],
                                            int (&w)[3], int (&tc)[3]) {
    tc[0] = (int)(t % g.nb[0]);
    tc[1] = (int)((t / g.nb[0]) % g.nb[1]);
    tc[2] = (int)(t / ((int64_t)g.nb[0] * g.nb[1]));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < g.dim) {
            s[a] = tile_start(tc[a], g.tq[a], g.tr[a]);
            w[a] = tile_start(tc[a] + 1, g.tq[a], g.tr[a]) - s[a];
        } else {
            s[a] = 0;
            w[a] = 1;
        }
    }
}

// Points of tile t are spread in FP32 plans in 32-bit fixed point with scale 2^s, s = min(21,
// clz(P) - 1) for P points, when P < kFixedMaxPoints (s >= 17: every contribution rounded to at
// most 2^-18, and no cell sum can reach 2^31 because every weight is at most 1); a more crowded
// tile accumulates float atomics. Double plans accumulate double atomics.
constexpr int kFixedMaxPoints = 1 << 14;

// Bank-residue schedule. A point's window starts at word b = i0_z E_xy + i0_y E_x + i0_x of the
// extended region, and every step of the window loop adds the same offset to the start of all
// lanes; so a warp whose 32 points have 32 distinct residues b mod 32 touches 32 distinct
// shared-memory banks at every step (no bank conflicts). The block counts its points per residue
// (cnt[j] points of residue j) and lists them level by level: level q holds the (q+1)-th point
// of every residue with more than q points, in residue order, and the levels follow each other
// without gaps. Consecutive runs of 32 list entries then hold 32 distinct residues where they lie
// inside one level and at most two points of a residue where they span two (the few short levels
// at the end, where only the most crowded residues are left, conflict more), and every lane of
// every warp round has a point but in the last round: lanes are not left idle for the residues
// with fewer points, as a residue-per-lane schedule would (the largest of 32 Poisson counts is
// ~1.3 times their mean at 50 points a tile, ~1.6 times at 13).
template <typename T, int W, int D>
__device__ __forceinline__ int window_of(const typename PT<T>::U (&u)[3], int Ex, int Exy,
                                         int (&i0)[3], T (&x1)[3]) {
    constexpr int HL = W / 2;
    i0[0] = i0[1] = i0[2] = 0;
    x1[0] = x1[1] = x1[2] = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int rel;
        T f;
        unpack_coord<T>(u[a], rel, f);
        i0[a] = rel + support_start<T, W>(f, x1[a]) + HL;
    }
    return (i0[2] * Exy + i0[1] * Ex + i0[0]) & 31;
}

// Levels the schedule tabulates; a tile with a residue of more points (clustered input) lists its
// points in arrival order instead (correct, with bank conflicts).
constexpr int kResidueLevels = 128;

// Shared state of the schedule. cnt must be zero (and visible to the block) before the call.
struct ResidueShared {
    int cnt[32];
    int cur[32];
    unsigned mask[kResidueLevels];   // residues with more than q points
    int pre[kResidueLevels];         // entries in the levels before q
    int levels;                      // largest count, or -1 beyond kResidueLevels
};

// Lists the block's points [p0, p1) in the level order above: put(slot, i0, x1, w3) stores the
// entry of one point at list position slot (w3: the caller index a float record carries, 0 for
// double records). Returns the number of entries, P = p1 - p0 (needs P <= list_cap); on return
// the entries are visible to the block.
template <typename T, int W, int D, typename Put>
__device__ __forceinline__ int residue_lists(const typename PT<T>::U *__restrict__ sorted, int p0,
                                             int p1, int Ex, int Exy, ResidueShared &rs,
                                             Put put) {
    using U = typename PT<T>::U;
    constexpr int IL = 4;   // records per thread in flight
    const int bs = blockDim.x;
    for (int p = p0 + threadIdx.x; p < p1; p += IL * bs) {
        U u[IL][3];
#pragma unroll
        for (int k = 0; k < IL; ++k)
            if (p + k * bs < p1) load_packed<T, D>(sorted, p + k * bs, u[k]);
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            if (p + k * bs >= p1) break;
            int i0[3];
            T x1[3];
            atomicAdd(&rs.cnt[window_of<T, W, D>(u[k], Ex, Exy, i0, x1)], 1);
        }
    }
    __syncthreads();
    {   // level masks (every warp takes every nw-th level), then their prefix sums (warp 0)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = bs >> 5;
        const int c = rs.cnt[lane];
        int m = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (m <= kResidueLevels) {
            for (int q = wid; q < m; q += nw) {
                const unsigned msk = __ballot_sync(0xffffffffu, c > q);
                if (lane == 0) rs.mask[q] = msk;
            }
        }
        if (threadIdx.x < 32) rs.cur[threadIdx.x] = 0;
        __syncthreads();
        if (wid == 0 && m <= kResidueLevels) {
            int run = 0;
            for (int q0 = 0; q0 < m; q0 += 32) {
                const int q = q0 + lane;
                const int v = q < m ? __popc(rs.mask[q]) : 0;
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (q < m) rs.pre[q] = run + x - v;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        if (threadIdx.x == 0) rs.levels = m <= kResidueLevels ? m : -1;
        __syncthreads();
    }
    const bool leveled = rs.levels >= 0;
    for (int p = p0 + threadIdx.x; p < p1; p += IL * bs) {
        U u[IL][3];
        unsigned w3[IL];
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            w3[k] = 0;
            if (p + k * bs < p1) {
                if constexpr (sizeof(T) == 4) {
                    const uint4 v = reinterpret_cast<const uint4 *>(sorted)[p + k * bs];
                    u[k][0] = v.x;
                    u[k][1] = v.y;
                    u[k][2] = v.z;
                    w3[k] = v.w;
                } else {
                    load_packed<T, D>(sorted, p + k * bs, u[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            if (p + k * bs >= p1) break;
            int i0[3];
            T x1[3];
            const int r = window_of<T, W, D>(u[k], Ex, Exy, i0, x1);
            int slot;
            if (leveled) {
                const int q = atomicAdd(&rs.cur[r], 1);
                slot = rs.pre[q] + __popc(rs.mask[q] & ((1u << r) - 1u));
            } else {
                slot = atomicAdd(&rs.cur[0], 1);
            }
            put(slot, i0, x1, w3[k]);
        }
    }
    __syncthreads();
    return p1 - p0;
}

template <typename T, int W, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_spread_own(
    Geom g, EsPoly<T> ep, const typename PT<T>::U *__restrict__ sorted,
    const int2 *__restrict__ tr, T *__restrict__ grid, T *__restrict__ ring,
    int64_t ring_slot) {
    using U = typename PT<T>::U;
    constexpr int HL = W / 2;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ ResidueShared s_rl;
    T *ftile = reinterpret_cast<T *>(sm_raw);
    int *itile = reinterpret_cast<int *>(sm_raw);
    // level-ordered entries: packed window start (10 bits per axis) and kernel offsets
    int *l_i0 = reinterpret_cast<int *>(sm_raw + spread_own_tile_bytes(g, sizeof(T)));
    float *l_x1 = reinterpret_cast<float *>(l_i0 + g.list_cap);
    const int64_t t = blockIdx.x;
    int s[3], w[3], tc[3];
    tile_extent(g, t, W, s, w, tc);
    const int Ex = w[0] + W, Ey = w[1] + W, Ez = D == 3 ? w[2] + W : 1;
    const int Exy = Ex * Ey, cells = Exy * Ez;
    const int p0 = tr[t].x, p1 = tr[t].y;
    const int P = p1 - p0;
    bool fixed = false;
    int sc = 0;
    if constexpr (sizeof(T) == 4) {
        fixed = P < kFixedMaxPoints;
        sc = fixed ? min(21, __clz(max(P, 1)) - 1) : 0;
    }
    {   // zero the region, 16 bytes per store (the region starts 16-byte aligned)
        const int words = cells * (int)(sizeof(T) / 4);
        uint4 *z4 = reinterpret_cast<uint4 *>(sm_raw);
        for (int i = threadIdx.x; i < words / 4; i += blockDim.x) z4[i] = make_uint4(0, 0, 0, 0);
        for (int i = (words & ~3) + threadIdx.x; i < words; i += blockDim.x) itile[i] = 0;
    }
    if (threadIdx.x < 32) s_rl.cnt[threadIdx.x] = 0;
    __syncthreads();
    const float fscale = __int_as_float((127 + sc) << 23);   // 2^sc
    const bool listed = sizeof(T) == 4 && fixed && P <= g.list_cap;
    if (listed) {
        const int cap = g.list_cap;
        const int n = residue_lists<T, W, D>(
            sorted, p0, p1, Ex, Exy, s_rl,
            [&](int slot, const int (&i0)[3], const T (&x1)[3], unsigned) {
                l_i0[slot] = i0[0] | (i0[1] << 10) | (i0[2] << 20);
#pragma unroll
                for (int a = 0; a < D; ++a) l_x1[a * cap + slot] = (float)x1[a];
            });
        for (int h = threadIdx.x; h < n; h += blockDim.x) {
            const int pk = l_i0[h];
            const int i0[3] = {pk & 1023, (pk >> 10) & 1023, pk >> 20};
            T x1[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int a = 0; a < D; ++a) x1[a] = (T)l_x1[a * cap + h];
            spread_point_own<T, W, D>(ep, i0, x1, Ex, Exy, ftile, itile, true, fscale);
        }
    } else {
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            U u[3];
            load_packed<T, D>(sorted, p, u);
            int i0[3];
            T x1[3];
            window_of<T, W, D>(u, Ex, Exy, i0, x1);
            spread_point_own<T, W, D>(ep, i0, x1, Ex, Exy, ftile, itile, fixed, fscale);
        }
    }
    __syncthreads();
    const float finv = __int_as_float((127 - sc) << 23);     // 2^-sc
    T *myring = ring + t * ring_slot;
    if constexpr (D == 2) {
        // one warp per row of the region (rows of at least W + 2 cells, most several warps wide):
        // the cells inside the tile go to the grid, the others to the ring, whose cells of one
        // row are contiguous
        const int lane = threadIdx.x & 31;
        for (int ey = threadIdx.x >> 5; ey < Ey; ey += blockDim.x >> 5) {
            const bool through = ey >= HL && ey < HL + w[1];
            const int64_t gbase = (int64_t)(s[1] + ey - HL) * g.nf[0] + s[0] - HL;
            T *rrow = myring + ring_index<W, D>(0, ey, 0, w[0], w[1], w[2]);
            for (int ex = lane; ex < Ex; ex += 32) {
                const int i = ey * Ex + ex;
                T v;
                if constexpr (sizeof(T) == 4) v = fixed ? (float)itile[i] * finv : ftile[i];
                else v = ftile[i];
                if (!through) rrow[ex] = v;
                else if (ex < HL) rrow[ex] = v;
                else if (ex >= HL + w[0]) rrow[ex - w[0]] = v;
                else grid[gbase + ex] = v;
            }
        }
    } else {
        // 3D rows are short (a warp's lanes would mostly idle per row): one cell per thread and
        // step, its row and plane by multiply-high division
        const FastDiv fex = tile_div<0, true>(g, w[0]), fey = tile_div<1, true>(g, w[1]);
        const int64_t gorg =
            ((int64_t)(s[2] - HL) * g.nf[1] + (s[1] - HL)) * g.nf[0] + s[0] - HL;
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            const int row = fex.div(i), ex = i - row * Ex;
            const int ez = fey.div(row), ey = row - ez * Ey;
            T v;
            if constexpr (sizeof(T) == 4) v = fixed ? (float)itile[i] * finv : ftile[i];
            else v = ftile[i];
            const bool through = ez >= HL && ez < HL + w[2] && ey >= HL && ey < HL + w[1];
            if (through && ex >= HL && ex < HL + w[0]) {
                grid[gorg + ((int64_t)ez * g.nf[1] + ey) * g.nf[0] + ex] = v;
            } else {
                const int r = ring_index<W, D>(0, ey, ez, w[0], w[1], w[2]);
                myring[r + (through && ex >= HL + w[0] ? ex - w[0] : ex)] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// 3D column spread: one block walks a segment of g.zseg tiles of one (x, y) column along z and
// keeps the planes of the current tile's extended region in a circular buffer of NP = tmax_z + W
// planes in shared memory. The w planes a tile shares with the next (its top halo and the next
// tile's bottom halo) stay in the buffer, so the z halo between the tiles of a segment is summed
// on chip; a plane is written out once no later point of the segment can reach it: its cells
// inside the column go to the grid, its x/y halo cells to the ring of the tile that owns the
// plane, and the planes beyond the segment's ends to the z halo planes of the first / last tile's
// ring. The rings are then folded z first (segment ends only), then x, then y. The plane stride
// is a multiple of 32 words, so a window's bank residue does not depend on its plane and the
// residue schedule stays conflict free across the wrap of the buffer. All tiles of a segment use
// one fixed-point scale, set by the three most crowded consecutive tiles that can reach a plane.
// Where one plane of a column's buffer goes: its slot in the circular buffer, whether it lies in
// its owner tile along z, its owner's ring plane (offset into the ring buffer) and the grid cell
// of its extended region's first row and column.
struct ColPlane {
    int slot;
    int zin;
    int64_t roff;
    int64_t goff;
};

__host__ __device__ inline int col_plane_stride(const Geom &g) {
    return ((g.tmax[0] + g.width) * (g.tmax[1] + g.width) + 31) & ~31;
}
__host__ __device__ inline size_t spread_col_tile_bytes(const Geom &g, size_t esize) {
    const size_t words = (size_t)(g.tmax[2] + g.width) * col_plane_stride(g);
    return (words * (esize > 4 ? esize : 4) + 15) & ~(size_t)15;
}

template <typename T, int W>
__device__ __forceinline__ void spread_point_col(const EsPoly<T> &ep, const int (&i0)[3],
                                                 const T (&x1)[3], int Ex, int Sxy, int NP,
                                                 int plane0, T *ftile, int *itile, bool fixed,
                                                 float fscale) {
    T wx[W], wy[W], wz[W];
    es_weights<T, W>(ep, x1[0], wx);
    es_weights<T, W>(ep, x1[1], wy);
    es_weights<T, W>(ep, x1[2], wz);
    const int oxy = i0[1] * Ex + i0[0];
    if constexpr (sizeof(T) == 4) {
        if (fixed) {
            const unsigned base = smem_addr(itile) + 4u * (unsigned)oxy;
            const unsigned step = 4u * (unsigned)Ex;
#pragma unroll (W <= 8 ? W : 1)
            for (int c = 0; c < W; ++c) {
                int pl = plane0 + c;
                pl -= pl >= NP ? NP : 0;
                unsigned row = base + 4u * (unsigned)(pl * Sxy);
                const float wzs = wz[c] * fscale;
#pragma unroll
                for (int b = 0; b < W; ++b, row += step)
                    red_row_fixed<W>(row, wzs * wy[b], wx, std::make_integer_sequence<int, W>{});
            }
            return;
        }
    }
#pragma unroll 1
    for (int c = 0; c < W; ++c) {
        int pl = plane0 + c;
        pl -= pl >= NP ? NP : 0;
        T *plane = ftile + (int64_t)pl * Sxy + oxy;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const T wzy = wz[c] * wy[b];
#pragma unroll
            for (int a = 0; a < W; ++a) atomicAdd(plane + b * Ex + a, wzy * wx[a]);
        }
    }
}

template <typename T, int W>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_spread_col(
    Geom g, EsPoly<T> ep, const typename PT<T>::U *__restrict__ sorted,
    const int2 *__restrict__ tr, T *__restrict__ grid, T *__restrict__ ring,
    int64_t ring_slot) {
    using U = typename PT<T>::U;
    constexpr int D = 3, HL = W / 2, HR = W - HL;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ ResidueShared s_rl;
    __shared__ ColPlane s_pl[kColMaxPlanes];
    __shared__ int s_pmax;
    T *ftile = reinterpret_cast<T *>(sm_raw);
    int *itile = reinterpret_cast<int *>(sm_raw);
    const int cap = g.list_cap;
    int *l_i0 = reinterpret_cast<int *>(sm_raw + spread_col_tile_bytes(g, sizeof(T)));
    float *l_x1 = reinterpret_cast<float *>(l_i0 + cap);
    const int bid = blockIdx.x;
    const int tx = bid % g.nb[0], ty = (bid / g.nb[0]) % g.nb[1];
    const int tz0 = (bid / (g.nb[0] * g.nb[1])) * g.zseg;
    const int nz = min(g.zseg, g.nb[2] - tz0);
    const int sx = tile_start(tx, g.tq[0], g.tr[0]);
    const int wx = tile_start(tx + 1, g.tq[0], g.tr[0]) - sx;
    const int sy = tile_start(ty, g.tq[1], g.tr[1]);
    const int wy = tile_start(ty + 1, g.tq[1], g.tr[1]) - sy;
    const int Ex = wx + W, Ey = wy + W;
    const int Sxy = col_plane_stride(g), NP = g.tmax[2] + W;
    const int zfirst = tile_start(tz0, g.tq[2], g.tr[2]);
    const int zend = tile_start(tz0 + nz, g.tq[2], g.tr[2]);
    const int zlast = tile_start(tz0 + nz - 1, g.tq[2], g.tr[2]);
    const int zbase = zfirst - HL;   // plane zbase is slot 0
    auto tile_id = [&](int tz) -> int64_t {
        return ((int64_t)tz * g.nb[1] + ty) * g.nb[0] + tx;
    };
    if (threadIdx.x == 0) s_pmax = 0;
    __syncthreads();
    if ((int)threadIdx.x < nz) {
        const int64_t t = tile_id(tz0 + threadIdx.x);
        atomicMax(&s_pmax, tr[t].y - tr[t].x);
    }
    {   // zero the buffer, 16 bytes per store
        const int words = NP * Sxy * (int)(sizeof(T) / 4);
        uint4 *z4 = reinterpret_cast<uint4 *>(sm_raw);
        for (int i = threadIdx.x; i < words / 4; i += blockDim.x) z4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    const int P3 = 3 * s_pmax;
    bool fixed = false;
    int sc = 0;
    if constexpr (sizeof(T) == 4) {
        fixed = P3 < kFixedMaxPoints;
        sc = fixed ? min(21, __clz(max(P3, 1)) - 1) : 0;
    }
    const float fscale = __int_as_float((127 + sc) << 23);   // 2^sc
    const float finv = __int_as_float((127 - sc) << 23);     // 2^-sc
    for (int k = 0; k < nz; ++k) {
        const int tz = tz0 + k;
        const int64_t t = tile_id(tz);
        const int zk = tile_start(tz, g.tq[2], g.tr[2]);
        const int wz = tile_start(tz + 1, g.tq[2], g.tr[2]) - zk;
        const int r0 = (zk - HL - zbase) % NP;     // buffer plane of the region's first plane
        const int p0 = tr[t].x, p1 = tr[t].y;
        if ((int)threadIdx.x < (k + 1 < nz ? wz : wz + W)) {
            // destinations of the plane this thread describes (written out after this tile)
            const int pz = zk - HL + (int)threadIdx.x;
            int owner, ez, wo;
            if (pz < zfirst) {
                owner = tz0;
                ez = pz - (zfirst - HL);
                wo = tile_start(tz0 + 1, g.tq[2], g.tr[2]) - zfirst;
            } else if (pz >= zend) {
                owner = tz0 + nz - 1;
                ez = pz - (zlast - HL);
                wo = zend - zlast;
            } else {
                owner = pz < zk ? tz - 1 : tz;
                const int zo = owner == tz ? zk : tile_start(owner, g.tq[2], g.tr[2]);
                ez = pz - zo + HL;
                wo = (owner == tz ? zk + wz : zk) - zo;
            }
            ColPlane &pl = s_pl[threadIdx.x];
            pl.zin = ez >= HL && ez < HL + wo;
            pl.slot = (r0 + (int)threadIdx.x) % NP;
            pl.roff = tile_id(owner) * ring_slot + ring_index<W, D>(0, 0, ez, wx, wy, wo);
            const int64_t gz = pz < 0 ? pz + g.nf[2] : (pz >= g.nf[2] ? pz - g.nf[2] : pz);
            pl.goff = (gz * g.nf[1] + sy - HL) * g.nf[0] + sx - HL;
        }
        if (threadIdx.x < 32) s_rl.cnt[threadIdx.x] = 0;
        __syncthreads();
        if (fixed && p1 - p0 <= cap) {
            const int n = residue_lists<T, W, D>(
                sorted, p0, p1, Ex, Sxy, s_rl,
                [&](int slot, const int (&i0)[3], const T (&x1)[3], unsigned) {
                    l_i0[slot] = i0[0] | (i0[1] << 10) | (i0[2] << 20);
#pragma unroll
                    for (int a = 0; a < D; ++a) l_x1[a * cap + slot] = (float)x1[a];
                });
            for (int h = threadIdx.x; h < n; h += blockDim.x) {
                const int pk = l_i0[h];
                const int i0[3] = {pk & 1023, (pk >> 10) & 1023, pk >> 20};
                const T x1[3] = {(T)l_x1[h], (T)l_x1[cap + h], (T)l_x1[2 * cap + h]};
                int pl = r0 + i0[2];
                pl -= pl >= NP ? NP : 0;
                spread_point_col<T, W>(ep, i0, x1, Ex, Sxy, NP, pl, ftile, itile, true, fscale);
            }
        } else {
            for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
                U u[3];
                load_packed<T, D>(sorted, p, u);
                int i0[3];
                T x1[3];
                window_of<T, W, D>(u, Ex, Sxy, i0, x1);
                spread_point_col<T, W>(ep, i0, x1, Ex, Sxy, NP, (r0 + i0[2]) % NP, ftile, itile,
                                       fixed, fscale);
            }
        }
        __syncthreads();
        // planes no later point of the segment reaches: [zk - HL, zk + wz - HL), or to the end.
        // Every plane's destinations (its owner tile's ring plane, or its grid plane, and its
        // buffer slot) are worked out once (s_pl, filled before the spread loop's barrier), then
        // the threads take the cells of all these planes one per step.
        const int pz0 = zk - HL;
        const int npl = k + 1 < nz ? wz : wz + W;
        const int pcells = Ex * Ey;
        const FastDiv fpc = g.fdp[wx - g.tq[0]][wy - g.tq[1]], fex = tile_div<0, true>(g, wx);
        for (int i = threadIdx.x; i < npl * pcells; i += blockDim.x) {
            const int q = fpc.div(i), rem = i - q * pcells;
            const int ey = fex.div(rem), ex = rem - ey * Ex;
            const ColPlane &pl = s_pl[q];
            const int c = pl.slot * Sxy + rem;
            T v;
            if constexpr (sizeof(T) == 4) {
                v = fixed ? (float)itile[c] * finv : ftile[c];
                itile[c] = 0;
            } else {
                v = ftile[c];
                ftile[c] = T(0);
            }
            // rows outside the tile (or planes outside it in z) are stored whole in the ring, rows
            // through it only their W halo cells; the cells inside go to the grid
            const bool yin = pl.zin && ey >= HL && ey < HL + wy;
            const bool xin = ex >= HL && ex < HL + wx;
            if (yin && xin) {
                grid[pl.goff + (int64_t)ey * g.nf[0] + ex] = v;
            } else {
                const int r = !pl.zin || ey < HL
                                  ? ey * Ex + ex
                                  : (ey < HL + wy ? HL * Ex + (ey - HL) * W + (ex < HL ? ex : ex - wx)
                                                  : HL * Ex + wy * W + (ey - HL - wy) * Ex + ex);
                ring[pl.roff + r] = v;
            }
        }
        __syncthreads();
    }
}

// Folds the rings into the grid, one axis A at a time (x, then y, then z). In the pass along A
// every tile adds the cells of its extended region that lie in its halo bands along A (the W/2
// cells below the tile and the W - W/2 above it) and inside the tile along the axes already
// folded (b < A) to the cells of its neighbour along A that they overlap; those lie in the
// neighbour's own band along A, either inside the neighbour along every axis (a grid cell) or in
// its halo along a later axis (one of its ring cells, folded in a later pass). A corner of the
// region thus reaches its tile in up to D hops. Within one pass the cells read (halo bands along
// A) and written (own bands along A) are disjoint; SIDES = 1 moves the low bands only, 2 the high
// bands only, 3 both in one launch, which needs tiles at least W wide along A (the cells a tile
// receives from below and from above are then disjoint). So no cell is written twice in a
// launch: the passes are race-free and the sums are in a fixed order.
//
// FM is the set of axes folded before A (bit b: axis b); the default order x, y, z has FM = the
// axes below A. Tiles spread by z-columns (k_spread_col) fold z first (FM = 0), then x ({z}),
// then y ({x, z}), and along z only the ends of a column segment have rings: with zseg > 0 the z
// pass moves the low band of a tile only if it starts a segment (tz % zseg == 0) and the high
// band only if it ends one.
template <typename T, int W, int D, int A, int SIDES, int FM>
__global__ void __launch_bounds__(256) k_halo_fold(Geom g, T *ring, int64_t ring_slot,
                                                   T *__restrict__ grid) {
    constexpr int HL = W / 2;
    const int64_t t = blockIdx.x;
    int s[3], w[3], tc[3];
    tile_extent(g, t, W, s, w, tc);
    bool do_low = SIDES != 2, do_high = SIDES != 1;
    if (A == 2 && g.zseg > 0) {
        do_low = do_low && tc[2] % g.zseg == 0;
        do_high = do_high && (tc[2] % g.zseg == g.zseg - 1 || tc[2] == g.nb[2] - 1);
        if (!do_low && !do_high) return;
    }
    // extents of the cells moved: NA along A, the tile along folded axes, the region otherwise
    constexpr int HR = W - HL;
    constexpr int NA = SIDES == 3 ? W : (SIDES == 1 ? HL : HR);   // cells moved along A
    int ext[3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
        ext[b] = b >= D ? 1 : (b == A ? NA : ((FM >> b) & 1 ? w[b] : w[b] + W));
    // neighbours along A
    const int lo_t = tc[A] == 0 ? g.nb[A] - 1 : tc[A] - 1;
    const int hi_t = tc[A] == g.nb[A] - 1 ? 0 : tc[A] + 1;
    const int lo_s = tile_start(lo_t, g.tq[A], g.tr[A]);
    const int lo_w = tile_start(lo_t + 1, g.tq[A], g.tr[A]) - lo_s;
    const int hi_s = tile_start(hi_t, g.tq[A], g.tr[A]);
    const int hi_w = tile_start(hi_t + 1, g.tq[A], g.tr[A]) - hi_s;
    int64_t stride_t[3] = {1, g.nb[0], (int64_t)g.nb[0] * g.nb[1]};
    const int64_t t_lo = t + (int64_t)(lo_t - tc[A]) * stride_t[A];
    const int64_t t_hi = t + (int64_t)(hi_t - tc[A]) * stride_t[A];
    const T *src_ring = ring + t * ring_slot;
    const int count = ext[0] * ext[1] * ext[2];
    // cell i of the moved block: the extent along A is a constant, the others take a
    // multiply-high division where they are needed
    const FastDiv f0 = (FM & 1) ? tile_div<0, false>(g, w[0]) : tile_div<0, true>(g, w[0]);
    const FastDiv f1 = (FM & 2) ? tile_div<1, false>(g, w[1]) : tile_div<1, true>(g, w[1]);
    // IL cells per thread and step: their source loads, then their destinations' loads, then the
    // stores, so that each thread keeps several memory accesses in flight (a cell read here is
    // never written in the same pass, and no cell is written twice)
    constexpr int IL = 4;
    for (int i0 = threadIdx.x; i0 < count; i0 += IL * blockDim.x) {
        T v[IL];
        T *dst[IL];
#pragma unroll
        for (int k = 0; k < IL; ++k) {
            dst[k] = nullptr;
            v[k] = T(0);
            const int i = i0 + k * blockDim.x;
            if (i >= count) continue;
            int e[3];
            if constexpr (A == 0) {
                const int q = i / NA;
                e[0] = i - q * NA;
                e[2] = D == 3 ? f1.div(q) : 0;
                e[1] = q - e[2] * ext[1];
            } else if constexpr (A == 1) {
                const int q = f0.div(i);
                e[0] = i - q * ext[0];
                e[2] = q / NA;
                e[1] = q - e[2] * NA;
            } else {
                const int q = f0.div(i);
                e[0] = i - q * ext[0];
                e[2] = f1.div(q);
                e[1] = q - e[2] * ext[1];
            }
            // e along folded axes counts from the tile's first cell
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if ((FM >> b) & 1) e[b] += HL;
            if (SIDES == 2) e[A] += HL;   // high band only
            const bool low = e[A] < HL;
            if (low ? !do_low : !do_high) continue;
            if (!low) e[A] += w[A];      // high band: HL + w .. w + W - 1
            v[k] = src_ring[ring_index<W, D>(e[0], e[1], e[2], w[0], w[1], w[2])];
            // the same cell in the neighbour's extended region
            int f[3] = {e[0], e[1], e[2]}, fw[3] = {w[0], w[1], w[2]};
            int64_t u;
            if (low) {
                f[A] = e[A] + lo_w;
                fw[A] = lo_w;
                u = t_lo;
            } else {
                f[A] = e[A] - w[A];
                fw[A] = hi_w;
                u = t_hi;
            }
            bool inside = true;
#pragma unroll
            for (int b = 0; b < D; ++b)
                if (b != A && !((FM >> b) & 1)) inside = inside && f[b] >= HL && f[b] < HL + fw[b];
            if (inside) {
                int gc[3] = {0, 0, 0};
#pragma unroll
                for (int b = 0; b < D; ++b)
                    gc[b] = (b == A ? (low ? lo_s : hi_s) : s[b]) + f[b] - HL;
                dst[k] = grid + ((int64_t)gc[2] * g.nf[1] + gc[1]) * g.nf[0] + gc[0];
            } else {
                dst[k] = ring + u * ring_slot +
                         ring_index<W, D>(f[0], f[1], f[2], fw[0], fw[1], fw[2]);
            }
        }
        T d[IL];
#pragma unroll
        for (int k = 0; k < IL; ++k) d[k] = dst[k] ? *dst[k] : T(0);
#pragma unroll
        for (int k = 0; k < IL; ++k)
            if (dst[k]) *dst[k] = d[k] + v[k];
    }
}

}  // namespace fresco
