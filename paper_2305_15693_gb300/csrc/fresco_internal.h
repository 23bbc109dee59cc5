// Internal declarations shared by the host code and the kernel translation units of libfresco.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "fresco.h"

namespace fresco {

constexpr int kMaxWidth = 16;     // largest ES kernel width instantiated
constexpr int kMinWidth = 2;
constexpr int kMaxTileEdge = 255; // tile-relative cell must fit the 8-bit field of a packed coordinate
constexpr int kTileCursors = 4;   // placement cursors per tile of a single plan (Geom.sub)
constexpr int kZSegment = 6;      // 3D single plans: tiles per z-column segment (Geom.zseg)
constexpr int kColMaxPlanes = 64; // column spread: tiles with tmax_z + w above this spread one by one
constexpr int kDirectPointsPerThread = 8;   // points in flight per thread of k_place_direct
// fresco_loss_grad_host copies the points in up to kHostChunks pieces of at least
// kHostChunkBytes, binning each piece while the next one is in flight
constexpr int kHostChunks = 8;
constexpr int64_t kHostChunkBytes = 32ll << 20;

// Geometry of the fine grid and its tiling, passed by value to kernels.
// Axis 0 is x, the contiguous axis of every grid. With q = nf / nb and r = nf % nb, tile b on an
// axis covers fine cells [start(b), start(b+1)), start(b) = b q + min(b, r): the first r tiles
// are q + 1 cells wide, the others q.
// Division of non-negative ints by a divisor d (1 <= d < 2^31) fixed for a loop, as a multiply-
// high, an add and a shift (the round-up method of Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> l for 0 <= n < 2^31 (umulhi(n, m) < n, so the sum fits 32 bits).
// The magic numbers of a plan's tile extents are computed on the host (Geom.fdw, Geom.fdp).
struct FastDiv {
    unsigned m;
    int l;
    FastDiv() = default;
    __host__ explicit FastDiv(int d) {
        l = 0;
        while ((1LL << l) < d) ++l;
        m = (unsigned)((((unsigned long long)((1ULL << l) - (unsigned long long)d)) << 32) /
                       (unsigned long long)d + 1ULL);
    }
    __host__ __device__ int div(int n) const {
#ifdef __CUDA_ARCH__
        return (int)((__umulhi((unsigned)n, m) + (unsigned)n) >> l);
#else
        return (int)((unsigned)((((unsigned long long)(unsigned)n * m) >> 32) + (unsigned)n) >> l);
#endif
    }
};

struct Geom {
    int dim;
    int nf[3];          // fine grid size per axis (1 for unused axes)
    int nb[3];          // tiles per axis (1 for unused axes)
    int tmax[3];        // widest tile per axis (1 for unused axes)
    int tq[3], tr[3];   // nf / nb and nf % nb per axis
    float tinv[3];      // nb / nf (estimate of the tile of a cell, corrected exactly)
    int64_t n_tiles;
    int list_cap;       // entries of the spread kernel's compacted point list (shared memory)
    int sub;            // bins per tile. Ensemble plans: 3^dim, per axis the low border strip
                        // (cells that can reach the previous tile), the interior, the high border
                        // strip. Single plans: kTileCursors placement cursors (bin = tile * sub +
                        // caller index mod sub)
    int strips[3];      // 1 if every tile on the axis is at least w cells wide (strips disjoint)
    int zseg;           // 3D single plans: tiles per z-column segment of the column spread (0:
                        // tiles spread one by one)
    int64_t n_bins;     // n_tiles * sub: the sort key space
    int tcap;           // single plans: records per tile of the direct binning form (0: the plan
                        // bins in the compact form only)
    int tma;            // single FP32 kernel-derivative plans: 1 if interpolation tiles are staged
                        // by TMA box loads of tbox elements (x, y, z)
    int tbox[3];
    int64_t n_points;
    int width;          // ES kernel width w
    double beta;        // ES kernel shape
    double s_hi[3];     // n_f / L split as s_hi + s_lo (s_hi exact in the working precision)
    double s_lo[3];
    FastDiv fdw[3][4];  // per axis, division by tq, tq + 1, tq + width, tq + 1 + width
    FastDiv fdp[2][2];  // division by (x tile width + width) (y tile width + width), the x and
                        // y widths tq or tq + 1
};

// Fills g.fdw and g.fdp from g.tq and g.width (host).
inline void set_tile_divisors(Geom &g) {
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 4; ++k) {
            const int d = std::max(1, g.tq[a] + (k & 1) + (k >= 2 ? g.width : 0));
            g.fdw[a][k] = FastDiv(d);
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            g.fdp[i][j] = FastDiv(std::max(1, (g.tq[0] + i + g.width) * (g.tq[1] + j + g.width)));
}

// The divisor of a tile extent along axis A: the tile width w (tq or tq + 1), plus the kernel
// width if PLUS.
template <int A, bool PLUS>
__host__ __device__ __forceinline__ FastDiv tile_div(const Geom &g, int w) {
    return w == g.tq[A] ? g.fdw[A][PLUS ? 2 : 0] : g.fdw[A][PLUS ? 3 : 1];
}

__host__ __device__ inline int tile_start(int b, int q, int r) { return b * q + (b < r ? b : r); }
__host__ __device__ inline int tile_of_cell(int c, int q, int r, float inv) {
    int b = (int)((float)c * inv);
    while (b > 0 && tile_start(b, q, r) > c) --b;
    while (tile_start(b + 1, q, r) <= c) ++b;
    return b;
}

// Geometry of the mask and the spectra.
struct MaskGeom {
    int dim;
    int nf[3];
    int kx;              // max n_x over representatives (>= 0)
    int64_t n_rep;
    int64_t half_row;    // nf[0] / 2 + 1: row length of the forward half spectrum
    int64_t hc_row;      // columns of the compact backward spectrum: 2 kx + 2 (n_x = -kx-1 .. kx)
                         // in the direct gradient mode, kx + 1 (n_x = 0 .. kx) in the kderiv mode
    int kderiv;          // the backward spectrum is the scalar E / Psi (kernel-derivative mode)
    int64_t plane;       // nf[1] * nf[2]: length of one transposed column (all (z, y) for one x)
    double inv_n;        // 1 / N
    double kscale[3];    // 2 pi / L_a
};

// Piecewise-polynomial form of the ES kernel: on the k-th unit interval of its support,
// psi(x1 + k) = sum_j c[k][j] tau^j with tau = 2 (x1 + W/2) - 1 in [-1, 1), fitted at plan time by
// Chebyshev interpolation in FP64 (degree 8 for float, 14 for double; maximum deviation from
// psi about 4e-8 for w = 7 and 5e-14 for w = 13). Passed by value to the spread/interp kernels,
// so the coefficients are read from the kernel parameter bank.
template <typename T> struct PolyDeg { static constexpr int value = 8; };
template <> struct PolyDeg<double> { static constexpr int value = 14; };
template <typename T>
struct EsPoly {
    T c[kMaxWidth][PolyDeg<T>::value + 1];
};

// One instance of an ensemble (batch plan): its geometry and where its data sit in the packed
// buffers. Instances are listed in the caller's order; point, sub-bin, tile, mask-block and
// representative offsets grow in that order. Grid and spectrum offsets follow the FFT size classes
// (instances of a class are contiguous there, so cuFFT transforms a class in one batch).
struct BInst {
    Geom g;
    MaskGeom m;
    int64_t po;        // first point
    int64_t bo;        // first sub-bin
    int64_t go;        // first fine-grid cell (real grid)
    int64_t ato;       // transposed forward spectrum
    int64_t hco;       // transposed compact backward spectrum (and the buffer after its y pass)
    int64_t ro;        // R and G of the direct gradient mode (complex elements)
    int64_t reo;       // first representative
    int64_t ipo[3];    // 1 / Psi tables per axis
    double loss_const;
};

// Device tables of a batch plan, passed to the ensemble launchers.
struct BTables {
    const BInst *inst;
    const int64_t *pt_first;     // [n_inst + 1]
    const int64_t *tile_first;   // [n_inst + 1]
    const int64_t *mblk_first;   // [n_inst + 1]
    int n_inst;
    int dim;
    int width;
    int list_cap;                // spread list entries (the same for every instance)
    int64_t n_points, n_tiles, n_mblk;
    int tmax[3];                 // widest tile over all instances (shared-memory sizing)
};

enum Stage { ST_SORT = 0, ST_SPREAD, ST_FFT_FWD, ST_MASK, ST_LOSS, ST_FFT_INV, ST_INTERP,
             ST_COUNT };

// Per-stage device time: a pool of CUDA events, one (start, end) pair per recorded stage,
// accumulated when read.
struct StageProfile {
    struct EvRec { int stage; cudaEvent_t a, b; };
    bool on = false;
    std::vector<EvRec> used;
    std::vector<cudaEvent_t> spare;
    double ms[ST_COUNT] = {};
    int64_t calls[ST_COUNT] = {};
    cudaEvent_t take();
    // fold the recorded pairs into ms / calls (the stream must be synchronised), copy them out
    // and reset
    void read(double *ms_out, int64_t *calls_out);
    void release();
};

// Records the events around one stage on a stream while it is in scope.
struct StageScope {
    StageProfile &p;
    cudaStream_t s;
    cudaEvent_t b = nullptr;
    StageScope(StageProfile &p_, cudaStream_t s_, int stage) : p(p_), s(s_) {
        if (!p.on) return;
        cudaEvent_t a = p.take();
        b = p.take();
        if (a && b) {
            cudaEventRecord(a, s);
            p.used.push_back({stage, a, b});
        } else {
            b = nullptr;
        }
    }
    ~StageScope() {
        if (b) cudaEventRecord(b, s);
    }
};

// Launchers, instantiated for T = float and T = double. All take the plan's stream and
// return the cudaError_t of the launch. Element layouts are documented in fresco_kernels.cuh.
template <typename T>
struct Launch {
    // exclusive prefix sum of cnt into off[0..n] (off[n] = total); when cur is not null it
    // receives a copy of off[0..n) (the placement cursors of k_place)
    // (with a guard, not null: the passes do nothing unless *guard != 0)
    static cudaError_t scan(const int *cnt, int *off, int *block_sums, int64_t n, cudaStream_t s,
                            int *launches, int *cur = nullptr, const int *guard = nullptr);
    // single plans (tiles without border sub-bins), compact form: points per bin, then placement
    // by cursor (guard as for scan)
    static cudaError_t count(const Geom &g, const T *points, int *cnt, int *err, cudaStream_t s,
                             const int *guard = nullptr);
    static cudaError_t place(const Geom &g, const T *points, int *cur, void *sorted, int *perm,
                             cudaStream_t s, const int *guard = nullptr);
    // direct form: g.n_points points starting at caller index j0 (points points at that point)
    // into tile slots of capacity g.tcap; tcur [n_tiles + 1] zero before the first chunk, its
    // last entry the overflow word
    static cudaError_t place_direct(const Geom &g, const T *points, int64_t j0, int *tcur,
                                    void *sorted, int *perm, int *err, cudaStream_t s);
    // tr[t] = record range of tile t from the direct form (tcur) unless it overflowed or tcur is
    // null, else from the compact offsets off
    static cudaError_t tile_ranges(const Geom &g, const int *tcur, const int *off, int2 *tr,
                                   cudaStream_t s);
    // own-points spread into the grid plus per-tile rings, then the ring sums into the grid
    static cudaError_t spread_own(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                  const int2 *tr, T *grid, T *ring, int64_t ring_slot,
                                  cudaStream_t s, int *launches);
    static int spread_own_smem(const Geom &g);
    static int64_t ring_slot(const Geom &g);

    static cudaError_t mask(const MaskGeom &m, const int *rep_n, const T *rep_s0, const T *rep_w,
                            const void *spec, const T *ip0, const T *ip1, const T *ip2,
                            void *hc0, void *hc1, double *partial, int n_blocks, cudaStream_t s);
    static cudaError_t finalize(const double *partial, int n_blocks, double loss_const,
                                double *loss, cudaStream_t s);
    static cudaError_t interp(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                              const int *perm, const int2 *tr, const void *g0, const void *g1,
                              const double *grad_out, T *grad, cudaStream_t s);
    // kernel-derivative mode: h is the real field, dscale[a] = -2 n_f[a] / L[a]; a plan with
    // g.tma stages its tiles by TMA box loads through map (the field h as a tensor), and latches
    // a timed-out load in *err (bit 4)
    static cudaError_t interp_kd(const Geom &g, const EsPoly<T> &ep, const void *sorted,
                                 const int *perm, const int2 *tr, const T *h,
                                 const double *grad_out, const double dscale[3], T *grad,
                                 cudaStream_t s, const CUtensorMap *map = nullptr,
                                 int *err = nullptr);
    static int interp_kd_smem(const Geom &g);
    // real transforms of even length 2M along x as complex transforms of length M: split the
    // forward result into the half spectrum (columns 0..kx, transposed), and merge a transposed
    // half spectrum into the complex rows of the inverse; tw[k] = exp(-2 pi i k / 2M), k <= M/2
    static cudaError_t rfft_split(const void *z, void *xt, const void *tw, int64_t rows, int M,
                                  int kx, cudaStream_t s, int batch = 1, int64_t z_stride = 0,
                                  int64_t xt_stride = 0);
    static cudaError_t rfft_merge(const void *xt, void *z, const void *tw, int64_t rows, int M,
                                  int kx, cudaStream_t s, int batch = 1, int64_t xt_stride = 0,
                                  int64_t z_stride = 0);
    static cudaError_t rows_to_half(const void *bt, void *r, int64_t rows, int64_t half_row,
                                    int kx, cudaStream_t s, int batch = 1, int64_t bt_stride = 0,
                                    int64_t r_stride = 0);
    static cudaError_t interp_kd_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                   const int *perm, const int *off, const T *h,
                                   const double *grad_out, T *grad, cudaStream_t s);
    static cudaError_t cols_to_rows(const void *a, void *at, int64_t rows, int64_t lda,
                                    int ncols, cudaStream_t s, int batch = 1,
                                    int64_t a_stride = 0, int64_t at_stride = 0);
    static cudaError_t rows_to_cols(const void *bt, void *r, int64_t rows, int nf0, int kx,
                                    cudaStream_t s, int batch = 1, int64_t bt_stride = 0,
                                    int64_t r_stride = 0);
    // ensemble (batched) launchers: one launch over every instance of a batch plan
    static cudaError_t bin_b(const BTables &b, const T *points, int *cnt, int *key, int *slot,
                             int *err, cudaStream_t s);
    static cudaError_t scatter_b(const BTables &b, const T *points, const int *key,
                                 const int *slot, const int *off, void *sorted, int *perm,
                                 cudaStream_t s);
    static cudaError_t spread_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                const int *off, T *grid, cudaStream_t s);
    static cudaError_t mask_b(const BTables &b, const int *rep_n, const T *rep_s0,
                              const T *rep_w, const void *spec, const T *ip, void *hc0, void *hc1,
                              double *partial, cudaStream_t s);
    static cudaError_t finalize_b(const BTables &b, const double *partial, double *losses,
                                  cudaStream_t s);
    static cudaError_t interp_b(const BTables &b, const EsPoly<T> &ep, const void *sorted,
                                const int *perm, const int *off, const void *g0, const void *g1,
                                const double *grad_out, T *grad, cudaStream_t s);
    static cudaError_t rho_s(const MaskGeom &m, const int *mask_n, int64_t n_k, const void *spec,
                             const T *ip0, const T *ip1, const T *ip2, T *rho, T *S,
                             cudaStream_t s);
    static int spread_smem(const Geom &g);
    static int interp_smem(const Geom &g);
};

// A point set spread onto a periodic fine grid by the plan machinery (own-points tiles, sorted
// records), for transforms other than fresco_plan's: its geometry, kernel polynomials and
// buffers. point_side_build chooses the tiles and allocates; point_side_spread bins the points and
// spreads them (unit strengths) into `grid`; Launch<T>::interp_kd interpolates a field at them.
struct PointSide {
    Geom g{};
    EsPoly<float> p32{};
    EsPoly<double> p64{};
    int precision = FRESCO_F32;
    void *sorted = nullptr;
    int *perm = nullptr, *cnt = nullptr, *off = nullptr, *bsum = nullptr, *err = nullptr;
    int2 *tr = nullptr;   // record range of every tile (compact binning only: Geom.tcap = 0)
    void *grid = nullptr, *ring = nullptr;
    int64_t ring_slot = 0;
    int64_t device_bytes = 0;
    std::vector<void *> allocs;
};
fresco_status point_side_build(PointSide &ps, int dim, const int nf[3], const double box[3],
                               int64_t n_points, int width, double beta, int precision,
                               cudaStream_t s);
void point_side_free(PointSide &ps);
template <typename T>
fresco_status point_side_spread(PointSide &ps, const T *pts, cudaStream_t s, int64_t *launches);
// Psi(theta) = integral psi(u) cos(theta u) du of the kernel of width w (u in cells), at n real
// frequencies theta (radians per cell).
void kernel_ft_at(int w, double beta, const double *theta, int64_t n, double *out);
// Entry points that launch work call this first: it clears a pending (non-sticky) launch error of
// earlier, unrelated work on the calling thread, so that the error they report after their own
// launches is theirs.
inline void clear_pending_error() { (void)cudaGetLastError(); }
// The piecewise polynomials of the kernel of width w and shape beta that es_weights evaluates.
void es_poly_table(int w, double beta, EsPoly<float> &out);
void es_poly_table(int w, double beta, EsPoly<double> &out);

#ifdef __CUDACC__
// Knuth's two-sum: s + e == a + b exactly (round to nearest, no overflow)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// One thread's running sum of products a_i b_i. FP32 operands: each product exactly as a float
// pair (fmaf), summed into an unevaluated float pair by two-sum, and converted to FP64 once, so
// the sum keeps about 48 bits without the narrow FP64 pipe in the loop; FP64 operands: FMA in
// FP64.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float pe = fmaf(a, b, -p);
        float s, e;
        two_sum(hi, p, s, e);
        hi = s;
        lo += e + pe;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <>
struct DotAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double value() const { return v; }
};
#endif

}  // namespace fresco

// The plan object behind fresco_plan_t.
struct fresco_plan_s {
    int dim = 0;
    int precision = FRESCO_F32;
    size_t esize = 4;                // sizeof(T)
    double box[3] = {1, 1, 1};
    int64_t n_points = 0;
    int64_t n_k = 0;
    fresco::Geom geom{};
    fresco::MaskGeom mgeom{};
    fresco_info info{};
    cudaStream_t stream = nullptr;

    // host copy of the mask as given (for fresco_get_rho_S)
    std::vector<int32_t> h_mask;

    // device buffers (owned)
    void *d_sorted = nullptr;        // sorted records: packed tile-relative coordinates (and, for
                                     // float plans, the caller index)
    int *d_perm = nullptr;           // double plans: sorted position -> caller index
    void *d_ring = nullptr;          // [n_tiles][ring_slot] spread rings (own-points spread)
    int64_t ring_slot = 0;
    int *d_cnt = nullptr;            // [n_bins] points per bin, then the placement cursors
    int *d_off = nullptr;            // [n_bins + 1] exclusive prefix sum of the counts
    int *d_tcur = nullptr;           // [n_tiles + 1] direct-form cursors, then the overflow word
    int2 *d_tr = nullptr;            // [n_tiles] record range of every tile
    CUtensorMap tmap{};              // geom.tma: the interpolated real field as a TMA tensor
    int *d_block_sums = nullptr;     // scan scratch
    void *d_grid = nullptr;          // real fine grid (spread output)
    void *d_tw = nullptr;            // exp(-2 pi i k / nf0), k = 0..nf0/4 (real-row split/merge)
    void *d_specT = nullptr;         // its columns x = 0..kx transposed: [kx+1][plane]
    void *d_hc[2] = {nullptr, nullptr};   // transposed compact backward spectra [2kx+2][plane]
    void *d_bt[2] = {nullptr, nullptr};   // after the (z,)y pass, still transposed
    void *d_r[2] = {nullptr, nullptr};    // transposed back to [plane][nf0]; other columns zero
    void *d_g[2] = {nullptr, nullptr};    // complex gradient grids (components packed re/im)
    int *d_rep_n = nullptr;          // [n_rep][dim] half-space representatives
    void *d_rep_s0 = nullptr;        // [n_rep] folded S0'
    void *d_rep_w = nullptr;         // [n_rep] folded W'
    void *d_ip[3] = {nullptr, nullptr, nullptr};  // 1 / Psi_a(nu), nu = 0..k_max[a]
    double *d_partial = nullptr;     // per-block loss partial sums
    int *d_err = nullptr;            // device error word
    int *d_mask_orig = nullptr;      // lazily uploaded mask (fresco_get_rho_S)
    void *d_fft_work = nullptr;
    void *d_stage_pts = nullptr;     // staging for fresco_loss_grad_host
    void *d_stage_grad = nullptr;
    double *d_stage_loss = nullptr;
    cudaStream_t copy_stream = nullptr;  // host-to-device chunks of fresco_loss_grad_host
    cudaEvent_t copy_ev[fresco::kHostChunks + 1] = {};  // one per chunk, plus the start of the copy
    fresco::EsPoly<float> poly32{};
    fresco::EsPoly<double> poly64{};
    int n_mask_blocks = 0;
    int n_pipes = 1;                 // complex gradient pipelines: ceil(dim / 2), 1 in kderiv
    double dscale[3] = {0, 0, 0};    // kderiv mode: -2 n_f[a] / L[a]
    int64_t device_bytes = 0;

    // cuFFT plans
    cufftHandle fft_rows = 0;        // x pass: every real row as a complex row of nf0/2, in place
    cufftHandle fft_cols = 0;        // C2C forward over the other axes, columns x in [0, kx]
    cufftHandle ifft_cols = 0;       // C2C inverse over the other axes, kx + 1 columns
    cufftHandle ifft_rows = 0;       // C2C inverse along x, all rows (kderiv: nf0/2, in place)
    bool have_fft[4] = {false, false, false, false};

    fresco::StageProfile prof;
    int64_t launches = 0;
    bool forward_done = false;
};

// An ensemble of independent 2D problems evaluated by one set of launches.
struct fresco_batch_s {
    struct Cls {
        int nf[2] = {0, 0};
        int kx = 0;
        int count = 0;
        int64_t go0 = 0, ato0 = 0, hco0 = 0, ro0 = 0, two0 = 0;
        cufftHandle h[4] = {0, 0, 0, 0};   // rows fwd, cols fwd, cols inv, rows inv
        bool have[4] = {false, false, false, false};
    };
    int dim = 0;
    int precision = FRESCO_F32;
    size_t esize = 4;
    int n_inst = 0;
    cudaStream_t stream = nullptr;
    std::vector<double> boxes;       // [n_inst][dim]
    std::vector<fresco_info> infos;  // per instance, as fresco_get_info reports a plan
    std::vector<fresco::BInst> inst;
    std::vector<Cls> cls;
    std::vector<int64_t> pt_first, tile_first, mblk_first;
    fresco::BTables tab{};
    fresco::EsPoly<float> poly32{};
    fresco::EsPoly<double> poly64{};
    int64_t n_points = 0, n_bins = 0, n_rep = 0;
    int64_t cells = 0, n_specT = 0, n_hc = 0, n_tw = 0;
    // device
    fresco::BInst *d_inst = nullptr;
    int64_t *d_pt_first = nullptr, *d_tile_first = nullptr, *d_mblk_first = nullptr;
    void *sorted = nullptr;
    int *perm = nullptr, *key = nullptr, *slot = nullptr, *cnt = nullptr, *off = nullptr;
    int *bsum = nullptr, *err = nullptr;
    void *grid = nullptr, *specT = nullptr, *hc = nullptr, *bt = nullptr;
    void *r = nullptr, *g = nullptr;
    void *tw = nullptr;              // per class: exp(-2 pi i k / nf0), k = 0..nf0/4
    int *rep_n = nullptr;
    void *rep_s0 = nullptr, *rep_w = nullptr, *ip = nullptr;
    double *partial = nullptr;
    void *work = nullptr;
    std::vector<void *> allocs;
    int64_t device_bytes = 0;
    int64_t launches = 0;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    fresco::StageProfile prof;
    int kderiv = 0;                  // gradient mode FRESCO_GRAD_KDERIV
    int64_t n_r = 0;                 // complex elements of the row-order backward buffer
};
