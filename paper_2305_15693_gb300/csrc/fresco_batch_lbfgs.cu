// L-BFGS over an ensemble: every instance of a batch plan runs its own minimisation (the
// optimiser of the main text after Eq. 4: L-BFGS with a maximal step and a backtracking line
// search), and all of them advance together, one loss+gradient evaluation of the whole ensemble
// per step.
//
// Each instance is a small state machine kept in device memory. A step is
//   evaluate the ensemble at the trial points xt
//   -> decide, per instance: first evaluation / Armijo accept / halve the step / give up
//   -> accepted instances store the pair (s, y) = (xt - x, g(xt) - g(x)), move to xt, and build
//      the next direction d = -H g by the two-loop recursion over their own history
//   -> every running instance writes its next trial point xt = x + t d.
// The step is a fixed sequence of launches (2 m + 8 for history m, plus the evaluation), with
// all per-instance branching done on the device, so it is captured once as a CUDA graph and
// replayed. Instances never wait for one another: one may be backtracking while its neighbour
// takes a new direction.
//
// Vectors live in the plan's precision, packed like the points (instance after instance); inner
// products keep FP64 accuracy (fresco::DotAcc: float pairs per thread for FP32 vectors, FP64
// from there on). The packed vector is cut into chunks that never straddle two
// instances; a chunk kernel writes one partial per chunk, and whoever needs an instance's sum
// adds that instance's partials in a fixed order (deterministic, and the same in every block).
//
// Per instance the iteration is the one of the single-problem solver (Nocedal & Wright,
// Numerical Optimization, Alg. 7.4 / 7.5): H0 = (s.y)/(y.y) I from the newest stored pair, a
// pair stored only if s.y > 0, steepest descent when g.d >= 0, t0 = min(1, max_step / max|d|),
// halving until L(x + t d) <= L(x) + c1 t g.d.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fresco.h"
#include "fresco_internal.h"

namespace {

constexpr int kChunk = 8192;     // elements of the packed vector per chunk (one block each)
constexpr int kThreads = 256;

enum Act { ACT_BACKTRACK = 0, ACT_ACCEPT = 1, ACT_IDLE = 2, ACT_INIT = 3 };

struct BLState {
    double fx;          // loss at x
    double t;           // current step along d
    double gd;          // g.d
    double gg;          // g.g
    double gmax;        // max |g_j|
    double gamma;       // (s.y)/(y.y) of the newest stored pair
    double max_step;
    int64_t n_el;       // elements of this instance (N dim)
    int64_t iters, evals;
    int phase;          // 0 first evaluation pending, 1 line search running, 2 stopped
    int act;            // what the current step does (Act)
    int restart;        // d replaced by -g in this step
    int restore;        // line search gave up: put x back into xt
    int count, head, k_bt;
    int status;         // fresco_lbfgs_report.status codes
};

struct BLParams {
    int m;
    int max_backtrack;
    double c1, gtol, ftol;
    int64_t max_iter;
};

// Sum (or max) of part[c0 .. c1) by one warp in a fixed order; the result in every lane.
__device__ __forceinline__ double warp_reduce_range(const double *__restrict__ part, int64_t c0,
                                                    int64_t c1, bool is_max) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int64_t c = c0 + lane; c < c1; c += 32) v = is_max ? fmax(v, part[c]) : v + part[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, u) : v + u;
    }
    return v;
}

// Instance sum of chunk partials, broadcast to the whole block.
__device__ __forceinline__ double block_inst_sum(const double *__restrict__ part, int64_t c0,
                                                 int64_t c1) {
    __shared__ double bc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const double v = warp_reduce_range(part, c0, c1, false);
        if (threadIdx.x == 0) bc = v;
    }
    __syncthreads();
    return bc;
}

// Block reduction of one partial per thread into out[blockIdx.x]; fixed order.
__device__ __forceinline__ void block_store(double v, bool is_max, double *__restrict__ out) {
    __shared__ double ws[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_down_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, u) : v + u;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s = is_max ? fmax(s, ws[w]) : s + ws[w];
        out[blockIdx.x] = s;
    }
}

__device__ __forceinline__ bool running(int act) { return act == ACT_ACCEPT || act == ACT_INIT; }

// ---- step kernels -----------------------------------------------------------------------------

// One thread per instance: read the trial loss and decide what this step does.
__global__ void k_decide(BLState *__restrict__ st, int n_inst, const double *__restrict__ loss_t,
                         BLParams P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    BLState s = st[i];
    s.restore = 0;   // consumed by the previous step's trial kernel
    if (s.phase == 2) {
        s.act = ACT_IDLE;
    } else if (s.phase == 0) {
        s.act = ACT_INIT;
        s.fx = loss_t[i];
        s.evals += 1;
    } else {
        const double ft = loss_t[i];
        s.evals += 1;
        if (isfinite(ft) && ft <= s.fx + P.c1 * s.t * s.gd) {
            s.act = ACT_ACCEPT;
            s.fx = ft;
            s.iters += 1;
        } else if (s.k_bt >= P.max_backtrack) {
            s.act = ACT_IDLE;
            s.phase = 2;
            s.status = 4;
            s.restore = 1;
        } else {
            s.act = ACT_BACKTRACK;
            s.k_bt += 1;
            s.t *= 0.5;
        }
    }
    st[i] = s;
}

// Accepted instances: new pair into ring slot head, x = xt, g = gt, q = g; partial s.y, y.y,
// g.g, max|g|.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_accept(
    const BLState *__restrict__ st, const int *__restrict__ chunk_inst,
    const int64_t *__restrict__ chunk_lo, T *__restrict__ x, T *__restrict__ g,
    const T *__restrict__ xt, const T *__restrict__ gt, T *__restrict__ q, T *const *Sv,
    T *const *Yv, double *__restrict__ p_sy, double *__restrict__ p_yy,
    double *__restrict__ p_gg, double *__restrict__ p_gmax) {
    const int c = blockIdx.x;
    const BLState &s = st[chunk_inst[c]];
    fresco::DotAcc<T> sy, yy, gg;
    T gm = T(0);
    if (running(s.act)) {
        const bool pair = s.act == ACT_ACCEPT;
        T *S = Sv[s.head], *Y = Yv[s.head];
        for (int64_t e = chunk_lo[c] + threadIdx.x; e < chunk_lo[c + 1]; e += kThreads) {
            const T xn = xt[e], gn = gt[e];
            if (pair) {
                const T se = xn - x[e], ye = gn - g[e];
                S[e] = se;
                Y[e] = ye;
                sy.add(se, ye);
                yy.add(ye, ye);
            }
            x[e] = xn;
            g[e] = gn;
            q[e] = gn;
            gg.add(gn, gn);
            gm = fmax(gm, fabs(gn));
        }
    }
    block_store(sy.value(), false, p_sy);
    block_store(yy.value(), false, p_yy);
    block_store(gg.value(), false, p_gg);
    block_store((double)gm, true, p_gmax);
}

// One warp per instance: store the pair (or not), convergence tests.
__global__ void k_pair(BLState *__restrict__ st, int n_inst, const int64_t *__restrict__ ic_first,
                       const double *__restrict__ p_sy, const double *__restrict__ p_yy,
                       const double *__restrict__ p_gg, const double *__restrict__ p_gmax,
                       double *__restrict__ rho, BLParams P) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n_inst) return;
    if (!running(st[i].act)) return;
    const int64_t c0 = ic_first[i], c1 = ic_first[i + 1];
    const double gg = warp_reduce_range(p_gg, c0, c1, false);
    const double gm = warp_reduce_range(p_gmax, c0, c1, true);
    const double sy = warp_reduce_range(p_sy, c0, c1, false);
    const double yy = warp_reduce_range(p_yy, c0, c1, false);
    if ((threadIdx.x & 31) != 0) return;
    BLState s = st[i];
    s.gg = gg;
    s.gmax = gm;
    if (s.act == ACT_ACCEPT) {
        if (sy > 0.0) {
            rho[(int64_t)i * P.m + s.head] = 1.0 / sy;
            s.gamma = yy > 0.0 ? sy / yy : 1.0;
            s.head = (s.head + 1) % P.m;
            s.count = min(s.count + 1, P.m);
        } else if (s.count == P.m) {
            s.count = P.m - 1;   // the rejected pair overwrote the oldest one's slot
        }
    }
    s.phase = 1;
    const double grms = sqrt(gg / (double)s.n_el);
    if (P.gtol > 0.0 && grms < P.gtol) { s.status = 1; s.phase = 2; s.act = ACT_IDLE; }
    else if (P.ftol > 0.0 && s.fx < P.ftol) { s.status = 2; s.phase = 2; s.act = ACT_IDLE; }
    else if (P.max_iter > 0 && s.iters >= P.max_iter) { s.status = 3; s.phase = 2; s.act = ACT_IDLE; }
    st[i] = s;
}

__device__ __forceinline__ int ring(int head, int k, int m) { return ((head - 1 - k) % m + m) % m; }

// First loop of the recursion, newest pair first. Launch k (0..m): finish pair k-1
// (alpha = rho s.q from its partials, q -= alpha y), then start pair k (partial s.q).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_loop1(
    const BLState *__restrict__ st, const int *__restrict__ chunk_inst,
    const int64_t *__restrict__ chunk_lo, const int64_t *__restrict__ ic_first,
    const double *__restrict__ rho, T *__restrict__ q, T *const *Sv, T *const *Yv,
    double *const *p_a, int k, int m, int64_t n_chunks) {
    const int c = blockIdx.x;
    const int i = chunk_inst[c];
    const BLState &s = st[i];
    if (!running(s.act) || k > s.count) return;
    const int64_t lo = chunk_lo[c], hi = chunk_lo[c + 1];
    if (k >= 1) {
        const int idx = ring(s.head, k - 1, m);
        const double alpha = rho[(int64_t)i * m + idx] * block_inst_sum(p_a[k - 1], ic_first[i],
                                                                        ic_first[i + 1]);
        const T a = (T)alpha;
        const T *Y = Yv[idx];
        for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) q[e] = fma(-a, Y[e], q[e]);
    }
    if (k < s.count) {
        const T *S = Sv[ring(s.head, k, m)];
        fresco::DotAcc<T> v;
        for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) v.add(S[e], q[e]);
        block_store(v.value(), false, p_a[k]);
    }
}

// Second loop, oldest pair first. Launch j (0..m): j = 0 scales r = gamma q; j >= 1 finishes
// pair p = count - j (beta = rho y.r, r += (alpha - beta) s); j < count starts pair
// p = count - 1 - j (partial y.r).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_loop2(
    const BLState *__restrict__ st, const int *__restrict__ chunk_inst,
    const int64_t *__restrict__ chunk_lo, const int64_t *__restrict__ ic_first,
    const double *__restrict__ rho, T *__restrict__ r, T *const *Sv, T *const *Yv,
    double *const *p_a, double *const *p_b, int j, int m) {
    const int c = blockIdx.x;
    const int i = chunk_inst[c];
    const BLState &s = st[i];
    if (!running(s.act) || j > s.count) return;
    const int64_t lo = chunk_lo[c], hi = chunk_lo[c + 1];
    if (j == 0) {
        if (s.count > 0) {
            const T gm = (T)s.gamma;
            for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) r[e] *= gm;
        }
    } else {
        const int p = s.count - j;
        const int idx = ring(s.head, p, m);
        const double rh = rho[(int64_t)i * m + idx];
        const double beta = rh * block_inst_sum(p_b[j - 1], ic_first[i], ic_first[i + 1]);
        const double alpha = rh * block_inst_sum(p_a[p], ic_first[i], ic_first[i + 1]);
        const T cf = (T)(alpha - beta);
        const T *S = Sv[idx];
        for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) r[e] = fma(cf, S[e], r[e]);
    }
    if (j < s.count) {
        const T *Y = Yv[ring(s.head, s.count - 1 - j, m)];
        fresco::DotAcc<T> v;
        for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) v.add(Y[e], r[e]);
        block_store(v.value(), false, p_b[j]);
    }
}

// d = -r; partial g.d and max|d|.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dir(const BLState *__restrict__ st,
                                                  const int *__restrict__ chunk_inst,
                                                  const int64_t *__restrict__ chunk_lo,
                                                  const T *__restrict__ g, T *__restrict__ d,
                                                  double *__restrict__ p_gd,
                                                  double *__restrict__ p_dmax) {
    const int c = blockIdx.x;
    const BLState &s = st[chunk_inst[c]];
    fresco::DotAcc<T> gd;
    T dm = T(0);
    if (running(s.act)) {
        for (int64_t e = chunk_lo[c] + threadIdx.x; e < chunk_lo[c + 1]; e += kThreads) {
            const T de = -d[e];
            d[e] = de;
            gd.add(g[e], de);
            dm = fmax(dm, fabs(de));
        }
    }
    block_store(gd.value(), false, p_gd);
    block_store((double)dm, true, p_dmax);
}

// One warp per instance: descent check, first step of the line search.
__global__ void k_line(BLState *__restrict__ st, int n_inst, const int64_t *__restrict__ ic_first,
                       const double *__restrict__ p_gd, const double *__restrict__ p_dmax) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n_inst) return;
    if (!running(st[i].act)) return;
    const int64_t c0 = ic_first[i], c1 = ic_first[i + 1];
    double gd = warp_reduce_range(p_gd, c0, c1, false);
    double dm = warp_reduce_range(p_dmax, c0, c1, true);
    if ((threadIdx.x & 31) != 0) return;
    BLState s = st[i];
    s.restart = 0;
    if (!(gd < 0.0)) {   // not a descent direction: drop the history, d = -g
        s.restart = 1;
        s.count = 0;
        s.head = 0;
        gd = -s.gg;
        dm = s.gmax;
    }
    if (!(dm > 0.0)) {   // zero gradient: a stationary point
        s.status = 1;
        s.phase = 2;
        s.act = ACT_IDLE;
    } else {
        s.gd = gd;
        s.t = fmin(1.0, s.max_step / dm);
        s.k_bt = 0;
    }
    st[i] = s;
}

// Next trial point xt = x + t d for every instance still searching.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_trial(BLState *__restrict__ st,
                                                    const int *__restrict__ chunk_inst,
                                                    const int64_t *__restrict__ chunk_lo,
                                                    const T *__restrict__ x, const T *__restrict__ g,
                                                    T *__restrict__ d, T *__restrict__ xt) {
    const int c = blockIdx.x;
    const int i = chunk_inst[c];
    const BLState s = st[i];
    const int64_t lo = chunk_lo[c], hi = chunk_lo[c + 1];
    if (s.restore) {   // the line search gave up: the trial buffer holds x again
        for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) xt[e] = x[e];
    } else if (s.phase == 1 && s.act != ACT_IDLE) {
        const T t = (T)s.t;
        const bool neg_g = s.restart && s.act != ACT_BACKTRACK;
        for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) {
            T de = d[e];
            if (neg_g) {
                de = -g[e];
                d[e] = de;
            }
            xt[e] = fma(t, de, x[e]);
        }
    }
}

}  // namespace

struct fresco_batch_lbfgs_s {
    fresco_batch_t b = nullptr;
    BLParams P{};
    int n_inst = 0;
    int64_t n_el = 0, n_chunks = 0;
    size_t es = 4;
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    BLState *st = nullptr;
    double *rho = nullptr, *loss_t = nullptr;
    int *chunk_inst = nullptr;
    int64_t *chunk_lo = nullptr, *ic_first = nullptr;
    void *x = nullptr, *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr;
    void **Sv = nullptr, **Yv = nullptr;          // device arrays of the history pointers
    double *p_sy = nullptr, *p_yy = nullptr, *p_gg = nullptr, *p_gmax = nullptr;
    double *p_gd = nullptr, *p_dmax = nullptr;
    double **p_a = nullptr, **p_b = nullptr;      // device arrays of m partial arrays each
    std::vector<double> max_step;
    bool started = false;
    int64_t steps = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
};

namespace {

bool lalloc(fresco_batch_lbfgs_s *s, void **p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    s->allocs.push_back(*p);
    return true;
}

void bl_free(fresco_batch_lbfgs_s *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    for (void *p : s->allocs) cudaFree(p);
    delete s;
}

fresco_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return FRESCO_OK;
    return e == cudaErrorMemoryAllocation ? FRESCO_ERR_OOM : FRESCO_ERR_CUDA;
}

// The update half of a step (everything after the evaluation).
template <typename T>
cudaError_t update(fresco_batch_lbfgs_s *s) {
    cudaStream_t q = s->stream;
    const int n = s->n_inst, m = s->P.m;
    const unsigned cb = (unsigned)s->n_chunks;
    const unsigned ib = (unsigned)((n + 255) / 256), wb = (unsigned)((n * 32 + 255) / 256);
    k_decide<<<ib, 256, 0, q>>>(s->st, n, s->loss_t, s->P);
    k_accept<T><<<cb, kThreads, 0, q>>>(s->st, s->chunk_inst, s->chunk_lo, (T *)s->x, (T *)s->g,
                                        (const T *)s->xt, (const T *)s->gt, (T *)s->d,
                                        (T *const *)s->Sv, (T *const *)s->Yv, s->p_sy, s->p_yy,
                                        s->p_gg, s->p_gmax);
    k_pair<<<wb, 256, 0, q>>>(s->st, n, s->ic_first, s->p_sy, s->p_yy, s->p_gg, s->p_gmax,
                              s->rho, s->P);
    for (int k = 0; k <= m; ++k)
        k_loop1<T><<<cb, kThreads, 0, q>>>(s->st, s->chunk_inst, s->chunk_lo, s->ic_first, s->rho,
                                           (T *)s->d, (T *const *)s->Sv, (T *const *)s->Yv,
                                           s->p_a, k, m, s->n_chunks);
    for (int j = 0; j <= m; ++j)
        k_loop2<T><<<cb, kThreads, 0, q>>>(s->st, s->chunk_inst, s->chunk_lo, s->ic_first, s->rho,
                                           (T *)s->d, (T *const *)s->Sv, (T *const *)s->Yv,
                                           s->p_a, s->p_b, j, m);
    k_dir<T><<<cb, kThreads, 0, q>>>(s->st, s->chunk_inst, s->chunk_lo, (const T *)s->g,
                                     (T *)s->d, s->p_gd, s->p_dmax);
    k_line<<<wb, 256, 0, q>>>(s->st, n, s->ic_first, s->p_gd, s->p_dmax);
    k_trial<T><<<cb, kThreads, 0, q>>>(s->st, s->chunk_inst, s->chunk_lo, (const T *)s->x,
                                       (const T *)s->g, (T *)s->d, (T *)s->xt);
    return cudaGetLastError();
}

fresco_status one_step(fresco_batch_lbfgs_s *s) {
    fresco_status st = fresco_batch_loss_grad(s->b, s->xt, s->loss_t, s->gt);
    if (st) return st;
    return cuda_st(s->es == 8 ? update<double>(s) : update<float>(s));
}

}  // namespace

extern "C" {

fresco_status fresco_batch_lbfgs_create(fresco_batch_lbfgs_t *out, fresco_batch_t b,
                                        const fresco_lbfgs_opts *opts, int64_t max_iter) {
    if (!out || !b || max_iter < 0) return FRESCO_ERR_ARG;
    *out = nullptr;
    fresco_lbfgs_opts o;
    fresco_lbfgs_opts_default(&o);
    if (opts) o = *opts;
    for (int i = 0; i < 3; ++i)
        if (o.reserved[i]) return FRESCO_ERR_ARG;
    // the ensemble solver keeps its instances' vectors in caller order (tile_order is 0)
    if (o.tile_order != 0) return FRESCO_ERR_ARG;
    if (o.history < 1 || o.history > 64 || o.max_backtrack < 0 || o.max_backtrack > 60 ||
        !(o.c1 > 0.0 && o.c1 < 1.0) || o.max_step < 0.0 || o.gtol < 0.0 || o.ftol < 0.0)
        return FRESCO_ERR_ARG;
    fresco_batch_lbfgs_s *s = new (std::nothrow) fresco_batch_lbfgs_s();
    if (!s) return FRESCO_ERR_OOM;
    s->b = b;
    s->P.m = o.history;
    s->P.max_backtrack = o.max_backtrack;
    s->P.c1 = o.c1;
    s->P.gtol = o.gtol;
    s->P.ftol = o.ftol;
    s->P.max_iter = max_iter;
    s->n_inst = b->n_inst;
    s->es = b->esize;
    s->stream = b->stream;
    const int dim = b->dim, n = b->n_inst, m = o.history;
    s->n_el = b->n_points * dim;
    // chunks: instance ranges cut into pieces of at most kChunk elements
    std::vector<int> ci;
    std::vector<int64_t> clo, icf(n + 1, 0);
    s->max_step.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        const int64_t e0 = b->pt_first[i] * dim, e1 = b->pt_first[i + 1] * dim;
        icf[i] = (int64_t)ci.size();
        for (int64_t e = e0; e < e1; e += kChunk) {
            ci.push_back(i);
            clo.push_back(e);
        }
        double lmin = 1e300;
        for (int a = 0; a < dim; ++a) lmin = std::min(lmin, b->boxes[(size_t)i * dim + a]);
        const double np = (double)(e1 - e0) / dim;
        s->max_step[i] = o.max_step > 0.0 ? o.max_step : 0.1 * lmin * std::pow(np, -1.0 / dim);
    }
    icf[n] = (int64_t)ci.size();
    clo.push_back(s->n_el);
    s->n_chunks = (int64_t)ci.size();
    const size_t vb = s->es * (size_t)s->n_el, pb = sizeof(double) * (size_t)s->n_chunks;
    bool ok = lalloc(s, (void **)&s->st, sizeof(BLState) * n) &&
              lalloc(s, (void **)&s->rho, sizeof(double) * (size_t)n * m) &&
              lalloc(s, (void **)&s->loss_t, sizeof(double) * n) &&
              lalloc(s, (void **)&s->chunk_inst, sizeof(int) * ci.size()) &&
              lalloc(s, (void **)&s->chunk_lo, sizeof(int64_t) * clo.size()) &&
              lalloc(s, (void **)&s->ic_first, sizeof(int64_t) * icf.size()) &&
              lalloc(s, &s->x, vb) && lalloc(s, &s->g, vb) && lalloc(s, &s->d, vb) &&
              lalloc(s, &s->xt, vb) && lalloc(s, &s->gt, vb) &&
              lalloc(s, (void **)&s->Sv, sizeof(void *) * m) &&
              lalloc(s, (void **)&s->Yv, sizeof(void *) * m) &&
              lalloc(s, (void **)&s->p_sy, pb) && lalloc(s, (void **)&s->p_yy, pb) &&
              lalloc(s, (void **)&s->p_gg, pb) && lalloc(s, (void **)&s->p_gmax, pb) &&
              lalloc(s, (void **)&s->p_gd, pb) && lalloc(s, (void **)&s->p_dmax, pb) &&
              lalloc(s, (void **)&s->p_a, sizeof(double *) * m) &&
              lalloc(s, (void **)&s->p_b, sizeof(double *) * m);
    std::vector<void *> S(m), Y(m);
    std::vector<double *> pa(m), pbv(m);
    for (int k = 0; ok && k < m; ++k)
        ok = lalloc(s, &S[k], vb) && lalloc(s, &Y[k], vb) && lalloc(s, (void **)&pa[k], pb) &&
             lalloc(s, (void **)&pbv[k], pb);
    if (!ok) {
        bl_free(s);
        return FRESCO_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(s->chunk_inst, ci.data(), sizeof(int) * ci.size(),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->chunk_lo, clo.data(), sizeof(int64_t) * clo.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->ic_first, icf.data(), sizeof(int64_t) * icf.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->Sv, S.data(), sizeof(void *) * m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->Yv, Y.data(), sizeof(void *) * m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->p_a, pa.data(), sizeof(double *) * m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->p_b, pbv.data(), sizeof(double *) * m, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        bl_free(s);
        return cuda_st(e);
    }
    *out = s;
    return FRESCO_OK;
}

fresco_status fresco_batch_lbfgs_start(fresco_batch_lbfgs_t s, const void *d_points) {
    fresco::clear_pending_error();
    if (!s || !d_points) return FRESCO_ERR_ARG;
    const int n = s->n_inst, dim = s->b->dim;
    std::vector<BLState> h(n);
    for (int i = 0; i < n; ++i) {
        BLState &q = h[i];
        std::memset(&q, 0, sizeof(q));
        q.gamma = 1.0;
        q.max_step = s->max_step[i];
        q.n_el = (s->b->pt_first[i + 1] - s->b->pt_first[i]) * dim;
        q.act = ACT_IDLE;
    }
    cudaError_t e = cudaMemcpyAsync(s->st, h.data(), sizeof(BLState) * n, cudaMemcpyHostToDevice,
                                    s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->xt, d_points, s->es * (size_t)s->n_el, cudaMemcpyDeviceToDevice,
                            s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->x, d_points, s->es * (size_t)s->n_el, cudaMemcpyDeviceToDevice,
                            s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);   // h goes out of scope
    s->started = e == cudaSuccess;
    s->steps = 0;
    return cuda_st(e);
}

fresco_status fresco_batch_lbfgs_step(fresco_batch_lbfgs_t s, int64_t n_steps) {
    fresco::clear_pending_error();
    if (!s || !s->started || n_steps < 0) return FRESCO_ERR_ARG;
    for (int64_t k = 0; k < n_steps; ++k) {
        if (!s->stream || (!s->gexec && s->steps == 0)) {
            // no stream to capture on, or the first step: run the launches directly (the first
            // one also settles kernel attributes and the FFT plans before any capture)
            fresco_status st = one_step(s);
            if (st) return st;
        } else {
            if (!s->gexec) {
                const bool prof_on = s->b->prof.on;   // no event records inside the graph
                s->b->prof.on = false;
                cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) {
                    s->b->prof.on = prof_on;
                    return cuda_st(e);
                }
                fresco_status st = one_step(s);
                cudaGraph_t graph = nullptr;
                e = cudaStreamEndCapture(s->stream, &graph);
                s->b->prof.on = prof_on;
                if (st) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                if (e != cudaSuccess) return cuda_st(e);
                s->graph = graph;
                if ((e = cudaGraphInstantiate(&s->gexec, graph, 0)) != cudaSuccess) {
                    s->gexec = nullptr;
                    return cuda_st(e);
                }
            }
            cudaError_t e = cudaGraphLaunch(s->gexec, s->stream);
            if (e != cudaSuccess) return cuda_st(e);
        }
        ++s->steps;
    }
    return FRESCO_OK;
}

fresco_status fresco_batch_lbfgs_read(fresco_batch_lbfgs_t s, void *d_points,
                                      fresco_lbfgs_report *reports, int64_t *n_running) {
    fresco::clear_pending_error();
    if (!s || !s->started) return FRESCO_ERR_ARG;
    cudaError_t e = cudaSuccess;
    if (d_points)
        e = cudaMemcpyAsync(d_points, s->x, s->es * (size_t)s->n_el, cudaMemcpyDeviceToDevice,
                            s->stream);
    std::vector<BLState> h(s->n_inst);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), s->st, sizeof(BLState) * h.size(), cudaMemcpyDeviceToHost,
                            s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_st(e);
    int64_t run = 0;
    for (int i = 0; i < s->n_inst; ++i) {
        const BLState &q = h[i];
        if (q.phase != 2) ++run;
        if (reports) {
            reports[i].iterations = q.iters;
            reports[i].evaluations = q.evals;
            reports[i].loss = q.fx;
            reports[i].grad_rms = q.n_el > 0 ? std::sqrt(q.gg / (double)q.n_el) : 0.0;
            reports[i].status = q.status;
        }
    }
    if (n_running) *n_running = run;
    return FRESCO_OK;
}

fresco_status fresco_batch_lbfgs_destroy(fresco_batch_lbfgs_t s) {
    bl_free(s);
    return FRESCO_OK;
}

}  // extern "C"
