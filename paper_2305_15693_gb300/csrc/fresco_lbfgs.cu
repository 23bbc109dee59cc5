// Device-resident L-BFGS minimisation of the FReSCo loss (the optimiser of the main text after
// Eq. 4: L-BFGS with a maximal step size and a backtracking line search).
//
// All vectors (positions, gradients, search direction, the m (s, y) history pairs) stay on the
// device in the plan's precision; every inner product keeps FP64 accuracy (per thread a float
// pair for FP32 vectors, fresco::DotAcc) and is reduced in FP64 in a fixed two-stage order. The two-loop recursion keeps its scalars (rho_i, alpha_i, beta, gamma) in
// device memory, so it runs without host round trips; the host reads back two scalars per
// line-search trial (the trial loss and, once per iteration, the slope and the step bound).
//
// Algorithm (Nocedal & Wright, Numerical Optimization, Alg. 7.4 / 7.5):
//   d = -H g by the two-loop recursion over the stored pairs, H0 = (s.y)/(y.y) I;
//   if g.d >= 0 the history is dropped and d = -g;
//   t0 = min(1, max_step / max_j |d_j|)        (no coordinate moves more than max_step);
//   t = t0, t0/2, ... until L(x + t d) <= L(x) + c1 t g.d (at most max_backtrack halvings);
//   s = t d, y = g(x + t d) - g(x); the pair is stored only if s.y > 0.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fresco.h"
#include "fresco_internal.h"

namespace {

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

enum Slot {
    SL_TMP = 0,     // scratch dot
    SL_GAMMA_NUM,   // s.y of the newest pair
    SL_GAMMA_DEN,   // y.y of the newest pair
    SL_BETA,
    SL_GD,          // g.d
    SL_DMAX,        // max |d_j|
    SL_GG,          // g.g
    SL_SY,          // s.y of the candidate pair
    SL_RHO0,        // rho_i at SL_RHO0 + i, alpha_i at SL_RHO0 + m + i, i = 0..m-1
};

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_dot_part(const T *__restrict__ a,
                                                          const T *__restrict__ b, int64_t n,
                                                          double *__restrict__ part) {
    __shared__ double ws[kRedThreads / 32];
    fresco::DotAcc<T> dot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dot.add(a[i], b[i]);
    double acc = dot.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) s += ws[w];
        part[blockIdx.x] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_absmax_part(const T *__restrict__ a, int64_t n,
                                                             double *__restrict__ part) {
    __shared__ double ws[kRedThreads / 32];
    T mt = T(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        mt = fmax(mt, fabs(a[i]));
    double m = (double)mt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) s = fmax(s, ws[w]);
        part[blockIdx.x] = s;
    }
}

// out = (sum or max of part[0..nb)) * (mul ? *mul : 1); fixed order
__global__ void __launch_bounds__(256) k_final(const double *__restrict__ part, int nb, int is_max,
                                               const double *__restrict__ mul,
                                               double *__restrict__ out) {
    __shared__ double sm[256];
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) v = is_max ? fmax(v, part[i]) : v + part[i];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            sm[threadIdx.x] = is_max ? fmax(sm[threadIdx.x], sm[threadIdx.x + o])
                                     : sm[threadIdx.x] + sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0] * (mul ? *mul : 1.0);
}

// y += sign * (*a - (b ? *b : 0)) * x
template <typename T>
__global__ void k_axpy_dev(T *__restrict__ y, const T *__restrict__ x, int64_t n,
                           const double *__restrict__ a, const double *__restrict__ b,
                           double sign) {
    const T c = (T)(sign * (*a - (b ? *b : 0.0)));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(c, x[i], y[i]);
}

// y = scale * x, scale = (num ? *num / *den : s0); non-positive denominators give scale 1
template <typename T>
__global__ void k_scale_copy(T *y, const T *x, int64_t n,
                             const double *__restrict__ num, const double *__restrict__ den,
                             double s0) {
    double c = s0;
    if (num) c = (*den > 0.0 && *num > 0.0) ? *num / *den : 1.0;
    const T ct = (T)c;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = ct * x[i];
}

// z = a + t * b
template <typename T>
__global__ void k_lincomb(T *__restrict__ z, const T *__restrict__ a, const T *__restrict__ b,
                          int64_t n, double t) {
    const T tt = (T)t;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        z[i] = fma(tt, b[i], a[i]);
}

__global__ void k_set(double *__restrict__ p, double v) { *p = v; }

}  // namespace

struct fresco_lbfgs_s {
    fresco_plan_t plan = nullptr;
    fresco_pair_t pair = nullptr;
    fresco_lbfgs_opts opts{};
    int64_t n = 0;          // N * dim
    size_t es = 4;
    cudaStream_t stream = nullptr;
    int *order = nullptr;   // tile_order: solver position i holds caller point order[i]
    int *tpre = nullptr;    // tile_order: first solver position of every tile's points
    void *xs = nullptr;     // tile_order: the points in solver order
    bool have_order = false;
    void *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr;
    std::vector<void *> S, Y;
    double *scal = nullptr;   // device scalars
    double *part = nullptr;   // reduction partials
    double *loss_x = nullptr, *loss_t = nullptr;   // device losses
    int count = 0, head = 0;  // stored pairs, index of the next slot
    int64_t evals = 0, iters = 0;
};

namespace {

template <typename T>
struct Ops {
    fresco_lbfgs_s *s;
    int grid() const {
        int64_t b = (s->n + kRedThreads - 1) / kRedThreads;
        return (int)std::max<int64_t>(1, std::min<int64_t>(b, kRedBlocks));
    }
    void dot(const void *a, const void *b, double *out, const double *mul = nullptr) {
        k_dot_part<T><<<grid(), kRedThreads, 0, s->stream>>>((const T *)a, (const T *)b, s->n,
                                                             s->part);
        k_final<<<1, 256, 0, s->stream>>>(s->part, grid(), 0, mul, out);
    }
    void absmax(const void *a, double *out) {
        k_absmax_part<T><<<grid(), kRedThreads, 0, s->stream>>>((const T *)a, s->n, s->part);
        k_final<<<1, 256, 0, s->stream>>>(s->part, grid(), 1, nullptr, out);
    }
    void axpy(void *y, const void *x, const double *a, const double *b, double sign) {
        k_axpy_dev<T><<<grid(), kRedThreads, 0, s->stream>>>((T *)y, (const T *)x, s->n, a, b,
                                                             sign);
    }
    void scale_copy(void *y, const void *x, const double *num, const double *den, double s0) {
        k_scale_copy<T><<<grid(), kRedThreads, 0, s->stream>>>((T *)y, (const T *)x, s->n, num,
                                                               den, s0);
    }
    void lincomb(void *z, const void *a, const void *b, double t) {
        k_lincomb<T><<<grid(), kRedThreads, 0, s->stream>>>((T *)z, (const T *)a, (const T *)b,
                                                            s->n, t);
    }
};

// Solver positions of the tiles: pre[t] = points of tiles 0 .. t-1 (the tiles' record ranges tr
// may have gaps between them), one block scanning the counts 1024 tiles at a time.
__global__ void __launch_bounds__(1024) k_tile_prefix(const int2 *__restrict__ tr, int64_t n_tiles,
                                                      int *__restrict__ pre) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < n_tiles; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const int v = t < n_tiles ? tr[t].y - tr[t].x : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int incl = x + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (t < n_tiles) pre[t] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
}

// order[pre[t] + k] = caller index of the k-th record of tile t (the index a float record
// carries, or the double plans' separate permutation); one warp per tile
template <typename T>
__global__ void __launch_bounds__(256) k_order_from_plan(const void *__restrict__ sorted,
                                                         const int *__restrict__ perm,
                                                         const int2 *__restrict__ tr,
                                                         const int *__restrict__ pre,
                                                         int64_t n_tiles, int *__restrict__ order) {
    const int lane = threadIdx.x & 31;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tiles;
         t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int2 r = tr[t];
        const int o = pre[t] - r.x;
        for (int i = r.x + lane; i < r.y; i += 32)
            order[o + i] = sizeof(T) == 4 ? (int)reinterpret_cast<const uint4 *>(sorted)[i].w
                                          : perm[i];
    }
}

// to_solver: y[i] = x[order[i]]; else x[order[i]] = y[i] (points of dim coordinates)
template <typename T>
__global__ void __launch_bounds__(256) k_permute(const int *__restrict__ order, int64_t n,
                                                 int dim, T *__restrict__ x, T *__restrict__ y,
                                                 int to_solver) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = order[i];
        for (int a = 0; a < dim; ++a) {
            if (to_solver) y[i * dim + a] = x[j * dim + a];
            else x[j * dim + a] = y[i * dim + a];
        }
    }
}

fresco_status cerr(cudaError_t e) {
    if (e == cudaSuccess) return FRESCO_OK;
    return e == cudaErrorMemoryAllocation ? FRESCO_ERR_OOM : FRESCO_ERR_CUDA;
}

double host_read(fresco_lbfgs_s *s, const double *dev) {
    double v = 0.0;
    cudaMemcpyAsync(&v, dev, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    cudaStreamSynchronize(s->stream);
    return v;
}

// loss and gradient of the minimised function: the structure-factor loss, plus the pair term
fresco_status evaluate(fresco_lbfgs_s *s, const void *x, double *loss, void *grad) {
    fresco_status st = fresco_loss_grad(s->plan, x, loss, grad);
    if (st || !s->pair) return st;
    return fresco_pair_energy_grad(s->pair, x, loss, grad, 1);
}

template <typename T>
fresco_status run_impl(fresco_lbfgs_s *s, void *x_caller, int64_t max_iter,
                       fresco_lbfgs_report *rep) {
    Ops<T> op{s};
    const int m = s->opts.history;
    double *sc = s->scal;
    fresco_status st;
    const int dim = s->plan->dim;
    const int64_t np = s->n / dim;
    const unsigned pb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, 152 * 8));
    void *x = x_caller;
    // loss and gradient at the start point
    if (s->opts.tile_order && !s->have_order) {
        // evaluate in caller order once; its tile order becomes the solver's order
        if ((st = evaluate(s, x_caller, s->loss_x, s->gt))) return st;
        const int64_t nt = s->plan->geom.n_tiles;
        k_tile_prefix<<<1, 1024, 0, s->stream>>>(s->plan->d_tr, nt, s->tpre);
        k_order_from_plan<T><<<pb, 256, 0, s->stream>>>(s->plan->d_sorted, s->plan->d_perm,
                                                         s->plan->d_tr, s->tpre, nt, s->order);
        k_permute<T><<<pb, 256, 0, s->stream>>>(s->order, np, dim, (T *)x_caller, (T *)s->xs, 1);
        k_permute<T><<<pb, 256, 0, s->stream>>>(s->order, np, dim, (T *)s->gt, (T *)s->g, 1);
        s->have_order = true;
        x = s->xs;
    } else if (s->opts.tile_order) {
        k_permute<T><<<pb, 256, 0, s->stream>>>(s->order, np, dim, (T *)x_caller, (T *)s->xs, 1);
        x = s->xs;
        if ((st = evaluate(s, x, s->loss_x, s->g))) return st;
    } else {
        if ((st = evaluate(s, x, s->loss_x, s->g))) return st;
    }
    ++s->evals;
    double fx = host_read(s, s->loss_x);
    int status = 0;
    for (int64_t it = 0; it < max_iter; ++it) {
        op.dot(s->g, s->g, sc + SL_GG);
        const double gg = host_read(s, sc + SL_GG);
        const double grms = std::sqrt(gg / (double)s->n);
        if (s->opts.gtol > 0.0 && grms < s->opts.gtol) { status = 1; break; }
        if (s->opts.ftol > 0.0 && fx < s->opts.ftol) { status = 2; break; }
        // two-loop recursion: d = -H g
        if (s->count == 0) {
            op.scale_copy(s->d, s->g, nullptr, nullptr, -1.0);
        } else {
            op.scale_copy(s->d, s->g, nullptr, nullptr, 1.0);   // q = g
            for (int k = 0; k < s->count; ++k) {     // newest to oldest
                const int i = (s->head - 1 - k + m) % m;
                double *a_i = sc + SL_RHO0 + m + i;  // alpha_i stored after the rho block
                op.dot(s->S[i], s->d, a_i, sc + SL_RHO0 + i);   // alpha_i = rho_i s_i.q
                op.axpy(s->d, s->Y[i], a_i, nullptr, -1.0);     // q -= alpha_i y_i
            }
            const int newest = (s->head - 1 + m) % m;
            op.dot(s->S[newest], s->Y[newest], sc + SL_GAMMA_NUM);
            op.dot(s->Y[newest], s->Y[newest], sc + SL_GAMMA_DEN);
            op.scale_copy(s->d, s->d, sc + SL_GAMMA_NUM, sc + SL_GAMMA_DEN, 1.0);  // r = gamma q
            for (int k = s->count - 1; k >= 0; --k) {    // oldest to newest
                const int i = (s->head - 1 - k + m) % m;
                op.dot(s->Y[i], s->d, sc + SL_BETA, sc + SL_RHO0 + i);   // beta = rho_i y_i.r
                op.axpy(s->d, s->S[i], sc + SL_RHO0 + m + i, sc + SL_BETA, 1.0);
            }
            op.scale_copy(s->d, s->d, nullptr, nullptr, -1.0);   // d = -r
        }
        op.dot(s->g, s->d, sc + SL_GD);
        double gd = host_read(s, sc + SL_GD);
        if (!(gd < 0.0)) {   // not a descent direction: restart from steepest descent
            s->count = 0;
            s->head = 0;
            op.scale_copy(s->d, s->g, nullptr, nullptr, -1.0);
            gd = -gg;
        }
        op.absmax(s->d, sc + SL_DMAX);
        const double dmax = host_read(s, sc + SL_DMAX);
        if (!(dmax > 0.0)) { status = 1; break; }
        double t = std::min(1.0, s->opts.max_step / dmax);
        bool accepted = false;
        double ft = fx;
        for (int k = 0; k <= s->opts.max_backtrack; ++k) {
            op.lincomb(s->xt, x, s->d, t);
            if ((st = evaluate(s, s->xt, s->loss_t, s->gt))) return st;
            ++s->evals;
            ft = host_read(s, s->loss_t);
            if (std::isfinite(ft) && ft <= fx + s->opts.c1 * t * gd) {
                accepted = true;
                break;
            }
            t *= 0.5;
        }
        if (cudaGetLastError() != cudaSuccess) return FRESCO_ERR_CUDA;
        if (!accepted) { status = 4; break; }
        // new pair in the ring slot head: s = xt - x, y = gt - g
        const int h = s->head;
        op.lincomb(s->S[h], s->xt, x, -1.0);
        op.lincomb(s->Y[h], s->gt, s->g, -1.0);
        op.dot(s->S[h], s->Y[h], sc + SL_SY);
        const double sy = host_read(s, sc + SL_SY);
        if (sy > 0.0) {
            k_set<<<1, 1, 0, s->stream>>>(sc + SL_RHO0 + h, 1.0 / sy);
            s->head = (h + 1) % m;
            s->count = std::min(s->count + 1, m);
        } else if (s->count == m) {
            s->count = m - 1;   // the oldest pair's slot was overwritten by the rejected one
        }
        // accept: x = xt, g = gt
        if (cudaMemcpyAsync(x, s->xt, s->es * (size_t)s->n, cudaMemcpyDeviceToDevice,
                            s->stream) != cudaSuccess)
            return FRESCO_ERR_CUDA;
        std::swap(s->g, s->gt);
        std::swap(s->loss_x, s->loss_t);
        fx = ft;
        ++s->iters;
        if (it + 1 == max_iter) status = 3;
    }
    if (s->opts.tile_order)   // the result back in caller order
        k_permute<T><<<pb, 256, 0, s->stream>>>(s->order, np, dim, (T *)x_caller, (T *)x, 0);
    if (rep) {
        op.dot(s->g, s->g, sc + SL_GG);
        const double gg = host_read(s, sc + SL_GG);
        rep->iterations = s->iters;
        rep->evaluations = s->evals;
        rep->loss = fx;
        rep->grad_rms = std::sqrt(gg / (double)s->n);
        rep->status = status;
    }
    return cerr(cudaGetLastError());
}

void lbfgs_free(fresco_lbfgs_s *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    void *bufs[] = {s->g, s->d, s->xt, s->gt, s->scal, s->part, s->loss_x, s->loss_t,
                    s->order, s->tpre, s->xs};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (void *b : s->S)
        if (b) cudaFree(b);
    for (void *b : s->Y)
        if (b) cudaFree(b);
    delete s;
}

}  // namespace

extern "C" {

void fresco_lbfgs_opts_default(fresco_lbfgs_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->history = 10;
    o->max_step = 0.0;
    o->c1 = 1e-4;
    o->max_backtrack = 20;
}

fresco_status fresco_lbfgs_create(fresco_lbfgs_t *out, fresco_plan_t plan,
                                  const fresco_lbfgs_opts *opts) {
    if (!out || !plan) return FRESCO_ERR_ARG;
    *out = nullptr;
    fresco_lbfgs_opts o;
    fresco_lbfgs_opts_default(&o);
    if (opts) o = *opts;
    for (int i = 0; i < 3; ++i)
        if (o.reserved[i]) return FRESCO_ERR_ARG;
    if (o.tile_order != 0 && o.tile_order != 1) return FRESCO_ERR_ARG;
    if (o.history < 1 || o.history > 64 || o.max_backtrack < 0 || o.max_backtrack > 60 ||
        !(o.c1 > 0.0 && o.c1 < 1.0) || o.max_step < 0.0 || o.gtol < 0.0 || o.ftol < 0.0)
        return FRESCO_ERR_ARG;
    fresco_info info;
    fresco_status st = fresco_get_info(plan, &info);
    if (st) return st;
    if (o.max_step == 0.0) {   // a tenth of the mean spacing along the shortest box side
        double lmin = 1e300;
        for (int a = 0; a < info.dim; ++a) lmin = std::min(lmin, plan->box[a]);
        o.max_step = 0.1 * lmin * std::pow((double)info.n_points, -1.0 / info.dim);
    }
    fresco_lbfgs_s *s = new (std::nothrow) fresco_lbfgs_s();
    if (!s) return FRESCO_ERR_OOM;
    s->plan = plan;
    s->opts = o;
    s->n = info.n_points * info.dim;
    s->es = info.precision == FRESCO_F64 ? 8 : 4;
    s->stream = plan->stream;
    const size_t vb = s->es * (size_t)s->n;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return true;
    };
    bool ok = alloc(&s->g, vb) && alloc(&s->d, vb) && alloc(&s->xt, vb) && alloc(&s->gt, vb) &&
              alloc((void **)&s->scal, sizeof(double) * (SL_RHO0 + 2 * o.history)) &&
              alloc((void **)&s->part, sizeof(double) * kRedBlocks) &&
              alloc((void **)&s->loss_x, sizeof(double)) &&
              alloc((void **)&s->loss_t, sizeof(double));
    s->S.assign(o.history, nullptr);
    s->Y.assign(o.history, nullptr);
    for (int i = 0; ok && i < o.history; ++i) ok = alloc(&s->S[i], vb) && alloc(&s->Y[i], vb);
    if (ok && o.tile_order)
        ok = alloc((void **)&s->order, sizeof(int) * (size_t)info.n_points) && alloc(&s->xs, vb) &&
             alloc((void **)&s->tpre, sizeof(int) * (size_t)plan->geom.n_tiles);
    if (!ok) {
        lbfgs_free(s);
        return FRESCO_ERR_OOM;
    }
    cudaMemsetAsync(s->scal, 0, sizeof(double) * (SL_RHO0 + 2 * o.history), s->stream);
    *out = s;
    return FRESCO_OK;
}

fresco_status fresco_lbfgs_run(fresco_lbfgs_t s, void *d_points, int64_t max_iter,
                               fresco_lbfgs_report *report) {
    fresco::clear_pending_error();
    if (!s || !d_points || max_iter < 0) return FRESCO_ERR_ARG;
    s->stream = s->plan->stream;
    if (s->es == 8) return run_impl<double>(s, d_points, max_iter, report);
    return run_impl<float>(s, d_points, max_iter, report);
}

fresco_status fresco_lbfgs_set_pair(fresco_lbfgs_t s, fresco_pair_t p) {
    if (!s) return FRESCO_ERR_ARG;
    s->pair = p;
    return FRESCO_OK;
}

fresco_status fresco_lbfgs_reset(fresco_lbfgs_t s) {
    if (!s) return FRESCO_ERR_ARG;
    s->have_order = false;
    s->count = 0;
    s->head = 0;
    s->iters = 0;
    s->evals = 0;
    return FRESCO_OK;
}

fresco_status fresco_lbfgs_destroy(fresco_lbfgs_t s) {
    lbfgs_free(s);
    return FRESCO_OK;
}

}  // extern "C"
