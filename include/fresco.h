/*
 * fresco.h -- C ABI of libfresco: one evaluation of the FReSCo structure-factor loss and its
 * position gradient on a GB300 GPU (sm_103a), through a type-1 / type-2 nonuniform FFT pair.
 *
 * What is computed (arXiv 2305.15693):
 *   points r_j in a periodic box [0, L_0) x ... x [0, L_{d-1}), d = 2 or 3, weights c_j = 1;
 *   mask: integer wavevectors n (k = 2 pi n / L, componentwise), given with S0(n) and W(n);
 *   rho(n)  = sum_j exp(-i k . r_j)                      (Eq. 1 and Methods Eq. M-ft; e^{-ik.r}
 *                                                          convention, i.e. the paper's rho conjugated)
 *   S(n)    = |rho(n)|^2 / N                               (Eq. 1)
 *   L       = sum_{n in mask} W(n) (S(n) - S0(n))^2        (Eq. 2, with W = w / S0^2 for the
 *                                                          relative form of Eq. 3, Methods
 *                                                          "Analytical gradients")
 *   dL/dr_j = Re sum_n 4 i k W (S - S0) rho(n) / N e^{+i k . r_j}    (Eq. 4)
 * rho is obtained by a type-1 NUFFT (spread with the exponential-of-semicircle kernel, FFT,
 * deconvolve), the gradient by d type-2 NUFFTs (deconvolve, inverse FFT, interpolate), the
 * transforms of Methods "Algorithm parameters" and "NUwU".
 *
 * Conventions shared by every entry point:
 *   - Arrays are row-major. Points are [N][d]: column a is the coordinate along axis a, which
 *     pairs with box[a] and with column a of the mask.
 *   - Precision: a plan is FRESCO_F32 or FRESCO_F64. Device point and gradient arrays have that
 *     element type (float or double). The loss is always a device double.
 *   - All calls that take a plan run asynchronously on the plan's stream (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream) and perform no host synchronisation, except
 *     fresco_status_check, fresco_get_info and the *_host variants.
 *   - Errors: argument errors are returned synchronously. Launch failures return
 *     FRESCO_ERR_CUDA / FRESCO_ERR_CUFFT. Problems only the device sees (non-finite coordinates)
 *     are latched in a device error word that fresco_status_check reads. No C++ exception
 *     crosses this interface.
 *   - Ownership: the caller owns every pointer it passes (points, gradient, loss, stream);
 *     a plan owns copies of the mask, S0 and W, all grids, cuFFT plans and workspaces, and
 *     frees them in fresco_destroy. A plan is not thread safe; use one plan per host thread.
 */
#ifndef FRESCO_H
#define FRESCO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fresco_plan_s *fresco_plan_t;

typedef enum {
    FRESCO_OK = 0,
    FRESCO_ERR_ARG = 1,          /* invalid argument (null pointer, size, dimension, mask) */
    FRESCO_ERR_OOM = 2,          /* a device or host allocation failed */
    FRESCO_ERR_CUFFT = 3,        /* a cuFFT call failed */
    FRESCO_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    FRESCO_ERR_NONFINITE = 5,    /* a coordinate was NaN or infinite (device-detected) */
    FRESCO_ERR_BOUNDS = 6,       /* an index check failed (device-detected) */
    FRESCO_ERR_TIMEOUT = 7,      /* a bounded device wait gave up */
    FRESCO_ERR_UNSUPPORTED = 8   /* a valid request outside what the library implements */
} fresco_status;

enum { FRESCO_F32 = 0, FRESCO_F64 = 1 };

/* Plan options. Zero-initialise (or call fresco_opts_default) and set what you need. */
typedef struct {
    int precision;       /* FRESCO_F32 (default) or FRESCO_F64 */
    double tol;          /* NUFFT relative tolerance eps; 0 -> 1e-6 (F32) or 1e-12 (F64). Sets the
                            kernel width w = ceil(ln(1/eps) / (pi sqrt(1 - 1/sigma))), at least 2;
                            a tolerance needing w > 16 is FRESCO_ERR_UNSUPPORTED */
    double upsample;     /* fine-grid oversampling sigma; 0 -> 2.0; must be in [1.25, 3] */
    int width_override;  /* kernel width w in fine-grid cells (2..16); 0 -> from tol */
    int tile[3];         /* spread/interp tile edge per axis in fine cells; 0 -> default */
    int grad_mode;       /* FRESCO_GRAD_DIRECT (default) or FRESCO_GRAD_KDERIV, see below */
    int reserved[3];     /* must be zero */
} fresco_opts;

/* Gradient modes (the adjoint half of the evaluation, Eq. 4).
 * FRESCO_GRAD_DIRECT: the d gradient components i k_d E(k) / Psi(k) are transformed to the fine
 *   grid (in 2D as one complex field G_x + i G_y; in 3D as that plus G_z) and interpolated with
 *   the kernel psi.
 * FRESCO_GRAD_KDERIV: one real field, the inverse transform of E(k) / Psi(k) (Hermitian, so a
 *   single complex-to-real FFT), interpolated with the kernel's derivative psi' along each axis:
 *   the gradient of the type-2 interpolant. It needs one real FFT instead of d real FFTs' worth
 *   and reads one real grid, at an accuracy slightly below the direct mode's (the derivative
 *   amplifies the kernel's aliasing error). Batch plans support both modes. */
#define FRESCO_GRAD_DIRECT 0
#define FRESCO_GRAD_KDERIV 1

/* Plan parameters, filled by fresco_plan_query and fresco_get_info. */
typedef struct {
    int dim;
    int precision;
    int width;             /* kernel width w (fine cells) */
    int n_fine[3];         /* fine grid size per axis (axis 0 = x, the contiguous one) */
    int k_max[3];          /* max |n_a| over the mask */
    int tile[3];           /* tile edge per axis used by spread / interp */
    int n_tiles[3];        /* tiles per axis */
    double beta;           /* ES kernel shape: psi(u) = exp(beta (sqrt(1 - (2u/w)^2) - 1)) */
    double upsample;
    double loss_const;     /* constant added back after folding +-n pairs (see fresco_plan) */
    int64_t n_points;
    int64_t n_modes;       /* mask entries as given */
    int64_t n_rep;         /* half-space representatives after folding */
    int64_t device_bytes;  /* device memory the plan holds (0 from fresco_plan_query) */
    int grad_mode;         /* FRESCO_GRAD_DIRECT or FRESCO_GRAD_KDERIV */
} fresco_info;

/* Fill *opts with the defaults (F32, eps = 1e-6, sigma = 2). */
void fresco_opts_default(fresco_opts *opts);

/* Create a plan for N points in a periodic box with a fixed wavevector mask (Eq. 2's region K).
 *   out      : receives the plan handle (set to NULL on failure)
 *   dim      : 2 or 3
 *   box      : host [dim] box side lengths L_a > 0
 *   n_points : N >= 1
 *   mask     : host int32 [n_k][dim], integer wavevectors n; any order; n = 0 is rejected (S(0) = N
 *              is fixed, cannot be constrained); |n_a| must stay below n_fine[a] / 2
 *   n_k      : number of mask rows, >= 1; duplicates are allowed and count separately
 *   S0, W    : host double [n_k] target and weight per row; W >= 0 and finite, S0 finite
 *   opts     : NULL for defaults
 *   stream   : cudaStream_t (as void*) every later call runs on; NULL = default stream
 * Folding (S(n) = S(-n) for real weights, Friedel's law, Eq. 3 text): rows n and -n share S, so
 * the plan merges them into one half-space representative with W' = sum W, S0' = sum W S0 / W'.
 * The loss is unchanged up to the constant sum W S0^2 - sum W' S0'^2, which the plan adds back.
 * Copies mask, S0 and W; allocates every device buffer and cuFFT plan the evaluations need, so
 * later calls allocate nothing. Synchronous. Returns FRESCO_ERR_ARG, _OOM, _CUFFT or _CUDA. */
fresco_status fresco_plan(fresco_plan_t *out, int dim, const double *box, int64_t n_points,
                          const int32_t *mask, int64_t n_k, const double *S0, const double *W,
                          const fresco_opts *opts, void *stream);

/* Host only (no GPU touched): validate the same arguments as fresco_plan and report the plan
 * parameters it would choose (fine grid, kernel width and shape, folded count, loss constant). */
fresco_status fresco_plan_query(int dim, const double *box, int64_t n_points, const int32_t *mask,
                                int64_t n_k, const double *S0, const double *W,
                                const fresco_opts *opts, fresco_info *info);

/* Host only: Fourier transform of the ES kernel on the fine grid,
 *   out[i] = integral_{-w/2}^{w/2} psi(u) cos(2 pi nu_i u / n_fine) du,  nu_i = i, i < n_nu,
 * by Gauss-Legendre quadrature in FP64 (the deconvolution factors of the type-1/type-2 NUFFT). */
fresco_status fresco_kernel_ft(int width, double beta, int n_fine, int64_t n_nu, double *out);

/* Copy the plan parameters into *info. */
fresco_status fresco_get_info(fresco_plan_t p, fresco_info *info);

/* Run later calls on another stream (cudaStream_t as void*). */
fresco_status fresco_set_stream(fresco_plan_t p, void *stream);

/* Loss and gradient in one call (Eq. 2 and Eq. 4).
 *   d_points: device [N][dim] positions (float for F32 plans, double for F64); any real values,
 *             wrapped into the box modulo L internally; the array is not modified
 *   d_loss  : device double, receives L
 *   d_grad  : device [N][dim] same type as d_points, receives dL/dr in the caller's point order;
 *             may be NULL (loss only) */
fresco_status fresco_loss_grad(fresco_plan_t p, const void *d_points, double *d_loss,
                               void *d_grad);

/* First half of fresco_loss_grad: sort, spread, FFT, deconvolve, S and the loss (type-1 NUFFT,
 * Eq. 1-2). Also prepares the gradient coefficients C(k) of Eq. 4 inside the plan, so a
 * fresco_backward on the same plan can follow. d_points must stay unchanged until then. */
fresco_status fresco_forward(fresco_plan_t p, const void *d_points, double *d_loss);

/* Second half: d_grad = g * dL/dr, g = *d_grad_out (device double; NULL means 1), by the
 * inverse FFT and interpolation of the type-2 NUFFT (Eq. 4). Requires a preceding fresco_forward. */
fresco_status fresco_backward(fresco_plan_t p, const double *d_grad_out, void *d_grad);

/* After fresco_forward: rho (interleaved re, im: device [n_k][2]) and S (device [n_k]) for the
 * mask rows in the order given to fresco_plan, in the plan's precision. Either may be NULL.
 * The first call uploads the mask (allocates once). */
fresco_status fresco_get_rho_S(fresco_plan_t p, void *d_rho, void *d_S);

/* End-to-end variant on host buffers: copies h_points (host, [N][dim] plan type) to the device,
 * evaluates, and copies the loss (host double) and, if h_grad is not NULL, the gradient back.
 * Synchronises the plan's stream before returning. Uses staging buffers the plan allocates on
 * first use. Points of 64 MB or more are copied in up to 8 chunks on a second stream that the
 * plan creates on first use, and each chunk is binned while the next is in flight; the result is
 * the same as that of fresco_loss_grad on a device copy. Page-locked h_points and h_grad give
 * the full copy rate. */
fresco_status fresco_loss_grad_host(fresco_plan_t p, const void *h_points, double *h_loss,
                                    void *h_grad);

/* Synchronise the plan's stream and return the first device-detected error, clearing it
 * (FRESCO_ERR_NONFINITE for a NaN/inf coordinate; FRESCO_ERR_TIMEOUT if an interpolation tile's
 * TMA load did not complete within its bounded wait, the gradient then being undefined), or a
 * pending CUDA error. */
fresco_status fresco_status_check(fresco_plan_t p);

/* Per-stage timing with CUDA events on the plan's stream. enable != 0 records events around
 * each stage of every later call; fresco_profile_read returns accumulated milliseconds and
 * call counts per stage (synchronises first) and resets them. Stages, in order:
 * 0 sort, 1 spread, 2 forward FFT, 3 mask/loss, 4 loss finalize, 5 inverse FFT, 6 interpolate.
 * ms and counts have room for FRESCO_N_STAGES entries each (counts may be NULL). */
#define FRESCO_N_STAGES 7
fresco_status fresco_profile(fresco_plan_t p, int enable);
fresco_status fresco_profile_read(fresco_plan_t p, double *ms, int64_t *counts);

/* Number of libfresco kernels launched through this plan so far (cuFFT's own not included). */
int64_t fresco_launch_count(fresco_plan_t p);

/* Measured shared-memory throughput of the current device, the denominator of the spread's and
 * the interpolation's roofline (both are bound by shared memory, not by HBM; the paper has no
 * counterpart, it is measurement support). op FRESCO_SMEM_ATOMIC_ADD: 32-bit integer atomic adds
 * (the spread's fixed-point accumulation); FRESCO_SMEM_LOAD: 32-bit loads (the interpolation's
 * window reads). Every warp instruction of the probe addresses 32 distinct banks, the pipe's best
 * case. d_sink: device int array of at least 8 x (multiprocessor count) entries (never read back);
 * stream: cudaStream_t (as void*), NULL = default stream. Launches a few untimed and ten timed
 * kernels (about a millisecond in all) and synchronises; *ops_per_s = lane operations per
 * second. FRESCO_ERR_ARG for a bad op or pointer, FRESCO_ERR_CUDA if a launch fails. */
#define FRESCO_SMEM_ATOMIC_ADD 0
#define FRESCO_SMEM_LOAD 1
fresco_status fresco_smem_peak(int op, void *d_sink, void *stream, double *ops_per_s);

/* Allocation-free loss: *d_loss = sum_{q < n_k} W[q] (S[q] - S0[q])^2, FP64 per-block partial
 * sums plus a fixed-order final stage: bitwise repeatable, and equal to a plan's loss for the same
 * S within the precision's tolerance.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate device
 * memory at call time -- code running under a device-memory budget fixed at start-up, or inside
 * a framework whose allocator already owns the device memory, where a cudaMalloc would fail or
 * is not allowed. It calls no cudaMalloc, cudaFree or allocating library routine.
 *   precision : FRESCO_F32 (d_S is float) or FRESCO_F64 (d_S is double)
 *   n_k       : number of rows, 1 <= n_k <= FRESCO_LOSS_NOALLOC_MAX_ROWS; larger sizes return
 *               FRESCO_ERR_UNSUPPORTED before any device work
 *   d_S       : device [n_k] structure factor (e.g. from fresco_get_rho_S)
 *   d_S0, d_W : device double [n_k] target and weight
 *   d_loss    : device double, receives the loss
 *   stream    : cudaStream_t (as void*), NULL = default stream
 * Its scratch (512 KiB of per-block partial sums) is one array compiled into the library. CUDA
 * loads modules lazily by default, so that array takes its device memory on a device at the
 * first call there (the call loads the module while it looks up the array's device address with
 * cudaGetSymbolAddress, the device current); from then on the GPU holds it until the process
 * exits. Make one warm-up call per device at start-up, before the memory budget is fixed and
 * before any stream capture (or run with CUDA_MODULE_LOADING=EAGER, which loads it with the
 * context). All calls on a device share the array: calls that overlap on the GPU (different
 * streams, no ordering between them) race and give wrong results; calls ordered on one stream are
 * safe. A pending launch error of earlier work on the thread is cleared on entry. Asynchronous;
 * returns FRESCO_ERR_ARG for bad arguments, FRESCO_ERR_CUDA if the address lookup or a launch
 * fails. */
#define FRESCO_LOSS_NOALLOC_MAX_ROWS ((int64_t)65536 * 4096)
fresco_status fresco_loss_noalloc(int precision, int64_t n_k, const void *d_S, const double *d_S0,
                                  const double *d_W, double *d_loss, void *stream);

/* ---- Repulsive pair term of the hybrid loss (Eq. 6) ----------------------------------------
 * E = sum_{m<n} U(|r_m - r_n|), minimum-image distance in the periodic box,
 * U(r) = (eps / alpha)(1 - r / sigma)^alpha for r < sigma, 0 beyond (alpha = 2.5: the Hertzian
 * potential of Eq. 6; alpha = 2: harmonic soft spheres), by a cell list (cells >= sigma wide). */
typedef struct fresco_pair_s *fresco_pair_t;

/* dim 2 or 3; box host [dim]; sigma < min(L) / 2; eps >= 0; alpha > 1; precision FRESCO_F32 or
 * FRESCO_F64 (type of points and gradient); stream as for fresco_plan. Allocates the cell list
 * (one int per cell, five per point) and a sorted copy of the points. */
fresco_status fresco_pair_plan(fresco_pair_t *out, int dim, const double *box, int64_t n_points,
                               double sigma, double eps, double alpha, int precision,
                               void *stream);

/* *d_energy = E and d_grad = dE/dr (device, [N][dim], caller order); with accumulate != 0 both
 * are added to what the arrays hold (e.g. after fresco_loss_grad, for the hybrid loss of Eq. 6).
 * The energy is summed in FP64 in a fixed order. Asynchronous. */
fresco_status fresco_pair_energy_grad(fresco_pair_t p, const void *d_points, double *d_energy,
                                      void *d_grad, int accumulate);

fresco_status fresco_pair_set_stream(fresco_pair_t p, void *stream);
fresco_status fresco_pair_destroy(fresco_pair_t p);

/* ---- Minimisation (the optimiser of the main text after Eq. 4: L-BFGS with a maximal step
 * size and a backtracking line search) ------------------------------------------------------
 * A solver owns device vectors (gradient, direction, trial point, m (s, y) pairs) in the plan's
 * precision and runs on the plan's stream; inner products are accumulated in FP64. Each
 * iteration: d = -H g by the two-loop recursion (H0 = (s.y)/(y.y) I; steepest descent when the
 * history is empty or d is not a descent direction); step t0 = min(1, max_step / max_j |d_j|);
 * backtracking t = t0, t0/2, ... until L(x + t d) <= L(x) + c1 t g.d; the pair (s, y) is kept when
 * s.y > 0. The host reads one or two scalars per line-search trial. */
typedef struct fresco_lbfgs_s *fresco_lbfgs_t;

typedef struct {
    int history;          /* stored pairs m, 1..64 (default 10) */
    double max_step;      /* largest displacement of any coordinate per iteration; 0 -> a tenth
                             of the mean point spacing, 0.1 min(L) N^(-1/d) */
    double c1;            /* Armijo constant in (0, 1) (default 1e-4) */
    int max_backtrack;    /* halvings per line search, 0..60 (default 20) */
    double gtol;          /* stop when the RMS gradient sqrt(g.g / (N d)) < gtol (0: off) */
    double ftol;          /* stop when the loss < ftol (0: off) */
    int tile_order;       /* 1: keep the solver's vectors in the plan's tile order. The first run
                             after create / reset evaluates the start points, takes the tile order
                             of that evaluation as a fixed permutation, and every run gathers the
                             caller's points into it, iterates there, and scatters the result back
                             (the returned points are in caller order). The points move little per
                             iteration, so every evaluation then sees nearly sorted points: the
                             binning's and the gradient's writes become nearly sequential instead
                             of random. The steps equal those of tile_order 0 up to the order of
                             the floating-point sums. Costs 4 bytes per point and one vector. */
    int reserved[3];      /* must be zero */
} fresco_lbfgs_opts;

typedef struct {
    int64_t iterations;   /* accepted steps since create / reset */
    int64_t evaluations;  /* loss+gradient evaluations since create / reset */
    double loss;          /* loss at the returned points */
    double grad_rms;      /* RMS gradient at the returned points */
    int status;           /* 1 gradient below gtol (or zero step), 2 loss below ftol,
                             3 iteration limit, 4 line search failed */
} fresco_lbfgs_report;

void fresco_lbfgs_opts_default(fresco_lbfgs_opts *opts);

/* Create a solver for a plan (the plan must outlive it). Allocates (2m + 4) vectors of N * dim
 * elements of the plan's precision. Returns FRESCO_ERR_ARG or FRESCO_ERR_OOM. */
fresco_status fresco_lbfgs_create(fresco_lbfgs_t *out, fresco_plan_t plan,
                                  const fresco_lbfgs_opts *opts);

/* Run up to max_iter iterations from the device points d_points ([N][dim], plan precision),
 * which are updated in place; the history persists across calls (continue a run by calling
 * again). report (host) may be NULL. Synchronises the plan's stream. */
fresco_status fresco_lbfgs_run(fresco_lbfgs_t s, void *d_points, int64_t max_iter,
                               fresco_lbfgs_report *report);

/* Minimise the hybrid loss of Eq. 6 from now on: every evaluation adds the pair term of p (same
 * points, precision and stream as the plan) to the structure-factor loss. NULL removes it. */
fresco_status fresco_lbfgs_set_pair(fresco_lbfgs_t s, fresco_pair_t p);

/* Drop the stored pairs, zero the counters and forget the tile order (tile_order: the next run
 * takes a new one). */
fresco_status fresco_lbfgs_reset(fresco_lbfgs_t s);

fresco_status fresco_lbfgs_destroy(fresco_lbfgs_t s);

/* ---- Ensembles: many independent problems in one set of launches ---------------------------
 * A batch plan holds n_inst independent 2D problems (points, box, mask, S0, W each their own,
 * the same precision and tolerance). Their points are packed one instance after the other in a
 * single device array; every stage (sort, spread, mask, interpolation) runs as one launch over
 * all instances, and the uniform FFTs run per size class (fine grids rounded up to 2^k or 3 2^k),
 * one batched cuFFT call per class and direction. The result for instance i is exactly what
 * fresco_plan / fresco_loss_grad give for that problem alone (up to the larger fine grid). */
typedef struct fresco_batch_s *fresco_batch_t;

/* boxes: host [n_inst][dim]; n_points, n_modes: host [n_inst]; masks: host int32, the instances'
 * masks concatenated ([sum n_modes][dim]); S0, W: host double, concatenated. dim must be 2
 * (3D returns FRESCO_ERR_UNSUPPORTED). Argument rules as for fresco_plan, per instance. */
fresco_status fresco_batch_plan(fresco_batch_t *out, int dim, int n_inst, const double *boxes,
                                const int64_t *n_points, const int64_t *n_modes,
                                const int32_t *masks, const double *S0, const double *W,
                                const fresco_opts *opts, void *stream);

/* d_points: device [sum N][dim] (instance after instance); d_losses: device double [n_inst];
 * d_grad: device [sum N][dim] or NULL (losses only). Asynchronous. */
fresco_status fresco_batch_loss_grad(fresco_batch_t b, const void *d_points, double *d_losses,
                                     void *d_grad);

/* Record one fresco_batch_loss_grad on these (fixed) pointers as a CUDA graph, after running it
 * once normally; fresco_batch_graph_launch replays it on the plan's stream. The plan needs a
 * non-default stream for capture. */
fresco_status fresco_batch_graph_capture(fresco_batch_t b, const void *d_points, double *d_losses,
                                         void *d_grad);
fresco_status fresco_batch_graph_launch(fresco_batch_t b);

/* Any argument may be NULL. */
fresco_status fresco_batch_info(fresco_batch_t b, int64_t *total_points, int *n_classes,
                                int64_t *device_bytes, int64_t *launches);
/* Geometry of instance i (0 <= i < n_inst) as fresco_get_info reports a plan: its own fine
 * grid (after rounding up to the size class), k_max, tiles, n_rep; device_bytes is 0. */
fresco_status fresco_batch_get_info(fresco_batch_t b, int i, fresco_info *info);
fresco_status fresco_batch_status_check(fresco_batch_t b);
/* Per-stage device time of ordinary (not graph-replayed) evaluations, as fresco_profile /
 * fresco_profile_read: ms and counts [FRESCO_N_STAGES], summed since the last read. */
fresco_status fresco_batch_profile(fresco_batch_t b, int enable);
fresco_status fresco_batch_profile_read(fresco_batch_t b, double *ms, int64_t *counts);
fresco_status fresco_batch_destroy(fresco_batch_t b);

/* L-BFGS over an ensemble: every instance of a batch plan minimises its own loss (the optimiser
 * of the main text after Eq. 4, with the rules of fresco_lbfgs_run, per instance), and all
 * instances advance together. One step = one loss+gradient evaluation of the whole ensemble at
 * the instances' trial points, then, per instance on the device, the Armijo decision (accept, or
 * halve the step, or give up after max_backtrack halvings), the new (s, y) pair and the next
 * direction by the two-loop recursion over that instance's own history. From the second step
 * on, a step is one replay of a CUDA graph when the batch plan has a non-default stream.
 * opts: as for fresco_lbfgs_create, with tile_order 0 (NULL = defaults; max_step 0 = a tenth of
 * each instance's mean spacing L N^(-1/d)); max_iter: accepted iterations per instance (0 = no
 * limit).
 * The solver owns its trial and history buffers ((5 + 2 history) x sum N x dim values). */
typedef struct fresco_batch_lbfgs_s *fresco_batch_lbfgs_t;
fresco_status fresco_batch_lbfgs_create(fresco_batch_lbfgs_t *out, fresco_batch_t b,
                                        const fresco_lbfgs_opts *opts, int64_t max_iter);
/* Copy the start points (device, packed like the batch's points) and reset every instance. */
fresco_status fresco_batch_lbfgs_start(fresco_batch_lbfgs_t s, const void *d_points);
/* Run n_steps steps, asynchronously on the batch plan's stream. Stopped instances (converged,
 * max_iter reached, line search failed) stay where they are while the others continue. */
fresco_status fresco_batch_lbfgs_step(fresco_batch_lbfgs_t s, int64_t n_steps);
/* Synchronising read-back: the accepted points into d_points (device, may be NULL), one report
 * per instance into reports (host [n_inst], may be NULL; status 0 = still running, others as in
 * fresco_lbfgs_report) and the number of instances still running. */
fresco_status fresco_batch_lbfgs_read(fresco_batch_lbfgs_t s, void *d_points,
                                      fresco_lbfgs_report *reports, int64_t *n_running);
fresco_status fresco_batch_lbfgs_destroy(fresco_batch_lbfgs_t s);

/* ---- Weights on a uniform grid (UwU, Methods "Analytical gradients") --------------------------
 * The weight-gradient form of the method: real weights c_m sit at the cells r_m = m L / M of a
 * periodic grid of M_0 x M_1 (x M_2) cells and the constraints are on integer wavevectors n,
 *   rho(n) = sum_m c_m e^{-2 pi i n.m / M},  rho0 = sum_m c_m^2,  S = |rho|^2 / rho0,
 *   L = sum_mask W (S - S0)^2,
 *   dL/dc_m = Re sum_mask [4 W (S - S0) rho / rho0] e^{+2 pi i n.m / M}
 *             - (4 c_m / rho0) sum_mask W S (S - S0)
 * (the weight gradient of Methods, in this library's e^{-ik.r} convention). Both FFTs are exact
 * transforms of the grid: no NUFFT kernel, so results are exact up to rounding. The box size does
 * not enter. grid: host [dim] cell counts, even, >= 4; mask entries need |n_a| < M_a / 2 and n != 0
 * (FRESCO_ERR_ARG otherwise); mask, S0, W as for fresco_plan (folded the same way). */
typedef struct fresco_uwu_s *fresco_uwu_t;
fresco_status fresco_uwu_plan(fresco_uwu_t *out, int dim, const int64_t *grid, const int32_t *mask,
                              int64_t n_k, const double *S0, const double *W, int precision,
                              void *stream);
/* d_c: device [M_{d-1}]..[M_0] of the plan's precision (x fastest, not all zero); d_loss: device
 * double; d_grad: device, same layout as d_c, or NULL. Asynchronous on the plan's stream. The loss
 * is summed in a fixed order and the type-1 spread adds in fixed point (integers scaled per tile
 * by a power of two below the tile's largest possible cell sum), so repeated calls agree bitwise. */
fresco_status fresco_uwu_loss_grad(fresco_uwu_t u, const void *d_c, double *d_loss, void *d_grad);
fresco_status fresco_uwu_destroy(fresco_uwu_t u);

/* ---- Weights on a uniform grid, constraints at real frequencies (UwNU, Methods "Analytical
 * gradients") ---------------------------------------------------------------------------------
 * The same weighted grid as fresco_uwu_plan with free boundaries: constraint q sits at a real
 * frequency nu_q (cycles per grid length along each axis; any value, not only integers),
 *   rho(nu) = sum_m c_m e^{-2 pi i sum_a nu_a m_a / M_a},  rho0 = sum_m c_m^2,  S = |rho|^2 / rho0,
 *   L = sum_q W_q (S_q - S0_q)^2,
 *   dL/dc_m = Re sum_q [4 W (S - S0) rho / rho0]_q e^{+2 pi i sum_a nu_qa m_a / M_a}
 *             - (4 c_m / rho0) sum_q W S (S - S0).
 * As Methods states for this variant, S comes from one type-2 NUFFT of the weights (deconvolve,
 * inverse FFT on the oversampled grid, interpolate at the constraints) and the gradient from one
 * type-1 NUFFT of the per-constraint coefficients (spread, forward FFT, deconvolve), both with the
 * exponential-of-semicircle kernel: accurate to the tolerance, not exact. At integer nu the
 * quantities are those of fresco_uwu_plan. Constraints are not folded: +nu and -nu are separate
 * terms if both are given.
 * grid: host [dim] cell counts, 2 .. 2^20 each (odd allowed); nu: host [n_k][dim] double, finite;
 * S0, W: host [n_k] (W >= 0); opts: precision, tol (0: 1e-6 F32, 1e-12 F64) and upsample (0: 2.0,
 * in [1.25, 3]) are used, the other fields are ignored; NULL = defaults. The fine grid per axis is
 * the smallest even 2-3-5-7-smooth size >= max(sigma M_a, 2 w). FRESCO_ERR_ARG for invalid
 * arguments, FRESCO_ERR_UNSUPPORTED when the fine grid exceeds 4e9 cells or w > 16. The plan owns
 * copies of the constraints, its fine grid and its cuFFT plan; it computes asynchronously on
 * `stream`. At plan time the host orders the constraints by the tile of the fine grid that holds
 * them (32 x 32 cells in 2D, 16 x 8 x 8 in 3D, at most half of each axis) and lists for every
 * tile the constraints whose kernel support meets it: the interpolation runs in that order, and
 * the spread runs one block per tile, accumulating in shared memory and storing each cell once.
 * That host work grows as n_k w^d (the tiles' cover counts): about 0.5 s per 10^6 constraints at
 * w = 7 in 2D. The tile lists hold fewer than 2^31 entries (FRESCO_ERR_UNSUPPORTED beyond). */
typedef struct fresco_uwnu_s *fresco_uwnu_t;
fresco_status fresco_uwnu_plan(fresco_uwnu_t *out, int dim, const int64_t *grid, int64_t n_k,
                               const double *nu, const double *S0, const double *W,
                               const fresco_opts *opts, void *stream);
/* d_c: device [M_{d-1}]..[M_0] of the plan's precision (x fastest, not all zero); d_loss: device
 * double; d_grad: device, same layout as d_c, or NULL. Asynchronous on the plan's stream. The loss
 * is summed in a fixed order and the type-1 spread adds in fixed point (integers scaled per tile
 * by a power of two below the tile's largest possible cell sum), so repeated calls agree bitwise. */
fresco_status fresco_uwnu_loss_grad(fresco_uwnu_t u, const void *d_c, double *d_loss,
                                    void *d_grad);
/* After fresco_uwnu_loss_grad: S at the constraints into d_S (device [n_k], plan precision, in
 * the order given to the plan). FRESCO_ERR_ARG before the first evaluation. */
fresco_status fresco_uwnu_get_S(fresco_uwnu_t u, void *d_S);
/* Kernel width, shape parameter beta and fine grid (n_fine[3], 1 beyond dim); any may be NULL. */
fresco_status fresco_uwnu_get_info(fresco_uwnu_t u, int *width, double *beta, int *n_fine);
fresco_status fresco_uwnu_destroy(fresco_uwnu_t u);
/* Per-stage timing with CUDA events on the plan's stream, as fresco_profile: enable != 0 records
 * events around each stage of every later evaluation; _read synchronises, returns accumulated
 * milliseconds and call counts per stage and resets them. ms and counts have room for
 * FRESCO_UWNU_N_STAGES entries (counts may be NULL). Stages, in order: 0 the points onto their
 * grid (point plans only), 1 the weights onto the fine grid and the inverse FFT, 2 the
 * interpolation at the constraints (S, loss, strengths), 3 the strengths onto the fine grid,
 * 4 the forward FFT and the gradient on the grid, 5 the gradient at the points (point plans). */
#define FRESCO_UWNU_N_STAGES 6
fresco_status fresco_uwnu_profile(fresco_uwnu_t u, int enable);
fresco_status fresco_uwnu_profile_read(fresco_uwnu_t u, double *ms, int64_t *counts);
/* Number of libfresco kernels launched through this plan so far (cuFFT's own not included). */
int64_t fresco_uwnu_launch_count(fresco_uwnu_t u);

/* ---- Points at free positions, constraints at real wavevectors (NUwNU, Methods "Analytical
 * gradients": type-3 transforms of the positions; the main text's quasicrystal targets have
 * Bragg peaks at non-integer k) -------------------------------------------------------------
 * rho(k_q) = sum_j exp(-i k_q . r_j), S_q = |rho_q|^2 / N, L = sum_q W_q (S_q - S0_q)^2,
 * dL/dr_j = Re sum_q (4 i k_q W_q (S_q - S0_q) rho_q / N) exp(+i k_q . r_j) (Eq. 4 without a
 * periodic box). Points lie in [-L_a/2, L_a/2] per axis (free boundaries, no wrapping); k_q are
 * real wavevectors (radians per unit length), none folded.
 * The type-3 transform runs as a spread of the points onto a grid of spacing h_a = pi / (sigma
 * K_a) (K_a = max_q |k_q,a|) and n1_a > L_a / h_a + w + 2 cells, followed by the type-2 transform
 * of that grid at theta_q = k_q h (a grid upsampled by sigma, the weights-on-a-grid machinery
 * above) and a division by the spreading kernel's Fourier transform at theta_q; the gradient by
 * the adjoint type-1 transform and the derivative of the spreading kernel at the points.
 *   dim 2 or 3; box host [dim] (L_a > 0); n_points N >= 1; kvec host [n_k][dim]; S0, W host
 *   [n_k] (W >= 0); opts: precision, tol (0: 1e-6 F32, 1e-12 F64), upsample (0: 2.0, in
 *   [1.25, 3]); other fields ignored; NULL = defaults. FRESCO_ERR_ARG for invalid arguments,
 *   FRESCO_ERR_UNSUPPORTED when a grid exceeds 4e9 cells or w > 16. The plan owns copies of the
 *   constraints, both grids, the points' sort buffers and a cuFFT plan; asynchronous on `stream`. */
typedef struct fresco_nuwnu_s *fresco_nuwnu_t;
fresco_status fresco_nuwnu_plan(fresco_nuwnu_t *out, int dim, const double *box, int64_t n_points,
                                int64_t n_k, const double *kvec, const double *S0, const double *W,
                                const fresco_opts *opts, void *stream);
/* d_points: device [N][dim] of the plan's precision, caller order; d_loss: device double;
 * d_grad: device [N][dim], caller order, or NULL. A point farther than L_a/2 + h_a/2 from the
 * origin on some axis is latched in the device error word (FRESCO_ERR_BOUNDS from
 * fresco_nuwnu_status_check), a NaN or infinite coordinate as
 * FRESCO_ERR_NONFINITE; the results are then undefined. Asynchronous on the plan's stream. The
 * loss repeats bitwise; the constraint-side spread adds in fixed point, and the points' spread and
 * gradient are those of the single plans. */
fresco_status fresco_nuwnu_loss_grad(fresco_nuwnu_t p, const void *d_points, double *d_loss,
                                     void *d_grad);
/* After fresco_nuwnu_loss_grad: S at the constraints into d_S (device [n_k], plan precision, in
 * the order given). */
fresco_status fresco_nuwnu_get_S(fresco_nuwnu_t p, void *d_S);
/* Synchronise and return the first device-detected error (clearing it) or a pending CUDA error. */
fresco_status fresco_nuwnu_status_check(fresco_nuwnu_t p);
/* Kernel width, cells per axis of the points' grid (n_grid[3]) and of the type-2 grid
 * (n_fine[3]), libfresco kernels launched so far; any pointer may be NULL. */
fresco_status fresco_nuwnu_get_info(fresco_nuwnu_t p, int *width, int *n_grid, int *n_fine,
                                    int64_t *launches);
fresco_status fresco_nuwnu_destroy(fresco_nuwnu_t p);
/* Per-stage timing of the plan's evaluations, stages as fresco_uwnu_profile. */
fresco_status fresco_nuwnu_profile(fresco_nuwnu_t p, int enable);
fresco_status fresco_nuwnu_profile_read(fresco_nuwnu_t p, double *ms, int64_t *counts);

/* Free everything the plan owns. Synchronises its stream first. NULL is accepted. */
fresco_status fresco_destroy(fresco_plan_t p);

/* Static description of a status code. */
const char *fresco_status_string(fresco_status s);

#ifdef __cplusplus
}
#endif

#endif /* FRESCO_H */
