/*
 * FReSCo reference oracle: the structure-factor loss and its position gradient written out
 * as plain direct (non-fast) Fourier sums in FP64.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the checker for the GPU library, not part of it:
 * only the tests, the smoke check and the bench's CPU-baseline leg load it. It shares no
 * code, header or table with the CUDA path.
 *
 * Definitions followed (arXiv 2305.15693):
 *   rho(k)  = sum_j c_j exp(-i k . r_j), c_j = 1, k = 2 pi n / L      (Eq. 1 text, Methods Eq. M-ft;
 *             the exponent sign is flipped to the e^{-ik.r} convention -- S, the loss and the
 *             gradient do not depend on it, rho is conjugated)
 *   S(k)    = |rho(k)|^2 / N                                          (Eq. 1)
 *   L_S     = sum_{k in mask} W(k) (S(k) - S0(k))^2                   (Eq. 2 with the weight
 *             W = w / S0^2 folded in as in Methods "Analytical gradients")
 *   dL/dr_j = Re sum_{k in mask} (4 i k W (S - S0) rho(k) / N) e^{+i k . r_j}
 *             (Eq. 4 / Methods, conjugate form for the e^{-ik.r} convention; the coefficient
 *             uses W, the weight that appears in the loss)
 *
 * Every phase is evaluated directly from its definition with cos/sin; no recurrences, no
 * tables, no fast transforms. Sums run over the mask exactly as given (no folding of +-n).
 * Cost is O(N * N_K); it is meant for small problems or sampled outputs.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* k . r for mask entry q and point j: sum_a (2 pi n_a / L_a) r_a */
static double k_dot_r(int dim, const int32_t *n, const double *r, const double *box)
{
    double s = 0.0;
    for (int a = 0; a < dim; ++a)
        s += TWO_PI * (double)n[a] / box[a] * r[a];
    return s;
}

/* rho(n_q) = sum_j exp(-i k_q . r_j) for every mask entry q.
 * r: [n_points][dim] row-major; mask: [n_k][dim]; box: [dim] side lengths. */
int oracle_rho(int dim, int64_t n_points, const double *r, const double *box,
               int64_t n_k, const int32_t *mask, double *rho_re, double *rho_im)
{
    if (dim < 1 || dim > 3 || n_points < 0 || n_k < 0) return 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_k; ++q) {
        double complex acc = 0.0;
        for (int64_t j = 0; j < n_points; ++j) {
            double ph = k_dot_r(dim, mask + q * dim, r + j * dim, box);
            acc += cexp(-I * ph);
        }
        rho_re[q] = creal(acc);
        rho_im[q] = cimag(acc);
    }
    return 0;
}

/* S, the loss and, optionally, the gradient at a chosen set of points.
 *   S0, W        : [n_k] target and weight per mask entry
 *   loss         : out, scalar
 *   S            : out [n_k] or NULL
 *   rho_re/rho_im: out [n_k] or NULL
 *   n_sel, sel   : gradient wanted at points sel[0..n_sel-1] (sel == NULL: all points)
 *   grad         : out [n_sel][dim] (or [n_points][dim] when sel == NULL), or NULL */
int oracle_loss_grad(int dim, int64_t n_points, const double *r, const double *box,
                     int64_t n_k, const int32_t *mask, const double *S0, const double *W,
                     double *loss, double *S_out, double *rho_re_out, double *rho_im_out,
                     int64_t n_sel, const int64_t *sel, double *grad)
{
    if (dim < 1 || dim > 3 || n_points <= 0 || n_k < 0) return 1;
    double *re = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *im = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    if (!re || !im || !S) { free(re); free(im); free(S); return 2; }

    oracle_rho(dim, n_points, r, box, n_k, mask, re, im);

    /* Eq. 1 and Eq. 2 */
    double N = (double)n_points;
    double total = 0.0;
    for (int64_t q = 0; q < n_k; ++q) {
        S[q] = (re[q] * re[q] + im[q] * im[q]) / N;
        double d = S[q] - S0[q];
        total += W[q] * d * d;
    }
    *loss = total;

    /* Eq. 4: dL/dr_j = Re sum_k C(k) e^{+i k . r_j}, C(k) = 4 i k W (S - S0) rho / N */
    if (grad) {
        int64_t n_out = sel ? n_sel : n_points;
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t t = 0; t < n_out; ++t) {
            int64_t j = sel ? sel[t] : t;
            double g[3] = {0.0, 0.0, 0.0};
            for (int64_t q = 0; q < n_k; ++q) {
                const int32_t *n = mask + q * dim;
                double complex rho = re[q] + I * im[q];
                double complex e = cexp(I * k_dot_r(dim, n, r + j * dim, box));
                double complex coef = 4.0 * W[q] * (S[q] - S0[q]) * rho / N;
                for (int a = 0; a < dim; ++a) {
                    double k_a = TWO_PI * (double)n[a] / box[a];
                    g[a] += creal(I * k_a * coef * e);
                }
            }
            for (int a = 0; a < dim; ++a) grad[t * dim + a] = g[a];
        }
    }

    if (S_out) for (int64_t q = 0; q < n_k; ++q) S_out[q] = S[q];
    if (rho_re_out) for (int64_t q = 0; q < n_k; ++q) rho_re_out[q] = re[q];
    if (rho_im_out) for (int64_t q = 0; q < n_k; ++q) rho_im_out[q] = im[q];
    free(re); free(im); free(S);
    return 0;
}

/* Repulsive pair term of the hybrid loss (Eq. 6): E = sum_{m<n} U(|r_m - r_n|) with the
 * minimum-image distance in the periodic box and U(r) = (eps / alpha) (1 - r / sigma)^alpha for
 * r < sigma, 0 otherwise (alpha = 2.5: the Hertzian potential of Eq. 6; alpha = 2: harmonic).
 * grad[j] = dE/dr_j = sum_{n != j} U'(r) (r_j - r_n) / r, U'(r) = -(eps / sigma)(1 - r/sigma)^(alpha-1).
 * Direct O(N^2) double loop; energy or grad may be NULL; sel/n_sel select the points whose
 * gradient is wanted (sel == NULL: all). */
int oracle_pair_energy_grad(int dim, int64_t n_points, const double *r, const double *box,
                            double sigma, double eps, double alpha, double *energy,
                            int64_t n_sel, const int64_t *sel, double *grad)
{
    if (dim < 1 || dim > 3 || n_points < 0 || !(sigma > 0.0) || !(alpha > 1.0)) return 1;
    double e = 0.0;
    int64_t n_e = energy ? n_points : 0;   /* energy == NULL: gradient rows only */
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : e)
    for (int64_t m = 0; m < n_e; ++m) {
        for (int64_t n = m + 1; n < n_points; ++n) {
            double d2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                double dx = r[m * dim + a] - r[n * dim + a];
                dx -= box[a] * nearbyint(dx / box[a]);
                d2 += dx * dx;
            }
            double rr = sqrt(d2);
            if (rr < sigma) e += eps / alpha * pow(1.0 - rr / sigma, alpha);
        }
    }
    if (energy) *energy = e;
    if (grad) {
        int64_t n_out = sel ? n_sel : n_points;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t t = 0; t < n_out; ++t) {
            int64_t j = sel ? sel[t] : t;
            double g[3] = {0.0, 0.0, 0.0};
            for (int64_t n = 0; n < n_points; ++n) {
                if (n == j) continue;
                double dx[3] = {0.0, 0.0, 0.0}, d2 = 0.0;
                for (int a = 0; a < dim; ++a) {
                    dx[a] = r[j * dim + a] - r[n * dim + a];
                    dx[a] -= box[a] * nearbyint(dx[a] / box[a]);
                    d2 += dx[a] * dx[a];
                }
                double rr = sqrt(d2);
                if (rr < sigma && rr > 0.0) {
                    double du = -eps / sigma * pow(1.0 - rr / sigma, alpha - 1.0);
                    for (int a = 0; a < dim; ++a) g[a] += du * dx[a] / rr;
                }
            }
            for (int a = 0; a < dim; ++a) grad[t * dim + a] = g[a];
        }
    }
    return 0;
}

/* Points at arbitrary real wavevectors (the position gradient with non-uniform k constraints and
 * free boundaries, NUwNU, Methods "Analytical gradients"): unit weights, each constraint a
 * wavevector k_q given directly (kvec [n_k][dim], any real values; nothing is periodic),
 *   rho(k_q) = sum_j exp(-i k_q . r_j),  S_q = |rho(k_q)|^2 / N,  L = sum_q W_q (S_q - S0_q)^2,
 * and the gradient by the chain rule per (point, wavevector) pair,
 *   dS_q/dr_j = (2 / N) Re[conj(rho_q) d rho_q / dr_j],  d rho_q / dr_j = -i k_q e^{-i k_q . r_j},
 *   dL/dr_j = sum_q 2 W_q (S_q - S0_q) dS_q/dr_j.
 * grad: out [n_points][dim] or NULL; the other outputs as oracle_loss_grad. */
int oracle_loss_grad_k(int dim, int64_t n_points, const double *r, int64_t n_k,
                       const double *kvec, const double *S0, const double *W, double *loss,
                       double *S_out, double *rho_re_out, double *rho_im_out, double *grad)
{
    if (dim < 1 || dim > 3 || n_points <= 0 || n_k < 0) return 1;
    double *re = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *im = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    if (!re || !im || !S) { free(re); free(im); free(S); return 2; }
    const double N = (double)n_points;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_k; ++q) {
        double complex acc = 0.0;
        for (int64_t j = 0; j < n_points; ++j) {
            double kr = 0.0;
            for (int a = 0; a < dim; ++a) kr += kvec[q * dim + a] * r[j * dim + a];
            acc += cexp(-I * kr);
        }
        re[q] = creal(acc);
        im[q] = cimag(acc);
    }
    double total = 0.0;
    for (int64_t q = 0; q < n_k; ++q) {
        S[q] = (re[q] * re[q] + im[q] * im[q]) / N;
        double d = S[q] - S0[q];
        total += W[q] * d * d;
    }
    *loss = total;
    if (grad) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t j = 0; j < n_points; ++j) {
            double g[3] = {0.0, 0.0, 0.0};
            for (int64_t q = 0; q < n_k; ++q) {
                double kr = 0.0;
                for (int a = 0; a < dim; ++a) kr += kvec[q * dim + a] * r[j * dim + a];
                const double complex conj_rho = re[q] - I * im[q];
                const double complex e = cexp(-I * kr);
                const double pre = 2.0 * W[q] * (S[q] - S0[q]) * 2.0 / N;
                for (int a = 0; a < dim; ++a) {
                    const double complex drho = -I * kvec[q * dim + a] * e;
                    g[a] += pre * creal(conj_rho * drho);
                }
            }
            for (int a = 0; a < dim; ++a) grad[j * dim + a] = g[a];
        }
    }
    if (S_out) for (int64_t q = 0; q < n_k; ++q) S_out[q] = S[q];
    if (rho_re_out) for (int64_t q = 0; q < n_k; ++q) rho_re_out[q] = re[q];
    if (rho_im_out) for (int64_t q = 0; q < n_k; ++q) rho_im_out[q] = im[q];
    free(re); free(im); free(S);
    return 0;
}

/* Threads the OpenMP runtime will use (1 without OpenMP). */
/* Weighted points (the "UwU" / "UwNU" weight-gradient forms of Methods "Analytical
 * gradients"): real weights c_j at fixed positions r_j,
 *   rho(k)   = sum_j c_j exp(-i k . r_j),   rho0 = sum_j c_j^2,   S(k) = |rho(k)|^2 / rho0,
 *   L_S      = sum_{k in mask} W(k) (S(k) - S0(k))^2,
 *   dL/dc_j  = sum_k 2 W (S - S0) dS/dc_j,
 *   dS/dc_j  = (d rho/dc_j conj(rho) + rho conj(d rho/dc_j)) / rho0 - |rho|^2 (2 c_j) / rho0^2
 *            = 2 Re[rho e^{+i k . r_j}] / rho0 - 2 c_j S / rho0
 * (the chain rule written out per (point, wavevector) pair, not the paper's regrouped form).
 *   c: [n_points]; grad: out [n_points] or NULL; other arguments as oracle_loss_grad. */
int oracle_weight_loss_grad(int dim, int64_t n_points, const double *r, const double *box,
                            const double *c, int64_t n_k, const int32_t *mask, const double *S0,
                            const double *W, double *loss, double *S_out, double *rho_re_out,
                            double *rho_im_out, double *grad)
{
    if (dim < 1 || dim > 3 || n_points <= 0 || n_k < 0) return 1;
    double *re = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *im = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    if (!re || !im || !S) { free(re); free(im); free(S); return 2; }
    double rho0 = 0.0;
    for (int64_t j = 0; j < n_points; ++j) rho0 += c[j] * c[j];
    if (!(rho0 > 0.0)) { free(re); free(im); free(S); return 3; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_k; ++q) {
        double complex acc = 0.0;
        for (int64_t j = 0; j < n_points; ++j)
            acc += c[j] * cexp(-I * k_dot_r(dim, mask + q * dim, r + j * dim, box));
        re[q] = creal(acc);
        im[q] = cimag(acc);
    }
    double total = 0.0;
    for (int64_t q = 0; q < n_k; ++q) {
        S[q] = (re[q] * re[q] + im[q] * im[q]) / rho0;
        double d = S[q] - S0[q];
        total += W[q] * d * d;
    }
    *loss = total;
    if (grad) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t j = 0; j < n_points; ++j) {
            double g = 0.0;
            for (int64_t q = 0; q < n_k; ++q) {
                double complex rho = re[q] + I * im[q];
                double complex e = cexp(I * k_dot_r(dim, mask + q * dim, r + j * dim, box));
                double dS = 2.0 * creal(rho * e) / rho0 - 2.0 * c[j] * S[q] / rho0;
                g += 2.0 * W[q] * (S[q] - S0[q]) * dS;
            }
            grad[j] = g;
        }
    }
    if (S_out) for (int64_t q = 0; q < n_k; ++q) S_out[q] = S[q];
    if (rho_re_out) for (int64_t q = 0; q < n_k; ++q) rho_re_out[q] = re[q];
    if (rho_im_out) for (int64_t q = 0; q < n_k; ++q) rho_im_out[q] = im[q];
    free(re); free(im); free(S);
    return 0;
}

/* Weighted points at arbitrary real wavevectors (the weight-gradient form of Methods
 * "Analytical gradients" with non-uniform k constraints, UwNU): the same quantities as
 * oracle_weight_loss_grad, but each constraint is a wavevector k_q given directly
 * (kvec [n_k][dim], any real values, free boundaries: no periodicity is assumed),
 *   rho(k_q) = sum_j c_j exp(-i k_q . r_j),  rho0 = sum_j c_j^2,  S_q = |rho(k_q)|^2 / rho0,
 *   L_S = sum_q W_q (S_q - S0_q)^2,
 *   dL/dc_j = sum_q 2 W_q (S_q - S0_q) [2 Re(rho(k_q) e^{+i k_q . r_j}) / rho0 - 2 c_j S_q / rho0].
 * Arguments as oracle_weight_loss_grad with kvec in place of (mask, box). */
int oracle_weight_loss_grad_k(int dim, int64_t n_points, const double *r, const double *c,
                              int64_t n_k, const double *kvec, const double *S0, const double *W,
                              double *loss, double *S_out, double *rho_re_out,
                              double *rho_im_out, double *grad)
{
    if (dim < 1 || dim > 3 || n_points <= 0 || n_k < 0) return 1;
    double *re = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *im = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(n_k > 0 ? n_k : 1));
    if (!re || !im || !S) { free(re); free(im); free(S); return 2; }
    double rho0 = 0.0;
    for (int64_t j = 0; j < n_points; ++j) rho0 += c[j] * c[j];
    if (!(rho0 > 0.0)) { free(re); free(im); free(S); return 3; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_k; ++q) {
        double complex acc = 0.0;
        for (int64_t j = 0; j < n_points; ++j) {
            double kr = 0.0;
            for (int a = 0; a < dim; ++a) kr += kvec[q * dim + a] * r[j * dim + a];
            acc += c[j] * cexp(-I * kr);
        }
        re[q] = creal(acc);
        im[q] = cimag(acc);
    }
    double total = 0.0;
    for (int64_t q = 0; q < n_k; ++q) {
        S[q] = (re[q] * re[q] + im[q] * im[q]) / rho0;
        double d = S[q] - S0[q];
        total += W[q] * d * d;
    }
    *loss = total;
    if (grad) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t j = 0; j < n_points; ++j) {
            double g = 0.0;
            for (int64_t q = 0; q < n_k; ++q) {
                double kr = 0.0;
                for (int a = 0; a < dim; ++a) kr += kvec[q * dim + a] * r[j * dim + a];
                double complex rho = re[q] + I * im[q];
                double dS = 2.0 * creal(rho * cexp(I * kr)) / rho0 - 2.0 * c[j] * S[q] / rho0;
                g += 2.0 * W[q] * (S[q] - S0[q]) * dS;
            }
            grad[j] = g;
        }
    }
    if (S_out) for (int64_t q = 0; q < n_k; ++q) S_out[q] = S[q];
    if (rho_re_out) for (int64_t q = 0; q < n_k; ++q) rho_re_out[q] = re[q];
    if (rho_im_out) for (int64_t q = 0; q < n_k; ++q) rho_im_out[q] = im[q];
    free(re); free(im); free(S);
    return 0;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
