// Host side of libfresco: plan construction (kernel parameters, mask folding, deconvolution
// tables, cuFFT plans, device buffers) and the C ABI declared in include/fresco.h.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fresco.h"
#include "fresco_internal.h"

using namespace fresco;

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;
// Dynamic shared memory a tile kernel may take: an SM holds 228 KB, a block reserves 1 KB and the
// kernels' static shared state (the residue schedule) takes up to 4 KB; one block may opt in to
// at most 227 KB in all.
constexpr size_t kSmemOptin = 223 * 1024;        // one block per SM
constexpr size_t kSmemTwoBlocks = 109 * 1024;    // two blocks per SM
constexpr double kTileHits = 2000.0;         // points per 2D tile (with halo) the default aims at

// ---- fine grid and kernel parameters --------------------------------------------------------

bool is_smooth_even(int64_t n) {
    if (n < 2 || (n & 1)) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Smallest even 2-3-5-7-smooth integer >= n.
int64_t next_smooth_even(int64_t n) {
    if (n < 2) n = 2;
    while (!is_smooth_even(n)) ++n;
    return n;
}

// Kernel width and shape for tolerance eps at oversampling sigma, from the error estimate of the
// exponential-of-semicircle kernel (Barnett, Magland, af Klinteberg, SIAM J. Sci. Comput. 2019,
// the NUFFT the paper uses, Methods "Algorithm parameters"): the aliasing error decays like
// exp(-pi w sqrt(1 - 1/sigma)); beta ~ 0.976 pi (1 - 1/(2 sigma)) w, i.e. 2.30 w at sigma = 2.
// Returns a width above kMaxWidth when eps cannot be reached at this sigma; the caller rejects it.
int es_width(double eps, double sigma) {
    double w = std::ceil(std::log(1.0 / eps) / (kPi * std::sqrt(1.0 - 1.0 / sigma)));
    if (w > 1000.0) w = 1000.0;
    int wi = (int)w;
    if (wi < kMinWidth) wi = kMinWidth;
    return wi;
}
double es_beta(int w, double sigma) { return 0.976 * kPi * (1.0 - 0.5 / sigma) * w; }

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the three-term
// recurrence, starting from the asymptotic root estimates).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &wts) {
    x.assign(n, 0.0);
    wts.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double t = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        {   // final derivative at the converged root
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        x[i] = -t;
        x[n - 1 - i] = t;
        double wq = 2.0 / ((1.0 - t * t) * dp * dp);
        wts[i] = wq;
        wts[n - 1 - i] = wq;
    }
}

// Psi(nu) = integral_{-w/2}^{w/2} psi(u) cos(2 pi nu u / nf) du for nu = 0..n_nu-1.
// With u = (w/2) sin(theta) the kernel becomes exp(beta (cos(theta) - 1)), analytic on
// theta in [0, pi/2] (the square-root edge of psi disappears), so Gauss-Legendre in theta
// converges geometrically.
void kernel_ft(int w, double beta, int nf, int64_t n_nu, double *out) {
    const int nq = 200;
    std::vector<double> x, wq;
    gauss_legendre(nq, x, wq);
    const double h = 0.25 * kPi;  // theta in [0, pi/2] = h (1 + t), t in [-1, 1]
    std::vector<double> u(nq), f(nq);
    for (int q = 0; q < nq; ++q) {
        const double th = h * (1.0 + x[q]);
        u[q] = 0.5 * w * std::sin(th);
        // factor 2: even integrand; du = (w/2) cos(theta) dtheta
        f[q] = 2.0 * h * wq[q] * std::exp(beta * (std::cos(th) - 1.0)) * 0.5 * w * std::cos(th);
    }
    for (int64_t nu = 0; nu < n_nu; ++nu) {
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += f[q] * std::cos(2.0 * kPi * (double)nu * u[q] / nf);
        out[nu] = s;
    }
}

// Chebyshev interpolation of psi on each unit interval of its support, converted to monomial
// coefficients in tau = 2 t - 1, t = x1 + w/2 in [0, 1): c[k][j], j = 0..deg.
template <typename T>
void es_poly(int w, double beta, EsPoly<T> &out) {
    const int deg = PolyDeg<T>::value;
    const int n = deg + 1;
    std::memset(&out, 0, sizeof(out));
    std::vector<double> nodes(n), f(n), a(n), tk(n), tkm1(n), tkp1(n), mono(n);
    for (int i = 0; i < n; ++i) nodes[i] = std::cos(kPi * (i + 0.5) / n);
    for (int k = 0; k < w; ++k) {
        for (int i = 0; i < n; ++i) {
            const double u = 0.5 * (nodes[i] + 1.0) - 0.5 * w + k;
            const double z = 2.0 * u / w;
            const double q = 1.0 - z * z;
            f[i] = q > 0.0 ? std::exp(beta * (std::sqrt(q) - 1.0)) : 0.0;
        }
        for (int j = 0; j < n; ++j) {   // Chebyshev coefficients
            double sj = 0.0;
            for (int i = 0; i < n; ++i) sj += f[i] * std::cos(j * kPi * (i + 0.5) / n);
            a[j] = (j == 0 ? 1.0 : 2.0) * sj / n;
        }
        // sum_j a_j T_j(tau) in monomials: T_0 = 1, T_1 = tau, T_{j+1} = 2 tau T_j - T_{j-1}
        std::fill(mono.begin(), mono.end(), 0.0);
        std::fill(tkm1.begin(), tkm1.end(), 0.0);
        std::fill(tk.begin(), tk.end(), 0.0);
        tkm1[0] = 1.0;   // T_0
        tk[1 < n ? 1 : 0] = 1.0;   // T_1
        mono[0] += a[0];
        if (n > 1)
            for (int m = 0; m < n; ++m) mono[m] += a[1] * tk[m];
        for (int j = 1; j + 1 < n; ++j) {
            for (int m = 0; m < n; ++m)
                tkp1[m] = (m > 0 ? 2.0 * tk[m - 1] : 0.0) - tkm1[m];
            for (int m = 0; m < n; ++m) mono[m] += a[j + 1] * tkp1[m];
            tkm1.swap(tk);
            tk.swap(tkp1);
        }
        for (int m = 0; m < n; ++m) out.c[k][m] = (T)mono[m];
    }
}

// ---- argument checks, parameters and mask folding -------------------------------------------

struct Folded {
    std::vector<int32_t> n;     // [n_rep][dim]
    std::vector<double> s0;     // S0'
    std::vector<double> w;      // W'
    double loss_const = 0.0;
};

struct Params {
    int dim, precision, width;
    int64_t n_points;
    int list_cap;     // spread list entries
    int grad_mode;    // fresco_opts.grad_mode
    double beta, sigma, tol;
    int kmax[3];
    int nf[3];
    int nb[3];
    int tmax[3];
};

bool canonical(const int32_t *n, int dim) {
    if (n[0] != 0) return n[0] > 0;
    if (n[1] != 0) return n[1] > 0;
    return dim == 3 && n[2] > 0;
}

int choose_tiles(int nf, int target, int minw) {
    if (target < minw) target = minw;
    int best = std::max(1, (int)std::lround((double)nf / target));
    // prefer an exact divisor of nf near the target edge
    for (int d = 0; d <= target / 4; ++d) {
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int e = target + sgn * d;
            if (e >= minw && e <= kMaxTileEdge && e <= nf && nf % e == 0) return nf / e;
        }
    }
    while (best > 1 && nf / best < minw) --best;
    while ((nf + best - 1) / best > kMaxTileEdge) ++best;
    return best;
}

// Tiles: the requested (or default) edge per axis, shrunk while the interpolation tile plus its
// halo, or the spread tile plus its point list, would not fit the shared-memory budget (2 blocks
// per SM by default, the opt-in maximum when the caller fixed the tiles). Needs P.nf, P.width,
// P.dim, P.precision.
fresco_status choose_tiling(Params &P, const int tile_req[3], bool own_tiles = false) {
    const int dim = P.dim, w = P.width;
    const size_t es = P.precision == FRESCO_F64 ? 8 : 4;
    const bool user_tiles = tile_req[0] > 0 || tile_req[1] > 0 || tile_req[2] > 0;
    // a tile is at least ceil(w / 2) cells wide: a point's window then reaches only the adjacent
    // tiles (the halo fold and the gathering spread rely on it)
    const int minw = (w + 1) / 2;
    size_t budget = user_tiles ? kSmemOptin : kSmemTwoBlocks;
    double cells_all = 1.0;
    for (int a = 0; a < dim; ++a) cells_all *= (double)P.nf[a];
    const double density = (double)P.n_points / cells_all;   // points per fine cell
    int target[3];
    auto reset_targets = [&]() {
        for (int a = 0; a < dim; ++a) {
            // 2D: a square tile whose halo-extended area holds about kTileHits points on
            // average (fewer points straddle tile borders than with small tiles; more than that
            // and the tile's shared memory limits residency), but enough tiles for about twelve
            // blocks per SM (one and a half waves of the interpolation kernel) where the grid
            // allows it. 3D: 24 x 24 x 12 (measured best of 18x18x8, 18^3, 24x24x12, 27x27x12, 24^3
            // on the 2^24-point workload), scaled down likewise on small grids
            int deft = a < 2 ? 24 : 12;
            if (dim == 3) {
                const double f = std::cbrt(cells_all / (12.0 * 152.0) / (24.0 * 24.0 * 12.0));
                if (f < 1.0) deft = std::max(a < 2 ? 8 : 4, (int)(deft * f));
            }
            if (dim == 2) {
                deft = (int)std::lround(std::sqrt(kTileHits / std::max(density, 1e-9))) - w;
                deft = std::min(deft, (int)std::sqrt(cells_all / (12.0 * 152.0)));
                deft = std::min(96, std::max(32, deft));
            }
            target[a] = tile_req[a] > 0 ? tile_req[a] : deft;
        }
    };
    reset_targets();
    for (int a = 0; a < dim; ++a)
        if (target[a] > kMaxTileEdge) return FRESCO_ERR_ARG;
    for (int iter = 0;; ++iter) {
        for (int a = 0; a < dim; ++a) {
            P.nb[a] = choose_tiles(P.nf[a], target[a], minw);
            P.tmax[a] = (P.nf[a] + P.nb[a] - 1) / P.nb[a];
        }
        // point lists: the expected points of a tile (with its halo for ensembles) plus five
        // standard deviations (Poisson) and 64; a tile beyond it takes the slower unlisted path
        // (single plans list a tile's own points; ensembles every point that reaches the tile)
        double hits = density;
        for (int a = 0; a < dim; ++a) hits *= (double)(P.tmax[a] + (own_tiles ? 0 : w));
        const double lmin = own_tiles ? 256.0 : 1024.0, lstep = own_tiles ? 32.0 : 256.0;
        P.list_cap = (int)std::min<double>(
            16384.0,
            std::max(lmin, std::ceil((hits + 5.0 * std::sqrt(hits) + 64.0) / lstep) * lstep));
        Geom tg{};
        tg.dim = dim;
        tg.width = w;
        tg.list_cap = P.list_cap;
        tg.zseg = own_tiles && dim == 3 && P.tmax[2] + w <= kColMaxPlanes ? kZSegment : 0;
        for (int a = 0; a < 3; ++a) tg.tmax[a] = a < dim ? P.tmax[a] : 1;
        // the interpolation form this plan uses (direct or kernel derivative)
        const bool kd = P.grad_mode == FRESCO_GRAD_KDERIV;
        const size_t interp =
            es == 8 ? (kd ? Launch<double>::interp_kd_smem(tg) : Launch<double>::interp_smem(tg))
                    : (kd ? Launch<float>::interp_kd_smem(tg) : Launch<float>::interp_smem(tg));
        const size_t spread =
            own_tiles ? (es == 8 ? Launch<double>::spread_own_smem(tg)
                                 : Launch<float>::spread_own_smem(tg))
                      : (es == 8 ? Launch<double>::spread_smem(tg) : Launch<float>::spread_smem(tg));
        if (interp <= budget && spread <= budget) break;
        int amax = 0;
        for (int a = 1; a < dim; ++a)
            if (P.tmax[a] > P.tmax[amax]) amax = a;
        if (target[amax] <= minw || iter > 256) {
            if (budget >= kSmemOptin) return FRESCO_ERR_UNSUPPORTED;
            budget = kSmemOptin;   // one block per SM rather than no plan
            reset_targets();
            iter = 0;
            continue;
        }
        target[amax] = std::max(minw, std::min(target[amax] - 1, (P.tmax[amax] * 3) / 4));
    }
    for (int a = P.dim; a < 3; ++a) {
        P.nb[a] = 1;
        P.tmax[a] = 1;
    }
    return FRESCO_OK;
}

fresco_status check_and_params(int dim, const double *box, int64_t n_points, const int32_t *mask,
                               int64_t n_k, const double *S0, const double *W,
                               const fresco_opts *opts_in, Params &P,
                               bool width_from_reached = true, bool own_tiles = true) {
    if (dim != 2 && dim != 3) return FRESCO_ERR_ARG;
    if (!box || !mask || !S0 || !W) return FRESCO_ERR_ARG;
    if (n_points < 1 || n_points > 2147483647LL) return FRESCO_ERR_ARG;
    if (n_k < 1) return FRESCO_ERR_ARG;
    fresco_opts o;
    fresco_opts_default(&o);
    if (opts_in) o = *opts_in;
    for (int i = 0; i < 3; ++i)
        if (o.reserved[i] != 0) return FRESCO_ERR_ARG;
    if (o.grad_mode != FRESCO_GRAD_DIRECT && o.grad_mode != FRESCO_GRAD_KDERIV)
        return FRESCO_ERR_ARG;
    if (o.precision != FRESCO_F32 && o.precision != FRESCO_F64) return FRESCO_ERR_ARG;
    double sigma = o.upsample == 0.0 ? 2.0 : o.upsample;
    if (!(sigma >= 1.25 && sigma <= 3.0)) return FRESCO_ERR_ARG;
    double tol = o.tol == 0.0 ? (o.precision == FRESCO_F64 ? 1e-12 : 1e-6) : o.tol;
    if (!(tol > 0.0 && tol < 1.0)) return FRESCO_ERR_ARG;
    for (int a = 0; a < dim; ++a)
        if (!(box[a] > 0.0) || !std::isfinite(box[a])) return FRESCO_ERR_ARG;
    int w = o.width_override ? o.width_override : es_width(tol, sigma);
    if (o.width_override && (w < kMinWidth || w > kMaxWidth)) return FRESCO_ERR_ARG;
    if (w > kMaxWidth) return FRESCO_ERR_UNSUPPORTED;   // tol unreachable at this sigma

    int kmax[3] = {0, 0, 0};
    for (int64_t q = 0; q < n_k; ++q) {
        const int32_t *n = mask + q * dim;
        bool zero = true;
        for (int a = 0; a < dim; ++a) {
            if (n[a] != 0) zero = false;
            if (n[a] <= -(1 << 28) || n[a] >= (1 << 28)) return FRESCO_ERR_ARG;
            kmax[a] = std::max(kmax[a], std::abs(n[a]));
        }
        if (zero) return FRESCO_ERR_ARG;
        if (!std::isfinite(S0[q]) || !std::isfinite(W[q]) || W[q] < 0.0) return FRESCO_ERR_ARG;
    }
    P.dim = dim;
    P.n_points = n_points;
    P.precision = o.precision;
    P.grad_mode = o.grad_mode;
    P.width = w;
    P.sigma = sigma;
    P.tol = tol;
    P.beta = es_beta(w, sigma);
    for (int a = 0; a < 3; ++a) {
        P.kmax[a] = a < dim ? kmax[a] : 0;
        if (a < dim) {
            int64_t need = (int64_t)std::ceil(sigma * (2.0 * kmax[a] + 1.0));
            need = std::max<int64_t>(need, 2 * w);
            need = std::max<int64_t>(need, 2 * (int64_t)kmax[a] + 2);
            int64_t nf = next_smooth_even(need);
            if (nf > (1 << 26)) return FRESCO_ERR_UNSUPPORTED;
            P.nf[a] = (int)nf;
        } else {
            P.nf[a] = 1;
            P.nb[a] = 1;
            P.tmax[a] = 1;
        }
    }
    if (!o.width_override && width_from_reached) {
        // rounding n_f up to an FFT-friendly size raises the oversampling actually reached; the
        // width rule applied to that ratio may then need fewer cells (never more)
        double sig_eff = 1e300;
        for (int a = 0; a < dim; ++a)
            sig_eff = std::min(sig_eff, (double)P.nf[a] / (2.0 * kmax[a] + 1.0));
        const int w_eff = std::max(kMinWidth, es_width(tol, sig_eff));
        if (w_eff < w) {
            w = w_eff;
            P.width = w;
            P.beta = es_beta(w, sig_eff);
        }
    }
    fresco_status st = choose_tiling(P, o.tile, own_tiles);
    if (st) return st;
    int64_t cells = (int64_t)P.nf[0] * P.nf[1] * P.nf[2];
    if (cells > (int64_t)1 << 36) return FRESCO_ERR_UNSUPPORTED;
    int64_t tiles = (int64_t)P.nb[0] * P.nb[1] * P.nb[2];
    if (tiles >= 2147483647LL) return FRESCO_ERR_UNSUPPORTED;
    return FRESCO_OK;
}

// Merge each +-n pair onto its half-space representative (first nonzero component > 0):
// W' = W(n) + W(-n), S0' = (W(n) S0(n) + W(-n) S0(-n)) / W', and the loss constant
// sum W S0^2 - W' S0'^2, so that sum_mask W (S - S0)^2 = sum_rep W' (S - S0')^2 + const
// whenever S(n) = S(-n). Representatives come out ordered by their address in the transposed
// forward spectrum (n_x major, then z, then y, each axis 0..k then -k..-1). Entries whose folded
// weight is zero are dropped (their terms are constants).
fresco_status fold_mask(const Params &P, const int32_t *mask, int64_t n_k, const double *S0,
                        const double *W, Folded &F) {
    const int dim = P.dim;
    const int kx = P.kmax[0], ky = P.kmax[1], kz = P.kmax[2];
    const int64_t ex = kx + 1, ey = 2 * (int64_t)ky + 1, ez = 2 * (int64_t)kz + 1;
    const int64_t box = ex * ey * ez;
    if (box > ((int64_t)1 << 31)) return FRESCO_ERR_UNSUPPORTED;
    std::vector<int32_t> slot;
    try {
        slot.assign((size_t)box, -1);
    } catch (...) {
        return FRESCO_ERR_OOM;
    }
    std::vector<double> sw, sws, sws2;
    std::vector<int32_t> nrep;
    for (int64_t q = 0; q < n_k; ++q) {
        int32_t n[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) n[a] = mask[q * dim + a];
        if (!canonical(n, dim))
            for (int a = 0; a < 3; ++a) n[a] = -n[a];
        const int64_t idx = ((int64_t)(n[2] + kz) * ey + (n[1] + ky)) * ex + n[0];
        int32_t s = slot[idx];
        if (s < 0) {
            s = (int32_t)sw.size();
            slot[idx] = s;
            sw.push_back(0.0);
            sws.push_back(0.0);
            sws2.push_back(0.0);
            for (int a = 0; a < dim; ++a) nrep.push_back(n[a]);
        }
        sw[s] += W[q];
        sws[s] += W[q] * S0[q];
        sws2[s] += W[q] * S0[q] * S0[q];
    }
    // emit in transposed-spectrum address order
    F.n.clear();
    F.s0.clear();
    F.w.clear();
    F.loss_const = 0.0;
    F.n.reserve(nrep.size());
    auto order = [](int k, int i) { return i <= k ? i : i - (2 * k + 1); };
    for (int x = 0; x <= kx; ++x) {
        for (int64_t iz = 0; iz < ez; ++iz) {
            const int z = order(kz, (int)iz);
            for (int64_t iy = 0; iy < ey; ++iy) {
                const int y = order(ky, (int)iy);
                const int32_t s = slot[((int64_t)(z + kz) * ey + (y + ky)) * ex + x];
                if (s < 0) continue;
                const double wp = sw[s];
                if (wp > 0.0) {
                    const double s0p = sws[s] / wp;
                    F.loss_const += sws2[s] - wp * s0p * s0p;
                    for (int a = 0; a < dim; ++a) F.n.push_back(nrep[(size_t)s * dim + a]);
                    F.s0.push_back(s0p);
                    F.w.push_back(wp);
                } else {
                    F.loss_const += sws2[s];
                }
            }
        }
    }
    return FRESCO_OK;
}

void fill_info(const Params &P, int64_t n_points, int64_t n_k, const Folded &F, fresco_info *info) {
    std::memset(info, 0, sizeof(*info));
    info->dim = P.dim;
    info->precision = P.precision;
    info->width = P.width;
    for (int a = 0; a < 3; ++a) {
        info->n_fine[a] = P.nf[a];
        info->k_max[a] = P.kmax[a];
        info->tile[a] = P.tmax[a];
        info->n_tiles[a] = P.nb[a];
    }
    info->beta = P.beta;
    info->upsample = P.sigma;
    info->loss_const = F.loss_const;
    info->n_points = n_points;
    info->n_modes = n_k;
    info->n_rep = (int64_t)F.s0.size();
    info->grad_mode = P.grad_mode;
}

// ---- device helpers --------------------------------------------------------------------------

fresco_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FRESCO_OK;
    if (e == cudaErrorMemoryAllocation) return FRESCO_ERR_OOM;
    return FRESCO_ERR_CUDA;
}

#define FR_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            fresco_status st_ = cuda_status(e_);              \
            return st_;                                       \
        }                                                     \
    } while (0)

#define FR_CUFFT(call)                                        \
    do {                                                      \
        cufftResult r_ = (call);                              \
        if (r_ != CUFFT_SUCCESS)                              \
            return r_ == CUFFT_ALLOC_FAILED ? FRESCO_ERR_OOM : FRESCO_ERR_CUFFT; \
    } while (0)

template <typename P>
fresco_status dalloc(fresco_plan_s *p, P **ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FRESCO_ERR_OOM;
    }
    p->device_bytes += (int64_t)bytes;
    *ptr = (P *)v;
    return FRESCO_OK;
}

void release(fresco_plan_s *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    void *bufs[] = {p->d_sorted, p->d_perm, p->d_ring, p->d_cnt, p->d_off, p->d_tcur, p->d_tr,
                    p->d_block_sums, p->d_grid, p->d_tw, p->d_specT, p->d_bt[0], p->d_bt[1],
                    p->d_hc[0], p->d_hc[1], p->d_r[0],
                    p->d_r[1], p->d_g[0], p->d_g[1], p->d_rep_n, p->d_rep_s0, p->d_rep_w,
                    p->d_ip[0], p->d_ip[1], p->d_ip[2], p->d_partial, p->d_err,
                    p->d_mask_orig, p->d_fft_work, p->d_stage_pts, p->d_stage_grad,
                    p->d_stage_loss};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : p->copy_ev)
        if (e) cudaEventDestroy(e);
    if (p->copy_stream) {
        cudaStreamSynchronize(p->copy_stream);
        cudaStreamDestroy(p->copy_stream);
    }
    cufftHandle hs[] = {p->fft_rows, p->fft_cols, p->ifft_cols, p->ifft_rows};
    for (int i = 0; i < 4; ++i)
        if (p->have_fft[i]) cufftDestroy(hs[i]);
    p->prof.release();
    delete p;
}

template <typename T>
cufftType c2r_type();
template <>
cufftType c2r_type<float>() { return CUFFT_C2R; }
template <>
cufftType c2r_type<double>() { return CUFFT_Z2D; }

template <typename T>
cufftType r2c_type();
template <>
cufftType r2c_type<float>() { return CUFFT_R2C; }
template <>
cufftType r2c_type<double>() { return CUFFT_D2Z; }
template <typename T>
cufftType c2c_type();
template <>
cufftType c2c_type<float>() { return CUFFT_C2C; }
template <>
cufftType c2c_type<double>() { return CUFFT_Z2Z; }

// Four cuFFT plans implement the pruned d-dimensional transforms, every one a batch of
// contiguous transforms (our kernels move the data in between):
//   forward: each real row of length nf0 as a complex row of length nf0/2, in place on the grid;
//            split into the half spectrum, whose columns x = 0..kx are written transposed to
//            [kx+1][plane] (k_rfft_split_cols); C2C over the contiguous (z,)y plane of each, in
//            place;
//   inverse: C2C over (z,)y for the transposed columns of the compact spectrum (out of place, so
//            its zeros survive); in the direct mode transposed back into R, whose other columns
//            were zeroed at plan time and are never written, and C2C along x; in the kderiv mode
//            merged into complex rows of length nf0/2 (k_rfft_merge_rows) and transformed in
//            place, which leaves the real field in R.
template <typename T>
fresco_status make_ffts(fresco_plan_s *p) {
    const int dim = p->dim;
    const int nf0 = p->geom.nf[0], nf1 = p->geom.nf[1], nf2 = p->geom.nf[2];
    const long long rows = (long long)nf1 * nf2;
    const long long kx = p->mgeom.kx;
    const long long hcw = p->mgeom.hc_row;
    size_t ws[4] = {0, 0, 0, 0};
    cufftHandle *hs[4] = {&p->fft_rows, &p->fft_cols, &p->ifft_cols, &p->ifft_rows};
    for (int i = 0; i < 4; ++i) {
        FR_CUFFT(cufftCreate(hs[i]));
        p->have_fft[i] = true;
        FR_CUFFT(cufftSetAutoAllocation(*hs[i], 0));
    }
    const long long mh = nf0 / 2;   // the real rows run as complex rows of half the length
    {   // rows, forward, in place on the grid
        long long n[1] = {mh};
        FR_CUFFT(cufftMakePlanMany64(p->fft_rows, 1, n, nullptr, 1, mh, nullptr, 1, mh,
                                     c2c_type<T>(), rows, &ws[0]));
    }
    long long cn[2];
    const int crank = dim - 1;
    if (dim == 2) {
        cn[0] = nf1;
    } else {
        cn[0] = nf2;
        cn[1] = nf1;
    }
    const long long plane = rows;
    // (z,)y transforms over contiguous planes of the transposed spectra
    FR_CUFFT(cufftMakePlanMany64(p->fft_cols, crank, cn, nullptr, 1, plane, nullptr, 1, plane,
                                 c2c_type<T>(), kx + 1, &ws[1]));
    FR_CUFFT(cufftMakePlanMany64(p->ifft_cols, crank, cn, nullptr, 1, plane, nullptr, 1, plane,
                                 c2c_type<T>(), hcw, &ws[2]));
    if (p->mgeom.kderiv) {   // rows, inverse, in place on the merged half-length rows
        long long n[1] = {mh};
        FR_CUFFT(cufftMakePlanMany64(p->ifft_rows, 1, n, nullptr, 1, mh, nullptr, 1, mh,
                                     c2c_type<T>(), rows, &ws[3]));
    } else {
        long long n[1] = {nf0};
        FR_CUFFT(cufftMakePlanMany64(p->ifft_rows, 1, n, nullptr, 1, nf0, nullptr, 1, nf0,
                                     c2c_type<T>(), rows, &ws[3]));
    }
    size_t wmax = std::max(std::max(ws[0], ws[1]), std::max(ws[2], ws[3]));
    fresco_status st = dalloc(p, &p->d_fft_work, wmax);
    if (st) return st;
    for (int i = 0; i < 4; ++i) {
        FR_CUFFT(cufftSetWorkArea(*hs[i], p->d_fft_work));
        FR_CUFFT(cufftSetStream(*hs[i], p->stream));
    }
    return FRESCO_OK;
}

// Blocks of a 256-thread tile kernel one SM holds at a given dynamic shared memory (each block
// also takes up to 4 KB of static shared state and 1 KB the hardware reserves; 228 KB per SM).
int tile_blocks_per_sm(size_t dyn) { return (int)((228 * 1024) / (dyn + 5 * 1024)); }

// TMA staging of the kernel-derivative interpolation (FP32 plans): the real field h, [nf2][nf1]
// [nf0] floats, as a tensor whose boxes cover a tile's region from the 16-byte boundary at or
// below its first column (rows up to 3 elements wider than the region). Sets g.tma and g.tbox
// and encodes p->tmap; leaves g.tma = 0 (the copy path) where the box or the tensor does not meet
// the TMA rules (box extents <= 256, rows a multiple of 16 bytes) or where the wider staged box
// would cost the interpolation kernel resident blocks.
void setup_interp_tma(fresco_plan_s *p, const void *field) {
    Geom &g = p->geom;
    g.tma = 0;
    if (p->precision != FRESCO_F32 || !p->mgeom.kderiv || (g.nf[0] * 4) % 16 != 0) return;
    const int w = g.width;
    Geom t = g;
    t.tbox[0] = (g.tmax[0] + w + 3 + 3) & ~3;
    t.tbox[1] = g.tmax[1] + w;
    t.tbox[2] = g.dim == 3 ? g.tmax[2] + w : 1;
    for (int a = 0; a < g.dim; ++a)
        if (t.tbox[a] > 256) return;
    const size_t before = (size_t)Launch<float>::interp_kd_smem(g);
    t.tma = 1;
    const size_t after = (size_t)Launch<float>::interp_kd_smem(t);
    if (after > kSmemOptin || tile_blocks_per_sm(after) < std::min(tile_blocks_per_sm(before), 3))
        return;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return;
    }
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t dims[3] = {(cuuint64_t)g.nf[0], (cuuint64_t)g.nf[1], (cuuint64_t)g.nf[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nf[0] * 4, (cuuint64_t)g.nf[0] * g.nf[1] * 4};
    const cuuint32_t box[3] = {(cuuint32_t)t.tbox[0], (cuuint32_t)t.tbox[1],
                               (cuuint32_t)t.tbox[2]};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(
        &p->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)g.dim, const_cast<void *>(field),
        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
    g = t;
}

// Records per tile of the direct binning form: the expected points of the widest tile (uniform
// density) plus eight Poisson standard deviations and 32, so that uniform and near-uniform inputs
// never overflow a tile. 0 (compact form only) where the slots would not be indexable in 32 bits
// or would take more than four times the points' records.
int direct_tile_capacity(const Geom &g) {
    double cells = 1.0, tile = 1.0;
    for (int a = 0; a < g.dim; ++a) {
        cells *= (double)g.nf[a];
        tile *= (double)g.tmax[a];
    }
    const double mu = (double)g.n_points / cells * tile;
    const double cap = std::ceil(mu + 8.0 * std::sqrt(mu) + 32.0);
    const double slots = cap * (double)g.n_tiles;
    if (slots >= 2147483647.0 || slots > 4.0 * (double)g.n_points + 1048576.0) return 0;
    return (int)cap;
}

template <typename T>
fresco_status build_plan(fresco_plan_s *p, const Params &P, const Folded &F) {
    using C2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const int dim = p->dim;
    Geom &g = p->geom;
    g.dim = dim;
    for (int a = 0; a < 3; ++a) {
        g.nf[a] = P.nf[a];
        g.nb[a] = P.nb[a];
        g.tmax[a] = P.tmax[a];
        g.tq[a] = P.nf[a] / P.nb[a];
        g.tr[a] = P.nf[a] % P.nb[a];
        g.tinv[a] = (float)P.nb[a] / (float)P.nf[a];
        double s = a < dim ? (double)P.nf[a] / p->box[a] : 0.0;
        double shi = (double)(T)s;
        long double slo = (long double)P.nf[a] / (long double)(a < dim ? p->box[a] : 1.0) -
                          (long double)shi;
        g.s_hi[a] = shi;
        g.s_lo[a] = a < dim ? (double)(T)(double)slo : 0.0;
    }
    es_poly<float>(P.width, P.beta, p->poly32);
    es_poly<double>(P.width, P.beta, p->poly64);
    g.n_tiles = (int64_t)P.nb[0] * P.nb[1] * P.nb[2];
    g.list_cap = P.list_cap;
    g.sub = kTileCursors;   // own-points spread: no border strips; sub-cursors per tile
    g.zseg = dim == 3 && P.tmax[2] + P.width <= kColMaxPlanes ? std::min(kZSegment, P.nb[2]) : 0;
    for (int a = 0; a < 3; ++a) g.strips[a] = 0;
    g.n_bins = g.n_tiles * g.sub;
    if (g.n_bins >= 2147483647LL) return FRESCO_ERR_UNSUPPORTED;
    g.n_points = p->n_points;
    g.width = P.width;
    g.beta = P.beta;
    g.tcap = direct_tile_capacity(g);
    set_tile_divisors(g);

    MaskGeom &m = p->mgeom;
    m.dim = dim;
    for (int a = 0; a < 3; ++a) {
        m.nf[a] = P.nf[a];
        m.kscale[a] = a < dim ? 2.0 * kPi / p->box[a] : 0.0;
    }
    m.kx = P.kmax[0];
    m.n_rep = (int64_t)F.s0.size();
    m.half_row = P.nf[0] / 2 + 1;
    m.kderiv = P.grad_mode == FRESCO_GRAD_KDERIV ? 1 : 0;
    m.hc_row = m.kderiv ? (int64_t)P.kmax[0] + 1 : 2 * (int64_t)P.kmax[0] + 2;
    m.plane = (int64_t)P.nf[1] * P.nf[2];
    m.inv_n = 1.0 / (double)p->n_points;
    p->n_pipes = (dim == 2 || m.kderiv) ? 1 : 2;
    for (int a = 0; a < 3; ++a)
        p->dscale[a] = a < dim ? -2.0 * (double)P.nf[a] / p->box[a] : 0.0;

    // shared memory budget
    int dev = 0;
    FR_CUDA(cudaGetDevice(&dev));
    int smem_optin = 0;
    FR_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int interp_bytes =
        m.kderiv ? Launch<T>::interp_kd_smem(g) : Launch<T>::interp_smem(g);
    if (Launch<T>::spread_own_smem(g) > smem_optin || interp_bytes > smem_optin)
        return FRESCO_ERR_UNSUPPORTED;

    const int64_t N = p->n_points;
    const int64_t cells = (int64_t)P.nf[0] * P.nf[1] * P.nf[2];
    const int64_t rows = (int64_t)P.nf[1] * P.nf[2];
    // sorted records: float plans keep the caller index inside each 16-byte record
    const int pw = sizeof(T) == 4 ? 4 : (dim == 3 ? 4 : 2);
    // record slots: the compact form's N, or the direct form's tcap per tile if more
    const int64_t slots = std::max<int64_t>(N, (int64_t)g.tcap * g.n_tiles);
    fresco_status st;
    if ((st = dalloc(p, &p->d_sorted, sizeof(T) * (size_t)slots * pw))) return st;
    if (sizeof(T) == 8 && (st = dalloc(p, &p->d_perm, sizeof(int) * (size_t)slots))) return st;
    if ((st = dalloc(p, &p->d_tcur, sizeof(int) * (size_t)(g.n_tiles + 1)))) return st;
    if ((st = dalloc(p, &p->d_tr, sizeof(int2) * (size_t)g.n_tiles))) return st;
    p->ring_slot = Launch<T>::ring_slot(g);
    if ((st = dalloc(p, &p->d_ring, sizeof(T) * (size_t)(g.n_tiles * p->ring_slot)))) return st;
    if ((st = dalloc(p, &p->d_cnt, sizeof(int) * (size_t)g.n_bins))) return st;
    if ((st = dalloc(p, &p->d_off, sizeof(int) * (size_t)(g.n_bins + 1)))) return st;
    if ((st = dalloc(p, &p->d_block_sums, sizeof(int) * (size_t)((g.n_bins + 1023) / 1024 + 1))))
        return st;

    if ((st = dalloc(p, &p->d_grid, sizeof(T) * (size_t)cells))) return st;
    {   // tau_k = exp(-2 pi i k / nf0), k = 0..nf0/4, for the real-row split and merge
        const int mh = g.nf[0] / 2;
        std::vector<C2> tw(mh / 2 + 1);
        for (int k = 0; k <= mh / 2; ++k) {
            const double a = 2.0 * M_PI * (double)k / (double)g.nf[0];
            tw[k].x = (T)std::cos(a);
            tw[k].y = (T)-std::sin(a);
        }
        if ((st = dalloc(p, &p->d_tw, sizeof(C2) * tw.size()))) return st;
        FR_CUDA(cudaMemcpy(p->d_tw, tw.data(), sizeof(C2) * tw.size(), cudaMemcpyHostToDevice));
    }
    if ((st = dalloc(p, &p->d_specT, sizeof(C2) * (size_t)(rows * (m.kx + 1))))) return st;
    // backward spectra: compact transposed [hc_row][plane], after the (z,)y pass, back in row
    // order (the direct mode's full complex rows, whose columns outside the mask stay zero from
    // here on; the kderiv mode's merged complex rows of nf0/2, every entry written per call), and
    // the direct mode's gradient grid(s)
    const size_t r_elems = m.kderiv ? (size_t)rows * (size_t)(g.nf[0] / 2) : (size_t)cells;
    // (the kderiv mode's inverse runs in place in R, whose rows then hold the real field)
    const size_t g_bytes = m.kderiv ? 0 : sizeof(C2) * (size_t)cells;
    for (int q = 0; q < p->n_pipes; ++q) {
        if ((st = dalloc(p, &p->d_hc[q], sizeof(C2) * (size_t)(rows * m.hc_row)))) return st;
        if ((st = dalloc(p, &p->d_bt[q], sizeof(C2) * (size_t)(rows * m.hc_row)))) return st;
        if ((st = dalloc(p, &p->d_r[q], sizeof(C2) * r_elems))) return st;
        if (g_bytes && (st = dalloc(p, &p->d_g[q], g_bytes))) return st;
        FR_CUDA(cudaMemsetAsync(p->d_hc[q], 0, sizeof(C2) * (size_t)(rows * m.hc_row), p->stream));
        FR_CUDA(cudaMemsetAsync(p->d_r[q], 0, sizeof(C2) * r_elems, p->stream));
    }
    const int64_t nrep = m.n_rep;
    if ((st = dalloc(p, &p->d_rep_n, sizeof(int) * (size_t)(nrep * dim)))) return st;
    if ((st = dalloc(p, &p->d_rep_s0, sizeof(T) * (size_t)nrep))) return st;
    if ((st = dalloc(p, &p->d_rep_w, sizeof(T) * (size_t)nrep))) return st;
    p->n_mask_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nrep + 255) / 256, 152 * 8));
    if ((st = dalloc(p, &p->d_partial, sizeof(double) * (size_t)p->n_mask_blocks))) return st;
    if ((st = dalloc(p, &p->d_err, sizeof(int)))) return st;
    FR_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream));

    {   // representatives
        std::vector<T> s0(nrep), w(nrep);
        for (int64_t i = 0; i < nrep; ++i) {
            s0[i] = (T)F.s0[i];
            w[i] = (T)F.w[i];
        }
        FR_CUDA(cudaMemcpy(p->d_rep_n, F.n.data(), sizeof(int) * (size_t)(nrep * dim),
                           cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(p->d_rep_s0, s0.data(), sizeof(T) * (size_t)nrep, cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(p->d_rep_w, w.data(), sizeof(T) * (size_t)nrep, cudaMemcpyHostToDevice));
    }
    for (int a = 0; a < dim; ++a) {   // 1 / Psi_a(nu), nu = 0..kmax[a]
        const int64_t n_nu = P.kmax[a] + 1;
        std::vector<double> ft(n_nu);
        kernel_ft(P.width, P.beta, P.nf[a], n_nu, ft.data());
        std::vector<T> ip(n_nu);
        for (int64_t i = 0; i < n_nu; ++i) ip[i] = (T)(1.0 / ft[i]);
        if ((st = dalloc(p, &p->d_ip[a], sizeof(T) * (size_t)n_nu))) return st;
        FR_CUDA(cudaMemcpy(p->d_ip[a], ip.data(), sizeof(T) * (size_t)n_nu, cudaMemcpyHostToDevice));
    }
    if ((st = make_ffts<T>(p))) return st;
    setup_interp_tma(p, p->d_r[0]);
    FR_CUDA(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    return FRESCO_OK;
}

// ---- evaluation ------------------------------------------------------------------------------

template <typename T>
const EsPoly<T> &poly_of(const fresco_plan_s *p);
template <>
const EsPoly<float> &poly_of<float>(const fresco_plan_s *p) { return p->poly32; }
template <>
const EsPoly<double> &poly_of<double>(const fresco_plan_s *p) { return p->poly64; }

// Host points into the device staging buffer, overlapped with the binning: the copy runs in
// chunks on a second stream and the plan's stream bins each chunk as soon as it has landed (the
// direct form places it, the compact form counts it). The slots within a tile come from atomics
// in any case and the fixed-point spread does not depend on them, so the result is the same as
// binning all points at once. The caller zeroes the counts (compact) or cursors (direct).
template <typename T>
fresco_status stage_and_bin(fresco_plan_s *p, const T *h_pts, T *d_pts) {
    const Geom &g = p->geom;
    const int64_t n = g.n_points, d = g.dim;
    const int64_t bytes = (int64_t)sizeof(T) * n * d;
    const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(kHostChunks, bytes / kHostChunkBytes));
    if (!p->copy_stream) FR_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t &e : p->copy_ev)
        if (!e) FR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    FR_CUDA(cudaEventRecord(p->copy_ev[kHostChunks], p->stream));
    FR_CUDA(cudaStreamWaitEvent(p->copy_stream, p->copy_ev[kHostChunks], 0));
    // chunks start at multiples of the cursors per tile, so a point's bin (which depends on its
    // caller index modulo g.sub) is the same whether it is counted in its chunk or placed later
    const int64_t per = ((n + chunks - 1) / chunks + g.sub - 1) / g.sub * g.sub;
    for (int c = 0; c < chunks; ++c) {
        const int64_t j0 = c * per, cnt = std::min(per, n - j0);
        if (cnt <= 0) break;
        FR_CUDA(cudaMemcpyAsync(d_pts + j0 * d, h_pts + j0 * d, sizeof(T) * (size_t)(cnt * d),
                                cudaMemcpyHostToDevice, p->copy_stream));
        FR_CUDA(cudaEventRecord(p->copy_ev[c], p->copy_stream));
        FR_CUDA(cudaStreamWaitEvent(p->stream, p->copy_ev[c], 0));
        Geom gc = g;
        gc.n_points = cnt;
        if (g.tcap)
            FR_CUDA(Launch<T>::place_direct(gc, d_pts + j0 * d, j0, p->d_tcur, p->d_sorted,
                                            p->d_perm, p->d_err, p->stream));
        else
            FR_CUDA(Launch<T>::count(gc, d_pts + j0 * d, p->d_cnt, p->d_err, p->stream));
        p->launches += 1;
    }
    return FRESCO_OK;
}

// h_pts, when not null, is the host copy of the points that pts (the staging buffer) receives.
template <typename T>
fresco_status forward_impl(fresco_plan_s *p, const T *pts, double *loss,
                           const T *h_pts = nullptr) {
    using C2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const Geom &g = p->geom;
    const MaskGeom &m = p->mgeom;
    cudaStream_t s = p->stream;
    {
        StageScope sc(p->prof, p->stream, ST_SORT);
        int nl = 0;
        // the direct form (one pass), then the compact form: always in a plan without the direct
        // form, else only if a tile overflowed (its kernels read the overflow word as a guard)
        const int *guard = nullptr;
        if (g.tcap) {
            FR_CUDA(cudaMemsetAsync(p->d_tcur, 0, sizeof(int) * (size_t)(g.n_tiles + 1), s));
            guard = p->d_tcur + g.n_tiles;
        }
        FR_CUDA(cudaMemsetAsync(p->d_cnt, 0, sizeof(int) * (size_t)g.n_bins, s));
        if (h_pts) {
            fresco_status st = stage_and_bin<T>(p, h_pts, const_cast<T *>(pts));
            if (st) return st;
        } else if (g.tcap) {
            FR_CUDA(Launch<T>::place_direct(g, pts, 0, p->d_tcur, p->d_sorted, p->d_perm, p->d_err,
                                            s));
            nl += 1;
        }
        if (!h_pts || g.tcap) {
            FR_CUDA(Launch<T>::count(g, pts, p->d_cnt, p->d_err, s, guard));
            nl += 1;
        }
        // the counts become the placement cursors (a copy of the tile offsets)
        FR_CUDA(Launch<T>::scan(p->d_cnt, p->d_off, p->d_block_sums, g.n_bins, s, &nl, p->d_cnt,
                                guard));
        FR_CUDA(Launch<T>::place(g, pts, p->d_cnt, p->d_sorted, p->d_perm, s, guard));
        FR_CUDA(Launch<T>::tile_ranges(g, g.tcap ? p->d_tcur : nullptr, p->d_off, p->d_tr, s));
        nl += 2;
        p->launches += nl;
    }
    {
        StageScope sc(p->prof, p->stream, ST_SPREAD);
        int nl = 0;
        FR_CUDA(Launch<T>::spread_own(g, poly_of<T>(p), p->d_sorted, p->d_tr, (T *)p->d_grid,
                                      (T *)p->d_ring, p->ring_slot, s, &nl));
        p->launches += nl;
    }
    {
        StageScope sc(p->prof, p->stream, ST_FFT_FWD);
        const int64_t rows = m.plane;
        if (sizeof(T) == 4)
            FR_CUFFT(cufftExecC2C(p->fft_rows, (cufftComplex *)p->d_grid,
                                  (cufftComplex *)p->d_grid, CUFFT_FORWARD));
        else
            FR_CUFFT(cufftExecZ2Z(p->fft_rows, (cufftDoubleComplex *)p->d_grid,
                                  (cufftDoubleComplex *)p->d_grid, CUFFT_FORWARD));
        FR_CUDA(Launch<T>::rfft_split(p->d_grid, p->d_specT, p->d_tw, rows, g.nf[0] / 2, m.kx, s));
        p->launches += 1;
        if (sizeof(T) == 4)
            FR_CUFFT(cufftExecC2C(p->fft_cols, (cufftComplex *)p->d_specT,
                                  (cufftComplex *)p->d_specT, CUFFT_FORWARD));
        else
            FR_CUFFT(cufftExecZ2Z(p->fft_cols, (cufftDoubleComplex *)p->d_specT,
                                  (cufftDoubleComplex *)p->d_specT, CUFFT_FORWARD));
    }
    {
        StageScope sc(p->prof, p->stream, ST_MASK);
        FR_CUDA(Launch<T>::mask(m, p->d_rep_n, (const T *)p->d_rep_s0, (const T *)p->d_rep_w,
                                p->d_specT, (const T *)p->d_ip[0], (const T *)p->d_ip[1],
                                (const T *)p->d_ip[2], p->d_hc[0], p->d_hc[1], p->d_partial,
                                p->n_mask_blocks, s));
        p->launches += 1;
    }
    {
        StageScope sc(p->prof, p->stream, ST_LOSS);
        FR_CUDA(Launch<T>::finalize(p->d_partial, p->n_mask_blocks, p->info.loss_const, loss, s));
        p->launches += 1;
    }
    (void)sizeof(C2);
    p->forward_done = true;
    return FRESCO_OK;
}

template <typename T>
fresco_status backward_impl(fresco_plan_s *p, const double *grad_out, T *grad) {
    const Geom &g = p->geom;
    const MaskGeom &m = p->mgeom;
    cudaStream_t s = p->stream;
    if (m.kderiv) {
        {
            StageScope sc(p->prof, p->stream, ST_FFT_INV);
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(p->ifft_cols, (cufftComplex *)p->d_hc[0],
                                      (cufftComplex *)p->d_bt[0], CUFFT_INVERSE));
            else
                FR_CUFFT(cufftExecZ2Z(p->ifft_cols, (cufftDoubleComplex *)p->d_hc[0],
                                      (cufftDoubleComplex *)p->d_bt[0], CUFFT_INVERSE));
            FR_CUDA(Launch<T>::rfft_merge(p->d_bt[0], p->d_r[0], p->d_tw, m.plane, g.nf[0] / 2,
                                          m.kx, s));
            p->launches += 1;
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(p->ifft_rows, (cufftComplex *)p->d_r[0],
                                      (cufftComplex *)p->d_r[0], CUFFT_INVERSE));
            else
                FR_CUFFT(cufftExecZ2Z(p->ifft_rows, (cufftDoubleComplex *)p->d_r[0],
                                      (cufftDoubleComplex *)p->d_r[0], CUFFT_INVERSE));
        }
        StageScope sc(p->prof, p->stream, ST_INTERP);
        FR_CUDA(Launch<T>::interp_kd(g, poly_of<T>(p), p->d_sorted, p->d_perm, p->d_tr,
                                     (const T *)p->d_r[0], grad_out, p->dscale, grad, s,
                                     g.tma ? &p->tmap : nullptr, p->d_err));
        p->launches += 1;
        return FRESCO_OK;
    }
    {
        StageScope sc(p->prof, p->stream, ST_FFT_INV);
        for (int q = 0; q < p->n_pipes; ++q) {
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(p->ifft_cols, (cufftComplex *)p->d_hc[q],
                                      (cufftComplex *)p->d_bt[q], CUFFT_INVERSE));
            else
                FR_CUFFT(cufftExecZ2Z(p->ifft_cols, (cufftDoubleComplex *)p->d_hc[q],
                                      (cufftDoubleComplex *)p->d_bt[q], CUFFT_INVERSE));
            FR_CUDA(Launch<T>::rows_to_cols(p->d_bt[q], p->d_r[q], m.plane, g.nf[0], m.kx, s));
            p->launches += 1;
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(p->ifft_rows, (cufftComplex *)p->d_r[q],
                                      (cufftComplex *)p->d_g[q], CUFFT_INVERSE));
            else
                FR_CUFFT(cufftExecZ2Z(p->ifft_rows, (cufftDoubleComplex *)p->d_r[q],
                                      (cufftDoubleComplex *)p->d_g[q], CUFFT_INVERSE));
        }
    }
    {
        StageScope sc(p->prof, p->stream, ST_INTERP);
        FR_CUDA(Launch<T>::interp(g, poly_of<T>(p), p->d_sorted, p->d_perm, p->d_tr, p->d_g[0],
                                  p->d_g[1], grad_out, grad, s));
        p->launches += 1;
    }
    return FRESCO_OK;
}

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

fresco_status check_point_ptr(fresco_plan_s *p, const void *ptr) {
    if (!ptr) return FRESCO_ERR_ARG;
    size_t a = p->esize * (p->dim == 2 ? 2 : 1);
    return aligned(ptr, a) ? FRESCO_OK : FRESCO_ERR_ARG;
}

}  // namespace

// ---- profiling event pool --------------------------------------------------------------------
// ---- point sets spread for other transforms (type-3 plans) -------------------------------------

void fresco::es_poly_table(int w, double beta, EsPoly<float> &out) {
    es_poly<float>(w, beta, out);
}
void fresco::es_poly_table(int w, double beta, EsPoly<double> &out) {
    es_poly<double>(w, beta, out);
}

void fresco::kernel_ft_at(int w, double beta, const double *theta, int64_t n, double *out) {
    const int nq = 200;
    std::vector<double> x, wq;
    gauss_legendre(nq, x, wq);
    const double h = 0.25 * kPi;
    std::vector<double> u(nq), f(nq);
    for (int q = 0; q < nq; ++q) {
        const double th = h * (1.0 + x[q]);
        u[q] = 0.5 * w * std::sin(th);
        f[q] = 2.0 * h * wq[q] * std::exp(beta * (std::cos(th) - 1.0)) * 0.5 * w * std::cos(th);
    }
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += f[q] * std::cos(theta[i] * u[q]);
        out[i] = s;
    }
}

namespace {
bool ps_alloc(fresco::PointSide &ps, void **p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    ps.allocs.push_back(*p);
    ps.device_bytes += (int64_t)bytes;
    return true;
}
}  // namespace

void fresco::point_side_free(PointSide &ps) {
    for (void *p : ps.allocs) cudaFree(p);
    ps.allocs.clear();
}

fresco_status fresco::point_side_build(PointSide &ps, int dim, const int nf[3], const double box[3],
                                       int64_t n_points, int width, double beta, int precision,
                                       cudaStream_t s) {
    Params P{};
    P.dim = dim;
    P.precision = precision;
    P.width = width;
    P.beta = beta;
    P.n_points = n_points;
    P.grad_mode = FRESCO_GRAD_KDERIV;
    for (int a = 0; a < 3; ++a) {
        P.nf[a] = a < dim ? nf[a] : 1;
        P.kmax[a] = 0;
    }
    const int no_req[3] = {0, 0, 0};
    fresco_status st = choose_tiling(P, no_req, true);
    if (st) return st;
    Geom &g = ps.g;
    g = Geom{};
    g.dim = dim;
    const size_t es = precision == FRESCO_F64 ? 8 : 4;
    for (int a = 0; a < 3; ++a) {
        g.nf[a] = P.nf[a];
        g.nb[a] = P.nb[a];
        g.tmax[a] = P.tmax[a];
        g.tq[a] = P.nf[a] / P.nb[a];
        g.tr[a] = P.nf[a] % P.nb[a];
        g.tinv[a] = (float)P.nb[a] / (float)P.nf[a];
        const double sc = a < dim ? (double)P.nf[a] / box[a] : 0.0;
        const double shi = es == 4 ? (double)(float)sc : sc;
        const long double slo = a < dim ? (long double)P.nf[a] / (long double)box[a] - shi : 0.0L;
        g.s_hi[a] = shi;
        g.s_lo[a] = es == 4 ? (double)(float)(double)slo : (double)slo;
    }
    es_poly<float>(width, beta, ps.p32);
    es_poly<double>(width, beta, ps.p64);
    g.n_tiles = (int64_t)P.nb[0] * P.nb[1] * P.nb[2];
    g.list_cap = P.list_cap;
    g.sub = kTileCursors;
    g.zseg = dim == 3 && P.tmax[2] + width <= kColMaxPlanes ? std::min(kZSegment, P.nb[2]) : 0;
    g.n_bins = g.n_tiles * g.sub;
    g.n_points = n_points;
    g.width = width;
    g.beta = beta;
    set_tile_divisors(g);
    ps.precision = precision;
    const int64_t cells = (int64_t)g.nf[0] * g.nf[1] * g.nf[2];
    const int pw = es == 4 ? 4 : (dim == 3 ? 4 : 2);
    ps.ring_slot = es == 8 ? Launch<double>::ring_slot(g) : Launch<float>::ring_slot(g);
    bool ok = ps_alloc(ps, &ps.sorted, es * (size_t)n_points * pw) &&
              (es == 4 || ps_alloc(ps, (void **)&ps.perm, sizeof(int) * (size_t)n_points)) &&
              ps_alloc(ps, (void **)&ps.cnt, sizeof(int) * (size_t)g.n_bins) &&
              ps_alloc(ps, (void **)&ps.off, sizeof(int) * (size_t)(g.n_bins + 1)) &&
              ps_alloc(ps, (void **)&ps.tr, sizeof(int2) * (size_t)g.n_tiles) &&
              ps_alloc(ps, (void **)&ps.bsum, sizeof(int) * (size_t)((g.n_bins + 1023) / 1024 + 1)) &&
              ps_alloc(ps, (void **)&ps.err, sizeof(int)) &&
              ps_alloc(ps, &ps.grid, es * (size_t)cells) &&
              ps_alloc(ps, &ps.ring, es * (size_t)(g.n_tiles * ps.ring_slot));
    if (!ok) {
        point_side_free(ps);
        return FRESCO_ERR_OOM;
    }
    if (cudaMemsetAsync(ps.err, 0, sizeof(int), s) != cudaSuccess) return FRESCO_ERR_CUDA;
    return FRESCO_OK;
}

template <typename T>
fresco_status fresco::point_side_spread(PointSide &ps, const T *pts, cudaStream_t s,
                                        int64_t *launches) {
    const Geom &g = ps.g;
    FR_CUDA(cudaMemsetAsync(ps.cnt, 0, sizeof(int) * (size_t)g.n_bins, s));
    FR_CUDA(Launch<T>::count(g, pts, ps.cnt, ps.err, s));
    int nl = 1;
    FR_CUDA(Launch<T>::scan(ps.cnt, ps.off, ps.bsum, g.n_bins, s, &nl, ps.cnt));
    FR_CUDA(Launch<T>::place(g, pts, ps.cnt, ps.sorted, ps.perm, s));
    FR_CUDA(Launch<T>::tile_ranges(g, nullptr, ps.off, ps.tr, s));
    nl += 2;
    const EsPoly<T> &ep = *reinterpret_cast<const EsPoly<T> *>(sizeof(T) == 4 ? (const void *)&ps.p32
                                                                              : (const void *)&ps.p64);
    FR_CUDA(Launch<T>::spread_own(g, ep, ps.sorted, ps.tr, (T *)ps.grid, (T *)ps.ring,
                                  ps.ring_slot, s, &nl));
    if (launches) *launches += nl;
    return FRESCO_OK;
}

template fresco_status fresco::point_side_spread<float>(PointSide &, const float *, cudaStream_t,
                                                        int64_t *);
template fresco_status fresco::point_side_spread<double>(PointSide &, const double *, cudaStream_t,
                                                         int64_t *);

cudaEvent_t fresco::StageProfile::take() {
    if (!spare.empty()) {
        cudaEvent_t e = spare.back();
        spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void fresco::StageProfile::read(double *ms_out, int64_t *calls_out) {
    for (auto &r : used) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ms[r.stage] += t;
            calls[r.stage] += 1;
        }
        spare.push_back(r.a);
        spare.push_back(r.b);
    }
    used.clear();
    for (int i = 0; i < ST_COUNT; ++i) {
        if (ms_out) ms_out[i] = ms[i];
        if (calls_out) calls_out[i] = calls[i];
        ms[i] = 0.0;
        calls[i] = 0;
    }
}

void fresco::StageProfile::release() {
    for (auto &r : used) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    used.clear();
    for (auto e : spare) cudaEventDestroy(e);
    spare.clear();
}

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

void fresco_opts_default(fresco_opts *opts) {
    if (!opts) return;
    std::memset(opts, 0, sizeof(*opts));
    opts->precision = FRESCO_F32;
    opts->tol = 0.0;
    opts->upsample = 2.0;
}

const char *fresco_status_string(fresco_status s) {
    switch (s) {
        case FRESCO_OK: return "ok";
        case FRESCO_ERR_ARG: return "invalid argument";
        case FRESCO_ERR_OOM: return "out of memory";
        case FRESCO_ERR_CUFFT: return "cuFFT error";
        case FRESCO_ERR_CUDA: return "CUDA error";
        case FRESCO_ERR_NONFINITE: return "non-finite coordinate";
        case FRESCO_ERR_BOUNDS: return "index out of bounds";
        case FRESCO_ERR_TIMEOUT: return "device wait timed out";
        case FRESCO_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

fresco_status fresco_kernel_ft(int width, double beta, int n_fine, int64_t n_nu, double *out) {
    if (width < kMinWidth || width > kMaxWidth || !(beta > 0.0) || n_fine < 2 * width ||
        n_nu < 0 || (n_nu > 0 && !out))
        return FRESCO_ERR_ARG;
    kernel_ft(width, beta, n_fine, n_nu, out);
    return FRESCO_OK;
}

fresco_status fresco_plan_query(int dim, const double *box, int64_t n_points, const int32_t *mask,
                                int64_t n_k, const double *S0, const double *W,
                                const fresco_opts *opts, fresco_info *info) {
    if (!info) return FRESCO_ERR_ARG;
    Params P;
    fresco_status st = check_and_params(dim, box, n_points, mask, n_k, S0, W, opts, P);
    if (st) return st;
    Folded F;
    if ((st = fold_mask(P, mask, n_k, S0, W, F))) return st;
    fill_info(P, n_points, n_k, F, info);
    return FRESCO_OK;
}

fresco_status fresco_plan(fresco_plan_t *out, int dim, const double *box, int64_t n_points,
                          const int32_t *mask, int64_t n_k, const double *S0, const double *W,
                          const fresco_opts *opts, void *stream) {
    if (!out) return FRESCO_ERR_ARG;
    *out = nullptr;
    Params P;
    fresco_status st = check_and_params(dim, box, n_points, mask, n_k, S0, W, opts, P);
    if (st) return st;
    Folded F;
    if ((st = fold_mask(P, mask, n_k, S0, W, F))) return st;
    if (F.s0.empty()) return FRESCO_ERR_ARG;   // every weight zero: nothing to evaluate
    fresco_plan_s *p = new (std::nothrow) fresco_plan_s();
    if (!p) return FRESCO_ERR_OOM;
    p->dim = dim;
    p->precision = P.precision;
    p->esize = P.precision == FRESCO_F64 ? 8 : 4;
    for (int a = 0; a < dim; ++a) p->box[a] = box[a];
    p->n_points = n_points;
    p->n_k = n_k;
    p->stream = (cudaStream_t)stream;
    fill_info(P, n_points, n_k, F, &p->info);
    try {
        p->h_mask.assign(mask, mask + n_k * dim);
    } catch (...) {
        delete p;
        return FRESCO_ERR_OOM;
    }
    st = P.precision == FRESCO_F64 ? build_plan<double>(p, P, F) : build_plan<float>(p, P, F);
    if (st) {
        release(p);
        return st;
    }
    p->info.device_bytes = p->device_bytes;
    *out = p;
    return FRESCO_OK;
}

fresco_status fresco_get_info(fresco_plan_t p, fresco_info *info) {
    if (!p || !info) return FRESCO_ERR_ARG;
    *info = p->info;
    info->device_bytes = p->device_bytes;
    return FRESCO_OK;
}

fresco_status fresco_set_stream(fresco_plan_t p, void *stream) {
    if (!p) return FRESCO_ERR_ARG;
    p->stream = (cudaStream_t)stream;
    cufftHandle hs[] = {p->fft_rows, p->fft_cols, p->ifft_cols, p->ifft_rows};
    for (int i = 0; i < 4; ++i)
        if (p->have_fft[i] && cufftSetStream(hs[i], p->stream) != CUFFT_SUCCESS)
            return FRESCO_ERR_CUFFT;
    return FRESCO_OK;
}

fresco_status fresco_forward(fresco_plan_t p, const void *d_points, double *d_loss) {
    fresco::clear_pending_error();
    if (!p || !d_loss) return FRESCO_ERR_ARG;
    fresco_status st = check_point_ptr(p, d_points);
    if (st) return st;
    if (p->precision == FRESCO_F64) return forward_impl<double>(p, (const double *)d_points, d_loss);
    return forward_impl<float>(p, (const float *)d_points, d_loss);
}

fresco_status fresco_backward(fresco_plan_t p, const double *d_grad_out, void *d_grad) {
    fresco::clear_pending_error();
    if (!p || !p->forward_done) return FRESCO_ERR_ARG;
    fresco_status st = check_point_ptr(p, d_grad);
    if (st) return st;
    if (p->precision == FRESCO_F64) return backward_impl<double>(p, d_grad_out, (double *)d_grad);
    return backward_impl<float>(p, d_grad_out, (float *)d_grad);
}

fresco_status fresco_loss_grad(fresco_plan_t p, const void *d_points, double *d_loss, void *d_grad) {
    fresco_status st = fresco_forward(p, d_points, d_loss);
    if (st || !d_grad) return st;
    return fresco_backward(p, nullptr, d_grad);
}

fresco_status fresco_get_rho_S(fresco_plan_t p, void *d_rho, void *d_S) {
    fresco::clear_pending_error();
    if (!p || !p->forward_done) return FRESCO_ERR_ARG;
    if (!d_rho && !d_S) return FRESCO_OK;
    if (!p->d_mask_orig) {
        fresco_status st = dalloc(p, &p->d_mask_orig, sizeof(int) * p->h_mask.size());
        if (st) return st;
        FR_CUDA(cudaMemcpyAsync(p->d_mask_orig, p->h_mask.data(), sizeof(int) * p->h_mask.size(),
                                cudaMemcpyHostToDevice, p->stream));
    }
    cudaError_t e;
    if (p->precision == FRESCO_F64)
        e = Launch<double>::rho_s(p->mgeom, p->d_mask_orig, p->n_k, p->d_specT,
                                  (const double *)p->d_ip[0], (const double *)p->d_ip[1],
                                  (const double *)p->d_ip[2], (double *)d_rho, (double *)d_S,
                                  p->stream);
    else
        e = Launch<float>::rho_s(p->mgeom, p->d_mask_orig, p->n_k, p->d_specT,
                                 (const float *)p->d_ip[0], (const float *)p->d_ip[1],
                                 (const float *)p->d_ip[2], (float *)d_rho, (float *)d_S,
                                 p->stream);
    p->launches += 1;
    return cuda_status(e);
}

fresco_status fresco_loss_grad_host(fresco_plan_t p, const void *h_points, double *h_loss,
                                    void *h_grad) {
    fresco::clear_pending_error();
    if (!p || !h_points || !h_loss) return FRESCO_ERR_ARG;
    const size_t bytes = p->esize * (size_t)p->n_points * p->dim;
    fresco_status st;
    if (!p->d_stage_pts && (st = dalloc(p, &p->d_stage_pts, bytes))) return st;
    if (!p->d_stage_grad && (st = dalloc(p, &p->d_stage_grad, bytes))) return st;
    if (!p->d_stage_loss && (st = dalloc(p, &p->d_stage_loss, sizeof(double)))) return st;
    st = p->precision == FRESCO_F64
             ? forward_impl<double>(p, (const double *)p->d_stage_pts, p->d_stage_loss,
                                    (const double *)h_points)
             : forward_impl<float>(p, (const float *)p->d_stage_pts, p->d_stage_loss,
                                   (const float *)h_points);
    if (!st && h_grad) st = fresco_backward(p, nullptr, p->d_stage_grad);
    if (st) return st;
    FR_CUDA(cudaMemcpyAsync(h_loss, p->d_stage_loss, sizeof(double), cudaMemcpyDeviceToHost,
                            p->stream));
    if (h_grad)
        FR_CUDA(cudaMemcpyAsync(h_grad, p->d_stage_grad, bytes, cudaMemcpyDeviceToHost, p->stream));
    FR_CUDA(cudaStreamSynchronize(p->stream));
    return FRESCO_OK;
}

fresco_status fresco_status_check(fresco_plan_t p) {
    if (!p) return FRESCO_ERR_ARG;
    FR_CUDA(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    int err = 0;
    FR_CUDA(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        int zero = 0;
        FR_CUDA(cudaMemcpy(p->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        if (err & 1) return FRESCO_ERR_NONFINITE;
        if (err & 4) return FRESCO_ERR_TIMEOUT;
        return FRESCO_ERR_BOUNDS;   // (bit 2: a point beyond the box; bit 8: a misaligned TMA box)
    }
    return cuda_status(cudaGetLastError());
}

fresco_status fresco_profile(fresco_plan_t p, int enable) {
    if (!p) return FRESCO_ERR_ARG;
    p->prof.on = enable != 0;
    return FRESCO_OK;
}

fresco_status fresco_profile_read(fresco_plan_t p, double *ms, int64_t *counts) {
    if (!p || !ms) return FRESCO_ERR_ARG;
    FR_CUDA(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    p->prof.read(ms, counts);
    return FRESCO_OK;
}

int64_t fresco_launch_count(fresco_plan_t p) { return p ? p->launches : -1; }

fresco_status fresco_destroy(fresco_plan_t p) {
    release(p);
    return FRESCO_OK;
}

}  // extern "C"

// ============================================================================================
// Ensembles: many independent problems evaluated by one set of launches
// ============================================================================================


namespace {

bool balloc(fresco_batch_s *b, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    b->allocs.push_back(*p);
    b->device_bytes += (int64_t)bytes;
    return true;
}

void batch_free(fresco_batch_s *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &c : b->cls)
        for (int i = 0; i < 4; ++i)
            if (c.have[i]) cufftDestroy(c.h[i]);
    for (void *p : b->allocs) cudaFree(p);
    b->prof.release();
    delete b;
}

// FFT size class of a fine-grid size: the smallest 2^k or 3 * 2^k (k >= 3) not below it
int class_size(int nf) {
    int best = 1 << 30;
    for (int64_t p = 8; p < (1 << 27); p *= 2) {
        if (p >= nf && p < best) best = (int)p;
        if (3 * p / 2 >= nf && 3 * p / 2 < best && (3 * p / 2) % 2 == 0) best = (int)(3 * p / 2);
    }
    return best;
}

template <typename T>
fresco_status batch_build(fresco_batch_s *b, const std::vector<Params> &P,
                          const std::vector<Folded> &F, const double *boxes,
                          const int64_t *n_points) {
    using C2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const int dim = b->dim;
    const int n = b->n_inst;
    // ---- classes (by fine grid size), per-class kx
    std::vector<int> cls_of(n);
    for (int i = 0; i < n; ++i) {
        int found = -1;
        for (size_t c = 0; c < b->cls.size(); ++c)
            if (b->cls[c].nf[0] == P[i].nf[0] && b->cls[c].nf[1] == P[i].nf[1]) found = (int)c;
        if (found < 0) {
            fresco_batch_s::Cls c;
            c.nf[0] = P[i].nf[0];
            c.nf[1] = P[i].nf[1];
            b->cls.push_back(c);
            found = (int)b->cls.size() - 1;
        }
        cls_of[i] = found;
        b->cls[found].kx = std::max(b->cls[found].kx, P[i].kmax[0]);
        b->cls[found].count += 1;
    }
    // ---- caller-order offsets
    b->inst.assign(n, BInst{});
    b->pt_first.assign(n + 1, 0);
    b->tile_first.assign(n + 1, 0);
    b->mblk_first.assign(n + 1, 0);
    int64_t bo = 0, reo = 0, ipo = 0;
    int tmax[3] = {1, 1, 1};
    for (int i = 0; i < n; ++i) {
        BInst &I = b->inst[i];
        const Params &p = P[i];
        const int64_t nt = (int64_t)p.nb[0] * p.nb[1] * p.nb[2];
        const int64_t nrep = (int64_t)F[i].s0.size();
        b->pt_first[i + 1] = b->pt_first[i] + n_points[i];
        b->tile_first[i + 1] = b->tile_first[i] + nt;
        b->mblk_first[i + 1] =
            b->mblk_first[i] + std::max<int64_t>(1, std::min<int64_t>((nrep + 1023) / 1024, 64));
        I.po = b->pt_first[i];
        I.bo = bo;
        I.reo = reo;
        for (int a = 0; a < 3; ++a) {
            I.ipo[a] = ipo;
            if (a < dim) ipo += p.kmax[a] + 1;
            tmax[a] = std::max(tmax[a], p.tmax[a]);
        }
        bo += nt * (dim == 3 ? 27 : 9);
        reo += nrep;
        I.loss_const = F[i].loss_const;
    }
    b->n_points = b->pt_first[n];
    b->n_bins = bo;
    b->n_rep = reo;
    if (b->n_points > 2147483647LL || b->n_bins > 2147483647LL) return FRESCO_ERR_UNSUPPORTED;
    // ---- class-order offsets (grids and spectra of a class are contiguous)
    int64_t go = 0, ato = 0, hco = 0, ro = 0, two = 0;
    for (size_t c = 0; c < b->cls.size(); ++c) {
        auto &K = b->cls[c];
        K.go0 = go; K.ato0 = ato; K.hco0 = hco; K.ro0 = ro; K.two0 = two;
        const int64_t plane = K.nf[1], cells = (int64_t)K.nf[0] * K.nf[1];
        two += K.nf[0] / 4 + 1;
        for (int i = 0; i < n; ++i) {
            if (cls_of[i] != (int)c) continue;
            BInst &I = b->inst[i];
            I.go = go; I.ato = ato; I.hco = hco; I.ro = ro;
            go += cells;
            ato += plane * (K.kx + 1);
            // kderiv: scalar half spectrum [kx+1][plane], merged and transformed in the grid's
            // place; direct: [2kx+2][plane] and full complex rows
            hco += plane * (b->kderiv ? (int64_t)K.kx + 1 : 2 * (int64_t)K.kx + 2);
            ro += b->kderiv ? 0 : cells;
        }
    }
    b->n_r = ro;
    b->cells = go;
    b->n_specT = ato;
    b->n_tw = two;
    b->n_hc = hco;
    // ---- per-instance geometry (one spread list size for all: the largest any instance needs)
    int cap_max = 1024;
    for (int i = 0; i < n; ++i) cap_max = std::max(cap_max, P[i].list_cap);
    std::vector<double> ip_h((size_t)std::max<int64_t>(ipo, 1));
    for (int i = 0; i < n; ++i) {
        BInst &I = b->inst[i];
        const Params &p = P[i];
        const auto &K = b->cls[cls_of[i]];
        Geom &g = I.g;
        g.dim = dim;
        for (int a = 0; a < 3; ++a) {
            g.nf[a] = p.nf[a];
            g.nb[a] = p.nb[a];
            g.tmax[a] = p.tmax[a];
            g.tq[a] = p.nf[a] / p.nb[a];
            g.tr[a] = p.nf[a] % p.nb[a];
            g.tinv[a] = (float)p.nb[a] / (float)p.nf[a];
            const double L = a < dim ? boxes[(size_t)i * dim + a] : 1.0;
            double sc = a < dim ? (double)p.nf[a] / L : 0.0;
            double shi = (double)(T)sc;
            long double slo = (long double)p.nf[a] / (long double)L - (long double)shi;
            g.s_hi[a] = shi;
            g.s_lo[a] = a < dim ? (double)(T)(double)slo : 0.0;
            I.m.nf[a] = p.nf[a];
            I.m.kscale[a] = a < dim ? 2.0 * kPi / L : 0.0;
        }
        g.n_tiles = (int64_t)p.nb[0] * p.nb[1] * p.nb[2];
        g.list_cap = cap_max;
        g.sub = dim == 3 ? 27 : 9;
        for (int a = 0; a < 3; ++a) g.strips[a] = a < dim && p.nf[a] / p.nb[a] >= p.width ? 1 : 0;
        g.n_bins = g.n_tiles * g.sub;
        g.n_points = n_points[i];
        g.width = p.width;
        g.beta = p.beta;
        set_tile_divisors(g);
        I.m.dim = dim;
        I.m.kx = K.kx;
        I.m.n_rep = (int64_t)F[i].s0.size();
        I.m.half_row = p.nf[0] / 2 + 1;
        I.m.hc_row = b->kderiv ? (int64_t)K.kx + 1 : 2 * (int64_t)K.kx + 2;
        I.m.kderiv = b->kderiv;
        I.m.plane = (int64_t)p.nf[1] * p.nf[2];
        I.m.inv_n = 1.0 / (double)n_points[i];
        for (int a = 0; a < dim; ++a) {
            std::vector<double> ft(p.kmax[a] + 1);
            kernel_ft(p.width, p.beta, p.nf[a], (int64_t)ft.size(), ft.data());
            for (size_t k = 0; k < ft.size(); ++k) ip_h[I.ipo[a] + k] = 1.0 / ft[k];
        }
    }
    es_poly<float>(P[0].width, P[0].beta, b->poly32);
    es_poly<double>(P[0].width, P[0].beta, b->poly64);
    // ---- device buffers
    const size_t N = (size_t)b->n_points;
    const int rw = sizeof(T) == 4 ? 4 : (dim == 3 ? 4 : 2);
    bool ok = balloc(b, (void **)&b->d_inst, sizeof(BInst) * n) &&
              balloc(b, (void **)&b->d_pt_first, sizeof(int64_t) * (n + 1)) &&
              balloc(b, (void **)&b->d_tile_first, sizeof(int64_t) * (n + 1)) &&
              balloc(b, (void **)&b->d_mblk_first, sizeof(int64_t) * (n + 1)) &&
              balloc(b, &b->sorted, sizeof(T) * N * rw) &&
              (sizeof(T) == 4 || balloc(b, (void **)&b->perm, sizeof(int) * N)) &&
              balloc(b, (void **)&b->key, sizeof(int) * N) &&
              balloc(b, (void **)&b->slot, sizeof(int) * N) &&
              balloc(b, (void **)&b->cnt, sizeof(int) * b->n_bins) &&
              balloc(b, (void **)&b->off, sizeof(int) * (b->n_bins + 1)) &&
              balloc(b, (void **)&b->bsum, sizeof(int) * ((b->n_bins + 1023) / 1024 + 1)) &&
              balloc(b, (void **)&b->err, sizeof(int)) &&
              balloc(b, &b->grid, sizeof(T) * b->cells) &&
              balloc(b, &b->tw, sizeof(C2) * b->n_tw) &&
              balloc(b, &b->specT, sizeof(C2) * b->n_specT) &&
              balloc(b, &b->hc, sizeof(C2) * b->n_hc) && balloc(b, &b->bt, sizeof(C2) * b->n_hc) &&
              (b->kderiv || balloc(b, &b->r, sizeof(C2) * b->n_r)) &&
              (b->kderiv || balloc(b, &b->g, sizeof(C2) * b->cells)) &&
              balloc(b, (void **)&b->rep_n, sizeof(int) * b->n_rep * dim) &&
              balloc(b, &b->rep_s0, sizeof(T) * b->n_rep) &&
              balloc(b, &b->rep_w, sizeof(T) * b->n_rep) &&
              balloc(b, &b->ip, sizeof(T) * ip_h.size()) &&
              balloc(b, (void **)&b->partial, sizeof(double) * b->mblk_first[n]);
    if (!ok) return FRESCO_ERR_OOM;
    {
        std::vector<int32_t> rn;
        std::vector<T> s0, w;
        rn.reserve((size_t)b->n_rep * dim);
        s0.reserve((size_t)b->n_rep);
        w.reserve((size_t)b->n_rep);
        for (int i = 0; i < n; ++i) {
            rn.insert(rn.end(), F[i].n.begin(), F[i].n.end());
            for (size_t k = 0; k < F[i].s0.size(); ++k) {
                s0.push_back((T)F[i].s0[k]);
                w.push_back((T)F[i].w[k]);
            }
        }
        std::vector<T> ipt(ip_h.size());
        for (size_t k = 0; k < ip_h.size(); ++k) ipt[k] = (T)ip_h[k];
        FR_CUDA(cudaMemcpy(b->rep_n, rn.data(), sizeof(int) * rn.size(), cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(b->rep_s0, s0.data(), sizeof(T) * s0.size(), cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(b->rep_w, w.data(), sizeof(T) * w.size(), cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(b->ip, ipt.data(), sizeof(T) * ipt.size(), cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(b->d_pt_first, b->pt_first.data(), sizeof(int64_t) * (n + 1),
                           cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(b->d_tile_first, b->tile_first.data(), sizeof(int64_t) * (n + 1),
                           cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(b->d_mblk_first, b->mblk_first.data(), sizeof(int64_t) * (n + 1),
                           cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemset(b->hc, 0, sizeof(C2) * b->n_hc));
        if (b->r) FR_CUDA(cudaMemset(b->r, 0, sizeof(C2) * b->n_r));
        std::vector<C2> tw((size_t)b->n_tw);
        for (auto &K : b->cls)
            for (int k = 0; k <= K.nf[0] / 4; ++k) {
                const double a = 2.0 * M_PI * (double)k / (double)K.nf[0];
                tw[(size_t)(K.two0 + k)].x = (T)std::cos(a);
                tw[(size_t)(K.two0 + k)].y = (T)-std::sin(a);
            }
        FR_CUDA(cudaMemcpy(b->tw, tw.data(), sizeof(C2) * tw.size(), cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemset(b->err, 0, sizeof(int)));
    }
    BTables &t = b->tab;
    t.inst = b->d_inst;
    t.pt_first = b->d_pt_first;
    t.tile_first = b->d_tile_first;
    t.mblk_first = b->d_mblk_first;
    t.n_inst = n;
    t.dim = dim;
    t.width = P[0].width;
    t.list_cap = cap_max;
    t.n_points = b->n_points;
    t.n_tiles = b->tile_first[n];
    t.n_mblk = b->mblk_first[n];
    for (int a = 0; a < 3; ++a) t.tmax[a] = tmax[a];
    {   // shared memory of the ensemble kernels must fit every instance's tiles
        int dev = 0, optin = 0;
        FR_CUDA(cudaGetDevice(&dev));
        FR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        Geom tg{};
        tg.dim = dim;
        tg.width = t.width;
        tg.list_cap = cap_max;
        for (int a = 0; a < 3; ++a) tg.tmax[a] = tmax[a];
        const int interp_bytes =
            b->kderiv ? Launch<T>::interp_kd_smem(tg) : Launch<T>::interp_smem(tg);
        if (Launch<T>::spread_smem(tg) > optin || interp_bytes > optin)
            return FRESCO_ERR_UNSUPPORTED;
    }
    // ---- cuFFT plans per class (all transforms of a class in one batch)
    size_t wmax = 0;
    for (auto &K : b->cls) {
        size_t ws = 0;
        for (int i = 0; i < 4; ++i) {
            FR_CUFFT(cufftCreate(&K.h[i]));
            K.have[i] = true;
            FR_CUFFT(cufftSetAutoAllocation(K.h[i], 0));
        }
        // the real rows of length n0 run as complex rows of length n0 / 2, in place
        long long n0 = K.nf[0], n1 = K.nf[1], mh = K.nf[0] / 2, cnt = K.count;
        FR_CUFFT(cufftMakePlanMany64(K.h[0], 1, &mh, nullptr, 1, mh, nullptr, 1, mh,
                                     c2c_type<T>(), cnt * n1, &ws));
        wmax = std::max(wmax, ws);
        FR_CUFFT(cufftMakePlanMany64(K.h[1], 1, &n1, nullptr, 1, n1, nullptr, 1, n1, c2c_type<T>(),
                                     cnt * (K.kx + 1), &ws));
        wmax = std::max(wmax, ws);
        FR_CUFFT(cufftMakePlanMany64(K.h[2], 1, &n1, nullptr, 1, n1, nullptr, 1, n1, c2c_type<T>(),
                                     cnt * (b->kderiv ? (long long)K.kx + 1
                                                      : 2 * (long long)K.kx + 2), &ws));
        wmax = std::max(wmax, ws);
        if (b->kderiv)
            FR_CUFFT(cufftMakePlanMany64(K.h[3], 1, &mh, nullptr, 1, mh, nullptr, 1, mh,
                                         c2c_type<T>(), cnt * n1, &ws));
        else
            FR_CUFFT(cufftMakePlanMany64(K.h[3], 1, &n0, nullptr, 1, n0, nullptr, 1, n0,
                                         c2c_type<T>(), cnt * n1, &ws));
        wmax = std::max(wmax, ws);
    }
    if (!balloc(b, &b->work, wmax)) return FRESCO_ERR_OOM;
    for (auto &K : b->cls)
        for (int i = 0; i < 4; ++i) {
            FR_CUFFT(cufftSetWorkArea(K.h[i], b->work));
            FR_CUFFT(cufftSetStream(K.h[i], b->stream));
        }
    FR_CUDA(cudaDeviceSynchronize());
    return FRESCO_OK;
}

template <typename T>
const EsPoly<T> &bpoly(const fresco_batch_s *b);
template <>
const EsPoly<float> &bpoly<float>(const fresco_batch_s *b) { return b->poly32; }
template <>
const EsPoly<double> &bpoly<double>(const fresco_batch_s *b) { return b->poly64; }

template <typename T>
fresco_status batch_eval(fresco_batch_s *b, const T *pts, double *losses, T *grad) {
    using C2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    cudaStream_t s = b->stream;
    const BTables &t = b->tab;
    {
        StageScope sc(b->prof, s, ST_SORT);
        FR_CUDA(cudaMemsetAsync(b->cnt, 0, sizeof(int) * (size_t)b->n_bins, s));
        FR_CUDA(Launch<T>::bin_b(t, pts, b->cnt, b->key, b->slot, b->err, s));
        int nl = 0;
        FR_CUDA(Launch<T>::scan(b->cnt, b->off, b->bsum, b->n_bins, s, &nl));
        FR_CUDA(Launch<T>::scatter_b(t, pts, b->key, b->slot, b->off, b->sorted, b->perm, s));
        b->launches += 2 + nl;
    }
    {
        StageScope sc(b->prof, s, ST_SPREAD);
        FR_CUDA(Launch<T>::spread_b(t, bpoly<T>(b), b->sorted, b->off, (T *)b->grid, s));
        b->launches += 1;
    }
    {
        StageScope sc(b->prof, s, ST_FFT_FWD);
        for (auto &K : b->cls) {   // forward FFT of each size class
            const int64_t plane = K.nf[1];
            const int mh = K.nf[0] / 2;
            C2 *A = (C2 *)((T *)b->grid + K.go0), *AT = (C2 *)b->specT + K.ato0;
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(K.h[0], (cufftComplex *)A, (cufftComplex *)A,
                                      CUFFT_FORWARD));
            else
                FR_CUFFT(cufftExecZ2Z(K.h[0], (cufftDoubleComplex *)A, (cufftDoubleComplex *)A,
                                      CUFFT_FORWARD));
            FR_CUDA(Launch<T>::rfft_split(A, AT, (C2 *)b->tw + K.two0, plane, mh, K.kx, s,
                                          K.count, plane * mh, plane * (K.kx + 1)));
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(K.h[1], (cufftComplex *)AT, (cufftComplex *)AT,
                                      CUFFT_FORWARD));
            else
                FR_CUFFT(cufftExecZ2Z(K.h[1], (cufftDoubleComplex *)AT, (cufftDoubleComplex *)AT,
                                      CUFFT_FORWARD));
            b->launches += 1;
        }
    }
    {
        StageScope sc(b->prof, s, ST_MASK);
        FR_CUDA(Launch<T>::mask_b(t, b->rep_n, (const T *)b->rep_s0, (const T *)b->rep_w,
                                  b->specT, (const T *)b->ip, b->hc, nullptr, b->partial, s));
        b->launches += 1;
    }
    {
        StageScope sc(b->prof, s, ST_LOSS);
        FR_CUDA(Launch<T>::finalize_b(t, b->partial, losses, s));
        b->launches += 1;
    }
    if (!grad) return FRESCO_OK;
    if (b->kderiv) {
        {
            StageScope sc(b->prof, s, ST_FFT_INV);
            for (auto &K : b->cls) {   // scalar spectrum -> real field (in the spread grid's place)
                const int64_t plane = K.nf[1];
                const int mh = K.nf[0] / 2;
                C2 *H = (C2 *)b->hc + K.hco0, *BT = (C2 *)b->bt + K.hco0;
                C2 *Z = (C2 *)((T *)b->grid + K.go0);
                if (sizeof(T) == 4)
                    FR_CUFFT(cufftExecC2C(K.h[2], (cufftComplex *)H, (cufftComplex *)BT,
                                          CUFFT_INVERSE));
                else
                    FR_CUFFT(cufftExecZ2Z(K.h[2], (cufftDoubleComplex *)H,
                                          (cufftDoubleComplex *)BT, CUFFT_INVERSE));
                FR_CUDA(Launch<T>::rfft_merge(BT, Z, (C2 *)b->tw + K.two0, plane, mh, K.kx, s,
                                              K.count, plane * ((int64_t)K.kx + 1), plane * mh));
                if (sizeof(T) == 4)
                    FR_CUFFT(cufftExecC2C(K.h[3], (cufftComplex *)Z, (cufftComplex *)Z,
                                          CUFFT_INVERSE));
                else
                    FR_CUFFT(cufftExecZ2Z(K.h[3], (cufftDoubleComplex *)Z,
                                          (cufftDoubleComplex *)Z, CUFFT_INVERSE));
                b->launches += 1;
            }
        }
        StageScope sc(b->prof, s, ST_INTERP);
        FR_CUDA(Launch<T>::interp_kd_b(t, bpoly<T>(b), b->sorted, b->perm, b->off,
                                       (const T *)b->grid, nullptr, grad, s));
        b->launches += 1;
        return FRESCO_OK;
    }
    {
        StageScope sc(b->prof, s, ST_FFT_INV);
        for (auto &K : b->cls) {   // inverse FFT of each size class
            const int64_t plane = K.nf[1];
            C2 *H = (C2 *)b->hc + K.hco0, *BT = (C2 *)b->bt + K.hco0, *R = (C2 *)b->r + K.ro0;
            C2 *G = (C2 *)b->g + K.ro0;
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(K.h[2], (cufftComplex *)H, (cufftComplex *)BT,
                                      CUFFT_INVERSE));
            else
                FR_CUFFT(cufftExecZ2Z(K.h[2], (cufftDoubleComplex *)H, (cufftDoubleComplex *)BT,
                                      CUFFT_INVERSE));
            FR_CUDA(Launch<T>::rows_to_cols(BT, R, plane, K.nf[0], K.kx, s, K.count,
                                            plane * (2 * (int64_t)K.kx + 2),
                                            (int64_t)K.nf[0] * plane));
            if (sizeof(T) == 4)
                FR_CUFFT(cufftExecC2C(K.h[3], (cufftComplex *)R, (cufftComplex *)G,
                                      CUFFT_INVERSE));
            else
                FR_CUFFT(cufftExecZ2Z(K.h[3], (cufftDoubleComplex *)R, (cufftDoubleComplex *)G,
                                      CUFFT_INVERSE));
            b->launches += 1;
        }
    }
    {
        StageScope sc(b->prof, s, ST_INTERP);
        FR_CUDA(Launch<T>::interp_b(t, bpoly<T>(b), b->sorted, b->perm, b->off, b->g, nullptr,
                                    nullptr, grad, s));
        b->launches += 1;
    }
    return FRESCO_OK;
}

}  // namespace

extern "C" {

fresco_status fresco_batch_plan(fresco_batch_t *out, int dim, int n_inst, const double *boxes,
                                const int64_t *n_points, const int64_t *n_modes,
                                const int32_t *masks, const double *S0, const double *W,
                                const fresco_opts *opts, void *stream) {
    if (!out) return FRESCO_ERR_ARG;
    *out = nullptr;
    if (dim != 2 && dim != 3) return FRESCO_ERR_ARG;
    if (dim != 2) return FRESCO_ERR_UNSUPPORTED;
    if (n_inst < 1 || !boxes || !n_points || !n_modes || !masks || !S0 || !W)
        return FRESCO_ERR_ARG;
    std::vector<Params> P(n_inst);
    std::vector<Folded> F(n_inst);
    int64_t m0 = 0;
    fresco_opts o;
    fresco_opts_default(&o);
    if (opts) o = *opts;
    for (int i = 0; i < n_inst; ++i) {
        if (n_modes[i] < 1) return FRESCO_ERR_ARG;
        // one kernel serves every instance: the width rule at the requested oversampling
        fresco_status st = check_and_params(dim, boxes + (size_t)i * dim, n_points[i],
                                            masks + m0 * dim, n_modes[i], S0 + m0, W + m0, &o,
                                            P[i], false, false);
        if (st) return st;
        if (i > 0 && P[i].width != P[0].width) return FRESCO_ERR_UNSUPPORTED;
        for (int a = 0; a < dim; ++a) P[i].nf[a] = class_size(P[i].nf[a]);
        if ((st = choose_tiling(P[i], o.tile))) return st;
        if ((st = fold_mask(P[i], masks + m0 * dim, n_modes[i], S0 + m0, W + m0, F[i]))) return st;
        if (F[i].s0.empty()) return FRESCO_ERR_ARG;
        m0 += n_modes[i];
    }
    fresco_batch_s *b = new (std::nothrow) fresco_batch_s();
    if (!b) return FRESCO_ERR_OOM;
    b->dim = dim;
    b->precision = o.precision;
    b->kderiv = o.grad_mode == FRESCO_GRAD_KDERIV ? 1 : 0;
    b->esize = o.precision == FRESCO_F64 ? 8 : 4;
    b->n_inst = n_inst;
    b->stream = (cudaStream_t)stream;
    b->boxes.assign(boxes, boxes + (size_t)n_inst * dim);
    b->infos.resize(n_inst);
    for (int i = 0; i < n_inst; ++i) fill_info(P[i], n_points[i], n_modes[i], F[i], &b->infos[i]);
    fresco_status st = o.precision == FRESCO_F64 ? batch_build<double>(b, P, F, boxes, n_points)
                                                 : batch_build<float>(b, P, F, boxes, n_points);
    if (st) {
        batch_free(b);
        return st;
    }
    *out = b;
    return FRESCO_OK;
}

fresco_status fresco_batch_loss_grad(fresco_batch_t b, const void *d_points, double *d_losses,
                                     void *d_grad) {
    fresco::clear_pending_error();
    if (!b || !d_points || !d_losses) return FRESCO_ERR_ARG;
    if (b->precision == FRESCO_F64)
        return batch_eval<double>(b, (const double *)d_points, d_losses, (double *)d_grad);
    return batch_eval<float>(b, (const float *)d_points, d_losses, (float *)d_grad);
}

fresco_status fresco_batch_graph_capture(fresco_batch_t b, const void *d_points, double *d_losses,
                                         void *d_grad) {
    fresco::clear_pending_error();
    if (!b || !d_points || !d_losses || !b->stream) return FRESCO_ERR_ARG;
    // one ordinary evaluation first (sets kernel attributes, warms the cuFFT plans)
    fresco_status st = fresco_batch_loss_grad(b, d_points, d_losses, d_grad);
    if (st) return st;
    FR_CUDA(cudaStreamSynchronize(b->stream));
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    const bool prof_on = b->prof.on;   // no event records inside the graph
    b->prof.on = false;
    FR_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    st = fresco_batch_loss_grad(b, d_points, d_losses, d_grad);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    b->prof.on = prof_on;
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    FR_CUDA(e);
    b->graph = graph;
    FR_CUDA(cudaGraphInstantiate(&b->gexec, graph, 0));
    return FRESCO_OK;
}

fresco_status fresco_batch_graph_launch(fresco_batch_t b) {
    fresco::clear_pending_error();
    if (!b || !b->gexec) return FRESCO_ERR_ARG;
    FR_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    return FRESCO_OK;
}

fresco_status fresco_batch_info(fresco_batch_t b, int64_t *total_points, int *n_classes,
                                int64_t *device_bytes, int64_t *launches) {
    if (!b) return FRESCO_ERR_ARG;
    if (total_points) *total_points = b->n_points;
    if (n_classes) *n_classes = (int)b->cls.size();
    if (device_bytes) *device_bytes = b->device_bytes;
    if (launches) *launches = b->launches;
    return FRESCO_OK;
}

fresco_status fresco_batch_get_info(fresco_batch_t b, int i, fresco_info *info) {
    if (!b || !info || i < 0 || i >= b->n_inst) return FRESCO_ERR_ARG;
    *info = b->infos[i];
    return FRESCO_OK;
}

fresco_status fresco_batch_status_check(fresco_batch_t b) {
    if (!b) return FRESCO_ERR_ARG;
    FR_CUDA(b->stream ? cudaStreamSynchronize(b->stream) : cudaDeviceSynchronize());
    int err = 0;
    FR_CUDA(cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        int zero = 0;
        FR_CUDA(cudaMemcpy(b->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return FRESCO_ERR_NONFINITE;
    }
    return cuda_status(cudaGetLastError());
}

fresco_status fresco_batch_profile(fresco_batch_t b, int enable) {
    if (!b) return FRESCO_ERR_ARG;
    b->prof.on = enable != 0;
    return FRESCO_OK;
}

fresco_status fresco_batch_profile_read(fresco_batch_t b, double *ms, int64_t *counts) {
    if (!b || !ms) return FRESCO_ERR_ARG;
    FR_CUDA(b->stream ? cudaStreamSynchronize(b->stream) : cudaDeviceSynchronize());
    b->prof.read(ms, counts);
    return FRESCO_OK;
}

fresco_status fresco_batch_destroy(fresco_batch_t b) {
    batch_free(b);
    return FRESCO_OK;
}

}  // extern "C"

// ============================================================================================
// Weights on a uniform grid with uniform k constraints (UwU, Methods "Analytical gradients"):
// real weights c_m at the cells r_m = m L / M of a periodic grid,
//   rho(n) = sum_m c_m e^{-2 pi i n.m/M} (one forward FFT), rho0 = sum_m c_m^2,
//   S = |rho|^2 / rho0, L = sum_mask W (S - S0)^2,
//   dL/dc_m = Re sum_mask [4 W (S - S0) rho / rho0] e^{+2 pi i n.m/M}
//             - (4 c_m / rho0) sum_mask W S (S - S0).
// The first gradient term is one real inverse FFT of a Hermitian half spectrum (the layout of the
// kernel-derivative mode), the second a scalar times c. No NUFFT is involved: the grid is the
// field. The mask folds onto half-space representatives as for points (S(n) = S(-n) for real
// weights); both sums above fold the same way because only their real parts enter.
// ============================================================================================

namespace {

constexpr int kUwuBlocks = 1024;

__device__ __forceinline__ double uwu_block_sum(double v) {
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
__global__ void __launch_bounds__(256) k_uwu_sumsq(const T *__restrict__ c, int64_t n,
                                                   double *__restrict__ part) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc = fma((double)c[i], (double)c[i], acc);
    const double b = uwu_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// out[k] = sum of part[k * nb .. (k + 1) * nb) (+ add[k]) for k < n_out; fixed order
__global__ void __launch_bounds__(256) k_uwu_sum(const double *__restrict__ part, int nb,
                                                 int n_out, double add0, double *__restrict__ out) {
    for (int k = 0; k < n_out; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[(int64_t)k * nb + i];
        const double s = uwu_block_sum(v);
        if (threadIdx.x == 0) out[k] = s + (k == 0 ? add0 : 0.0);
        __syncthreads();
    }
}

// One pass over the folded representatives (n_x-major): S, the loss and F partials, and the
// Hermitian half spectrum (E/2) rho at n (and its conjugate at -n on the n_x = 0 column),
// E = 4 W' (S - S0') / rho0.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_uwu_mask(
    int64_t n_rep, const int *__restrict__ rep_n, const T *__restrict__ rep_s0,
    const T *__restrict__ rep_w, const typename std::conditional<sizeof(T) == 4, float2, double2>::type *__restrict__ spec,
    int nf1, int nf2, int64_t plane, const double *__restrict__ rho0p,
    typename std::conditional<sizeof(T) == 4, float2, double2>::type *__restrict__ hs,
    double *__restrict__ part) {
    using C = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const double rho0 = *rho0p;
    const T inv = (T)(1.0 / rho0);
    double lsum = 0.0, fsum = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_rep;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int nx = rep_n[e * D + 0], ny = rep_n[e * D + 1], nz = D == 3 ? rep_n[e * D + 2] : 0;
        const int ry = ny < 0 ? ny + nf1 : ny, rz = nz < 0 ? nz + nf2 : nz;
        const int64_t row = (int64_t)rz * nf1 + ry;
        const C F = spec[(int64_t)nx * plane + row];
        const T S = (F.x * F.x + F.y * F.y) * inv;
        const double d = (double)S - (double)rep_s0[e];
        const double wgt = (double)rep_w[e];
        lsum = fma(wgt * d, d, lsum);
        fsum = fma(wgt * (double)S, d, fsum);
        const T h = (T)(2.0 * wgt * d / rho0);   // E / 2
        hs[(int64_t)nx * plane + row] = C{h * F.x, h * F.y};
        if (nx == 0) {
            const int my = ny > 0 ? nf1 - ny : -ny, mz = nz > 0 ? nf2 - nz : -nz;
            hs[(int64_t)mz * nf1 + my] = C{h * F.x, -h * F.y};
        }
    }
    const double bl = uwu_block_sum(lsum);
    const double bf = uwu_block_sum(fsum);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bl;
        part[gridDim.x + blockIdx.x] = bf;
    }
}

// grad_m = h_m - (4 c_m / rho0) * fsum
template <typename T>
__global__ void __launch_bounds__(256) k_uwu_grad(const T *__restrict__ h, const T *__restrict__ c,
                                                  int64_t n, const double *__restrict__ scal,
                                                  const double *__restrict__ fsum,
                                                  T *__restrict__ grad) {
    const T coef = (T)(4.0 * (*fsum) / scal[0]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        grad[i] = h[i] - coef * c[i];
}

}  // namespace

struct fresco_uwu_s {
    int dim = 0, precision = FRESCO_F32;
    size_t esize = 4;
    int M[3] = {1, 1, 1};
    int kx = 0;
    int64_t cells = 0, plane = 0, half = 0, n_rep = 0, n_mask_blocks = 0;
    double loss_const = 0.0;
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    int *rep_n = nullptr;
    void *rep_s0 = nullptr, *rep_w = nullptr;
    void *spec = nullptr, *specT = nullptr, *hs = nullptr, *bt = nullptr, *r = nullptr, *h = nullptr;
    double *part = nullptr, *scal = nullptr;   // scal[0] = rho0, scal[1] = F sum
    void *work = nullptr;
    cufftHandle fft[4] = {0, 0, 0, 0};        // rows R2C, cols fwd, cols inv, rows C2R
    bool have[4] = {false, false, false, false};
};

namespace {

bool ualloc(fresco_uwu_s *u, void **p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    u->allocs.push_back(*p);
    return true;
}

void uwu_free(fresco_uwu_s *u) {
    if (!u) return;
    if (u->stream) cudaStreamSynchronize(u->stream);
    else cudaDeviceSynchronize();
    for (int i = 0; i < 4; ++i)
        if (u->have[i]) cufftDestroy(u->fft[i]);
    for (void *p : u->allocs) cudaFree(p);
    delete u;
}

template <typename T>
fresco_status uwu_build(fresco_uwu_s *u, const Folded &F) {
    using C2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const int dim = u->dim;
    u->plane = (int64_t)u->M[1] * u->M[2];
    u->half = u->M[0] / 2 + 1;
    u->cells = u->plane * u->M[0];
    u->n_rep = (int64_t)F.s0.size();
    u->n_mask_blocks = std::max<int64_t>(1, std::min<int64_t>((u->n_rep + 255) / 256, kUwuBlocks));
    const size_t specT_n = (size_t)(u->kx + 1) * (size_t)u->plane;
    bool ok = ualloc(u, (void **)&u->rep_n, sizeof(int) * F.n.size()) &&
              ualloc(u, &u->rep_s0, sizeof(T) * (size_t)u->n_rep) &&
              ualloc(u, &u->rep_w, sizeof(T) * (size_t)u->n_rep) &&
              ualloc(u, &u->spec, sizeof(C2) * (size_t)(u->plane * u->half)) &&
              ualloc(u, &u->specT, sizeof(C2) * specT_n) && ualloc(u, &u->hs, sizeof(C2) * specT_n) &&
              ualloc(u, &u->bt, sizeof(C2) * specT_n) &&
              ualloc(u, &u->r, sizeof(C2) * (size_t)(u->plane * u->half)) &&
              ualloc(u, &u->h, sizeof(T) * (size_t)u->cells) &&
              ualloc(u, (void **)&u->part, sizeof(double) * (size_t)std::max<int64_t>(2 * u->n_mask_blocks, kUwuBlocks)) &&
              ualloc(u, (void **)&u->scal, sizeof(double) * 4);
    if (!ok) return FRESCO_ERR_OOM;
    std::vector<T> s0(F.s0.size()), w(F.w.size());
    for (size_t i = 0; i < s0.size(); ++i) {
        s0[i] = (T)F.s0[i];
        w[i] = (T)F.w[i];
    }
    FR_CUDA(cudaMemcpy(u->rep_n, F.n.data(), sizeof(int) * F.n.size(), cudaMemcpyHostToDevice));
    FR_CUDA(cudaMemcpy(u->rep_s0, s0.data(), sizeof(T) * s0.size(), cudaMemcpyHostToDevice));
    FR_CUDA(cudaMemcpy(u->rep_w, w.data(), sizeof(T) * w.size(), cudaMemcpyHostToDevice));
    // entries outside the mask stay zero from here on
    FR_CUDA(cudaMemset(u->hs, 0, sizeof(C2) * specT_n));
    FR_CUDA(cudaMemset(u->r, 0, sizeof(C2) * (size_t)(u->plane * u->half)));
    // cuFFT: rows R2C, (z,)y columns forward over n_x = 0..kx, the same inverse, rows C2R
    long long n0 = u->M[0], half = u->half, rows = u->plane, cn[2];
    const int crank = dim - 1;
    if (dim == 2) cn[0] = u->M[1];
    else { cn[0] = u->M[2]; cn[1] = u->M[1]; }
    size_t ws[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) {
        FR_CUFFT(cufftCreate(&u->fft[i]));
        u->have[i] = true;
        FR_CUFFT(cufftSetAutoAllocation(u->fft[i], 0));
    }
    FR_CUFFT(cufftMakePlanMany64(u->fft[0], 1, &n0, nullptr, 1, n0, nullptr, 1, half,
                                 r2c_type<T>(), rows, &ws[0]));
    FR_CUFFT(cufftMakePlanMany64(u->fft[1], crank, cn, nullptr, 1, rows, nullptr, 1, rows,
                                 c2c_type<T>(), u->kx + 1, &ws[1]));
    FR_CUFFT(cufftMakePlanMany64(u->fft[2], crank, cn, nullptr, 1, rows, nullptr, 1, rows,
                                 c2c_type<T>(), u->kx + 1, &ws[2]));
    FR_CUFFT(cufftMakePlanMany64(u->fft[3], 1, &n0, nullptr, 1, half, nullptr, 1, n0,
                                 c2r_type<T>(), rows, &ws[3]));
    const size_t wmax = std::max(std::max(ws[0], ws[1]), std::max(ws[2], ws[3]));
    if (!ualloc(u, &u->work, wmax)) return FRESCO_ERR_OOM;
    for (int i = 0; i < 4; ++i) {
        FR_CUFFT(cufftSetWorkArea(u->fft[i], u->work));
        FR_CUFFT(cufftSetStream(u->fft[i], u->stream));
    }
    FR_CUDA(cudaDeviceSynchronize());
    return FRESCO_OK;
}

template <typename T>
fresco_status uwu_eval(fresco_uwu_s *u, const T *c, double *loss, T *grad) {
    using C2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    cudaStream_t s = u->stream;
    // rho0 = sum c^2
    k_uwu_sumsq<T><<<kUwuBlocks, 256, 0, s>>>(c, u->cells, u->part);
    k_uwu_sum<<<1, 256, 0, s>>>(u->part, kUwuBlocks, 1, 0.0, u->scal);
    // forward transform, columns n_x = 0..kx transposed
    if (sizeof(T) == 4)
        FR_CUFFT(cufftExecR2C(u->fft[0], (cufftReal *)c, (cufftComplex *)u->spec));
    else
        FR_CUFFT(cufftExecD2Z(u->fft[0], (cufftDoubleReal *)c, (cufftDoubleComplex *)u->spec));
    FR_CUDA(Launch<T>::cols_to_rows(u->spec, u->specT, u->plane, u->half, u->kx + 1, s));
    if (sizeof(T) == 4)
        FR_CUFFT(cufftExecC2C(u->fft[1], (cufftComplex *)u->specT, (cufftComplex *)u->specT,
                              CUFFT_FORWARD));
    else
        FR_CUFFT(cufftExecZ2Z(u->fft[1], (cufftDoubleComplex *)u->specT,
                              (cufftDoubleComplex *)u->specT, CUFFT_FORWARD));
    // S, loss and F partials, Hermitian half spectrum of the gradient field
    const unsigned nb = (unsigned)u->n_mask_blocks;
    if (u->dim == 2)
        k_uwu_mask<T, 2><<<nb, 256, 0, s>>>(u->n_rep, u->rep_n, (const T *)u->rep_s0,
                                            (const T *)u->rep_w, (const C2 *)u->specT, u->M[1],
                                            u->M[2], u->plane, u->scal, (C2 *)u->hs, u->part);
    else
        k_uwu_mask<T, 3><<<nb, 256, 0, s>>>(u->n_rep, u->rep_n, (const T *)u->rep_s0,
                                            (const T *)u->rep_w, (const C2 *)u->specT, u->M[1],
                                            u->M[2], u->plane, u->scal, (C2 *)u->hs, u->part);
    k_uwu_sum<<<1, 256, 0, s>>>(u->part, (int)nb, 2, u->loss_const, u->scal + 2);
    FR_CUDA(cudaMemcpyAsync(loss, u->scal + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (!grad) return cuda_status(cudaGetLastError());
    if (sizeof(T) == 4)
        FR_CUFFT(cufftExecC2C(u->fft[2], (cufftComplex *)u->hs, (cufftComplex *)u->bt,
                              CUFFT_INVERSE));
    else
        FR_CUFFT(cufftExecZ2Z(u->fft[2], (cufftDoubleComplex *)u->hs, (cufftDoubleComplex *)u->bt,
                              CUFFT_INVERSE));
    FR_CUDA(Launch<T>::rows_to_half(u->bt, u->r, u->plane, u->half, u->kx, s));
    if (sizeof(T) == 4)
        FR_CUFFT(cufftExecC2R(u->fft[3], (cufftComplex *)u->r, (cufftReal *)u->h));
    else
        FR_CUFFT(cufftExecZ2D(u->fft[3], (cufftDoubleComplex *)u->r, (cufftDoubleReal *)u->h));
    k_uwu_grad<T><<<(unsigned)std::min<int64_t>((u->cells + 255) / 256, 152 * 16), 256, 0, s>>>(
        (const T *)u->h, c, u->cells, u->scal, u->scal + 3, grad);
    return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

fresco_status fresco_uwu_plan(fresco_uwu_t *out, int dim, const int64_t *grid, const int32_t *mask,
                              int64_t n_k, const double *S0, const double *W, int precision,
                              void *stream) {
    if (!out) return FRESCO_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !grid || !mask || !S0 || !W || n_k < 1) return FRESCO_ERR_ARG;
    if (precision != FRESCO_F32 && precision != FRESCO_F64) return FRESCO_ERR_ARG;
    Params P{};
    P.dim = dim;
    P.precision = precision;
    for (int a = 0; a < 3; ++a) {
        P.nf[a] = 1;
        P.kmax[a] = 0;
    }
    for (int a = 0; a < dim; ++a) {
        if (grid[a] < 4 || grid[a] > (1 << 26) || grid[a] % 2) return FRESCO_ERR_ARG;
        P.nf[a] = (int)grid[a];
    }
    if ((double)P.nf[0] * P.nf[1] * P.nf[2] > 2147483647.0 * 8) return FRESCO_ERR_UNSUPPORTED;
    for (int64_t q = 0; q < n_k; ++q) {
        bool zero = true;
        for (int a = 0; a < dim; ++a) {
            const int32_t v = mask[q * dim + a];
            if (v != 0) zero = false;
            // each wavevector must be a distinct frequency of the grid: |n_a| < M_a / 2
            if (2 * (int64_t)std::abs((int64_t)v) >= P.nf[a]) return FRESCO_ERR_ARG;
            P.kmax[a] = std::max(P.kmax[a], std::abs(v));
        }
        if (zero) return FRESCO_ERR_ARG;
        if (!std::isfinite(S0[q]) || !std::isfinite(W[q]) || W[q] < 0.0) return FRESCO_ERR_ARG;
    }
    Folded F;
    fresco_status st = fold_mask(P, mask, n_k, S0, W, F);
    if (st) return st;
    if (F.s0.empty()) return FRESCO_ERR_ARG;
    fresco_uwu_s *u = new (std::nothrow) fresco_uwu_s();
    if (!u) return FRESCO_ERR_OOM;
    u->dim = dim;
    u->precision = precision;
    u->esize = precision == FRESCO_F64 ? 8 : 4;
    for (int a = 0; a < 3; ++a) u->M[a] = P.nf[a];
    u->kx = P.kmax[0];
    u->loss_const = F.loss_const;
    u->stream = (cudaStream_t)stream;
    st = precision == FRESCO_F64 ? uwu_build<double>(u, F) : uwu_build<float>(u, F);
    if (st) {
        uwu_free(u);
        return st;
    }
    *out = u;
    return FRESCO_OK;
}

fresco_status fresco_uwu_loss_grad(fresco_uwu_t u, const void *d_c, double *d_loss, void *d_grad) {
    fresco::clear_pending_error();
    if (!u || !d_c || !d_loss) return FRESCO_ERR_ARG;
    if (u->precision == FRESCO_F64)
        return uwu_eval<double>(u, (const double *)d_c, d_loss, (double *)d_grad);
    return uwu_eval<float>(u, (const float *)d_c, d_loss, (float *)d_grad);
}

fresco_status fresco_uwu_destroy(fresco_uwu_t u) {
    uwu_free(u);
    return FRESCO_OK;
}

}  // extern "C"
