"""Seeded synthetic inputs: point sets, wavevector masks, targets S0 and weights w.

This module is shared by the GPU tests, the bench and the oracle checks. It holds none
of the method's arithmetic (no Fourier sums, no loss, no gradient): only the problem
definitions the paper's workloads are made of.

* Points: i.i.d. uniform in the periodic box (the Poisson starts of the SI benchmark,
  "Benchmark of FReSCo"), or perfect square / cubic lattices (the Bragg-peak examples
  of SI "Saturating peaks" and the square lattice of SI "Born approximation").
* Masks: the integer wavevectors n != 0 with |n| <= K (k = 2 pi n / L), the constrained
  region of Eq. 2. K follows from the constraint ratio chi = N_K / (2 d N) of Methods
  "Algorithm parameters", with N_K counted over the full ball (both n and -n).
* Targets: stealthy (S0 = 0), power law S0 = (|n|/K)^2, and a peaked ring of Gaussian
  peaks of height N/10 (the "10-petaled flower" target of Fig. 1).

Random numbers come from numpy's Philox counter-based generator, which gives the same
stream on every platform.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    """Philox-backed generator for a seed (platform independent)."""
    return np.random.Generator(np.random.Philox(seed))


def uniform_points(n_points: int, dim: int, seed: int, dtype=np.float64,
                   box: float = 1.0) -> np.ndarray:
    """[n_points, dim] i.i.d. uniform positions in [0, box)^dim, row-major.

    Drawn directly in `dtype`, so FP32 inputs are uniform FP32 values in [0, 1) times box.
    """
    g = rng(seed)
    if np.dtype(dtype) == np.float32:
        x = g.random((n_points, dim), dtype=np.float32)
        if box != 1.0:
            x *= np.float32(box)
        return x
    x = g.random((n_points, dim), dtype=np.float64)
    if box != 1.0:
        x *= box
    return x.astype(dtype, copy=False)


def lattice_points(m: int, dim: int, box: float = 1.0, dtype=np.float64,
                   offset: float = 0.0) -> np.ndarray:
    """The m^dim points of a simple square (2D) / cubic (3D) lattice of spacing box/m.

    Point (i_0, ..., i_{d-1}) sits at ((i + offset) * box / m) in each coordinate.
    """
    axes = [np.arange(m, dtype=np.float64)] * dim
    grid = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([g.reshape(-1) for g in grid], axis=1)
    return ((pts + offset) * (box / m)).astype(dtype)


def ball_count(K: int, dim: int) -> int:
    """Number of integer vectors n != 0 with |n|^2 <= K^2 (the full ball, origin excluded)."""
    K = int(K)
    K2 = K * K
    total = 0
    if dim == 2:
        for nx in range(-K, K + 1):
            total += 2 * math.isqrt(K2 - nx * nx) + 1
    elif dim == 3:
        for nx in range(-K, K + 1):
            rx = K2 - nx * nx
            my = math.isqrt(rx)
            for ny in range(-my, my + 1):
                total += 2 * math.isqrt(rx - ny * ny) + 1
    else:
        raise ValueError("dim must be 2 or 3")
    return total - 1


def radius_for_chi(n_points: int, dim: int, chi: float) -> int:
    """Integer K whose full-ball count N_K is closest to 2 d N chi.

    The ratio chi = N_K / (2 d N) is the one of Methods "Algorithm parameters"; N_K counts
    both members of each +-n pair. With this reading the paper's own sizes come out:
    K = 5050 at N = 5e7 (2D, chi ~ 0.4), K = 142 at N = 5e6 (3D) and K ~ 71 at N = 1e4.
    """
    target = 2.0 * dim * n_points * chi
    if dim == 2:
        k0 = math.sqrt(target / math.pi)
    else:
        k0 = (3.0 * target / (4.0 * math.pi)) ** (1.0 / 3.0)
    best_k, best_err = None, None
    for K in range(max(1, int(k0) - 3), int(k0) + 5):
        err = abs(ball_count(K, dim) - target)
        if best_err is None or err < best_err:
            best_k, best_err = K, err
    return best_k


def ball_mask(K: int, dim: int) -> np.ndarray:
    """int32 [N_K, dim]: every n != 0 with |n| <= K, in lexicographic order of (n_0, n_1, ...).

    Column a is the component along coordinate a of the points (column 0 pairs with x).
    """
    K = int(K)
    K2 = K * K
    chunks = []
    if dim == 2:
        for n0 in range(-K, K + 1):
            m = math.isqrt(K2 - n0 * n0)
            n1 = np.arange(-m, m + 1, dtype=np.int32)
            c = np.empty((n1.size, 2), dtype=np.int32)
            c[:, 0] = n0
            c[:, 1] = n1
            chunks.append(c)
    elif dim == 3:
        for n0 in range(-K, K + 1):
            r0 = K2 - n0 * n0
            m1 = math.isqrt(r0)
            for n1 in range(-m1, m1 + 1):
                m2 = math.isqrt(r0 - n1 * n1)
                n2 = np.arange(-m2, m2 + 1, dtype=np.int32)
                c = np.empty((n2.size, 3), dtype=np.int32)
                c[:, 0] = n0
                c[:, 1] = n1
                c[:, 2] = n2
                chunks.append(c)
    else:
        raise ValueError("dim must be 2 or 3")
    mask = np.concatenate(chunks, axis=0)
    keep = np.any(mask != 0, axis=1)
    return np.ascontiguousarray(mask[keep])


def half_space(mask: np.ndarray) -> np.ndarray:
    """Boolean selector of the entries whose first nonzero component, scanning from column 0,
    is positive: exactly one of each +-n pair. Used by tests to build one-sided masks."""
    sel = np.zeros(mask.shape[0], dtype=bool)
    undecided = np.ones(mask.shape[0], dtype=bool)
    for a in range(mask.shape[1]):
        c = mask[:, a]
        sel |= undecided & (c > 0)
        undecided &= c == 0
    return sel


def stealthy_target(mask: np.ndarray) -> np.ndarray:
    """S0 = 0 on the whole mask (stealthy hyperuniform target)."""
    return np.zeros(mask.shape[0], dtype=np.float64)


def power_law_target(mask: np.ndarray, K: float, exponent: float = 2.0) -> np.ndarray:
    """S0(n) = (|n| / K)^exponent (power-law hyperuniform target)."""
    nn = np.sqrt(np.sum(mask.astype(np.float64) ** 2, axis=1))
    return (nn / float(K)) ** exponent


def peaked_target(mask: np.ndarray, n_points: int, K: float, n_peaks: int = 10,
                  width: float = 1.0) -> np.ndarray:
    """Ring of n_peaks Gaussian peaks of height N/10 and width `width` (grid units) at |n| = K/2.

    Peak p sits at (K/2)(cos 2 pi p / n_peaks, sin 2 pi p / n_peaks) in the (n_0, n_1)
    plane; with an even n_peaks the set is centrosymmetric, so S0(n) = S0(-n).
    """
    out = np.zeros(mask.shape[0], dtype=np.float64)
    h = n_points / 10.0
    # h exp(-d^2 / (2 width^2)) is exactly 0.0 in double once d^2 / (2 width^2) > 745 + ln h, so
    # evaluating it only inside that radius gives the same array as evaluating it everywhere.
    cut2 = 2.0 * width * width * (746.0 + math.log(max(h, 1.0)))
    for p in range(n_peaks):
        a = 2.0 * math.pi * p / n_peaks
        c0 = 0.5 * K * math.cos(a)
        c1 = 0.5 * K * math.sin(a)
        d2 = (mask[:, 0] - c0) ** 2 + (mask[:, 1] - c1) ** 2
        if mask.shape[1] == 3:
            d2 = d2 + mask[:, 2].astype(np.float64) ** 2
        near = np.nonzero(d2 < cut2)[0]
        out[near] += h * np.exp(-d2[near] / (2.0 * width * width))
    return out


def unit_weights(mask: np.ndarray) -> np.ndarray:
    """w = 1 on the whole mask."""
    return np.ones(mask.shape[0], dtype=np.float64)


@dataclass
class Workload:
    """One synthetic problem: N points in a periodic box with a ball mask and a target."""
    name: str
    dim: int
    n_points: int
    K: int
    target: str            # "stealthy" | "power_law" | "peaked"
    dtype: str             # "f64" | "f32"
    seed: int = 0
    box: float = 1.0
    tol: float = 1e-6
    upsample: float = 2.0
    grad_mode: str = "direct"   # "direct" or "kderiv" (gradient of the type-2 interpolant)
    extra: dict = field(default_factory=dict)

    @property
    def np_dtype(self):
        return np.float64 if self.dtype == "f64" else np.float32

    def points(self) -> np.ndarray:
        return uniform_points(self.n_points, self.dim, self.seed, self.np_dtype, self.box)

    def mask(self) -> np.ndarray:
        return ball_mask(self.K, self.dim)

    def targets(self, mask: np.ndarray):
        if self.target == "stealthy":
            s0 = stealthy_target(mask)
        elif self.target == "power_law":
            s0 = power_law_target(mask, self.K)
        elif self.target == "peaked":
            s0 = peaked_target(mask, self.n_points, self.K)
        else:
            raise ValueError(self.target)
        return s0, unit_weights(mask)


def workload(name: str) -> Workload:
    """The named synthetic workloads (sizes in the name; see the module docstring)."""
    if name == "stealthy2d_n1024_k20_f64":
        return Workload(name, 2, 1024, 20, "stealthy", "f64", seed=0, tol=1e-12)
    # the FP32 workloads take the gradient of the type-2 interpolant (one real inverse FFT, one
    # real grid to interpolate): 2.3x faster in 3D and 7% faster at 1e8 in 2D than the direct
    # mode, 2e-6 .. 6e-6 relative gradient difference
    if name == "stealthy2d_n1e6_chi045_f32":
        return Workload(name, 2, 10**6, radius_for_chi(10**6, 2, 0.45), "stealthy", "f32",
                        seed=0, tol=1e-6, grad_mode="kderiv")
    # 3D: the 3-smooth grid 648 = 2^3 3^4 (oversampling 1.6744 for K = 193, w = 7) instead of 784
    # at oversampling 2: 0.56x the cells, more points per staged tile; 31.6 -> 20.0 ms per
    # evaluation measured
    if name == "powerlaw3d_n2p24_chi03_f32":
        return Workload(name, 3, 2**24, radius_for_chi(2**24, 3, 0.3), "power_law", "f32",
                        seed=0, tol=1e-6, upsample=1.6744, grad_mode="kderiv")
    # the large 2D workloads: the fine grid is the 3-smooth 20736 = 2^8 3^4 (oversampling 1.6775
    # for K = 6180), the smallest size at which the tolerance 1e-6 needs only w = 7; its FFTs run
    # ~20% faster than those of 18750 (oversampling 1.5, w = 8) or 20480 = 2^12 5. The 1e7
    # stand-in used for profiling keeps the same kernel width (n_f = 6480, oversampling 1.6577)
    if name == "peaked2d_n1e8_chi03_f32":
        return Workload(name, 2, 10**8, radius_for_chi(10**8, 2, 0.3), "peaked", "f32",
                        seed=0, tol=1e-6, upsample=1.6775, grad_mode="kderiv")
    if name == "peaked2d_n1e7_chi03_f32":
        return Workload(name, 2, 10**7, radius_for_chi(10**7, 2, 0.3), "peaked", "f32",
                        seed=0, tol=1e-6, upsample=1.6577, grad_mode="kderiv")
    # 3D profiling stand-in: the same kernel width and point density per fine cell at 1/8 of the
    # points (n_f = 324 = 2^2 3^4, K = 97, oversampling 1.6615; fine grid 136 MB > L2)
    if name == "powerlaw3d_n2p21_chi03_f32":
        return Workload(name, 3, 2**21, radius_for_chi(2**21, 3, 0.3), "power_law", "f32",
                        seed=0, tol=1e-6, upsample=1.6615, grad_mode="kderiv")
    if name == "peaked2d_n1e8_chi03_f64":
        return Workload(name, 2, 10**8, radius_for_chi(10**8, 2, 0.3), "peaked", "f64",
                        seed=0, tol=1e-12, upsample=1.6775)
    raise KeyError(name)


@dataclass
class FreeWorkload:
    """Points at free positions in [-L/2, L/2]^d with constraints at real wavevectors (the
    NUwNU form): a quasicrystal-like target, a ring of n_peaks Gaussian Bragg peaks at a radius
    incommensurate with the box's reciprocal lattice."""
    name: str
    dim: int
    n_points: int
    n_k: int
    kmax: float            # wavevectors uniform in the ball |k| <= kmax (radians per length)
    dtype: str
    seed: int = 0
    box: float = 1.0
    tol: float = 1e-6
    upsample: float = 2.0
    n_peaks: int = 10

    def points(self) -> np.ndarray:
        dt = np.float64 if self.dtype == "f64" else np.float32
        g = rng(self.seed)
        return ((g.random((self.n_points, self.dim)) - 0.5) * self.box).astype(dt)

    def wavevectors(self) -> np.ndarray:
        g = rng(self.seed + 1)
        k = g.standard_normal((self.n_k, self.dim))
        k *= (self.kmax * g.random(self.n_k) ** (1.0 / self.dim)
              / np.linalg.norm(k, axis=1))[:, None]
        return k

    def targets(self, k: np.ndarray):
        r = self.kmax / (1.0 + np.sqrt(5.0))
        ang = 2 * np.pi * np.arange(self.n_peaks) / self.n_peaks
        c = np.zeros((self.n_peaks, self.dim))
        c[:, 0], c[:, 1] = r * np.cos(ang), r * np.sin(ang)
        width = 2 * np.pi / self.box
        S0 = np.zeros(k.shape[0])
        for p in range(self.n_peaks):
            S0 += (self.n_points / self.n_peaks) * np.exp(
                -((k - c[p]) ** 2).sum(1) / (2 * width ** 2))
        return S0, np.ones(k.shape[0])


def free_workload(name: str) -> FreeWorkload:
    """The named NUwNU workloads."""
    if name == "quasicrystal2d_n1e6_k1e6_f32":
        return FreeWorkload(name, 2, 10**6, 10**6, 2 * np.pi * 400, "f32", seed=11)
    raise KeyError(name)


@dataclass
class FieldWorkload:
    """Real weights on a uniform grid with constraints at real frequencies (the UwNU form): a
    density field of M^d pixels with weights uniform in [0, 1), n_k constraints at frequencies
    uniform in the ball |nu| <= nu_max (cycles per grid length), targets zero (a stealthy-like
    band) except a ring of n_peaks Gaussian peaks one cycle wide at radius nu_max / 4 (the
    six-fold target of the paper's UwNU fields, at real rather than lattice frequencies)."""
    name: str
    dim: int
    M: int                 # pixels per axis
    n_k: int
    nu_max: float
    dtype: str
    seed: int = 0
    tol: float = 1e-6
    upsample: float = 2.0
    n_peaks: int = 6
    peak_height: float = 10.0

    @property
    def shape(self):
        return (self.M,) * self.dim

    @property
    def n_weights(self) -> int:
        return self.M ** self.dim

    def weights(self) -> np.ndarray:
        """Weights [M]*dim (x the last, contiguous index)."""
        dt = np.float64 if self.dtype == "f64" else np.float32
        return rng(self.seed).random(self.shape).astype(dt)

    def frequencies(self) -> np.ndarray:
        g = rng(self.seed + 1)
        nu = g.standard_normal((self.n_k, self.dim))
        nu *= (self.nu_max * g.random(self.n_k) ** (1.0 / self.dim)
               / np.linalg.norm(nu, axis=1))[:, None]
        return nu

    def targets(self, nu: np.ndarray):
        r = 0.25 * self.nu_max
        ang = 2 * np.pi * np.arange(self.n_peaks) / self.n_peaks
        c = np.zeros((self.n_peaks, self.dim))
        c[:, 0], c[:, 1] = r * np.cos(ang), r * np.sin(ang)
        S0 = np.zeros(nu.shape[0])
        for p in range(self.n_peaks):
            S0 += self.peak_height * np.exp(-((nu - c[p]) ** 2).sum(1) / 2.0)
        return S0, np.ones(nu.shape[0])


def field_workload(name: str) -> FieldWorkload:
    """The named UwNU workloads."""
    if name == "hexfield2d_m1024_k1e6_f32":
        return FieldWorkload(name, 2, 1024, 10**6, 460.0, "f32", seed=13)
    raise KeyError(name)


@dataclass
class Ensemble:
    """Many independent 2D problems: instance i has n_points[i] uniform points in a periodic box
    boxes[i] (a square of that side) and the ball mask of radius K[i] (from chi[i]), with a
    stealthy target and unit weights."""
    name: str
    n_points: list
    K: list
    chi: list
    boxes: list
    dtype: str = "f32"
    seed: int = 7
    tol: float = 1e-6
    upsample: float = 2.0
    grad_mode: str = "direct"

    @property
    def n_inst(self) -> int:
        return len(self.n_points)

    @property
    def np_dtype(self):
        return np.float64 if self.dtype == "f64" else np.float32

    def instance_points(self, i: int) -> np.ndarray:
        # instance i draws from its own stream, so any one instance can be rebuilt alone
        return uniform_points(self.n_points[i], 2, self.seed * 1_000_003 + 1 + i, self.np_dtype,
                              self.boxes[i])

    def points(self) -> np.ndarray:
        """All instances' points packed one instance after the other: [sum N, 2]."""
        return np.ascontiguousarray(np.concatenate(
            [self.instance_points(i) for i in range(self.n_inst)], axis=0))

    def masks(self) -> list:
        return [ball_mask(k, 2) for k in self.K]

    def targets(self, masks: list):
        return [stealthy_target(m) for m in masks], [unit_weights(m) for m in masks]


def ensemble(n_inst: int, n_lo: float, n_hi: float, chi_lo: float, chi_hi: float, seed: int,
             dtype: str = "f32", box_lo: float = 1.0, box_hi: float = 1.0, tol: float = 1e-6,
             upsample: float = 2.0, name: str = "") -> Ensemble:
    """n_inst instances with N log-uniform in [n_lo, n_hi], chi uniform in [chi_lo, chi_hi] and
    box sides uniform in [box_lo, box_hi], all drawn from one seeded stream."""
    g = rng(seed)
    n = np.rint(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), n_inst))).astype(np.int64)
    chi = g.uniform(chi_lo, chi_hi, n_inst)
    box = g.uniform(box_lo, box_hi, n_inst) if box_hi > box_lo else np.full(n_inst, box_lo)
    K = [max(1, radius_for_chi(int(n[i]), 2, float(chi[i]))) for i in range(n_inst)]
    return Ensemble(name or "ensemble%d_seed%d" % (n_inst, seed), [int(x) for x in n], K,
                    [float(c) for c in chi], [float(b) for b in box], dtype, seed, tol, upsample)


def ensemble_workload(name: str) -> Ensemble:
    """The named ensembles: 512 stealthy 2D configurations, N log-uniform in [1e3, 1e5] and chi
    uniform in [0.1, 0.5], seed 7, unit square boxes."""
    if name == "stealthy2d_ens512_n1e3to1e5_f32":
        e = ensemble(512, 1e3, 1e5, 0.1, 0.5, 7, "f32", tol=1e-6, name=name)
        e.grad_mode = "kderiv"
        return e
    if name == "stealthy2d_ens512_n1e3to1e5_f64":
        return ensemble(512, 1e3, 1e5, 0.1, 0.5, 7, "f64", tol=1e-12, name=name)
    raise KeyError(name)
