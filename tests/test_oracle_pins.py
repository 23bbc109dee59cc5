"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, not by the oracle.

Each test below would fail for a plausible mistake in the oracle (a dropped term, a wrong
sign or index, a transposed operand, a wrong factor in the gradient):

* rho(0) = N (S(0) = N, Eq. 1);
* points on an M x M (x M) grid with random occupancy: rho equals numpy's FFT of the
  occupancy array (catches a wrong exponent sign, swapped axes or a wrong box scaling);
* square / cubic lattices: Bragg peaks S = N on the reciprocal lattice and 0 elsewhere
  (SI "Saturating peaks");
* Poisson points: E[S(n)] = 1 for integer n != 0;
* N = 1: S = 1 and zero gradient; N = 2: closed forms for S, the loss and the gradient;
* central finite differences of the oracle's own loss against its gradient;
* translation invariance: sum_j dL/dr_j = 0;
* lattice with spacing finer than the mask (m > K): L = 0 and dL/dr = 0 (stealthy ground
  state);
* weighted points at real wavevectors (non-uniform constraints): integer wavevectors reproduce
  the separately written mask form, one and two weights have closed forms off the lattice, and
  central differences pin the weight gradient;
* unit-weight points at real wavevectors (free boundaries): the same reduction to the mask form,
  N = 1 and N = 2 closed forms off the lattice (S and the forces), central differences in 3D and
  invariance under a rigid shift.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2305_15693_gb300 import inputs


def test_rho_at_origin_is_n():
    pts = inputs.uniform_points(333, 2, seed=3)
    mask = np.array([[0, 0], [1, 0]], dtype=np.int32)
    rho = oracle.rho(pts, mask)
    assert rho[0].real == pytest.approx(333.0, abs=1e-9)
    assert abs(rho[0].imag) < 1e-9


@pytest.mark.parametrize("dim,M,box", [(2, 12, (1.0, 2.5)), (3, 6, (1.5, 1.0, 0.75))])
def test_grid_occupancy_equals_numpy_fft(dim, M, box):
    g = inputs.rng(11)
    occ = g.random((M,) * dim) < 0.4          # occ[i_{d-1}, ..., i_0] (numpy axis 0 = last coord)
    idx = np.argwhere(occ)                    # rows (i_{d-1}, ..., i_0)
    coords = idx[:, ::-1].astype(np.float64)  # (i_0, ..., i_{d-1}) -> coordinate a uses i_a
    pts = coords / M * np.asarray(box)
    mask = g.integers(-2 * M, 2 * M, size=(40, dim)).astype(np.int32)
    rho = oracle.rho(pts, mask, box=box)
    F = np.fft.fftn(occ.astype(np.float64))   # sum occ[i] exp(-2 pi i k.i / M)
    want = np.array([F[tuple((n[::-1]) % M)] for n in mask])
    np.testing.assert_allclose(rho, want, rtol=0, atol=1e-9)


def test_square_lattice_bragg_peaks():
    m = 8
    pts = inputs.lattice_points(m, 2, offset=0.3)
    N = pts.shape[0]
    mask = inputs.ball_mask(20, 2)
    S0 = np.zeros(mask.shape[0])
    W = np.ones(mask.shape[0])
    _, _, S, _ = oracle.loss_grad(pts, mask, S0, W, want_grad=False)
    on = np.all(mask % m == 0, axis=1)
    assert on.sum() > 0
    np.testing.assert_allclose(S[on], N, rtol=1e-12)
    assert np.max(np.abs(S[~on])) < 1e-12 * N


def test_cubic_lattice_bragg_peaks():
    m = 5
    pts = inputs.lattice_points(m, 3, box=2.0, offset=0.1)
    N = pts.shape[0]
    mask = inputs.ball_mask(8, 3)
    S0 = np.zeros(mask.shape[0])
    W = np.ones(mask.shape[0])
    _, _, S, _ = oracle.loss_grad(pts, mask, S0, W, box=2.0, want_grad=False)
    on = np.all(mask % m == 0, axis=1)
    np.testing.assert_allclose(S[on], N, rtol=1e-12)
    assert np.max(np.abs(S[~on])) < 1e-12 * N


def test_poisson_mean_structure_factor_is_one():
    mask = inputs.ball_mask(20, 2)
    keep = inputs.half_space(mask)            # S(n) = S(-n): count each pair once
    half = mask[keep]
    vals = []
    for seed in range(64):
        pts = inputs.uniform_points(1024, 2, seed=1000 + seed)
        r = oracle.rho(pts, half)
        vals.append(np.abs(r) ** 2 / 1024.0)
    s = np.concatenate(vals)
    sigma = 1.0 / math.sqrt(s.size)           # S ~ Exp(1) for i.i.d. uniform points
    assert abs(s.mean() - 1.0) < 4.0 * sigma


def test_single_point():
    pts = np.array([[0.37, 0.81]])
    mask = inputs.ball_mask(5, 2)
    S0 = np.full(mask.shape[0], 0.25)
    W = np.linspace(0.5, 2.0, mask.shape[0])
    loss, grad, S, _ = oracle.loss_grad(pts, mask, S0, W)
    np.testing.assert_allclose(S, 1.0, rtol=1e-13)
    assert loss == pytest.approx(np.sum(W * 0.75 ** 2), rel=1e-13)
    assert np.max(np.abs(grad)) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_two_points_closed_form(dim):
    g = inputs.rng(5)
    pts = g.random((2, dim))
    box = 1.0 + g.random(dim)
    mask = inputs.ball_mask(3, dim)
    S0 = g.random(mask.shape[0]) * 2.0
    W = 0.5 + g.random(mask.shape[0])
    loss, grad, S, _ = oracle.loss_grad(pts, mask, S0, W, box=box)
    k = 2.0 * np.pi * mask / box                           # [n_k, dim]
    phi = k @ (pts[0] - pts[1])                            # k . (r_1 - r_2)
    S_cf = 1.0 + np.cos(phi)                               # |1 + e^{-i phi}|^2 / 2
    L_cf = np.sum(W * (S_cf - S0) ** 2)
    dS_dr1 = -np.sin(phi)[:, None] * k                     # d/dr_1 of 1 + cos(k.(r_1 - r_2))
    g1 = np.sum((2.0 * W * (S_cf - S0))[:, None] * dS_dr1, axis=0)
    np.testing.assert_allclose(S, S_cf, rtol=1e-12, atol=1e-12)
    assert loss == pytest.approx(L_cf, rel=1e-12)
    np.testing.assert_allclose(grad[0], g1, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(grad[1], -g1, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("dim,N,K", [(2, 16, 4), (3, 12, 3)])
def test_gradient_matches_central_differences(dim, N, K):
    g = inputs.rng(17 + dim)
    pts = g.random((N, dim))
    box = np.linspace(1.0, 1.3, dim)
    pts *= box
    mask = inputs.ball_mask(K, dim)
    S0 = g.random(mask.shape[0])
    W = 0.2 + g.random(mask.shape[0])
    _, grad, _, _ = oracle.loss_grad(pts, mask, S0, W, box=box)
    h = 1e-6
    fd = np.zeros_like(pts)
    for j in range(N):
        for a in range(dim):
            p = pts.copy()
            p[j, a] += h
            lp, _, _, _ = oracle.loss_grad(p, mask, S0, W, box=box, want_grad=False)
            p[j, a] -= 2 * h
            lm, _, _, _ = oracle.loss_grad(p, mask, S0, W, box=box, want_grad=False)
            fd[j, a] = (lp - lm) / (2 * h)
    err = np.linalg.norm(fd - grad) / np.linalg.norm(grad)
    assert err < 1e-7


def test_translation_invariance_and_selection():
    g = inputs.rng(23)
    pts = g.random((200, 2))
    mask = inputs.ball_mask(6, 2)
    S0 = g.random(mask.shape[0])
    W = g.random(mask.shape[0])
    loss, grad, _, _ = oracle.loss_grad(pts, mask, S0, W)
    assert np.linalg.norm(grad.sum(axis=0)) < 1e-11 * np.linalg.norm(grad)
    sel = np.array([5, 0, 199, 42])
    loss2, gsel, _, _ = oracle.loss_grad(pts, mask, S0, W, sel=sel)
    assert loss2 == loss
    np.testing.assert_array_equal(gsel, grad[sel])
    shifted = pts + np.array([0.3, -1.7])
    loss3, grad3, _, _ = oracle.loss_grad(shifted, mask, S0, W)
    assert loss3 == pytest.approx(loss, rel=1e-11)
    np.testing.assert_allclose(grad3, grad, rtol=1e-8, atol=1e-9 * np.abs(grad).max())


def test_lattice_ground_state_is_stealthy():
    m = 16
    pts = inputs.lattice_points(m, 2, offset=0.5)
    mask = inputs.ball_mask(10, 2)            # every |n| <= 10 < m: no reciprocal-lattice point
    loss, grad, S, _ = oracle.loss_grad(pts, mask, np.zeros(mask.shape[0]),
                                        np.ones(mask.shape[0]))
    assert loss < 1e-20
    assert np.max(np.abs(grad)) < 1e-9


# ---- repulsive pair term of the hybrid loss (Eq. 6) ------------------------------------------

@pytest.mark.parametrize("alpha", [2.0, 2.5])
def test_pair_two_points_closed_form_and_periodic_image(alpha):
    sigma, eps = 0.2, 1.7
    # direct distance 0.12 along y; 0.12 again through the periodic image along x for the second
    for pts, r in ((np.array([[0.3, 0.40], [0.3, 0.52]]), 0.12),
                   (np.array([[0.04, 0.5], [0.92, 0.5]]), 0.12)):
        e, g = oracle.pair_energy_grad(pts, sigma, eps, alpha, box=1.0)
        assert e == pytest.approx(eps / alpha * (1 - r / sigma) ** alpha, rel=1e-12)
        du = -eps / sigma * (1 - r / sigma) ** (alpha - 1)
        dx = pts[0] - pts[1]
        dx -= np.round(dx)
        np.testing.assert_allclose(g[0], du * dx / r, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(g[1], -g[0], rtol=1e-12, atol=1e-14)
    e, g = oracle.pair_energy_grad(np.array([[0.1, 0.1], [0.1, 0.35]]), sigma, eps, alpha)
    assert e == 0.0 and np.all(g == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_pair_gradient_central_differences_and_invariance(dim):
    g = inputs.rng(90 + dim)
    N = 40
    box = np.linspace(1.0, 1.2, dim)
    pts = g.random((N, dim)) * box
    sigma = 0.6 * (np.prod(box) / N) ** (1.0 / dim) * 2
    e, grad = oracle.pair_energy_grad(pts, sigma, 1.3, 2.5, box=box)
    assert e > 0
    h = 1e-7
    fd = np.zeros_like(pts)
    for j in range(N):
        for a in range(dim):
            p = pts.copy()
            p[j, a] += h
            ep, _ = oracle.pair_energy_grad(p, sigma, 1.3, 2.5, box=box, want_grad=False)
            p[j, a] -= 2 * h
            em, _ = oracle.pair_energy_grad(p, sigma, 1.3, 2.5, box=box, want_grad=False)
            fd[j, a] = (ep - em) / (2 * h)
    assert np.linalg.norm(fd - grad) / np.linalg.norm(grad) < 1e-6
    assert np.linalg.norm(grad.sum(axis=0)) < 1e-10 * np.linalg.norm(grad)
    e2, _ = oracle.pair_energy_grad(pts + 0.37, sigma, 1.3, 2.5, box=box, want_grad=False)
    assert e2 == pytest.approx(e, rel=1e-12)


# ---- weighted points: the weight gradient (Methods, "Analytical gradients", UwU / UwNU) -----

def _grid_problem(shape, K, seed):
    g = inputs.rng(seed)
    dim = len(shape)
    c = g.standard_normal(int(np.prod(shape)))
    mask = inputs.ball_mask(K, dim)
    S0 = g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    return oracle.grid_points(shape), c, mask, S0, W


@pytest.mark.parametrize("shape", [(12, 10), (6, 5, 4)])
def test_weighted_grid_rho_equals_numpy_fft(shape):
    pts, c, mask, S0, W = _grid_problem(shape, 2, 81)
    _, _, S, rho = oracle.weight_loss_grad(pts, c, mask, S0, W)
    F = np.fft.fftn(c.reshape(shape[::-1]))           # numpy axis 0 is the last coordinate
    want = np.array([F[tuple((n[::-1]) % np.array(shape[::-1]))] for n in mask])
    np.testing.assert_allclose(rho, want, rtol=0, atol=1e-10)
    np.testing.assert_allclose(S, np.abs(want) ** 2 / np.sum(c * c), rtol=1e-12)


def test_weight_gradient_matches_central_differences():
    pts, c, mask, S0, W = _grid_problem((8, 7), 3, 82)
    _, grad, _, _ = oracle.weight_loss_grad(pts, c, mask, S0, W)
    h = 1e-6
    fd = np.zeros_like(c)
    for j in range(c.size):
        cp, cm = c.copy(), c.copy()
        cp[j] += h
        cm[j] -= h
        lp, _, _, _ = oracle.weight_loss_grad(pts, cp, mask, S0, W, want_grad=False)
        lm, _, _, _ = oracle.weight_loss_grad(pts, cm, mask, S0, W, want_grad=False)
        fd[j] = (lp - lm) / (2 * h)
    assert np.linalg.norm(fd - grad) / np.linalg.norm(grad) < 1e-7


def test_weight_gradient_scale_invariance_and_single_weight():
    pts, c, mask, S0, W = _grid_problem((9, 8), 3, 83)
    loss, grad, _, _ = oracle.weight_loss_grad(pts, c, mask, S0, W)
    # S, hence L, is invariant under c -> alpha c, so sum_j c_j dL/dc_j = 0 (Euler)
    assert abs(np.dot(c, grad)) < 1e-11 * np.linalg.norm(c) * np.linalg.norm(grad)
    loss2, _, _, _ = oracle.weight_loss_grad(pts, -3.7 * c, mask, S0, W, want_grad=False)
    assert loss2 == pytest.approx(loss, rel=1e-12)
    # a single nonzero weight: S = 1 everywhere and no force on that weight
    one = np.zeros_like(c)
    one[17] = 2.5
    _, g1, S1, _ = oracle.weight_loss_grad(pts, one, mask, S0, W)
    np.testing.assert_allclose(S1, 1.0, rtol=1e-13)
    assert abs(g1[17]) < 1e-12


def test_unit_weights_reproduce_the_point_oracle():
    pts = inputs.uniform_points(300, 2, 84)
    mask = inputs.ball_mask(5, 2)
    g = inputs.rng(84)
    S0, W = g.random(mask.shape[0]), 0.5 + g.random(mask.shape[0])
    l1, _, S1, r1 = oracle.weight_loss_grad(pts, np.ones(300), mask, S0, W, want_grad=False)
    l2, _, S2, r2 = oracle.loss_grad(pts, mask, S0, W, want_grad=False)
    assert l1 == pytest.approx(l2, rel=1e-13)
    np.testing.assert_allclose(S1, S2, rtol=1e-12)


# ---- weighted points at arbitrary real wavevectors (UwNU, Methods "Analytical gradients") -------

def test_integer_wavevectors_reproduce_the_mask_form():
    """With k = 2 pi n / L for integer n, the wavevector form equals the separately written
    mask form on the same weighted grid (loss, gradient, S and rho)."""
    g = inputs.rng(41)
    shape, box = (7, 6), np.array([1.3, 0.8])
    pts = oracle.grid_points(shape, box)
    c = g.standard_normal(pts.shape[0])
    mask = np.array([[1, 0], [0, 2], [-3, 1], [2, -2], [3, 2]], dtype=np.int32)
    S0 = g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    l1, g1, S1, r1 = oracle.weight_loss_grad(pts, c, mask, S0, W, box=box)
    kvec = 2.0 * np.pi * mask / box
    l2, g2, S2, r2 = oracle.weight_loss_grad_k(pts, c, kvec, S0, W)
    assert l2 == pytest.approx(l1, rel=1e-12)
    np.testing.assert_allclose(g2, g1, rtol=1e-10, atol=1e-12 * np.abs(g1).max())
    np.testing.assert_allclose(S2, S1, rtol=1e-12)
    np.testing.assert_allclose(r2, r1, rtol=1e-12, atol=1e-12)


def test_wavevector_form_closed_forms_off_the_lattice():
    """One weight: S = 1 at every k and no force. Two weights c1, c2 at distance dr:
    S(k) = (c1^2 + c2^2 + 2 c1 c2 cos(k . dr)) / (c1^2 + c2^2) at non-integer k."""
    k = np.array([[0.37, -2.11], [5.5, 0.25], [-1.0, 3.3]])
    S0 = np.array([0.3, 1.2, 0.8])
    W = np.array([1.0, 0.5, 2.0])
    loss, grad, S, _ = oracle.weight_loss_grad_k(np.array([[0.4, -0.7]]), [2.5], k, S0, W)
    np.testing.assert_allclose(S, 1.0, rtol=1e-14)
    assert loss == pytest.approx(float(np.sum(W * (1.0 - S0) ** 2)), rel=1e-14)
    assert abs(grad[0]) < 1e-13
    r = np.array([[0.1, 0.2], [0.9, -0.4]])
    c = np.array([1.5, -0.7])
    _, _, S, _ = oracle.weight_loss_grad_k(r, c, k, S0, W, want_grad=False)
    dr = r[0] - r[1]
    ref = (c[0] ** 2 + c[1] ** 2 + 2 * c[0] * c[1] * np.cos(k @ dr)) / (c @ c)
    np.testing.assert_allclose(S, ref, rtol=1e-13)


def test_wavevector_form_gradient_matches_central_differences():
    g = inputs.rng(43)
    pts = oracle.grid_points((5, 4, 3))
    c = g.standard_normal(pts.shape[0])
    k = g.uniform(-9.0, 9.0, (11, 3))
    S0 = g.random(11)
    W = 0.5 + g.random(11)
    _, grad, _, _ = oracle.weight_loss_grad_k(pts, c, k, S0, W)
    h = 1e-6
    for j in (0, 7, 31, 59):
        cp, cm = c.copy(), c.copy()
        cp[j] += h
        cm[j] -= h
        lp = oracle.weight_loss_grad_k(pts, cp, k, S0, W, want_grad=False)[0]
        lm = oracle.weight_loss_grad_k(pts, cm, k, S0, W, want_grad=False)[0]
        assert grad[j] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-8)


# ---- points at arbitrary real wavevectors (NUwNU, free boundaries) ------------------------------

def test_point_form_at_integer_wavevectors_reproduces_the_mask_form():
    g = inputs.rng(51)
    box = np.array([1.3, 0.7])
    pts = g.random((40, 2)) * box
    mask = np.array([[1, 0], [0, 3], [-2, 1], [4, -1], [2, 2]], dtype=np.int32)
    S0 = g.random(5)
    W = 0.5 + g.random(5)
    l1, g1, S1, r1 = oracle.loss_grad(pts, mask, S0, W, box=box)
    l2, g2, S2, r2 = oracle.loss_grad_k(pts, 2.0 * np.pi * mask / box, S0, W)
    assert l2 == pytest.approx(l1, rel=1e-12)
    np.testing.assert_allclose(g2, g1, rtol=1e-10, atol=1e-12 * np.abs(g1).max())
    np.testing.assert_allclose(S2, S1, rtol=1e-12)
    np.testing.assert_allclose(r2, r1, rtol=1e-12, atol=1e-12)


def test_point_form_closed_forms_off_the_lattice():
    """N = 1: S = 1, no force. N = 2 at non-integer k: S = 1 + cos(k . dr) and
    dL/dr_1 = -sum_q 2 W (S - S0) sin(k . dr) k = -dL/dr_2."""
    k = np.array([[0.37, -2.11], [5.5, 0.25], [-1.0, 3.3]])
    S0 = np.array([0.3, 1.2, 0.8])
    W = np.array([1.0, 0.5, 2.0])
    loss, grad, S, _ = oracle.loss_grad_k(np.array([[0.4, -0.7]]), k, S0, W)
    np.testing.assert_allclose(S, 1.0, rtol=1e-14)
    assert loss == pytest.approx(float(np.sum(W * (1.0 - S0) ** 2)), rel=1e-14)
    assert np.abs(grad).max() < 1e-13
    r = np.array([[0.1, 0.2], [0.9, -0.4]])
    loss, grad, S, _ = oracle.loss_grad_k(r, k, S0, W)
    ph = k @ (r[0] - r[1])
    np.testing.assert_allclose(S, 1.0 + np.cos(ph), rtol=1e-13)
    assert loss == pytest.approx(float(np.sum(W * (1.0 + np.cos(ph) - S0) ** 2)), rel=1e-13)
    g1 = -(2.0 * W * (1.0 + np.cos(ph) - S0) * np.sin(ph)) @ k
    np.testing.assert_allclose(grad[0], g1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(grad[1], -g1, rtol=1e-12, atol=1e-14)


def test_point_form_central_differences_and_translation():
    g = inputs.rng(53)
    pts = g.random((30, 3)) * 2.0 - 0.5
    k = g.uniform(-12.0, 12.0, (17, 3))
    S0 = g.random(17)
    W = 0.5 + g.random(17)
    loss, grad, _, _ = oracle.loss_grad_k(pts, k, S0, W)
    h = 1e-6
    for j, a in ((0, 0), (7, 1), (29, 2)):
        pp, pm = pts.copy(), pts.copy()
        pp[j, a] += h
        pm[j, a] -= h
        lp = oracle.loss_grad_k(pp, k, S0, W, want_grad=False)[0]
        lm = oracle.loss_grad_k(pm, k, S0, W, want_grad=False)[0]
        assert grad[j, a] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-8)
    # a rigid shift multiplies every rho by a phase: L unchanged and the forces sum to zero
    shifted = oracle.loss_grad_k(pts + np.array([0.3, -1.7, 2.9]), k, S0, W, want_grad=False)[0]
    assert shifted == pytest.approx(loss, rel=1e-12)
    np.testing.assert_allclose(grad.sum(axis=0), 0.0, atol=1e-10 * np.abs(grad).max())
