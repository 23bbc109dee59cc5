"""GPU parity of the repulsive pair term of the hybrid loss (Eq. 6) against the oracle's direct
double loop, at small sizes and at the 3D workload's full size (2^24 points), and the hybrid
L-BFGS."""

import numpy as np
import pytest

import oracle
from paper_2305_15693_gb300 import inputs

from _parity import TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2305_15693_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()


def _gpu_pair(pts_np, box, sigma, eps, alpha, precision):
    import torch
    from paper_2305_15693_gb300 import fresco
    dt = torch.float64 if precision == "f64" else torch.float32
    pts = torch.from_numpy(np.ascontiguousarray(pts_np)).to("cuda", dt)
    with fresco.PairTerm(box, pts.shape[1], pts.shape[0], sigma, eps, alpha, precision) as pt:
        e, g = pt.energy_grad(pts)
        torch.cuda.synchronize()
        return e.item(), g.double().cpu().numpy()


@pytest.mark.parametrize("dim,N,alpha,precision", [
    (2, 4000, 2.0, "f64"), (2, 4000, 2.5, "f32"), (3, 5000, 2.0, "f32"), (3, 5000, 2.5, "f64")])
def test_pair_term_matches_oracle(dim, N, alpha, precision):
    g = inputs.rng(200 + dim)
    box = np.linspace(1.0, 1.25, dim)
    dt = np.float64 if precision == "f64" else np.float32
    pts = ((g.random((N, dim)) * 3.0 - 1.0) * box).astype(dt)      # some outside the box
    sigma = 1.5 * (np.prod(box) / N) ** (1.0 / dim)
    e_o, g_o = oracle.pair_energy_grad(pts, sigma, 0.7, alpha, box=box)
    e_g, g_g = _gpu_pair(pts, box, sigma, 0.7, alpha, precision)
    bar = 1e-11 if precision == "f64" else 2e-5
    assert e_o > 0
    assert abs(e_g - e_o) <= bar * e_o
    assert rel_l2(g_g, g_o) <= bar


def test_pair_term_with_two_cells_per_axis():
    g = inputs.rng(7)
    pts = g.random((300, 2))
    sigma = 0.4                                   # box / sigma = 2.5: two cells per axis
    e_o, g_o = oracle.pair_energy_grad(pts, sigma, 1.0, 2.0)
    e_g, g_g = _gpu_pair(pts, 1.0, sigma, 1.0, 2.0, "f64")
    assert abs(e_g - e_o) <= 1e-11 * e_o
    assert rel_l2(g_g, g_o) <= 1e-11


def test_pair_accumulates_onto_the_structure_factor_loss():
    import torch
    from paper_2305_15693_gb300 import fresco
    pts_np = inputs.uniform_points(2000, 3, 4)
    mask = inputs.ball_mask(6, 3)
    S0 = inputs.power_law_target(mask, 6)
    W = np.ones(mask.shape[0])
    sigma = 0.8 * (1.0 / 2000) ** (1 / 3)
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.Plan(1.0, mask, S0, W, 2000, precision="f64") as plan, \
            fresco.PairTerm(1.0, 3, 2000, sigma, 1.0, 2.0, "f64") as pair:
        loss, grad = plan.loss_grad(pts)
        l_s = loss.item()
        g_s = grad.cpu().numpy().copy()
        pair.energy_grad(pts, loss, grad, accumulate=True)
        torch.cuda.synchronize()
        e_p, g_p = oracle.pair_energy_grad(pts_np, sigma, 1.0, 2.0)
        assert loss.item() == pytest.approx(l_s + e_p, rel=1e-11)
        np.testing.assert_allclose(grad.cpu().numpy(), g_s + g_p, rtol=1e-9,
                                   atol=1e-11 * np.abs(g_s + g_p).max())


def test_hybrid_lbfgs_lowers_both_terms():
    import torch
    from paper_2305_15693_gb300 import fresco
    N = 3000
    pts_np = inputs.uniform_points(N, 3, 8)
    mask = inputs.ball_mask(5, 3)
    S0 = inputs.power_law_target(mask, 5)
    W = np.ones(mask.shape[0])
    sigma = 0.8 * (1.0 / N) ** (1 / 3)
    l0, _, _, _ = oracle.loss_grad(pts_np, mask, S0, W, want_grad=False)
    e0, _ = oracle.pair_energy_grad(pts_np, sigma, 1.0, 2.0, want_grad=False)
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.Plan(1.0, mask, S0, W, N, precision="f64") as plan, \
            fresco.PairTerm(1.0, 3, N, sigma, 1.0, 2.0, "f64") as pair:
        solver = fresco.LBFGS(plan)
        solver.set_pair(pair)
        rep = solver.run(pts, 60)
        solver.close()
    x = pts.cpu().numpy()
    l1, _, _, _ = oracle.loss_grad(x, mask, S0, W, want_grad=False)
    e1, _ = oracle.pair_energy_grad(x, sigma, 1.0, 2.0, want_grad=False)
    assert rep["loss"] == pytest.approx(l1 + e1, rel=1e-9)
    assert l1 + e1 < 0.2 * (l0 + e0)
    assert e1 < e0


@pytest.mark.slow
def test_pair_term_full_size_3d():
    """2^24 points in the unit cube, harmonic spheres of diameter 0.8 (L^3/N)^(1/3) (the 3D
    workload): FP32 against FP64 on the GPU, and the gradient at 64 sampled points against the
    oracle's direct sums over all points."""
    import torch
    from paper_2305_15693_gb300 import fresco
    wl = inputs.workload("powerlaw3d_n2p24_chi03_f32")
    pts_np = wl.points()
    N = wl.n_points
    sigma = 0.8 * (wl.box ** 3 / N) ** (1 / 3)
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.PairTerm(wl.box, 3, N, sigma, 1.0, 2.0, "f32") as p32:
        e32, g32 = p32.energy_grad(pts)
    with fresco.PairTerm(wl.box, 3, N, sigma, 1.0, 2.0, "f64") as p64:
        e64, g64 = p64.energy_grad(pts.double())
    torch.cuda.synchronize()
    assert abs(e32.item() - e64.item()) <= 1e-5 * e64.item()
    gerr = float(torch.linalg.vector_norm(g32.double() - g64) / torch.linalg.vector_norm(g64))
    assert gerr <= TOL["f32"]["grad"]
    sel = np.sort(inputs.rng(3).choice(N, 64, replace=False))
    _, g_or = oracle.pair_energy_grad(pts_np, sigma, 1.0, 2.0, box=wl.box, sel=sel,
                                      want_energy=False)
    assert rel_l2(g64.cpu().numpy()[sel], g_or) <= 1e-11
