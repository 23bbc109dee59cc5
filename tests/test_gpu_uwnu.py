"""GPU parity of the weight-gradient form with constraints at real frequencies (UwNU, Methods
"Analytical gradients": one type-2 NUFFT for S, one type-1 NUFFT for the gradient): S, the loss
and dL/dc through the C ABI against the oracle's direct sums on the same grid weights, in 2D and
3D, FP64 and FP32, with odd and even grids and frequencies beyond +-M/2; integer frequencies
reproduce the exact-transform UwU plan."""

import numpy as np
import pytest

import oracle
from paper_2305_15693_gb300 import inputs

from _parity import rel_l2

pytestmark = pytest.mark.gpu

# FP64 at tolerance 1e-12 and FP32 at 1e-6 (the FP32 bars of the point form)
BAR = {"f64": {"S": 1e-10, "loss": 1e-10, "grad": 1e-9},
       "f32": {"S": 1e-5, "loss": 1e-5, "grad": 1e-4}}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2305_15693_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()


def _problem(shape, n_k, seed, span):
    g = inputs.rng(seed)
    c = g.standard_normal(int(np.prod(shape)))
    nu = g.uniform(-span, span, (n_k, len(shape)))
    S0 = 0.5 * g.random(n_k)
    W = 0.5 + g.random(n_k)
    return c, nu, S0, W


def _run(shape, c, nu, S0, W, precision, **kw):
    import torch
    from paper_2305_15693_gb300 import fresco
    dt = torch.float64 if precision == "f64" else torch.float32
    c_dev = torch.from_numpy(c.reshape(shape[::-1])).to("cuda", dt)
    c_used = c_dev.double().cpu().numpy().reshape(-1)          # the values the GPU sees
    with fresco.Uwnu(shape, nu, S0, W, precision, **kw) as u:
        for _ in range(2):
            loss, grad = u.loss_grad(c_dev)
        S = u.S()
        torch.cuda.synchronize()
        info = u.info
        out = (loss.item(), grad.double().cpu().numpy().reshape(-1),
               S.double().cpu().numpy(), info)
    return c_used, out


@pytest.mark.parametrize("shape,precision", [((48, 40), "f64"), ((48, 40), "f32"),
                                             ((45, 33), "f32"), ((45, 33), "f64"),
                                             ((20, 18, 16), "f64"), ((20, 18, 16), "f32"),
                                             ((15, 12, 9), "f32")])
def test_uwnu_matches_oracle(shape, precision):
    c, nu, S0, W = _problem(shape, 160, 60 + sum(shape), span=0.7 * max(shape))
    c_used, (loss, grad, S, info) = _run(shape, c, nu, S0, W, precision)
    assert all(info["n_fine"][a] >= 2 * shape[a] for a in range(len(shape)))
    l_o, g_o, S_o, _ = oracle.weight_loss_grad_k(oracle.grid_points(shape), c_used,
                                                  2.0 * np.pi * nu, S0, W)
    bar = BAR[precision]
    assert rel_l2(S, S_o) <= bar["S"]
    assert abs(loss - l_o) <= bar["loss"] * abs(l_o)
    assert rel_l2(grad, g_o) <= bar["grad"]
    # L is invariant under c -> a c, so sum_m c_m dL/dc_m = 0
    assert abs(np.dot(c_used, grad)) <= 10 * bar["grad"] * np.linalg.norm(c_used) * \
        np.linalg.norm(grad)


@pytest.mark.parametrize("upsample", [1.25, 2.5])
def test_uwnu_other_oversampling(upsample):
    shape = (36, 30)
    c, nu, S0, W = _problem(shape, 90, 71, span=20.0)
    c_used, (loss, grad, S, info) = _run(shape, c, nu, S0, W, "f32", upsample=upsample)
    assert info["n_fine"][0] >= upsample * shape[0]
    l_o, g_o, S_o, _ = oracle.weight_loss_grad_k(oracle.grid_points(shape), c_used,
                                                  2.0 * np.pi * nu, S0, W)
    assert rel_l2(S, S_o) <= BAR["f32"]["S"]
    assert abs(loss - l_o) <= BAR["f32"]["loss"] * abs(l_o)
    assert rel_l2(grad, g_o) <= BAR["f32"]["grad"]


def test_integer_frequencies_reproduce_the_uniform_plan():
    """At integer nu (|nu_a| < M_a / 2, no +-n pair) the NUFFT form gives the UwU quantities,
    which that plan computes with exact transforms."""
    import torch
    from paper_2305_15693_gb300 import fresco
    shape = (32, 28)
    g = inputs.rng(77)
    mask = inputs.ball_mask(9, 2)
    mask = mask[(mask[:, 0] > 0) | ((mask[:, 0] == 0) & (mask[:, 1] > 0))]   # one of each +-n
    S0 = 0.5 * g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    c = torch.from_numpy(g.standard_normal(shape[::-1])).to("cuda", torch.float64)
    with fresco.Uwu(shape, mask, S0, W, "f64") as u:
        l1, g1 = u.loss_grad(c)
    c_used, (l2, g2, _, _) = _run(shape, c.cpu().numpy().reshape(-1), mask.astype(np.float64),
                                  S0, W, "f64")
    assert l2 == pytest.approx(l1.item(), rel=1e-10)
    assert rel_l2(g2, g1.cpu().numpy().reshape(-1)) <= 1e-9


def test_uwnu_rejects_bad_arguments():
    from paper_2305_15693_gb300 import fresco
    nu = np.array([[0.5, 1.5]])
    with pytest.raises(fresco.FrescoError):
        fresco.Uwnu((1, 8), nu, [0.0], [1.0])                     # grid too small
    with pytest.raises(fresco.FrescoError):
        fresco.Uwnu((8, 8), np.array([[np.nan, 0.0]]), [0.0], [1.0])
    with pytest.raises(fresco.FrescoError):
        fresco.Uwnu((8, 8), nu, [0.0], [-1.0])                    # negative weight
    with pytest.raises(fresco.FrescoError):
        fresco.Uwnu((8, 8), nu, [0.0], [1.0], upsample=4.0)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_uwnu_crowded_tile_and_seam(precision):
    """Constraints packed into one tile of the fine grid (a tile list longer than a block's
    threads), at integer and half-integer frequencies (supports that start on tile boundaries),
    and at frequencies whose support wraps across the grid's periodic seam."""
    shape = (64, 48)
    g = inputs.rng(81)
    crowd = 3.0 + 0.05 * g.random((700, 2))
    seam = np.array([[0.0, 0.0], [0.5, -0.5], [32.0, 24.0], [-32.0, -24.0], [31.9, 0.1],
                     [-0.01, 23.99], [-31.99, -23.9]])
    lattice = g.integers(-40, 40, (100, 2)).astype(np.float64) / 2
    nu = np.concatenate([crowd, seam, lattice])
    S0 = 0.5 * g.random(nu.shape[0])
    W = 0.5 + g.random(nu.shape[0])
    c = g.standard_normal(shape[0] * shape[1])
    c_used, (loss, grad, S, info) = _run(shape, c, nu, S0, W, precision)
    l_o, g_o, S_o, _ = oracle.weight_loss_grad_k(oracle.grid_points(shape), c_used,
                                                  2.0 * np.pi * nu, S0, W)
    bar = BAR[precision]
    assert rel_l2(S, S_o) <= bar["S"]
    assert abs(loss - l_o) <= bar["loss"] * abs(l_o)
    assert rel_l2(grad, g_o) <= bar["grad"]


def test_uwnu_profile_and_launch_count():
    import torch
    from paper_2305_15693_gb300 import fresco
    shape = (40, 36)
    c, nu, S0, W = _problem(shape, 50, 5, span=15.0)
    c_dev = torch.from_numpy(c.reshape(shape[::-1])).to("cuda", torch.float32)
    with fresco.Uwnu(shape, nu, S0, W, "f32") as u:
        n0 = u.launch_count()
        u.profile(True)
        u.loss_grad(c_dev)
        u.loss_grad(c_dev)
        st = u.profile_read()
        assert u.launch_count() - n0 == 14          # seven kernels per evaluation
        u.profile(False)
        u.loss_grad(c_dev, want_grad=False)
        assert u.launch_count() - n0 == 19          # five without the gradient
        torch.cuda.synchronize()
        assert u.profile_read()["interp"][1] == 0   # nothing recorded while off
    for name in ("type2", "interp", "spread", "type1"):
        assert st[name][1] == 2 and st[name][0] > 0.0
    assert st["point_spread"][1] == 0 and st["point_interp"][1] == 0


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_uwnu_repeats_bitwise(precision):
    """The spread adds in fixed point, so every output of a repeated call is bitwise equal."""
    import torch
    from paper_2305_15693_gb300 import fresco
    shape = (96, 80)
    c, nu, S0, W = _problem(shape, 3000, 83, span=40.0)
    dt = torch.float64 if precision == "f64" else torch.float32
    c_dev = torch.from_numpy(c.reshape(shape[::-1])).to("cuda", dt)
    with fresco.Uwnu(shape, nu, S0, W, precision) as u:
        l1, g1 = u.loss_grad(c_dev)
        S1 = u.S()
        l1, g1 = l1.clone(), g1.clone()
        l2, g2 = u.loss_grad(c_dev)
        S2 = u.S()
        torch.cuda.synchronize()
    assert l1.item() == l2.item()
    assert torch.equal(g1, g2) and torch.equal(S1, S2)
