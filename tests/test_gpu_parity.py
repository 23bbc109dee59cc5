"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

Sizes are small enough for the oracle's direct sums yet span many spread/interp tiles, ragged
tile widths and periodic wrap-around."""

import numpy as np
import pytest

import oracle
from paper_2305_15693_gb300 import inputs

from _parity import TOL, compare, gpu_eval, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2305_15693_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()


def _assert_within(err, precision, what=("rho", "loss", "grad")):
    assert err["status"] == 0, err
    for k in what:
        assert err[k] <= TOL[precision][k], (k, err[k], TOL[precision][k], err)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_stealthy_2d_n1024_k20(precision):
    wl = inputs.workload("stealthy2d_n1024_k20_f64")
    pts = inputs.uniform_points(wl.n_points, 2, wl.seed,
                                np.float64 if precision == "f64" else np.float32)
    mask = wl.mask()
    S0, W = wl.targets(mask)
    err = compare(pts, mask, S0, W, precision=precision)
    _assert_within(err, precision)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_power_law_3d_with_box_and_weights(precision):
    g = inputs.rng(31)
    dt = np.float64 if precision == "f64" else np.float32
    box = np.array([1.0, 1.3, 0.8])
    pts = (inputs.uniform_points(3000, 3, 32, np.float64) * box).astype(dt)
    mask = inputs.ball_mask(7, 3)
    S0 = inputs.power_law_target(mask, 7)
    W = 0.5 + g.random(mask.shape[0])
    err = compare(pts, mask, S0, W, box=box, precision=precision)
    _assert_within(err, precision)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_asymmetric_mask_duplicates_and_wrap(precision):
    """One-sided entries, +-n pairs with different S0/W, duplicate rows, a non-square box and
    coordinates far outside it (the library wraps them periodically)."""
    g = inputs.rng(41)
    dt = np.float64 if precision == "f64" else np.float32
    box = np.array([2.0, 0.5])
    full = inputs.ball_mask(16, 2)
    keep = g.random(full.shape[0]) < 0.6
    mask = np.vstack([full[keep], full[keep][:50]]).astype(np.int32)
    S0 = 3.0 * g.random(mask.shape[0])
    W = g.random(mask.shape[0])
    pts = ((g.random((1500, 2)) * 6.0 - 3.0) * box).astype(dt)
    err = compare(pts, mask, S0, W, box=box, precision=precision)
    _assert_within(err, precision)


@pytest.mark.parametrize("tile", [(10, 7), (5, 5), (84, 84), (13, 29)])
def test_tilings_with_ragged_edges(tile):
    pts = inputs.uniform_points(2048, 2, seed=3)
    mask = inputs.ball_mask(20, 2)
    g = inputs.rng(4)
    S0 = g.random(mask.shape[0])
    W = np.ones(mask.shape[0])
    err = compare(pts, mask, S0, W, precision="f64", tile=tile)
    _assert_within(err, "f64")
    assert err["info"]["n_tiles"][0] >= 1


@pytest.mark.parametrize("sigma,precision,tol,bar", [
    (1.25, "f64", 1e-9, {"rho": 1e-8, "loss": 1e-7, "grad": 1e-6}),
    (2.5, "f32", 0.0, TOL["f32"]),
    (1.5, "f32", 0.0, TOL["f32"]),
    (1.25, "f32", 0.0, TOL["f32"]),
])
def test_other_upsampling_factors(sigma, precision, tol, bar):
    """Lower oversampling trades grid size for kernel width; the accuracy follows the tolerance
    (at sigma = 1.25 the FP64 default 1e-12 would need w = 20 > 16, so 1e-9 is asked for)."""
    pts = inputs.uniform_points(1024, 2, 9, np.float64 if precision == "f64" else np.float32)
    mask = inputs.ball_mask(15, 2)
    S0 = np.full(mask.shape[0], 0.5)
    W = np.ones(mask.shape[0])
    err = compare(pts, mask, S0, W, precision=precision, upsample=sigma, tol=tol)
    assert err["status"] == 0
    for k in ("rho", "loss", "grad"):
        assert err[k] <= bar[k], (k, err)


def test_boundary_coordinates_and_tiny_problem():
    eps = np.finfo(np.float32).eps
    pts = np.array([[0.0, 0.0], [1.0 - eps / 2, 0.5], [-0.0, 1.0], [3.0, -2.0 + 1e-7],
                    [0.25, 1.0 - eps]], dtype=np.float32)
    mask = inputs.ball_mask(1, 2)
    S0 = np.array([0.5, 1.0, 1.5, 2.0])
    W = np.array([1.0, 2.0, 0.5, 1.0])
    err = compare(pts, mask, S0, W, precision="f32")
    _assert_within(err, "f32")


def test_single_point_has_unit_S_and_no_force():
    pts = np.array([[0.3, 0.7]])
    mask = inputs.ball_mask(6, 2)
    S0 = np.zeros(mask.shape[0])
    W = np.ones(mask.shape[0])
    loss, grad, rho, S, st, _ = gpu_eval(pts, mask, S0, W, precision="f64")
    assert st == 0
    np.testing.assert_allclose(S, 1.0, rtol=1e-11)
    assert loss == pytest.approx(mask.shape[0], rel=1e-11)
    assert np.max(np.abs(grad)) < 1e-9


def test_lattice_ground_state_is_stealthy_on_gpu():
    pts = inputs.lattice_points(32, 2, offset=0.25)
    mask = inputs.ball_mask(20, 2)
    loss, grad, rho, S, st, _ = gpu_eval(pts, mask, np.zeros(mask.shape[0]),
                                         np.ones(mask.shape[0]), precision="f64")
    assert st == 0
    assert loss < 1e-18 * 1024 ** 2
    assert np.max(np.abs(grad)) < 1e-8


def test_repeat_split_and_scaled_backward():
    import torch
    from paper_2305_15693_gb300 import fresco
    pts_np = inputs.uniform_points(4096, 2, 5, np.float32)
    mask = inputs.ball_mask(24, 2)
    g = inputs.rng(6)
    S0 = g.random(mask.shape[0])
    W = np.ones(mask.shape[0])
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.Plan(1.0, mask, S0, W, pts.shape[0]) as plan:
        l1, g1 = plan.loss_grad(pts)
        r1, _ = plan.rho_S()
        l2, g2 = plan.loss_grad(pts)          # zero regions of the spectra must survive a call
        r2, _ = plan.rho_S()
        l3 = plan.forward(pts)
        go = torch.tensor(2.5, dtype=torch.float64, device="cuda")
        g3 = plan.backward(go)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert plan.launch_count() > 0
    assert rel_l2(r2.cpu().numpy(), r1.cpu().numpy()) < 1e-6
    assert abs(l2.item() - l1.item()) <= 1e-6 * abs(l1.item())
    assert rel_l2(g2.cpu().numpy(), g1.cpu().numpy()) < 1e-5
    assert abs(l3.item() - l1.item()) <= 1e-6 * abs(l1.item())
    assert rel_l2(g3.cpu().numpy(), 2.5 * g1.cpu().numpy()) < 1e-5


def test_rho_in_caller_order_includes_conjugate_rows():
    pts = inputs.uniform_points(700, 2, 8)
    mask = inputs.ball_mask(9, 2)
    perm = inputs.rng(1).permutation(mask.shape[0])
    mask = np.ascontiguousarray(mask[perm])
    S0 = np.zeros(mask.shape[0])
    W = np.ones(mask.shape[0])
    _, _, rho, S, st, _ = gpu_eval(pts, mask, S0, W, precision="f64")
    want = oracle.rho(pts, mask)
    assert st == 0
    assert rel_l2(rho, want) < 1e-11
    np.testing.assert_allclose(S, np.abs(want) ** 2 / 700, rtol=1e-10, atol=1e-12)


def test_nonfinite_coordinate_is_reported_and_cleared():
    import torch
    from paper_2305_15693_gb300 import fresco
    pts_np = inputs.uniform_points(256, 2, 2, np.float32)
    pts_np[17, 1] = np.nan
    mask = inputs.ball_mask(5, 2)
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.Plan(1.0, mask, np.zeros(mask.shape[0]), np.ones(mask.shape[0]), 256) as plan:
        plan.loss_grad(pts)
        assert plan.status() == fresco.FRESCO_ERR_NONFINITE
        pts[17, 1] = 0.5
        plan.loss_grad(pts)
        assert plan.status() == 0


def test_host_buffer_entry_point_matches_device_call():
    import torch
    from paper_2305_15693_gb300 import fresco
    pts_np = inputs.uniform_points(3000, 2, 12, np.float32)
    mask = inputs.ball_mask(18, 2)
    S0 = np.full(mask.shape[0], 0.2)
    W = np.ones(mask.shape[0])
    with fresco.Plan(1.0, mask, S0, W, 3000) as plan:
        loss_d, grad_d = plan.loss_grad(torch.from_numpy(pts_np).cuda())
        grad_h = np.empty_like(pts_np)
        loss_h = plan.loss_grad_host(pts_np, grad_h)
        torch.cuda.synchronize()
    assert loss_h == pytest.approx(loss_d.item(), rel=1e-6)
    assert rel_l2(grad_h, grad_d.cpu().numpy()) < 1e-5


def test_host_buffer_entry_point_in_chunks_is_bit_identical():
    """72 MB of points: the host copy runs as two unequal chunks (4 500 001 and 4 500 000 points),
    each binned while the other is in flight; the fixed-point spread makes the result independent
    of the order in which the points reach their sub-bins."""
    import torch
    from paper_2305_15693_gb300 import fresco
    N = 9_000_001
    pts_np = inputs.uniform_points(N, 2, 31, np.float32)
    mask = inputs.ball_mask(1000, 2)
    S0 = np.full(mask.shape[0], 0.2)
    W = np.ones(mask.shape[0])
    with fresco.Plan(1.0, mask, S0, W, N, grad_mode="kderiv") as plan:
        loss_d, grad_d = plan.loss_grad(torch.from_numpy(pts_np).cuda())
        grad_h = np.empty_like(pts_np)
        loss_h = plan.loss_grad_host(pts_np, grad_h)
        loss_h2 = plan.loss_grad_host(pts_np, grad_h)
        assert plan.status() == 0
    assert loss_h == loss_d.item() == loss_h2
    np.testing.assert_array_equal(grad_h, grad_d.cpu().numpy())


def test_bad_pointer_alignment_is_an_argument_error():
    import torch
    from paper_2305_15693_gb300 import fresco
    mask = inputs.ball_mask(4, 2)
    with fresco.Plan(1.0, mask, np.zeros(mask.shape[0]), np.ones(mask.shape[0]), 10) as plan:
        buf = torch.zeros(64, dtype=torch.float32, device="cuda")
        loss = torch.zeros((), dtype=torch.float64, device="cuda")
        with pytest.raises(fresco.FrescoError) as e:
            fresco.fresco_loss_grad(plan.handle, buf.data_ptr() + 4, loss, None)
        assert e.value.status == fresco.FRESCO_ERR_ARG


@pytest.mark.parametrize("dim,precision", [(2, "f32"), (2, "f64"), (3, "f32"), (3, "f64")])
def test_kernel_derivative_gradient_mode_matches_oracle(dim, precision):
    """The kderiv gradient mode (one real inverse transform of E / Psi, interpolated with the
    kernel derivative) against the oracle, on a non-square box with wrapped coordinates and
    ragged tiles."""
    from paper_2305_15693_gb300 import fresco
    g = inputs.rng(70 + dim)
    dt = np.float64 if precision == "f64" else np.float32
    box = np.linspace(0.8, 1.3, dim)
    n = 3000 if dim == 2 else 2500
    pts = ((g.random((n, dim)) * 3.0 - 1.0) * box).astype(dt)
    mask = inputs.ball_mask(18 if dim == 2 else 6, dim)
    S0 = g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    err = compare(pts, mask, S0, W, box=box, precision=precision,
                  grad_mode=fresco.FRESCO_GRAD_KDERIV)
    assert err["info"]["grad_mode"] == fresco.FRESCO_GRAD_KDERIV
    _assert_within(err, precision)


@pytest.mark.parametrize("grad_mode", ["direct", "kderiv"])
@pytest.mark.parametrize("dim,precision", [(2, "f32"), (2, "f64"), (3, "f32"), (3, "f64")])
def test_odd_half_length_x_transform(dim, precision, grad_mode):
    """Fine grids whose x length is twice an odd number (90 in 2D, 42 in 3D): the real transforms
    along x run as complex transforms of odd length M = n_f / 2, where the pair (k, M - k) never
    meets itself, and the half spectrum must still match the oracle."""
    from paper_2305_15693_gb300 import fresco
    g = inputs.rng(90 + dim)
    dt = np.float64 if precision == "f64" else np.float32
    n = 2000
    pts = g.random((n, dim)).astype(dt)
    mask = inputs.ball_mask(22 if dim == 2 else 10, dim)
    S0 = g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    mode = fresco.FRESCO_GRAD_KDERIV if grad_mode == "kderiv" else fresco.FRESCO_GRAD_DIRECT
    err = compare(pts, mask, S0, W, precision=precision, grad_mode=mode)
    nf = err["info"]["n_fine"][0]
    assert nf == (90 if dim == 2 else 42) and (nf // 2) % 2 == 1
    _assert_within(err, precision)


def test_kernel_derivative_mode_follows_the_incoming_gradient():
    """backward(g_out) scales the kderiv gradient by g_out, as in the direct mode."""
    import torch
    from paper_2305_15693_gb300 import fresco
    pts_np = inputs.uniform_points(4000, 2, 71, np.float32)
    mask = inputs.ball_mask(25, 2)
    S0 = inputs.power_law_target(mask, 25)
    W = np.ones(mask.shape[0])
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.Plan(1.0, mask, S0, W, 4000, grad_mode="kderiv") as plan:
        loss, g1 = plan.loss_grad(pts)
        plan.forward(pts)
        gout = torch.tensor(-2.5, dtype=torch.float64, device="cuda")
        g2 = plan.backward(gout)
        torch.cuda.synchronize()
        np.testing.assert_allclose(g2.cpu().numpy(), -2.5 * g1.cpu().numpy(), rtol=1e-6,
                                   atol=1e-6 * float(g1.abs().max()))


@pytest.mark.parametrize("dim,precision", [(2, "f32"), (2, "f64"), (3, "f32")])
def test_clustered_points_overflow_the_tile_lists(dim, precision):
    """Most points in one small cluster: the tiles there receive far more points than the spread
    list sized from the mean density holds, so spreading takes the float-atomic path straight
    from the point lists; the result must not change."""
    g = inputs.rng(99 + dim)
    dt = np.float64 if precision == "f64" else np.float32
    n_cl, n_bg = (16000, 2000) if dim == 2 else (12000, 1500)
    cluster = 0.37 + 0.01 * g.standard_normal((n_cl, dim))
    pts = np.vstack([cluster, g.random((n_bg, dim))]).astype(dt)
    mask = inputs.ball_mask(20 if dim == 2 else 6, dim)
    S0 = g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    err = compare(pts, mask, S0, W, precision=precision)
    _assert_within(err, precision)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_one_crowded_tile_falls_back_to_compact_binning(dim, precision):
    """Uniform points plus a tight clump: one tile receives more points than the direct binning
    form's fixed capacity per tile (the uniform density's mean plus eight standard deviations), so
    the evaluation bins again in the compact form; both the device and the host-buffer entry point
    must match the oracle."""
    import torch
    from paper_2305_15693_gb300 import fresco
    g = inputs.rng(123 + dim)
    dt = np.float64 if precision == "f64" else np.float32
    n_bg, n_cl = (20000, 4000) if dim == 2 else (15000, 6000)
    pts = np.vstack([g.random((n_bg, dim)), 0.61 + 0.002 * g.random((n_cl, dim))]).astype(dt)
    mask = inputs.ball_mask(20 if dim == 2 else 6, dim)
    S0 = g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    err = compare(pts, mask, S0, W, precision=precision)
    _assert_within(err, precision)
    with fresco.Plan(1.0, mask, S0, W, pts.shape[0], precision=precision) as plan:
        loss_d, grad_d = plan.loss_grad(torch.from_numpy(pts).cuda())
        grad_h = np.empty_like(pts)
        loss_h = plan.loss_grad_host(pts, grad_h)
        assert plan.status() == 0
        loss_d, grad_d = float(loss_d.item()), grad_d.cpu().numpy()
    if precision == "f32" and dim == 2:
        # fixed-point spreading: the same sums whatever order the points are binned in
        assert loss_h == loss_d
        np.testing.assert_array_equal(grad_h, grad_d)
    else:
        # the crowded tile spreads with float atomics (FP64 plans; in 3D a z-column segment with
        # more than 16384 / 3 points a tile), whose sums depend on the order: equal to rounding
        tol = 1e-12 if precision == "f64" else 1e-5
        assert abs(loss_h - loss_d) <= tol * abs(loss_d)
        assert np.linalg.norm(grad_h - grad_d) <= tol * np.linalg.norm(grad_d)
