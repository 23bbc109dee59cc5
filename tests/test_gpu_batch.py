"""GPU parity of the batched ensemble path (many independent 2D problems in one set of launches):
every instance's loss and gradient against the oracle and against a plan of its own, CUDA-graph
replay against ordinary evaluation, and the 512-instance ensemble (N log-uniform in [1e3, 1e5],
chi uniform in [0.1, 0.5], seed 7) at full size."""

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


def _problem(ens):
    masks = ens.masks()
    S0s, Ws = ens.targets(masks)
    return masks, S0s, Ws


def _batch_eval(ens, masks, S0s, Ws, pts_np, **kw):
    import torch
    from paper_2305_15693_gb300 import fresco
    dt = torch.float64 if ens.dtype == "f64" else torch.float32
    pts = torch.from_numpy(pts_np).to("cuda", dt)
    kw.setdefault("grad_mode", ens.grad_mode)
    with fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws, precision=ens.dtype, tol=ens.tol,
                      upsample=ens.upsample, **kw) as b:
        losses, grad = b.loss_grad(pts)
        torch.cuda.synchronize()
        assert b.status() == fresco.FRESCO_OK
        return losses.cpu().numpy(), grad.double().cpu().numpy(), b.first, b.info


def _mixed_ensemble(dtype):
    # uneven sizes, boxes and radii, a single point and K = 1 included
    ens = inputs.ensemble(7, 200, 4000, 0.1, 0.5, 11, dtype, box_lo=0.7, box_hi=2.0,
                          tol=1e-12 if dtype == "f64" else 1e-6)
    ens.n_points[0], ens.K[0] = 1, 3
    ens.n_points[1], ens.K[1] = 37, 1
    return ens


@pytest.mark.parametrize("dtype,grad_mode", [("f64", "direct"), ("f32", "direct"),
                                             ("f64", "kderiv"), ("f32", "kderiv")])
def test_batch_matches_oracle_per_instance(dtype, grad_mode):
    ens = _mixed_ensemble(dtype)
    masks, S0s, Ws = _problem(ens)
    pts = ens.points()
    losses, grad, first, info = _batch_eval(ens, masks, S0s, Ws, pts, grad_mode=grad_mode)
    assert info["total_points"] == sum(ens.n_points)
    tol = TOL[dtype]
    for i in range(ens.n_inst):
        p = pts[first[i]:first[i + 1]]
        l_o, g_o, _, _ = oracle.loss_grad(p, masks[i], S0s[i], Ws[i], box=ens.boxes[i])
        assert abs(losses[i] - l_o) <= tol["loss"] * abs(l_o), i
        if ens.n_points[i] > 1:
            assert rel_l2(grad[first[i]:first[i + 1]], g_o) <= tol["grad"], i
        else:
            assert np.max(np.abs(grad[first[i]:first[i + 1]])) < 1e-3


def test_batch_matches_single_plans():
    """Same instances through fresco_plan one at a time: equal up to the batch's larger grids."""
    import torch
    from paper_2305_15693_gb300 import fresco
    ens = inputs.ensemble(9, 500, 20000, 0.1, 0.5, 5, "f64", tol=1e-12)
    masks, S0s, Ws = _problem(ens)
    pts = ens.points()
    losses, grad, first, info = _batch_eval(ens, masks, S0s, Ws, pts)
    assert 1 <= info["n_classes"] <= ens.n_inst
    for i in range(ens.n_inst):
        p = torch.from_numpy(pts[first[i]:first[i + 1]]).cuda()
        with fresco.Plan(ens.boxes[i], masks[i], S0s[i], Ws[i], p.shape[0], precision="f64",
                         tol=1e-12) as plan:
            l1, g1 = plan.loss_grad(p)
            assert abs(losses[i] - l1.item()) <= 1e-10 * abs(l1.item())
            assert rel_l2(grad[first[i]:first[i + 1]], g1.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("grad_mode", ["direct", "kderiv"])
def test_graph_replay_equals_eager_and_follows_the_points(grad_mode):
    import torch
    from paper_2305_15693_gb300 import fresco
    ens = inputs.ensemble(24, 300, 30000, 0.1, 0.5, 3, "f32")
    masks, S0s, Ws = _problem(ens)
    pts_np = ens.points()
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws, precision="f32",
                      grad_mode=grad_mode) as b:
        l_e, g_e = b.loss_grad(pts)
        l_e, g_e = l_e.clone(), g_e.clone()
        losses = torch.empty(ens.n_inst, dtype=torch.float64, device="cuda")
        grad = torch.empty_like(pts)
        b.capture(pts, losses, grad)
        for _ in range(3):
            b.launch()
        torch.cuda.synchronize()
        # spreading accumulates in fixed point and every sum runs in a fixed order: replays are
        # bit-identical to ordinary evaluation
        assert torch.equal(losses, l_e)
        assert torch.equal(grad, g_e)
        shifted = np.ascontiguousarray(pts_np + np.float32(0.013))
        pts.copy_(torch.from_numpy(shifted))
        b.launch()
        l_n, g_n = b.loss_grad(pts)
        torch.cuda.synchronize()
        assert torch.equal(losses, l_n) and torch.equal(grad, g_n)
        assert not torch.equal(l_n, l_e)
        assert b.status() == fresco.FRESCO_OK


def test_batch_rejects_bad_arguments():
    from paper_2305_15693_gb300 import fresco
    m = inputs.ball_mask(3, 2)
    s0, w = inputs.stealthy_target(m), inputs.unit_weights(m)
    with pytest.raises(fresco.FrescoError) as e:
        fresco.fresco_batch_plan([1.0, 1.0], [10, 0], [m, m], [s0, s0], [w, w])
    assert e.value.status == fresco.FRESCO_ERR_ARG
    m3 = inputs.ball_mask(2, 3)
    with pytest.raises(fresco.FrescoError) as e:
        fresco.fresco_batch_plan([1.0], [10], [m3], [inputs.stealthy_target(m3)],
                                 [inputs.unit_weights(m3)])
    assert e.value.status == fresco.FRESCO_ERR_UNSUPPORTED


@pytest.mark.slow
def test_ensemble_512_full_size():
    """The 512-instance ensemble: FP32 batch against the FP64 batch for every instance, the FP64
    batch against the oracle on the smallest instances and on sampled gradient rows of large
    ones."""
    e32 = inputs.ensemble_workload("stealthy2d_ens512_n1e3to1e5_f32")
    e64 = inputs.ensemble_workload("stealthy2d_ens512_n1e3to1e5_f64")
    masks, S0s, Ws = _problem(e32)
    pts32 = e32.points()
    l32, g32, first, info = _batch_eval(e32, masks, S0s, Ws, pts32)
    l64, g64, _, _ = _batch_eval(e64, masks, S0s, Ws, pts32.astype(np.float64))
    assert info["total_points"] == sum(e32.n_points)
    for i in range(e32.n_inst):
        sl = slice(first[i], first[i + 1])
        assert abs(l32[i] - l64[i]) <= TOL["f32"]["loss"] * l64[i], i
        assert rel_l2(g32[sl], g64[sl]) <= TOL["f32"]["grad"], i
    order = np.argsort(e32.n_points)
    for i in list(order[:3]):
        sl = slice(first[i], first[i + 1])
        l_o, g_o, _, _ = oracle.loss_grad(pts32[sl], masks[i], S0s[i], Ws[i])
        assert abs(l64[i] - l_o) <= TOL["f64"]["loss"] * l_o
        assert rel_l2(g64[sl], g_o) <= TOL["f64"]["grad"]
    i = int(order[len(order) // 2])
    sl = slice(first[i], first[i + 1])
    sel = np.sort(inputs.rng(5).choice(e32.n_points[i], 32, replace=False))
    l_o, g_o, _, _ = oracle.loss_grad(pts32[sl], masks[i], S0s[i], Ws[i], sel=sel)
    assert abs(l64[i] - l_o) <= TOL["f64"]["loss"] * l_o
    assert rel_l2(g64[sl][sel], g_o) <= TOL["f64"]["grad"]


# ---- L-BFGS over the ensemble ----------------------------------------------------------------

def test_batch_lbfgs_follows_reference_per_instance():
    """Each instance's first iterations on the device follow the numpy L-BFGS driven by the
    oracle (FP64), although instances accept, backtrack and stop at different steps."""
    import torch
    from paper_2305_15693_gb300 import fresco
    from _lbfgs_ref import lbfgs as lbfgs_ref
    ens = inputs.ensemble(5, 40, 400, 0.2, 0.5, 21, "f64", box_lo=0.8, box_hi=1.5, tol=1e-12)
    masks, S0s, Ws = _problem(ens)
    pts_np = ens.points()
    iters, m, step = 8, 5, 2e-3
    pts = torch.from_numpy(pts_np).cuda()
    with fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws, precision="f64",
                      tol=1e-12) as b, \
            fresco.BatchLBFGS(b, max_iter=iters, history=m, max_step=step) as opt:
        reps = opt.run(pts, 2000)
        first = b.first
    x = pts.cpu().numpy()
    for i in range(ens.n_inst):
        sl = slice(first[i], first[i + 1])

        def fg(p, i=i):
            loss, grad, _, _ = oracle.loss_grad(p, masks[i], S0s[i], Ws[i], box=ens.boxes[i])
            return loss, grad

        x_ref, trace = lbfgs_ref(fg, pts_np[sl], iters, m=m, max_step=step)
        assert reps[i]["iterations"] == iters and reps[i]["status"] == 3, (i, reps[i])
        assert reps[i]["loss"] == pytest.approx(trace[-1], rel=1e-8), i
        assert rel_l2(x[sl] - pts_np[sl], x_ref - pts_np[sl]) < 1e-6, i


def test_batch_lbfgs_lowers_every_instance_and_reports_true_losses():
    import torch
    from paper_2305_15693_gb300 import fresco
    ens = inputs.ensemble(48, 500, 20000, 0.1, 0.5, 8, "f32")
    masks, S0s, Ws = _problem(ens)
    pts = torch.from_numpy(ens.points()).cuda()
    with fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws, precision="f32") as b:
        l0, _ = b.loss_grad(pts, want_grad=False)
        l0 = l0.cpu().numpy()
        with fresco.BatchLBFGS(b) as opt:
            reps = opt.run(pts, 150)
        l1, _ = b.loss_grad(pts, want_grad=False)
        torch.cuda.synchronize()
        l1 = l1.cpu().numpy()
        assert b.status() == fresco.FRESCO_OK
    for i, r in enumerate(reps):
        assert r["evaluations"] <= 150
        assert r["loss"] == l1[i], i            # the reported loss is the loss at the points
        assert l1[i] < 0.1 * l0[i], (i, l0[i], l1[i])


def test_autotuner_times_every_candidate_and_keeps_the_fastest():
    import torch
    from paper_2305_15693_gb300 import fresco, tune
    ens = inputs.ensemble(16, 300, 5000, 0.1, 0.5, 4, "f32")
    masks, S0s, Ws = _problem(ens)
    pts = torch.from_numpy(ens.points()).cuda()
    best, table = tune.autotune_batch(ens.boxes, ens.n_points, masks, S0s, Ws, pts,
                                      upsamples=(1.5, 2.0), tiles=(32, 64), reps=3, warmup=1)
    assert len(table) == 4
    timed = [r for r in table if r["ms"] is not None]
    assert timed and all(r["ms"] > 0 for r in timed)
    assert best["ms"] == min(r["ms"] for r in timed)
    assert {r["width"] for r in timed if r["upsample"] == 1.5} == {8}   # eps 1e-6 at sigma 1.5
    # the chosen configuration is an ordinary batch plan with the same results as the default
    with fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws, upsample=best["upsample"],
                      tile=best["tile"]) as b, \
            fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws) as ref:
        l1, g1 = b.loss_grad(pts)
        l2, g2 = ref.loss_grad(pts)
        torch.cuda.synchronize()
        np.testing.assert_allclose(l1.cpu().numpy(), l2.cpu().numpy(), rtol=TOL["f32"]["loss"])
        assert rel_l2(g1.double().cpu().numpy(), g2.double().cpu().numpy()) <= TOL["f32"]["grad"]
