"""Parity at the full workload sizes, in the launch configuration the bench uses.

The oracle's direct sums cost O(N N_K) for the loss and gradient, out of reach at these sizes
(up to 1.2e16 pair terms), so each workload is checked on what can be computed one by one or
holds at any size:
* rho at seeded samples of mask rows, each an O(N) direct sum in the oracle (FP32 bar 1e-5);
* the FP32 loss and gradient against the all-FP64 GPU path (itself pinned to the oracle at
  sizes the oracle finishes), loss 1e-5 and gradient 1e-4;
* the directional derivative of the FP64 loss along a random direction (central difference)
  against the FP64 gradient, and the same for FP32 with a wider step.
"""

import numpy as np
import pytest

import oracle
from paper_2305_15693_gb300 import inputs

from _parity import TOL, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WORKLOADS = ["stealthy2d_n1e6_chi045_f32", "powerlaw3d_n2p24_chi03_f32", "peaked2d_n1e8_chi03_f32"]
# rho rows checked against the oracle's direct sums (each an O(N) sum: ~2.7 s on 16 host cores at
# 1e8 points, so the 1e8 workload's 64 rows take about three minutes)
N_SAMPLE_ROWS = {"stealthy2d_n1e6_chi045_f32": 128, "powerlaw3d_n2p24_chi03_f32": 64,
                 "peaked2d_n1e8_chi03_f32": 64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2305_15693_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()


@pytest.mark.parametrize("name", WORKLOADS)
def test_full_size_workload(name):
    import torch
    from paper_2305_15693_gb300 import fresco
    wl = inputs.workload(name)
    pts_np = wl.points()
    mask = wl.mask()
    S0, W = wl.targets(mask)
    N = wl.n_points
    pts = torch.from_numpy(pts_np).cuda()

    with fresco.Plan(wl.box, mask, S0, W, N, precision="f32", tol=wl.tol,
                     upsample=wl.upsample, grad_mode=wl.grad_mode) as plan:
        loss32, grad32 = plan.loss_grad(pts)
        rho32, _ = plan.rho_S()
        torch.cuda.synchronize()
        assert plan.status() == 0
        loss32 = loss32.item()
        grad32 = grad32.double()
        rng = inputs.rng(2)
        rows = np.sort(rng.choice(mask.shape[0], N_SAMPLE_ROWS[name], replace=False))
        rho32_s = rho32[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    del rho32
    torch.cuda.empty_cache()

    # rho at sampled rows against the oracle's direct sums: relative L2 over the rows, and no
    # single row off by more than 1e-4 of the rows' RMS |rho| (|rho| ~ sqrt(N) for these points)
    want = oracle.rho(pts_np, mask[rows], box=wl.box)
    got = rho32_s[:, 0] + 1j * rho32_s[:, 1]
    assert rel_l2(got, want) <= TOL["f32"]["rho"], rel_l2(got, want)
    rms = np.sqrt(np.mean(np.abs(want) ** 2))
    assert np.max(np.abs(got - want)) <= 1e-4 * rms, np.max(np.abs(got - want)) / rms

    # FP32 against the plain all-FP64 GPU path (direct gradient, oversampling 2) on the same points
    pts64 = pts.double()
    with fresco.Plan(wl.box, mask, S0, W, N, precision="f64", upsample=2.0) as p64:
        loss64, grad64 = p64.loss_grad(pts64)
        torch.cuda.synchronize()
        assert p64.status() == 0
        loss64 = loss64.item()
        assert abs(loss32 - loss64) <= TOL["f32"]["loss"] * abs(loss64)
        gerr = float(torch.linalg.vector_norm(grad32 - grad64) / torch.linalg.vector_norm(grad64))
        assert gerr <= TOL["f32"]["grad"], gerr

        # directional derivative of the FP64 loss along the normalised FP64 gradient: the central
        # difference must reproduce |grad L| (step 1e-5 box lengths keeps rounding noise of L,
        # ~1e-13 relative, well under the 1e-4 bar)
        v = grad64 / torch.linalg.vector_norm(grad64)
        h = 1e-5 * wl.box
        lp, _ = p64.loss_grad(pts64 + h * v, want_grad=False)
        lm, _ = p64.loss_grad(pts64 - h * v, want_grad=False)
        fd = (lp.item() - lm.item()) / (2 * h)
        dd = float(torch.linalg.vector_norm(grad64))
        assert abs(fd - dd) <= 1e-4 * dd, (fd, dd, loss64)
