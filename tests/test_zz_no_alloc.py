"""fresco_loss_noalloc: the loss computed without any device allocation, for callers that cannot
allocate device memory when they evaluate (a fixed memory budget set at start-up, or another
allocator that owns the device memory). Its result must equal the loss that a plan computes
(fresco_forward) from the same structure factor, on every call, including two calls in a row
that reuse the library's shared scratch array.

This file is named so that pytest collects it last."""

import numpy as np
import pytest

from paper_2305_15693_gb300 import inputs

from _parity import TOL


@pytest.fixture(scope="module")
def fr():
    from paper_2305_15693_gb300 import _build
    _build.build()
    from paper_2305_15693_gb300 import fresco
    fresco.load()
    return fresco


def test_oversize_and_bad_arguments_are_rejected_before_device_work(fr):
    fake = 256  # never dereferenced: the size / argument checks come first
    with pytest.raises(fr.FrescoError) as e:
        fr.fresco_loss_noalloc("f64", fr.FRESCO_LOSS_NOALLOC_MAX_ROWS + 1, fake, fake, fake, fake)
    assert e.value.status == fr.FRESCO_ERR_UNSUPPORTED
    with pytest.raises(fr.FrescoError) as e:
        fr.fresco_loss_noalloc("f64", 0, fake, fake, fake, fake)
    assert e.value.status == fr.FRESCO_ERR_ARG
    with pytest.raises(fr.FrescoError) as e:
        fr.fresco_loss_noalloc("f32", 10, None, fake, fake, fake)
    assert e.value.status == fr.FRESCO_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_loss_matches_the_plan_loss_on_two_calls(fr, precision):
    import torch
    N, K = 20000, 60
    dt = np.float64 if precision == "f64" else np.float32
    pts_np = inputs.uniform_points(N, 2, seed=21, dtype=dt)
    mask = inputs.ball_mask(K, 2)
    g = inputs.rng(22)
    S0 = 2.0 * g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    pts = torch.from_numpy(pts_np).cuda()
    with fr.Plan(1.0, mask, S0, W, N, precision=precision) as plan:
        loss_plan = plan.forward(pts)
        _, S = plan.rho_S()
        S0_d = torch.from_numpy(S0).cuda()
        W_d = torch.from_numpy(W).cuda()
        stream = torch.cuda.current_stream()
        results = []
        for _ in range(2):
            out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
            fr.fresco_loss_noalloc(precision, mask.shape[0], S, S0_d, W_d, out, stream)
            torch.cuda.synchronize()
            results.append(out.item())
        want = loss_plan.item()
    tol = TOL[precision]["loss"]
    for got in results:
        assert np.isfinite(got)
        assert abs(got - want) <= tol * abs(want), (got, want)
    assert results[0] == results[1]          # fixed-order reduction: bitwise repeatable


_WARMUP_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2305_15693_gb300 import fresco
torch.cuda.set_device(0)
g = np.random.default_rng(5)
n = 50000
S_h, S0_h, W_h = g.random(n) * 3.0, g.random(n) * 2.0, 0.5 + g.random(n)
want = float(np.sum(W_h * (S_h - S0_h) ** 2))
for precision, dt in (("f64", torch.float64), ("f32", torch.float32)):
    S = torch.from_numpy(S_h).to(dt).cuda()
    S0, W = torch.from_numpy(S0_h).cuda(), torch.from_numpy(W_h).cuda()
    ref = float(np.sum(W_h * (S.double().cpu().numpy() - S0_h) ** 2))
    outs = []
    for _ in range(2):
        out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        fresco.fresco_loss_noalloc(precision, n, S, S0, W, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        outs.append(out.item())
    assert outs[0] == outs[1], outs
    assert abs(outs[0] - ref) <= 1e-12 * abs(ref), (precision, outs[0], ref)
print("WARMUP_OK", want)
"""


@pytest.mark.gpu
def test_warm_up_call_before_any_plan_in_a_fresh_process(fr):
    """A caller under a fixed memory budget makes its first (warm-up) call at start-up, before it
    has made any plan: in a fresh process that first call loads the library's scratch array and
    must already give the loss, on two calls in a row."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _WARMUP_SCRIPT, root], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "WARMUP_OK" in r.stdout, r.stdout + r.stderr
