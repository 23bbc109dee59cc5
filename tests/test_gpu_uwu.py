"""GPU parity of the weight-gradient form on a uniform grid (UwU, Methods "Analytical
gradients"): loss and dL/dc through the C ABI against the oracle's direct sums on the same grid
weights, in 2D and 3D, FP64 and FP32. Both transforms are exact DFTs of the grid, so the FP64
path agrees with the oracle to rounding."""

import numpy as np
import pytest

import oracle
from paper_2305_15693_gb300 import inputs

from _parity import rel_l2

pytestmark = pytest.mark.gpu

BAR = {"f64": {"loss": 1e-11, "grad": 1e-10}, "f32": {"loss": 1e-5, "grad": 1e-4}}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2305_15693_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()


def _problem(shape, K, seed):
    g = inputs.rng(seed)
    c = g.standard_normal(int(np.prod(shape)))
    mask = inputs.ball_mask(K, len(shape))
    S0 = 0.5 * g.random(mask.shape[0])
    W = 0.5 + g.random(mask.shape[0])
    return c, mask, S0, W


@pytest.mark.parametrize("shape,K,precision", [((48, 40), 11, "f64"), ((48, 40), 11, "f32"),
                                               ((20, 18, 16), 5, "f64"), ((20, 18, 16), 5, "f32")])
def test_uwu_matches_oracle(shape, K, precision):
    import torch
    from paper_2305_15693_gb300 import fresco
    c, mask, S0, W = _problem(shape, K, 90 + len(shape))
    dt = torch.float64 if precision == "f64" else torch.float32
    c_dev = torch.from_numpy(c.reshape(shape[::-1])).to("cuda", dt)
    c_used = c_dev.double().cpu().numpy().reshape(-1)          # the values the GPU sees
    with fresco.Uwu(shape, mask, S0, W, precision) as u:
        for _ in range(2):
            loss, grad = u.loss_grad(c_dev)
        torch.cuda.synchronize()
        loss = loss.item()
        grad = grad.double().cpu().numpy().reshape(-1)
    l_o, g_o, _, _ = oracle.weight_loss_grad(oracle.grid_points(shape), c_used, mask, S0, W)
    assert abs(loss - l_o) <= BAR[precision]["loss"] * abs(l_o)
    assert rel_l2(grad, g_o) <= BAR[precision]["grad"]
    # L is invariant under c -> a c, so sum_m c_m dL/dc_m = 0
    assert abs(np.dot(c_used, grad)) <= 10 * BAR[precision]["grad"] * np.linalg.norm(c_used) * \
        np.linalg.norm(grad)


def test_uwu_rejects_aliased_or_zero_wavevectors():
    from paper_2305_15693_gb300 import fresco
    m = np.array([[3, 1], [12, 0]], dtype=np.int32)      # |n_x| = 12 = M_0 / 2 aliases
    with pytest.raises(fresco.FrescoError) as e:
        fresco.fresco_uwu_plan((24, 20), m, np.zeros(2), np.ones(2))
    assert e.value.status == fresco.FRESCO_ERR_ARG
    with pytest.raises(fresco.FrescoError) as e:
        fresco.fresco_uwu_plan((24, 20), np.array([[0, 0]], dtype=np.int32), [0.0], [1.0])
    assert e.value.status == fresco.FRESCO_ERR_ARG
