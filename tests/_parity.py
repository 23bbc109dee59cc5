"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI and measure its
error against the oracle on identical inputs."""

import numpy as np

# Tolerances. FP32 bars are the stated targets for the single-precision path (relative L2 of rho
# over the mask <= 1e-5, loss relative error <= 1e-5, gradient relative L2 <= 1e-4). For the FP64
# path rho must reach 1e-11; the loss is quadratic in S (relative error <= 2 |dS/S| <= 4 |drho/rho|
# times the conditioning |S / (S - S0)|), hence 1e-10, and the gradient carries one more factor of
# rho and the interpolation error, hence 1e-9.
TOL = {
    "f32": {"rho": 1e-5, "loss": 1e-5, "grad": 1e-4},
    "f64": {"rho": 1e-11, "loss": 1e-10, "grad": 1e-9},
}


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / den) if den > 0 else float(
        np.linalg.norm(a.ravel()))


def gpu_eval(points, mask, S0, W, box=1.0, precision="f64", tol=0.0, tile=None, upsample=2.0,
             want_rho=True, grad_mode=0):
    """One loss+gradient evaluation through the C ABI; returns (loss, grad, rho, S, status, info)."""
    import torch
    from paper_2305_15693_gb300 import fresco
    dt = torch.float64 if precision == "f64" else torch.float32
    pts = torch.from_numpy(np.ascontiguousarray(points)).to("cuda", dt)
    plan = fresco.Plan(box, mask, S0, W, pts.shape[0], precision=precision, tol=tol, tile=tile,
                       upsample=upsample, grad_mode=grad_mode)
    try:
        loss, grad = plan.loss_grad(pts)
        rho = S = None
        if want_rho:
            r, S = plan.rho_S()
            rho = (r[:, 0].double() + 1j * r[:, 1].double()).cpu().numpy()
            S = S.double().cpu().numpy()
        torch.cuda.synchronize()
        st = plan.status()
        out = (float(loss.item()), grad.double().cpu().numpy(), rho, S, st, plan.info)
    finally:
        plan.close()
    return out


def compare(points, mask, S0, W, box=1.0, precision="f64", tol=0.0, tile=None, upsample=2.0,
            grad_mode=0):
    """GPU vs oracle errors on the same inputs."""
    import oracle
    loss_g, grad_g, rho_g, S_g, st, info = gpu_eval(points, mask, S0, W, box, precision, tol,
                                                    tile, upsample, grad_mode=grad_mode)
    loss_o, grad_o, S_o, rho_o = oracle.loss_grad(points, mask, S0, W, box=box)
    return {
        "status": st,
        "rho": rel_l2(rho_g, rho_o),
        "S": rel_l2(S_g, S_o),
        "loss": abs(loss_g - loss_o) / abs(loss_o) if loss_o != 0 else abs(loss_g),
        "grad": rel_l2(grad_g, grad_o),
        "loss_gpu": loss_g,
        "loss_oracle": loss_o,
        "info": info,
    }
