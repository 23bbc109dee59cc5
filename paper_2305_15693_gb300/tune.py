"""Autotuner for batch plans: picks the fine-grid oversampling (and with it the kernel width the
tolerance needs) and the spread/interpolation tile edge by timing CUDA-graph replays of each
candidate on the caller's own ensemble.

A lower oversampling means smaller FFTs but a wider kernel (more spread/interp work per point);
the tile edge trades shared-memory halo overhead against the number of blocks. Which wins
depends on the mix of N and K in the ensemble, so the choice is measured, not modelled.
Timing uses CUDA events on the batch's stream around single graph launches; nothing here
computes a loss itself.
"""

from __future__ import annotations

import numpy as np

from . import fresco

DEFAULT_UPSAMPLES = (1.5, 2.0)
DEFAULT_TILES = (24, 32, 48, 64, 96)


def time_graph(batch, points, reps=10, warmup=3):
    """Per-launch device times (ms) of `reps` replays of one captured evaluation."""
    import torch
    losses = torch.empty(batch.n_inst, dtype=torch.float64, device=points.device)
    grad = torch.empty_like(points)
    batch.capture(points, losses, grad)
    s = batch.stream
    for _ in range(warmup):
        fresco.fresco_batch_graph_launch(batch.handle)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(s)
        fresco.fresco_batch_graph_launch(batch.handle)
        b.record(s)
    torch.cuda.synchronize()
    st = batch.status()
    if st != fresco.FRESCO_OK:
        raise fresco.FrescoError(st, "batch evaluation")
    return [a.elapsed_time(b) for a, b in evs]


def autotune_batch(boxes, n_points, masks, S0s, Ws, points, precision="f32", tol=0.0,
                   upsamples=DEFAULT_UPSAMPLES, tiles=DEFAULT_TILES, reps=10, warmup=3,
                   grad_mode="direct"):
    """Time every (upsample, tile) candidate; returns (best, table). `best` holds the keyword
    arguments (upsample, tile) for fresco.Batch and its median time; `table` lists every
    candidate with its median ms (None where the plan is unsupported)."""
    table = []
    for sigma in upsamples:
        for t in tiles:
            row = {"upsample": float(sigma), "tile": int(t), "ms": None}
            try:
                b = fresco.Batch(boxes, n_points, masks, S0s, Ws, precision=precision, tol=tol,
                                 upsample=sigma, tile=(t, t), grad_mode=grad_mode)
            except fresco.FrescoError as e:
                row["error"] = fresco.status_string(e.status)
                table.append(row)
                continue
            try:
                ms = time_graph(b, points, reps, warmup)
                row["ms"] = float(np.median(ms))
                row["width"] = fresco.fresco_batch_get_info(b.handle, 0)["width"]
                row["device_bytes"] = b.info["device_bytes"]
            finally:
                b.close()
            table.append(row)
    ok = [r for r in table if r["ms"] is not None]
    if not ok:
        raise RuntimeError("no candidate configuration could be planned")
    best = min(ok, key=lambda r: r["ms"])
    return {"upsample": best["upsample"], "tile": (best["tile"], best["tile"]),
            "ms": best["ms"]}, table
