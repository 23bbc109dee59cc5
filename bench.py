#!/usr/bin/env python3
"""Throughput of one FReSCo loss+gradient evaluation on the GPU (points/s), FP32 against the
all-FP64 GPU path, with per-stage CUDA-event timing, the HBM roofline of the dominant kernel,
an end-to-end figure through the host-buffer C entry point, and the CPU oracle as baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Default workload: 2D, N = 1e8 uniform FP32 points, ball mask |n| <= K with chi = 0.3 (K = 6180),
peaked ring target of 10 Gaussian peaks of height N/10, W = 1. Under torchrun each rank runs an
independent replica of the workload on its own GPU (no data-path collective; weak scaling); the
barrier and the max over ranks only frame the timing.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "peaked2d_n1e8_chi03_f32"
METRIC = "points/s per loss+grad eval (FP32 vs FP64 GPU, 2D N=1e8); % HBM roofline"
L2_BYTES = 129 * 2 ** 20


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.rows = []
        self.proc = None
        self.device_id = device_id
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.device_id:
            cmd += ["-i", self.device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # the timed region starts once the sampler is running (its first row has arrived), so
        # that even a region of a few tenths of a second is sampled every 50 ms
        t0 = time.perf_counter()
        while not self.rows and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _device_selector(dev_index: int) -> str | None:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------------------------------------
# algorithmic bytes per launch of every stage (the minimum each stage must move through HBM)

def stage_bytes(info: dict, n_points: int, esize: int) -> dict:
    d = info["dim"]
    nf = info["n_fine"][:d]
    cells = int(np.prod(nf))
    rows = cells // nf[0]
    half = nf[0] // 2 + 1
    kx = info["k_max"][0]
    hc_row = 2 * kx + 2
    pd = 4 if d == 3 else 2           # words per packed coordinate
    n_pipes = 1 if d == 2 else 2
    nrep = info["n_rep"]
    N = n_points
    c2 = 2 * esize                    # complex element
    out = {
        "sort": N * d * esize + N * pd * esize + 4 * N,
        "spread": N * pd * esize + cells * esize,
        "fft_fwd": cells * esize + rows * half * c2,
        "mask": nrep * (4 * d + 2 * esize + c2 + n_pipes * 2 * c2),
        "loss": 0,
        "fft_inv": n_pipes * (rows * hc_row * c2 + cells * c2),
        "interp": n_pipes * cells * c2 + N * pd * esize + 4 * N + N * d * esize,
    }
    if info.get("grad_mode", 0) == 1:
        # one scalar half spectrum [kx + 1][rows] in, one real grid out and back in
        out["mask"] = nrep * (4 * d + 2 * esize + c2 + c2)
        out["fft_inv"] = rows * (kx + 1) * c2 + cells * esize
        out["interp"] = cells * esize + N * pd * esize + 4 * N + N * d * esize
    return out


def load_peaks():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------------------------

def max_over_ranks(value: float, dist_on: bool, device=None) -> float:
    """Largest value over all ranks (the slowest replica sets the step time)."""
    if not dist_on:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(n_points: int, world: int, t_step: float) -> float:
    """Whole-job points/s when each of `world` ranks evaluates its own n_points-point replica in
    t_step seconds (weak scaling: no data crosses ranks)."""
    return world * n_points / t_step


def make_inputs(wl):
    t0 = time.time()
    pts = wl.points()
    mask = wl.mask()
    S0, W = wl.targets(mask)
    log("inputs: N=%d K=%d N_K=%d (%.1f s)" % (wl.n_points, wl.K, mask.shape[0], time.time() - t0))
    return pts, mask, S0, W


def time_device(plan, pts, steps, warmup, dist_on, profile=True):
    """Device-resident timing: W untimed steps, then K steps bracketed by barrier + sync."""
    import torch
    stream = torch.cuda.current_stream()
    loss = torch.empty((), dtype=torch.float64, device=pts.device)
    grad = torch.empty_like(pts)
    from paper_2305_15693_gb300 import fresco
    for _ in range(warmup):
        fresco.fresco_loss_grad(plan.handle, pts, loss, grad)
    torch.cuda.synchronize()
    if profile:
        plan.profile_read()           # drop warm-up records
        plan.profile(True)
    n0 = plan.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist_on:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        fresco.fresco_loss_grad(plan.handle, pts, loss, grad)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist_on:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = plan.launch_count() - n0
    stages = plan.profile_read() if profile else None
    plan.profile(False)
    st = plan.status()
    if st != 0:
        raise RuntimeError("device status after timing: %d" % st)
    return ms, launches, stages, float(loss.item()), grad


def time_e2e(plan, pts_np, steps, warmup):
    """Through fresco_loss_grad_host on pinned host buffers: H2D of the points, evaluation,
    D2H of the loss and the gradient, every step."""
    import torch
    h_pts = torch.from_numpy(pts_np).pin_memory()
    h_grad = torch.empty(pts_np.shape, dtype=h_pts.dtype).pin_memory()
    a_pts = h_pts.numpy()
    a_grad = h_grad.numpy()
    for _ in range(warmup):
        plan.loss_grad_host(a_pts, a_grad)
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.loss_grad_host(a_pts, a_grad)
    dt = (time.perf_counter() - t0) / steps
    return dt, a_pts.nbytes, a_grad.nbytes + 8


def oracle_sample_rows(threads: int) -> int:
    """Mask rows per timed oracle sample: the oracle hands rows to its threads four at a time, so
    four rows per host thread keep every core busy."""
    return 4 * max(1, threads)


def cpu_baseline(pts_np, mask, box, budget_s=12.0, seed=2, min_rows=None):
    """The oracle timed on the host cores on a bounded sample: rho at a seeded sample of mask rows
    (at least four per host thread, more while they fit the budget) over all N points (direct
    sums). A full evaluation costs rho over all N_K rows plus the gradient over all N points x N_K
    rows: about 2 N N_K pair terms at the same per-term cost."""
    import oracle
    N = pts_np.shape[0]
    n_k = mask.shape[0]
    threads = oracle.threads()
    if min_rows is None:
        min_rows = oracle_sample_rows(threads)
    g = np.random.Generator(np.random.Philox(seed))
    r64 = np.ascontiguousarray(pts_np, dtype=np.float64)
    probe = mask[g.choice(n_k, min(n_k, min_rows), replace=False)]
    t0 = time.perf_counter()
    oracle.rho(r64, probe, box)
    t_probe = max(time.perf_counter() - t0, 1e-6)
    per_row = t_probe / probe.shape[0]
    n_s = int(max(min(min_rows, n_k), min(4 * min_rows, n_k, budget_s / per_row)))
    rows = np.sort(g.choice(n_k, n_s, replace=False))
    sample = mask[rows]
    t0 = time.perf_counter()
    rho = oracle.rho(r64, sample, box)
    t = time.perf_counter() - t0
    rate = N * n_s / t                                  # pair terms / s
    t_eval = 2.0 * N * n_k / rate
    used = min(threads, (n_s + 3) // 4)
    return ({"value": N / t_eval, "unit": "points/s", "cores": used, "kind": "oracle",
             "sample": "rho at %d of %d mask rows over all %d points (%.1f s); full evaluation "
                       "extrapolated as 2*N*N_K pair terms at the measured %.3e terms/s"
                       % (n_s, n_k, N, t, rate),
             "seconds_per_eval_extrapolated": t_eval}, rows, rho)


def rho_error_report(got, want, rows_n, K, n_bins=4):
    """rho of the GPU against the oracle at sampled mask rows: relative L2 over the rows, the
    largest per-row error |got - want| relative to the rows' RMS |want| (|rho| ~ sqrt(N) for
    uniform points, so a single row's own |rho| can be near zero), and the relative L2 per bin of
    |n| / K."""
    got = np.asarray(got)
    want = np.asarray(want)
    err = np.abs(got - want)
    rms = float(np.sqrt(np.mean(np.abs(want) ** 2)))
    r = np.linalg.norm(np.asarray(rows_n, dtype=np.float64), axis=1) / float(K)
    edges = np.linspace(0.0, 1.0, n_bins + 1)
    bins = []
    for b in range(n_bins):
        sel = (r > edges[b]) & (r <= edges[b + 1]) if b else (r <= edges[b + 1])
        if np.any(sel):
            bins.append({"n_over_K": [float(edges[b]), float(edges[b + 1])],
                         "rows": int(sel.sum()),
                         "rel_l2": float(np.linalg.norm(got[sel] - want[sel]) /
                                         np.linalg.norm(want[sel]))})
    return {"rows": int(got.size),
            "rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
            "max_row_err_over_rms": float(err.max() / rms) if rms > 0 else None,
            "by_n_over_K": bins}


def smem_peaks(device="cuda"):
    """Conflict-free shared-memory 32-bit atomic adds and loads per second, measured now on this
    GPU (fresco_smem_peak)."""
    import torch
    from paper_2305_15693_gb300 import fresco
    sink = torch.zeros(8 * torch.cuda.get_device_properties(device).multi_processor_count,
                       dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream()
    return {"atomic_add": fresco.fresco_smem_peak(fresco.FRESCO_SMEM_ATOMIC_ADD, sink, stream),
            "load": fresco.fresco_smem_peak(fresco.FRESCO_SMEM_LOAD, sink, stream)}


def smem_rooflines(per_stage: dict, n_points: int, dim: int, width: int, peaks: dict) -> dict:
    """Spread and interpolation against the shared-memory pipe that binds them: every point costs
    w^d 32-bit atomic adds (spread) or w^d 32-bit loads (interpolation) of shared memory."""
    ops = float(n_points) * width ** dim
    out = {}
    for stage, op in (("spread", "atomic_add"), ("interp", "load")):
        if stage not in per_stage or op not in peaks:
            continue
        rate = ops / (per_stage[stage]["ms"] * 1e-3)
        out[stage] = {"op": "shared 32-bit " + op.replace("_", " "), "ops_per_launch": ops,
                      "achieved_ops_per_s": rate, "peak_ops_per_s": peaks[op],
                      "frac": round(rate / peaks[op], 4),
                      "peak_source": "fresco_smem_peak, measured in this run (conflict-free)"}
    return out


# ---------------------------------------------------------------------------------------------

def run_reference(args, wl, rank, world):
    """The oracle as the reference arm: each step is one bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    pts, mask, S0, W = make_inputs(wl)
    r64 = np.ascontiguousarray(pts, dtype=np.float64)
    g = np.random.Generator(np.random.Philox(3))
    N, n_k = pts.shape[0], mask.shape[0]
    n_s = min(n_k, max(int(args.ref_rows), oracle_sample_rows(oracle.threads())))
    for _ in range(args.warmup):
        oracle.rho(r64, mask[g.choice(n_k, n_s, replace=False)], wl.box)
    times = []
    for _ in range(args.steps):
        sample = mask[g.choice(n_k, n_s, replace=False)]
        t0 = time.perf_counter()
        oracle.rho(r64, sample, wl.box)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    rate = N * n_s / t
    t_eval = 2.0 * N * n_k / rate
    value = N / t_eval
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n_points": N, "K": wl.K, "n_modes": n_k,
                   "parallelism": "replicas"},
        # ms_per_step is the measured time of one step (the bounded sample); a full evaluation at
        # the measured pair-term rate would take this long:
        "ms_per_eval_extrapolated": 1e3 * t_eval,
        "cpu_baseline": {"value": value, "unit": "points/s",
                         "cores": min(oracle.threads(), (n_s + 3) // 4), "kind": "oracle",
                         "sample": "per step: rho at %d seeded mask rows over all %d points by "
                                   "direct sums (four rows per host thread); evaluation "
                                   "extrapolated as 2*N*N_K pair terms" % (n_s, N)},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# ensembles: many independent 2D problems per evaluation (configurations/s)

ENS_METRIC = ("configurations/s per loss+grad eval of a 512-instance 2D ensemble "
              "(N log-uniform in [1e3, 1e5]); p50/p99 ms per evaluation")


def ensemble_inputs(ens):
    t0 = time.time()
    masks = ens.masks()
    S0s, Ws = ens.targets(masks)
    pts = ens.points()
    log("ensemble: %d instances, %d points, %d modes (%.1f s)" % (
        ens.n_inst, pts.shape[0], sum(m.shape[0] for m in masks), time.time() - t0))
    return pts, masks, S0s, Ws


def ensemble_cpu_rate(ens, pts_np, masks, budget_s=12.0, seed=4):
    """Oracle pair terms per second on the host cores, from rho at sampled mask rows of a few
    seeded instances; a full ensemble evaluation is sum_i 2 N_i N_K,i such terms."""
    import oracle
    g = np.random.Generator(np.random.Philox(seed))
    first = np.concatenate([[0], np.cumsum(ens.n_points)])
    picks = g.choice(ens.n_inst, 3, replace=False)
    terms, t = 0.0, 0.0
    for i in picks:
        r64 = np.ascontiguousarray(pts_np[first[i]:first[i + 1]], dtype=np.float64)
        n_s = max(2, min(masks[i].shape[0], 64))
        rows = masks[i][g.choice(masks[i].shape[0], n_s, replace=False)]
        t0 = time.perf_counter()
        oracle.rho(r64, rows, ens.boxes[i])
        t += time.perf_counter() - t0
        terms += r64.shape[0] * n_s
        if t > budget_s:
            break
    rate = terms / t
    total = sum(2.0 * ens.n_points[i] * masks[i].shape[0] for i in range(ens.n_inst))
    return rate, total, [int(i) for i in picks]


def run_ensemble(args, ens, rank, world, local_rank, dist_on):
    import torch
    from paper_2305_15693_gb300 import fresco, tune
    pts_np, masks, S0s, Ws = ensemble_inputs(ens)
    pts = torch.from_numpy(pts_np).cuda()
    n_inst, n_tot = ens.n_inst, pts_np.shape[0]
    esize = 4 if ens.dtype == "f32" else 8

    # ---- autotuned oversampling and tile edge ----------------------------------------------
    table = None
    if args.tile:
        best = {"upsample": args.upsample or ens.upsample, "tile": tuple(args.tile[:2])}
    else:
        best, table = tune.autotune_batch(ens.boxes, ens.n_points, masks, S0s, Ws, pts,
                                          precision=ens.dtype, tol=ens.tol,
                                          grad_mode=ens.grad_mode)
        log("autotune: %s" % json.dumps(table))
    b = fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws, precision=ens.dtype, tol=ens.tol,
                     upsample=best["upsample"], tile=best["tile"], grad_mode=ens.grad_mode)
    infos = [fresco.fresco_batch_get_info(b.handle, i) for i in range(n_inst)]

    # launches of one evaluation (eager), then per-stage device time
    l0 = fresco.fresco_batch_info(b.handle)["launches"]
    b.loss_grad(pts)
    torch.cuda.synchronize()
    per_eval_launches = fresco.fresco_batch_info(b.handle)["launches"] - l0
    b.profile(True)
    for _ in range(3):
        b.loss_grad(pts)
    stages = b.profile_read()
    b.profile(False)

    # ---- graph replays: K evaluations, each bracketed by events -----------------------------
    losses = torch.empty(n_inst, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(pts)
    b.capture(pts, losses, grad)
    s = b.stream
    for _ in range(args.warmup):
        fresco.fresco_batch_graph_launch(b.handle)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(_device_selector(local_rank))
    clocks.start()
    if dist_on:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs[0].record(s)
    for k in range(args.steps):
        fresco.fresco_batch_graph_launch(b.handle)
        evs[k + 1].record(s)
    torch.cuda.synchronize()
    if dist_on:
        torch.distributed.barrier()
    clk = clocks.stop()
    per = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)])
    total_ms = evs[0].elapsed_time(evs[-1])
    t_step = max_over_ranks(total_ms / args.steps / 1e3, dist_on, "cuda")
    if b.status() != fresco.FRESCO_OK:
        raise RuntimeError("device status after timing")
    value = world * n_inst / t_step

    # ---- e2e: pinned host points in, losses and gradient out, every step --------------------
    h_pts = torch.from_numpy(pts_np).pin_memory()
    h_grad = torch.empty(pts_np.shape, dtype=h_pts.dtype).pin_memory()
    h_loss = torch.empty(n_inst, dtype=torch.float64).pin_memory()

    def e2e_step():
        with torch.cuda.stream(s):
            pts.copy_(h_pts, non_blocking=True)
            fresco.fresco_batch_graph_launch(b.handle)
            h_grad.copy_(grad, non_blocking=True)
            h_loss.copy_(losses, non_blocking=True)
        s.synchronize()
    e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    dt_e2e = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist_on, "cuda")

    # ---- one L-BFGS step per graph replay ----------------------------------------------------
    x = pts.clone()
    opt = fresco.BatchLBFGS(b)
    opt.start(x)
    opt.step(2)                       # the first step runs directly, the second is captured
    torch.cuda.synchronize()
    n_lb = max(args.steps, 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    opt.step(n_lb)
    e1.record(s)
    torch.cuda.synchronize()
    lbfgs_ms = e0.elapsed_time(e1) / n_lb
    reps, running = opt.read()
    opt.close()

    # ---- roofline of the slowest kernel stage ------------------------------------------------
    sb = {}
    for i in range(n_inst):
        for k, v in stage_bytes(infos[i], ens.n_points[i], esize).items():
            sb[k] = sb.get(k, 0) + v
    peaks = load_peaks() if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    per_stage = {}
    for name, (tot_ms, cnt) in stages.items():
        if cnt == 0:
            continue
        avg = tot_ms / cnt
        gbs = sb[name] / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        per_stage[name] = {"ms": round(avg, 4), "alg_bytes": int(sb[name]),
                           "GB/s": round(gbs, 1), "frac": round(gbs / hbm_peak, 4)}
    ours = {k: v for k, v in per_stage.items() if k in ("sort", "spread", "interp", "mask")}
    dom = max(ours, key=lambda k: ours[k]["ms"])
    roofline = {"bound": "hbm", "achieved": per_stage[dom]["GB/s"], "peak": hbm_peak,
                "unit": "GB/s", "frac": per_stage[dom]["frac"], "traffic": None, "kernel": dom,
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, burst)"}
    smem_roof = smem_rooflines(per_stage, n_tot, 2, infos[0]["width"], smem_peaks())
    b.close()

    # ---- all-FP64 batch on the same ensemble ------------------------------------------------
    f64 = None
    if ens.dtype == "f32" and args.f64_steps > 0:
        p64 = pts.double()
        b64 = fresco.Batch(ens.boxes, ens.n_points, masks, S0s, Ws, precision="f64", tol=1e-12,
                           upsample=best["upsample"], tile=best["tile"])
        ms64 = tune.time_graph(b64, p64, reps=args.f64_steps, warmup=3)
        b64.close()
        t64 = float(np.mean(ms64)) / 1e3
        f64 = {"value": world * n_inst / t64, "ms_per_step": 1e3 * t64,
               "speedup_f32_over_f64": t64 / t_step}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, terms, picks = ensemble_cpu_rate(ens, pts_np, masks)
        cpu = {"value": n_inst / (terms / rate), "unit": "configurations/s",
               "cores": __import__("oracle").threads(), "kind": "oracle",
               "sample": "rho at up to 64 sampled mask rows of instances %s by direct sums "
                         "(%.3e pair terms/s); a full ensemble evaluation extrapolated as "
                         "sum 2 N_i N_K,i = %.3e terms" % (picks, rate, terms)}

    if rank == 0:
        line = {
            "metric": ENS_METRIC, "value": value, "unit": "configurations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ens.dtype, "data": "synthetic",
            "config": {"workload": ens.name, "n_inst": n_inst, "total_points": n_tot,
                       "n_modes": int(sum(m.shape[0] for m in masks)), "tol": ens.tol,
                       "upsample": best["upsample"], "tile": list(best["tile"]),
                       "width": infos[0]["width"], "grad_mode": ens.grad_mode,
                       "autotune": table,
                       "parallelism": "replicas" if world > 1 else "single",
                       "timing": "CUDA-graph replay per evaluation",
                       "l2": "inputs larger than L2 (points %.0f MB + grids, %d MB L2)"
                             % (pts_np.nbytes / 1e6, L2_BYTES // 2 ** 20)},
            "latency_ms": {"p50": float(np.percentile(per, 50)),
                           "p99": float(np.percentile(per, 99)), "mean": float(per.mean())},
            "points_per_s": world * n_tot / t_step,
            "lbfgs_step_ms": lbfgs_ms,
            "lbfgs_after": {"steps": n_lb + 2, "running": running,
                            "iterations_median": float(np.median([r["iterations"]
                                                                  for r in reps]))},
            "roofline": roofline,
            "smem_roofline": smem_roof,
            "stages": per_stage,
            "fp64": f64,
            "cpu_baseline": cpu,
            "e2e": {"value": world * n_inst / dt_e2e, "unit": "configurations/s",
                    "h2d_bytes_per_step": int(pts_np.nbytes),
                    "d2h_bytes_per_step": int(pts_np.nbytes + 8 * n_inst),
                    "ms_per_step": 1e3 * dt_e2e},
            "clocks": clk,
            "gpu_launches": per_eval_launches * args.steps,
        }
        print(json.dumps(line), flush=True)


def run_reference_ensemble(args, ens, rank):
    """The oracle as the reference arm on an ensemble: each step is a bounded sample."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    pts_np, masks, _, _ = ensemble_inputs(ens)
    times, samples = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rate, terms, _ = ensemble_cpu_rate(ens, pts_np, masks, budget_s=5.0, seed=10 + k)
        if k >= args.warmup:
            times.append(terms / rate)
            samples.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = ens.n_inst / t
    line = {
        "impl": "reference", "metric": ENS_METRIC, "value": value, "unit": "configurations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(samples)), "ms_per_eval_extrapolated": 1e3 * t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": ens.name, "n_inst": ens.n_inst,
                   "total_points": int(sum(ens.n_points)), "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": "configurations/s", "cores": oracle.threads(),
                         "kind": "oracle",
                         "sample": "per step: rho at up to 64 sampled mask rows of 3 seeded "
                                   "instances; ensemble evaluation extrapolated as "
                                   "sum 2 N_i N_K,i pair terms"},
        "e2e": {"value": value, "unit": "configurations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_accuracy(args, wl):
    """Where the FP32 path's rho error comes from, on the same points: rho at seeded mask rows by
    the oracle's direct sums against (a) the FP32 plan, (b) an FP64 plan with the same grid and
    kernel width (FP64 arithmetic, the same truncation of the kernel), (c) the FP64 plan at
    tolerance 1e-12. (b) - oracle is the truncation error of the kernel at the plan's tolerance,
    (a) - (b) the FP32 arithmetic (fixed-point spread, FP32 transforms, deconvolution); both binned
    by |n| / K, where 1 / Psi grows toward the mask edge."""
    import torch
    import oracle
    from paper_2305_15693_gb300 import _build, fresco
    _build.build()
    oracle.build()
    pts_np, mask, S0, W = make_inputs(wl)
    N = wl.n_points
    g = np.random.Generator(np.random.Philox(args.accuracy_seed))
    rows = np.sort(g.choice(mask.shape[0], args.accuracy_rows, replace=False))
    sel = torch.from_numpy(rows).cuda()
    pts = torch.from_numpy(pts_np).cuda()
    out = {"workload": wl.name, "rows": int(len(rows)), "seed": args.accuracy_seed}

    def rho_at(precision, tol, upsample, width=0):
        p = pts if precision == wl.dtype else pts.double()
        with fresco.Plan(wl.box, mask, S0, W, N, precision=precision, tol=tol,
                         upsample=upsample, width=width, grad_mode=wl.grad_mode) as plan:
            plan.forward(p)
            r, _ = plan.rho_S()
            got = r[sel].double().cpu().numpy()
            info = plan.info
        return got[:, 0] + 1j * got[:, 1], info

    rho32, info32 = rho_at(wl.dtype, wl.tol, wl.upsample)
    rho64k, info64k = rho_at("f64", wl.tol, wl.upsample, width=info32["width"])
    rho64, info64 = rho_at("f64", 1e-12, 2.0)
    t0 = time.perf_counter()
    want = oracle.rho(np.ascontiguousarray(pts_np, dtype=np.float64), mask[rows], wl.box)
    out["oracle_seconds"] = time.perf_counter() - t0
    out["oracle_cores"] = oracle.threads()
    out["plans"] = {"f32": {"width": info32["width"], "n_fine": info32["n_fine"][:wl.dim]},
                    "f64_same_kernel": {"width": info64k["width"],
                                        "n_fine": info64k["n_fine"][:wl.dim]},
                    "f64_tol_1e-12": {"width": info64["width"],
                                      "n_fine": info64["n_fine"][:wl.dim]}}
    out["f32_vs_oracle"] = rho_error_report(rho32, want, mask[rows], wl.K)
    out["f64_same_kernel_vs_oracle"] = rho_error_report(rho64k, want, mask[rows], wl.K)
    out["f32_vs_f64_same_kernel"] = rho_error_report(rho32, rho64k, mask[rows], wl.K)
    out["f64_tol_1e-12_vs_oracle"] = rho_error_report(rho64, want, mask[rows], wl.K)
    out["bar"] = 1e-5
    print(json.dumps(out), flush=True)


NUWNU_METRIC = "points/s per NUwNU loss+grad eval (free boundaries, real wavevectors)"
UWNU_METRIC = "weights/s per UwNU loss+grad eval (grid weights, constraints at real frequencies)"


def constraint_side_bytes(dim: int, n_k: int, fine: int, esize: int, dq: bool) -> dict:
    """Algorithmic bytes of the constraint-side kernels of the UwNU / NUwNU plans, per launch:
    interp reads the fine grid once and each constraint's cell, position, target, weight
    (and deconvolution factor) and caller index, and writes its strength and S; spread reads
    each constraint's cell, position and strength and writes the fine grid once."""
    per_k_in = dim * 4 + dim * esize
    return {"interp": fine * 2 * esize + n_k * (per_k_in + 2 * esize + (esize if dq else 0) + 4
                                               + 3 * esize),
            "spread": n_k * (per_k_in + 2 * esize) + fine * 2 * esize}


def constraint_side_roofline(stages: dict, dim: int, n_k: int, fine: int, esize: int, dq: bool,
                             calls: int, workload: str) -> dict:
    """HBM roofline of the slower of the two constraint-side kernels (stage times from the
    plan's event timers, per evaluation; the interp stage also holds the partial-sum kernel).
    traffic: the ncu DRAM bytes of that kernel on this workload from profiles/traffic.json,
    when they were taken on the current sources of the weights-on-a-grid plans."""
    byt = constraint_side_bytes(dim, n_k, fine, esize, dq)
    peaks = load_peaks() if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    ms = {k: stages[k][0] / max(calls, 1) for k in ("interp", "spread")}
    dom = max(ms, key=ms.get)
    achieved = byt[dom] / (ms[dom] / 1e3) / 1e9
    traffic = None
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(path):
        with open(path) as f:
            entry = json.load(f).get(workload, {}).get(dom)
        try:
            current = _kernel_source_hash("uwnu")
        except OSError:
            current = None
        if entry and current and entry.get("source_hash") == current:
            traffic = entry.get("bytes_per_launch")
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": dom,
            "algorithmic_bytes": byt[dom], "ms_per_launch": ms[dom],
            "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs, burst)"}


def profile_stages(plan, steps: int, run) -> dict:
    """Per-stage device time of `steps` further evaluations, from the plan's event timers."""
    import torch
    plan.profile(True)
    plan.profile_read()
    for _ in range(steps):
        run()
    torch.cuda.synchronize()
    st = plan.profile_read()
    plan.profile(False)
    return st


def run_reference_free(args, fw, rank):
    """The oracle as the reference arm of a NUwNU workload: each step is the loss and gradient of
    a bounded sample of points (four per host thread x 64) at every wavevector."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    pts_np = fw.points()
    k = fw.wavevectors()
    S0, W = fw.targets(k)
    n_s = min(fw.n_points, 256 * oracle_sample_rows(oracle.threads()))
    times = []
    for step in range(args.warmup + args.steps):
        sub = pts_np[(step * n_s) % fw.n_points:][:n_s]
        t0 = time.perf_counter()
        oracle.loss_grad_k(sub, k, S0, W)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    rate = 2.0 * n_s * k.shape[0] / t
    t_eval = 2.0 * fw.n_points * k.shape[0] / rate
    value = fw.n_points / t_eval
    line = {
        "impl": "reference", "metric": NUWNU_METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
        "ms_per_eval_extrapolated": 1e3 * t_eval, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": fw.name, "n_points": fw.n_points, "n_modes": fw.n_k,
                   "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": oracle.threads(),
                         "kind": "oracle",
                         "sample": "per step: loss and gradient of %d points at all %d "
                                   "wavevectors by direct sums; evaluation extrapolated as "
                                   "2 N N_K pair terms" % (n_s, k.shape[0])},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_nuwnu(args, fw, rank, world, local_rank, dist_on):
    """Points at free positions with constraints at real wavevectors (fresco_nuwnu_*)."""
    import torch
    from paper_2305_15693_gb300 import fresco
    pts_np = fw.points()
    k = fw.wavevectors()
    S0, W = fw.targets(k)
    pts = torch.from_numpy(pts_np).cuda()
    plan = fresco.Nuwnu(fw.box, k, S0, W, fw.n_points, fw.dtype, tol=fw.tol,
                        upsample=fw.upsample)
    s = torch.cuda.current_stream()
    for _ in range(args.warmup):
        loss, grad = plan.loss_grad(pts)
    torch.cuda.synchronize()
    l0 = fresco.fresco_nuwnu_get_info(plan.handle)["launches"]
    clocks = ClockSampler(_device_selector(local_rank))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist_on:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.steps):
        loss, grad = plan.loss_grad(pts)
    e1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3, dist_on, "cuda")
    launches = fresco.fresco_nuwnu_get_info(plan.handle)["launches"] - l0
    if plan.status() != 0:
        raise RuntimeError("device status after timing")
    # e2e: pinned host points in, loss and gradient out, every step
    h_pts = torch.from_numpy(pts_np).pin_memory()
    h_grad = torch.empty(pts_np.shape, dtype=h_pts.dtype).pin_memory()
    h_loss = torch.empty((), dtype=torch.float64).pin_memory()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        pts.copy_(h_pts, non_blocking=True)
        loss, grad = plan.loss_grad(pts)
        h_grad.copy_(grad, non_blocking=True)
        h_loss.copy_(loss, non_blocking=True)
        s.synchronize()
    dt_e2e = max_over_ranks((time.perf_counter() - t0) / max(args.e2e_steps, 1), dist_on, "cuda")
    info = plan.info
    stages = profile_stages(plan, args.steps, lambda: plan.loss_grad(pts))
    esize = 4 if fw.dtype == "f32" else 8
    fine = int(np.prod(info["n_fine"][:fw.dim]))
    roof = constraint_side_roofline(stages, fw.dim, k.shape[0], fine, esize, True, args.steps,
                                    fw.name)
    # accuracy on a subsample the oracle finishes in seconds: 4096 points, all wavevectors
    acc = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        sub = pts_np[:4096]
        with fresco.Nuwnu(fw.box, k, S0, W, sub.shape[0], fw.dtype, tol=fw.tol,
                          upsample=fw.upsample) as p2:
            l_g, g_g = p2.loss_grad(torch.from_numpy(sub).cuda())
            S_g = p2.S().double().cpu().numpy()
            l_g, g_g = l_g.item(), g_g.double().cpu().numpy()
        t0 = time.perf_counter()
        l_o, g_o, S_o, _ = oracle.loss_grad_k(sub, k, S0, W)
        t_or = time.perf_counter() - t0
        acc = {"points": int(sub.shape[0]), "S_rel_l2": float(np.linalg.norm(S_g - S_o) /
                                                            np.linalg.norm(S_o)),
               "loss_rel": abs(l_g - l_o) / abs(l_o),
               "grad_rel_l2": float(np.linalg.norm(g_g - g_o) / np.linalg.norm(g_o))}
        rate = 2.0 * sub.shape[0] * k.shape[0] / t_or      # pair terms / s (rho and gradient)
        cpu = {"value": fw.n_points / (2.0 * fw.n_points * k.shape[0] / rate), "unit": "points/s",
               "cores": oracle.threads(), "kind": "oracle",
               "sample": "loss and gradient of the first 4096 points at all %d wavevectors "
                         "(%.1f s); full evaluation extrapolated as 2 N N_K pair terms"
                         % (k.shape[0], t_or)}
    plan.close()
    if rank == 0:
        line = {
            "metric": NUWNU_METRIC, "value": world * fw.n_points / t_step, "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": fw.dtype, "data": "synthetic",
            "config": {"workload": fw.name, "n_points": fw.n_points, "dim": fw.dim,
                       "n_modes": fw.n_k, "kmax": fw.kmax, "tol": fw.tol,
                       "upsample": fw.upsample, "width": info["width"],
                       "n_grid": info["n_grid"][:fw.dim], "n_fine": info["n_fine"][:fw.dim],
                       "parallelism": "replicas" if world > 1 else "single"},
            "accuracy_vs_oracle": acc,
            "stages_ms": {k_: round(v[0] / max(v[1], 1), 4) for k_, v in stages.items()},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": world * fw.n_points / dt_e2e, "unit": "points/s",
                    "h2d_bytes_per_step": int(pts_np.nbytes),
                    "d2h_bytes_per_step": int(pts_np.nbytes + 8), "ms_per_step": 1e3 * dt_e2e},
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)


def run_reference_field(args, fw, rank):
    """The oracle as the reference arm of a UwNU workload: each step is the loss and gradient of
    all weights at a bounded sample of the constraints (direct sums), extrapolated to all."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    c = fw.weights().astype(np.float64).reshape(-1)
    nu = fw.frequencies()
    S0, W = fw.targets(nu)
    pos = oracle.grid_points(fw.shape)
    n_s = min(fw.n_k, 8 * oracle_sample_rows(oracle.threads()))
    times = []
    for step in range(args.warmup + args.steps):
        sl = slice((step * n_s) % fw.n_k, (step * n_s) % fw.n_k + n_s)
        t0 = time.perf_counter()
        oracle.weight_loss_grad_k(pos, c, 2.0 * np.pi * nu[sl], S0[sl], W[sl])
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    rate = 2.0 * fw.n_weights * n_s / t
    t_eval = 2.0 * fw.n_weights * fw.n_k / rate
    value = fw.n_weights / t_eval
    line = {
        "impl": "reference", "metric": UWNU_METRIC, "value": value, "unit": "weights/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
        "ms_per_eval_extrapolated": 1e3 * t_eval, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": fw.name, "n_weights": fw.n_weights, "n_modes": fw.n_k,
                   "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": "weights/s", "cores": oracle.threads(),
                         "kind": "oracle",
                         "sample": "per step: loss and gradient of all %d weights at %d of the "
                                   "%d constraints by direct sums; evaluation extrapolated as "
                                   "2 M^d N_K pair terms" % (fw.n_weights, n_s, fw.n_k)},
        "e2e": {"value": value, "unit": "weights/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_uwnu(args, fw, rank, world, local_rank, dist_on):
    """Real weights on a uniform grid with constraints at real frequencies (fresco_uwnu_*)."""
    import torch
    from paper_2305_15693_gb300 import fresco
    c_np = fw.weights()
    nu = fw.frequencies()
    S0, W = fw.targets(nu)
    c = torch.from_numpy(c_np).cuda()
    plan = fresco.Uwnu(fw.shape, nu, S0, W, fw.dtype, tol=fw.tol, upsample=fw.upsample)
    s = torch.cuda.current_stream()
    for _ in range(args.warmup):
        loss, grad = plan.loss_grad(c)
    torch.cuda.synchronize()
    l0 = plan.launch_count()
    clocks = ClockSampler(_device_selector(local_rank))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist_on:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.steps):
        loss, grad = plan.loss_grad(c)
    e1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3, dist_on, "cuda")
    launches = plan.launch_count() - l0
    # e2e: pinned host weights in, loss and gradient out, every step
    h_c = torch.from_numpy(c_np).pin_memory()
    h_grad = torch.empty(c_np.shape, dtype=h_c.dtype).pin_memory()
    h_loss = torch.empty((), dtype=torch.float64).pin_memory()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        c.copy_(h_c, non_blocking=True)
        loss, grad = plan.loss_grad(c)
        h_grad.copy_(grad, non_blocking=True)
        h_loss.copy_(loss, non_blocking=True)
        s.synchronize()
    dt_e2e = max_over_ranks((time.perf_counter() - t0) / max(args.e2e_steps, 1), dist_on, "cuda")
    info = plan.info
    stages = profile_stages(plan, args.steps, lambda: plan.loss_grad(c))
    esize = 4 if fw.dtype == "f32" else 8
    fine = int(np.prod(info["n_fine"][:fw.dim]))
    roof = constraint_side_roofline(stages, fw.dim, fw.n_k, fine, esize, False, args.steps,
                                    fw.name)
    # accuracy and the oracle's rate on a sample the oracle finishes in seconds: every weight
    # at 512 of the constraints (a plan of its own on the GPU)
    acc = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        n_s = 512
        sub = slice(0, n_s)
        with fresco.Uwnu(fw.shape, nu[sub], S0[sub], W[sub], fw.dtype, tol=fw.tol,
                         upsample=fw.upsample) as p2:
            l_g, g_g = p2.loss_grad(c)
            S_g = p2.S().double().cpu().numpy()
            l_g, g_g = l_g.item(), g_g.double().cpu().numpy().reshape(-1)
        c_used = c.double().cpu().numpy().reshape(-1)
        t0 = time.perf_counter()
        l_o, g_o, S_o, _ = oracle.weight_loss_grad_k(oracle.grid_points(fw.shape), c_used,
                                                      2.0 * np.pi * nu[sub], S0[sub], W[sub])
        t_or = time.perf_counter() - t0
        acc = {"constraints": n_s, "S_rel_l2": float(np.linalg.norm(S_g - S_o) /
                                                     np.linalg.norm(S_o)),
               "loss_rel": abs(l_g - l_o) / abs(l_o),
               "grad_rel_l2": float(np.linalg.norm(g_g - g_o) / np.linalg.norm(g_o))}
        rate = 2.0 * fw.n_weights * n_s / t_or      # pair terms / s (rho and gradient)
        cpu = {"value": fw.n_weights / (2.0 * fw.n_weights * fw.n_k / rate), "unit": "weights/s",
               "cores": oracle.threads(), "kind": "oracle",
               "sample": "loss and gradient of all %d weights at the first %d constraints "
                         "(%.1f s); full evaluation extrapolated as 2 M^d N_K pair terms"
                         % (fw.n_weights, n_s, t_or)}
    plan.close()
    if rank == 0:
        line = {
            "metric": UWNU_METRIC, "value": world * fw.n_weights / t_step, "unit": "weights/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": fw.dtype, "data": "synthetic",
            "config": {"workload": fw.name, "n_weights": fw.n_weights, "dim": fw.dim,
                       "n_modes": fw.n_k, "nu_max": fw.nu_max, "tol": fw.tol,
                       "upsample": fw.upsample, "width": info["width"],
                       "n_fine": info["n_fine"][:fw.dim],
                       "l2": "fine grid (%.0f MB) below L2; inputs re-read from HBM each step"
                             % (fine * 2 * esize / 1e6),
                       "parallelism": "replicas" if world > 1 else "single"},
            "accuracy_vs_oracle": acc,
            "stages_ms": {k_: round(v[0] / max(v[1], 1), 4) for k_, v in stages.items()},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": world * fw.n_weights / dt_e2e, "unit": "weights/s",
                    "h2d_bytes_per_step": int(c_np.nbytes),
                    "d2h_bytes_per_step": int(c_np.nbytes + 8), "ms_per_step": 1e3 * dt_e2e},
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--f64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--ref-rows", type=int, default=0,
                    help="mask rows per reference step (at least four per host thread)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--upsample", type=float, default=0.0,
                    help="override the workload's fine-grid oversampling sigma")
    ap.add_argument("--tile", type=int, nargs="*", default=None,
                    help="override the spread/interp tile edge per axis")
    ap.add_argument("--grad-mode", default=None, choices=["direct", "kderiv"],
                    help="override the workload's gradient mode")
    ap.add_argument("--lbfgs-steps", type=int, default=0,
                    help="also time this many L-BFGS iterations (caller order and tile order)")
    ap.add_argument("--accuracy", action="store_true",
                    help="instead of timing: attribute the FP32 rho error at sampled mask rows")
    ap.add_argument("--accuracy-rows", type=int, default=64)
    ap.add_argument("--accuracy-seed", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3:
        log("warmup raised to 3")
        args.warmup = 3

    from paper_2305_15693_gb300 import inputs
    ens = None
    fw = None
    fld = None
    try:
        ens = inputs.ensemble_workload(args.workload)
    except KeyError:
        try:
            fw = inputs.free_workload(args.workload)
        except KeyError:
            try:
                fld = inputs.field_workload(args.workload)
            except KeyError:
                wl = inputs.workload(args.workload)
            if args.upsample:
                wl.upsample = args.upsample
            if args.grad_mode:
                wl.grad_mode = args.grad_mode

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.accuracy:
        if fw is not None or ens is not None or fld is not None:
            raise SystemExit("--accuracy takes a periodic single-problem workload")
        run_accuracy(args, wl)
        return

    if args.impl == "reference":
        if fld is not None:
            run_reference_field(args, fld, rank)
        elif ens is not None:
            run_reference_ensemble(args, ens, rank)
        elif fw is not None:
            run_reference_free(args, fw, rank)
        else:
            run_reference(args, wl, rank, world)
        return

    import torch
    from paper_2305_15693_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    dist_on = world > 1
    if dist_on:
        torch.distributed.init_process_group("nccl")
        _build.build()
    torch.cuda.set_device(local_rank)
    from paper_2305_15693_gb300 import fresco
    fresco.load()

    if fld is not None:
        run_uwnu(args, fld, rank, world, local_rank, dist_on)
        if dist_on:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    if fw is not None:
        run_nuwnu(args, fw, rank, world, local_rank, dist_on)
        if dist_on:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    if ens is not None:
        run_ensemble(args, ens, rank, world, local_rank, dist_on)
        if dist_on:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    pts_np, mask, S0, W = make_inputs(wl)
    N = wl.n_points
    pts = torch.from_numpy(pts_np).cuda()

    # ---- FP32 path: the headline -------------------------------------------------------------
    plan = fresco.Plan(wl.box, mask, S0, W, N, precision=wl.dtype, tol=wl.tol,
                       upsample=wl.upsample, tile=args.tile, grad_mode=wl.grad_mode)
    info = plan.info
    log("plan: n_fine=%s w=%d tiles=%s n_rep=%d device_bytes=%.2f GB" % (
        info["n_fine"][:wl.dim], info["width"], info["n_tiles"][:wl.dim], info["n_rep"],
        info["device_bytes"] / 1e9))
    clocks = ClockSampler(_device_selector(local_rank))
    clocks.start()
    ms, launches, stages, loss_val, grad32 = time_device(plan, pts, args.steps, args.warmup,
                                                         dist_on)
    clk = clocks.stop()
    t_step = max_over_ranks(ms / args.steps / 1e3, dist_on, "cuda")
    value = replica_throughput(N, world, t_step)

    # e2e through the host-buffer entry point (before the oracle leg, whose host threads and
    # allocations would share the host with the copies)
    dt_e2e, h2d, d2h = time_e2e(plan, pts_np, args.e2e_steps, 2)
    dt_e2e = max_over_ranks(dt_e2e, dist_on, "cuda")

    # the oracle on the host cores (a bounded sample of mask rows), and the GPU's rho at the same
    # rows for the accuracy report
    cpu, rho_err = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, rows, rho_oracle = cpu_baseline(pts_np, mask, wl.box)
        rho_dev, _ = plan.rho_S()
        got = rho_dev[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        del rho_dev
        got = got[:, 0] + 1j * got[:, 1]
        rho_err = rho_error_report(got, rho_oracle, mask[rows], wl.K)

    # L-BFGS iterations on the same plan, the solver's vectors in caller order and in tile order
    lbfgs = None
    if args.lbfgs_steps > 0:
        lbfgs = {}
        for tile_order in (False, True):
            x = pts.clone()
            solver = fresco.LBFGS(plan, tile_order=tile_order)
            solver.run(x, 2)                              # warm-up (history, tile order)
            torch.cuda.synchronize()
            plan.profile_read()
            plan.profile(True)
            t0 = time.perf_counter()
            rep0 = solver.run(x, 0)
            rep = solver.run(x, args.lbfgs_steps)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = plan.profile_read()
            plan.profile(False)
            solver.close()
            evals = rep["evaluations"] - rep0["evaluations"]
            lbfgs["tile_order" if tile_order else "caller_order"] = {
                "iterations": args.lbfgs_steps, "evaluations": evals,
                "ms_per_iteration": 1e3 * dt / args.lbfgs_steps,
                "ms_per_evaluation": 1e3 * dt / max(evals, 1), "loss": rep["loss"],
                "stages_ms": {k: round(v[0] / max(v[1], 1), 3) for k, v in st.items()}}
            del x

    plan.close()

    # ---- per-stage roofline ------------------------------------------------------------------
    esize = 4 if wl.dtype == "f32" else 8
    sb = stage_bytes(info, N, esize)
    peaks = load_peaks() if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    per_stage = {}
    for name, (tot_ms, cnt) in stages.items():
        if cnt == 0:
            continue
        avg = tot_ms / cnt
        gbs = sb[name] / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        per_stage[name] = {"ms": round(avg, 4), "alg_bytes": int(sb[name]),
                           "GB/s": round(gbs, 1), "frac": round(gbs / hbm_peak, 4)}
    # the roofline names the slowest libfresco stage (the FFT stages, cuFFT's own kernels plus a
    # transpose, keep their lines in "stages")
    ours = {k: v for k, v in per_stage.items() if k in ("sort", "spread", "interp", "mask")}
    dom = max(ours, key=lambda k: ours[k]["ms"])
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tr = json.load(f)
        entry = tr.get(wl.name, {}).get(dom)
        try:
            current = _kernel_source_hash()
        except OSError:   # a listed source is missing: the entry cannot be matched
            current = None
        if entry and current and entry.get("source_hash") == current:
            traffic = entry.get("bytes_per_launch")
    roofline = {"bound": "hbm", "achieved": per_stage[dom]["GB/s"], "peak": hbm_peak,
                "unit": "GB/s", "frac": per_stage[dom]["frac"], "traffic": traffic,
                "kernel": dom, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, burst)"}
    smem_roof = smem_rooflines(per_stage, N, wl.dim, info["width"], smem_peaks())

    # ---- all-FP64 GPU path on the same workload ----------------------------------------------
    f64 = None
    if wl.dtype == "f32" and args.f64_steps > 0:
        pts64 = pts.double()
        plan64 = fresco.Plan(wl.box, mask, S0, W, N, precision="f64", tol=1e-12,
                             upsample=wl.upsample, grad_mode=wl.grad_mode)
        ms64, _, st64, loss64, grad64 = time_device(plan64, pts64, args.f64_steps, 3, dist_on)
        plan64.close()
        del pts64
        grad_err = float(torch.linalg.vector_norm(grad32.double() - grad64) /
                         torch.linalg.vector_norm(grad64))
        del grad64
        t64 = ms64 / args.f64_steps / 1e3
        f64 = {"value": world * N / t64, "ms_per_step": 1e3 * t64, "width": None,
               "speedup_f32_over_f64": t64 / t_step,
               "loss_rel_diff_f32_vs_f64": abs(loss_val - loss64) / abs(loss64),
               "grad_rel_l2_f32_vs_f64": grad_err,
               "stages_ms": {k: round(v[0] / max(v[1], 1), 3) for k, v in st64.items()}}

    accuracy = {
        "fp32_vs_fp64_gpu": ({"loss_rel": f64["loss_rel_diff_f32_vs_f64"],
                              "grad_rel_l2": f64["grad_rel_l2_f32_vs_f64"]} if f64 else None),
        "rho_rel_l2_vs_oracle": rho_err["rel_l2"] if rho_err else None,
        "rho_rows_vs_oracle": rho_err["rows"] if rho_err else 0,
        "rho_vs_oracle": rho_err,
        "bars": {"rho": 1e-5, "loss": 1e-5, "grad": 1e-4},
    }

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": wl.dtype, "data": "synthetic",
            "config": {"workload": wl.name, "n_points": N, "dim": wl.dim, "K": wl.K,
                       "n_modes": int(mask.shape[0]), "target": wl.target, "tol": wl.tol,
                       "upsample": wl.upsample, "width": info["width"],
                       "grad_mode": wl.grad_mode,
                       "n_fine": info["n_fine"][:wl.dim], "tiles": info["n_tiles"][:wl.dim],
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (fine grid %.2f GB > %d MB)"
                             % (np.prod(info["n_fine"][:wl.dim]) * esize / 1e9,
                                L2_BYTES // 2 ** 20)},
            "roofline": roofline,
            "smem_roofline": smem_roof,
            "stages": per_stage,
            "fp64": f64,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": {"value": replica_throughput(N, world, dt_e2e), "unit": "points/s",
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * dt_e2e},
            "clocks": clk,
            "gpu_launches": launches,
            "loss": loss_val,
        }
        if lbfgs is not None:
            line["lbfgs"] = lbfgs
        print(json.dumps(line), flush=True)
    if dist_on:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


# Library sources that neither build nor size the single-plan kernels of the traffic entries
# (sort, spread, mask, interp): the solvers, the allocation-free entry point, the pair term, the
# shared-memory probe and the weights-on-a-grid / type-3 plans.
OTHER_PLAN_SOURCES = ("fresco_batch_lbfgs.cu", "fresco_lbfgs.cu", "fresco_noalloc.cu",
                      "fresco_pair.cu", "fresco_probe.cu", "fresco_uwnu.cu", "fresco_uwnu_tiles.h")


# The sources of the weights-on-a-grid / type-3 plans' constraint-side kernels (interp, spread).
UWNU_SOURCES = ("fresco_internal.h", "fresco_kernels.cuh", "fresco_uwnu.cu", "fresco_uwnu_tiles.h")


def traffic_sources(family: str = "single") -> list:
    """The sources that build (and size the launches of) the kernels the traffic entries
    describe: for the single plans every CUDA source and header of the library but
    OTHER_PLAN_SOURCES; for "uwnu" the constraint-side kernels' UWNU_SOURCES."""
    if family == "uwnu":
        return sorted(UWNU_SOURCES)
    import glob
    csrc = os.path.join(ROOT, "paper_2305_15693_gb300", "csrc")
    return sorted(os.path.basename(f) for f in glob.glob(os.path.join(csrc, "*"))
                  if f.endswith((".cu", ".cuh", ".h"))
                  and os.path.basename(f) not in OTHER_PLAN_SOURCES)


def _kernel_source_hash(family: str = "single") -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_15693_gb300", "csrc")
    for name in traffic_sources(family):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
