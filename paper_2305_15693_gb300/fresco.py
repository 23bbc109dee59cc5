"""Thin Python binding of libfresco (include/fresco.h): argument marshalling only.

Every function keeps the C name and forwards to the shared library; all numerical work runs in
the library's CUDA kernels and cuFFT. Device arrays are passed as torch CUDA tensors (or raw
integer addresses); torch serves only as the device allocator and stream provider. There is no
fallback path: if libfresco.so is missing or cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfresco.so")

FRESCO_OK = 0
FRESCO_ERR_ARG = 1
FRESCO_ERR_OOM = 2
FRESCO_ERR_CUFFT = 3
FRESCO_ERR_CUDA = 4
FRESCO_ERR_NONFINITE = 5
FRESCO_ERR_BOUNDS = 6
FRESCO_ERR_TIMEOUT = 7
FRESCO_ERR_UNSUPPORTED = 8
FRESCO_F32 = 0
FRESCO_F64 = 1
FRESCO_GRAD_DIRECT = 0
FRESCO_GRAD_KDERIV = 1
FRESCO_N_STAGES = 7
STAGES = ("sort", "spread", "fft_fwd", "mask", "loss", "fft_inv", "interp")
FRESCO_UWNU_N_STAGES = 6
UWNU_STAGES = ("point_spread", "type2", "interp", "spread", "type1", "point_interp")

# every entry point declared in include/fresco.h
EXPORTS = (
    "fresco_opts_default", "fresco_plan", "fresco_plan_query", "fresco_kernel_ft",
    "fresco_get_info", "fresco_set_stream", "fresco_loss_grad", "fresco_forward",
    "fresco_backward", "fresco_get_rho_S", "fresco_loss_grad_host", "fresco_status_check",
    "fresco_profile", "fresco_profile_read", "fresco_launch_count", "fresco_destroy",
    "fresco_status_string", "fresco_loss_noalloc", "fresco_lbfgs_opts_default",
    "fresco_lbfgs_create", "fresco_lbfgs_run", "fresco_lbfgs_reset", "fresco_lbfgs_destroy",
    "fresco_lbfgs_set_pair", "fresco_pair_plan", "fresco_pair_energy_grad",
    "fresco_pair_set_stream", "fresco_pair_destroy", "fresco_batch_plan",
    "fresco_batch_loss_grad", "fresco_batch_graph_capture", "fresco_batch_graph_launch",
    "fresco_batch_info", "fresco_batch_status_check", "fresco_batch_destroy",
    "fresco_batch_lbfgs_create", "fresco_batch_lbfgs_start", "fresco_batch_lbfgs_step",
    "fresco_batch_lbfgs_read", "fresco_batch_lbfgs_destroy", "fresco_batch_profile",
    "fresco_batch_profile_read", "fresco_batch_get_info",
    "fresco_uwu_plan", "fresco_uwu_loss_grad", "fresco_uwu_destroy",
    "fresco_uwnu_plan", "fresco_uwnu_loss_grad", "fresco_uwnu_get_S", "fresco_uwnu_get_info",
    "fresco_uwnu_destroy", "fresco_uwnu_profile", "fresco_uwnu_profile_read",
    "fresco_uwnu_launch_count", "fresco_smem_peak",
    "fresco_nuwnu_plan", "fresco_nuwnu_loss_grad", "fresco_nuwnu_get_S",
    "fresco_nuwnu_status_check", "fresco_nuwnu_get_info", "fresco_nuwnu_destroy",
    "fresco_nuwnu_profile", "fresco_nuwnu_profile_read",
)
FRESCO_LOSS_NOALLOC_MAX_ROWS = 65536 * 4096


class FrescoError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s (status %d)" % (what, status_string(status), status))
        self.status = status


class fresco_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("upsample", ctypes.c_double), ("width_override", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("grad_mode", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


class fresco_lbfgs_opts(ctypes.Structure):
    _fields_ = [("history", ctypes.c_int), ("max_step", ctypes.c_double), ("c1", ctypes.c_double),
                ("max_backtrack", ctypes.c_int), ("gtol", ctypes.c_double),
                ("ftol", ctypes.c_double), ("tile_order", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


class fresco_lbfgs_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("evaluations", ctypes.c_int64),
                ("loss", ctypes.c_double), ("grad_rms", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class fresco_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("precision", ctypes.c_int), ("width", ctypes.c_int),
                ("n_fine", ctypes.c_int * 3), ("k_max", ctypes.c_int * 3),
                ("tile", ctypes.c_int * 3), ("n_tiles", ctypes.c_int * 3),
                ("beta", ctypes.c_double), ("upsample", ctypes.c_double),
                ("loss_const", ctypes.c_double), ("n_points", ctypes.c_int64),
                ("n_modes", ctypes.c_int64), ("n_rep", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("grad_mode", ctypes.c_int)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if isinstance(v, ctypes.Array) else v
        return d


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libfresco.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FileNotFoundError(
                "libfresco.so not built: run paper_2305_15693_gb300._build.build() "
                "(or __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "fresco_opts_default": (None, [P]),
            "fresco_plan": (I, [P, I, P, I64, P, I64, P, P, P, P]),
            "fresco_plan_query": (I, [I, P, I64, P, I64, P, P, P, P]),
            "fresco_kernel_ft": (I, [I, D, I, I64, P]),
            "fresco_get_info": (I, [P, P]),
            "fresco_set_stream": (I, [P, P]),
            "fresco_loss_grad": (I, [P, P, P, P]),
            "fresco_forward": (I, [P, P, P]),
            "fresco_backward": (I, [P, P, P]),
            "fresco_get_rho_S": (I, [P, P, P]),
            "fresco_loss_grad_host": (I, [P, P, P, P]),
            "fresco_status_check": (I, [P]),
            "fresco_profile": (I, [P, I]),
            "fresco_profile_read": (I, [P, P, P]),
            "fresco_launch_count": (I64, [P]),
            "fresco_destroy": (I, [P]),
            "fresco_status_string": (ctypes.c_char_p, [I]),
            "fresco_loss_noalloc": (I, [I, I64, P, P, P, P, P]),
            "fresco_lbfgs_opts_default": (None, [P]),
            "fresco_lbfgs_create": (I, [P, P, P]),
            "fresco_lbfgs_run": (I, [P, P, I64, P]),
            "fresco_lbfgs_reset": (I, [P]),
            "fresco_lbfgs_destroy": (I, [P]),
            "fresco_lbfgs_set_pair": (I, [P, P]),
            "fresco_pair_plan": (I, [P, I, P, I64, D, D, D, I, P]),
            "fresco_pair_energy_grad": (I, [P, P, P, P, I]),
            "fresco_pair_set_stream": (I, [P, P]),
            "fresco_pair_destroy": (I, [P]),
            "fresco_batch_plan": (I, [P, I, I, P, P, P, P, P, P, P, P]),
            "fresco_batch_loss_grad": (I, [P, P, P, P]),
            "fresco_batch_graph_capture": (I, [P, P, P, P]),
            "fresco_batch_graph_launch": (I, [P]),
            "fresco_batch_info": (I, [P, P, P, P, P]),
            "fresco_batch_status_check": (I, [P]),
            "fresco_batch_destroy": (I, [P]),
            "fresco_batch_lbfgs_create": (I, [P, P, P, I64]),
            "fresco_batch_lbfgs_start": (I, [P, P]),
            "fresco_batch_lbfgs_step": (I, [P, I64]),
            "fresco_batch_lbfgs_read": (I, [P, P, P, P]),
            "fresco_batch_lbfgs_destroy": (I, [P]),
            "fresco_batch_profile": (I, [P, I]),
            "fresco_batch_profile_read": (I, [P, P, P]),
            "fresco_batch_get_info": (I, [P, I, P]),
        }
        sig.update({
            "fresco_uwu_plan": (I, [P, I, P, P, I64, P, P, I, P]),
            "fresco_uwu_loss_grad": (I, [P, P, P, P]),
            "fresco_uwu_destroy": (I, [P]),
            "fresco_uwnu_plan": (I, [P, I, P, I64, P, P, P, P, P]),
            "fresco_uwnu_loss_grad": (I, [P, P, P, P]),
            "fresco_uwnu_get_S": (I, [P, P]),
            "fresco_uwnu_get_info": (I, [P, P, P, P]),
            "fresco_uwnu_destroy": (I, [P]),
            "fresco_uwnu_profile": (I, [P, I]),
            "fresco_uwnu_profile_read": (I, [P, P, P]),
            "fresco_uwnu_launch_count": (I64, [P]),
            "fresco_smem_peak": (I, [I, P, P, P]),
            "fresco_nuwnu_plan": (I, [P, I, P, I64, I64, P, P, P, P, P]),
            "fresco_nuwnu_loss_grad": (I, [P, P, P, P]),
            "fresco_nuwnu_get_S": (I, [P, P]),
            "fresco_nuwnu_status_check": (I, [P]),
            "fresco_nuwnu_get_info": (I, [P, P, P, P, P]),
            "fresco_nuwnu_destroy": (I, [P]),
            "fresco_nuwnu_profile": (I, [P, I]),
            "fresco_nuwnu_profile_read": (I, [P, P, P]),
        })
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load().fresco_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != FRESCO_OK:
        raise FrescoError(status, what)


def _addr(x):
    """Device or host address of a torch tensor, numpy array or integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _host_arrays(box, mask, S0, W):
    mask = np.ascontiguousarray(np.asarray(mask, dtype=np.int32))
    if mask.ndim != 2:
        raise ValueError("mask must be [n_k, dim]")
    dim = mask.shape[1]
    box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (dim,)))
    S0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    if S0.size != mask.shape[0] or W.size != mask.shape[0]:
        raise ValueError("S0 and W need one value per mask row")
    return dim, box, mask, S0, W


def parse_precision(precision) -> int:
    """FRESCO_F32 or FRESCO_F64 from any accepted spelling ("f32", "float32", np.float32,
    torch.float32, FRESCO_F32, and the same for 64 bits); anything else raises ValueError."""
    if precision in (FRESCO_F32, FRESCO_F64) and not isinstance(precision, bool):
        return int(precision)
    name = getattr(precision, "__name__", None) or str(precision)
    name = name.replace("torch.", "").lower()
    if name in ("f32", "float32", "fp32", "single"):
        return FRESCO_F32
    if name in ("f64", "float64", "fp64", "double"):
        return FRESCO_F64
    raise ValueError("unknown precision %r (expected 'f32' or 'f64')" % (precision,))


def _torch_dtype(prec: int):
    import torch
    return torch.float64 if prec == FRESCO_F64 else torch.float32


def _check_dtype(name, x, dtype):
    """Raise if x is a torch tensor whose dtype is not `dtype` (raw addresses are not checked)."""
    dt = getattr(x, "dtype", None)
    if dt is not None and dt != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, dt))


def make_opts(precision="f32", tol=0.0, upsample=2.0, width=0, tile=None,
              grad_mode=FRESCO_GRAD_DIRECT) -> fresco_opts:
    o = fresco_opts()
    load().fresco_opts_default(ctypes.byref(o))
    o.precision = parse_precision(precision)
    o.tol = float(tol)
    o.upsample = float(upsample)
    o.width_override = int(width)
    if tile is not None:
        for a, t in enumerate(tile):
            o.tile[a] = int(t)
    o.grad_mode = {"direct": FRESCO_GRAD_DIRECT, "kderiv": FRESCO_GRAD_KDERIV}.get(
        grad_mode, grad_mode)
    return o


# ---- the C entry points, same names -----------------------------------------------------------

def fresco_plan(box, mask, S0, W, n_points, opts=None, stream=None):
    """Create a plan; returns the opaque handle (an int). See fresco_plan in include/fresco.h."""
    lib = load()
    dim, box, mask, S0, W = _host_arrays(box, mask, S0, W)
    h = ctypes.c_void_p()
    st = lib.fresco_plan(ctypes.byref(h), dim, box.ctypes.data, int(n_points), mask.ctypes.data,
                         mask.shape[0], S0.ctypes.data, W.ctypes.data,
                         ctypes.byref(opts) if opts is not None else None, _stream_handle(stream))
    _check(st, "fresco_plan")
    return h.value


def fresco_plan_query(box, mask, S0, W, n_points, opts=None) -> dict:
    """Host-only parameter query (no GPU touched)."""
    lib = load()
    dim, box, mask, S0, W = _host_arrays(box, mask, S0, W)
    info = fresco_info()
    st = lib.fresco_plan_query(dim, box.ctypes.data, int(n_points), mask.ctypes.data,
                               mask.shape[0], S0.ctypes.data, W.ctypes.data,
                               ctypes.byref(opts) if opts is not None else None,
                               ctypes.byref(info))
    _check(st, "fresco_plan_query")
    return info.as_dict()


def fresco_kernel_ft(width: int, beta: float, n_fine: int, n_nu: int) -> np.ndarray:
    out = np.empty(int(n_nu))
    _check(load().fresco_kernel_ft(int(width), float(beta), int(n_fine), int(n_nu),
                                   out.ctypes.data), "fresco_kernel_ft")
    return out


def fresco_get_info(plan) -> dict:
    info = fresco_info()
    _check(load().fresco_get_info(plan, ctypes.byref(info)), "fresco_get_info")
    return info.as_dict()


def fresco_set_stream(plan, stream):
    _check(load().fresco_set_stream(plan, _stream_handle(stream)), "fresco_set_stream")


def fresco_loss_grad(plan, points, loss, grad=None):
    _check(load().fresco_loss_grad(plan, _addr(points), _addr(loss), _addr(grad)),
           "fresco_loss_grad")


def fresco_forward(plan, points, loss):
    _check(load().fresco_forward(plan, _addr(points), _addr(loss)), "fresco_forward")


def fresco_backward(plan, grad_out, grad):
    _check(load().fresco_backward(plan, _addr(grad_out), _addr(grad)), "fresco_backward")


def fresco_get_rho_S(plan, rho, S):
    _check(load().fresco_get_rho_S(plan, _addr(rho), _addr(S)), "fresco_get_rho_S")


def fresco_loss_grad_host(plan, points: np.ndarray, grad: np.ndarray | None = None) -> float:
    loss = np.zeros(1)
    _check(load().fresco_loss_grad_host(plan, _addr(points), loss.ctypes.data, _addr(grad)),
           "fresco_loss_grad_host")
    return float(loss[0])


def fresco_status_check(plan) -> int:
    """Returns the status code (does not raise)."""
    return int(load().fresco_status_check(plan))


def fresco_profile(plan, enable: bool):
    _check(load().fresco_profile(plan, 1 if enable else 0), "fresco_profile")


def fresco_profile_read(plan):
    ms = np.zeros(FRESCO_N_STAGES)
    cnt = np.zeros(FRESCO_N_STAGES, dtype=np.int64)
    _check(load().fresco_profile_read(plan, ms.ctypes.data, cnt.ctypes.data),
           "fresco_profile_read")
    return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(STAGES)}


FRESCO_SMEM_ATOMIC_ADD = 0
FRESCO_SMEM_LOAD = 1


def fresco_smem_peak(op, sink, stream=None) -> float:
    """Shared-memory 32-bit atomic adds (op FRESCO_SMEM_ATOMIC_ADD) or loads (FRESCO_SMEM_LOAD)
    per second on the current device, conflict-free (the pipe's best case). sink: a device int
    tensor of at least 8 x the multiprocessor count entries."""
    v = ctypes.c_double()
    _check(load().fresco_smem_peak(int(op), _addr(sink), _stream_handle(stream), ctypes.byref(v)),
           "fresco_smem_peak")
    return v.value


def fresco_launch_count(plan) -> int:
    return int(load().fresco_launch_count(plan))


def fresco_destroy(plan):
    if plan:
        _check(load().fresco_destroy(plan), "fresco_destroy")


def fresco_status_string(status: int) -> str:
    return status_string(status)


def fresco_loss_noalloc(precision, n_k, S, S0, W, loss, stream=None):
    """sum W (S - S0)^2 into the device double `loss`, allocating nothing (see include/fresco.h:
    for callers that cannot allocate device memory at call time). S is float (precision "f32")
    or double ("f64"); S0 and W are device doubles."""
    import torch
    prec = parse_precision(precision)
    _check_dtype("S", S, _torch_dtype(prec))
    for name, x in (("S0", S0), ("W", W), ("loss", loss)):
        _check_dtype(name, x, torch.float64)
    _check(load().fresco_loss_noalloc(prec, int(n_k), _addr(S), _addr(S0), _addr(W), _addr(loss),
                                      _stream_handle(stream)), "fresco_loss_noalloc")


def fresco_lbfgs_opts_default() -> fresco_lbfgs_opts:
    o = fresco_lbfgs_opts()
    load().fresco_lbfgs_opts_default(ctypes.byref(o))
    return o


def fresco_lbfgs_create(plan, opts=None):
    h = ctypes.c_void_p()
    _check(load().fresco_lbfgs_create(ctypes.byref(h), plan,
                                      ctypes.byref(opts) if opts is not None else None),
           "fresco_lbfgs_create")
    return h.value


def fresco_lbfgs_run(solver, points, max_iter) -> dict:
    rep = fresco_lbfgs_report()
    _check(load().fresco_lbfgs_run(solver, _addr(points), int(max_iter), ctypes.byref(rep)),
           "fresco_lbfgs_run")
    return rep.as_dict()


def fresco_lbfgs_reset(solver):
    _check(load().fresco_lbfgs_reset(solver), "fresco_lbfgs_reset")


def fresco_lbfgs_destroy(solver):
    if solver:
        _check(load().fresco_lbfgs_destroy(solver), "fresco_lbfgs_destroy")


def fresco_pair_plan(box, dim, n_points, sigma, eps=1.0, alpha=2.0, precision="f32",
                     stream=None):
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (dim,)))
    h = ctypes.c_void_p()
    prec = parse_precision(precision)
    _check(load().fresco_pair_plan(ctypes.byref(h), int(dim), b.ctypes.data, int(n_points),
                                   float(sigma), float(eps), float(alpha), prec,
                                   _stream_handle(stream)), "fresco_pair_plan")
    return h.value


def fresco_pair_energy_grad(pair, points, energy, grad, accumulate=False):
    _check(load().fresco_pair_energy_grad(pair, _addr(points), _addr(energy), _addr(grad),
                                          1 if accumulate else 0), "fresco_pair_energy_grad")


def fresco_pair_set_stream(pair, stream):
    _check(load().fresco_pair_set_stream(pair, _stream_handle(stream)), "fresco_pair_set_stream")


def fresco_pair_destroy(pair):
    if pair:
        _check(load().fresco_pair_destroy(pair), "fresco_pair_destroy")


def fresco_lbfgs_set_pair(solver, pair):
    _check(load().fresco_lbfgs_set_pair(solver, pair), "fresco_lbfgs_set_pair")


def fresco_batch_plan(boxes, n_points, masks, S0s, Ws, opts=None, stream=None):
    """Batch plan over independent 2D problems: boxes [n_inst][dim] (or scalars), n_points
    [n_inst], and per instance a mask [n_k, dim], S0 [n_k], W [n_k] (lists of arrays)."""
    lib = load()
    n = len(n_points)
    if not (len(masks) == len(S0s) == len(Ws) == n) or n < 1:
        raise ValueError("one mask, S0 and W per instance")
    arrs = [_host_arrays(boxes[i], masks[i], S0s[i], Ws[i]) for i in range(n)]
    dim = arrs[0][0]
    if any(a[0] != dim for a in arrs):
        raise ValueError("all instances need the same dimension")
    box = np.ascontiguousarray(np.stack([a[1] for a in arrs]))
    mask = np.ascontiguousarray(np.concatenate([a[2] for a in arrs]))
    S0 = np.ascontiguousarray(np.concatenate([a[3] for a in arrs]))
    W = np.ascontiguousarray(np.concatenate([a[4] for a in arrs]))
    npts = np.ascontiguousarray(np.asarray(n_points, dtype=np.int64))
    nmod = np.ascontiguousarray(np.array([a[2].shape[0] for a in arrs], dtype=np.int64))
    h = ctypes.c_void_p()
    st = lib.fresco_batch_plan(ctypes.byref(h), dim, n, box.ctypes.data, npts.ctypes.data,
                               nmod.ctypes.data, mask.ctypes.data, S0.ctypes.data, W.ctypes.data,
                               ctypes.byref(opts) if opts is not None else None,
                               _stream_handle(stream))
    _check(st, "fresco_batch_plan")
    return h.value


def fresco_batch_loss_grad(batch, points, losses, grad=None):
    _check(load().fresco_batch_loss_grad(batch, _addr(points), _addr(losses), _addr(grad)),
           "fresco_batch_loss_grad")


def fresco_batch_graph_capture(batch, points, losses, grad=None):
    _check(load().fresco_batch_graph_capture(batch, _addr(points), _addr(losses), _addr(grad)),
           "fresco_batch_graph_capture")


def fresco_batch_graph_launch(batch):
    _check(load().fresco_batch_graph_launch(batch), "fresco_batch_graph_launch")


def fresco_batch_info(batch) -> dict:
    tp, nc = ctypes.c_int64(), ctypes.c_int()
    db, nl = ctypes.c_int64(), ctypes.c_int64()
    _check(load().fresco_batch_info(batch, ctypes.byref(tp), ctypes.byref(nc), ctypes.byref(db),
                                    ctypes.byref(nl)), "fresco_batch_info")
    return {"total_points": tp.value, "n_classes": nc.value, "device_bytes": db.value,
            "launches": nl.value}


def fresco_batch_get_info(batch, i: int) -> dict:
    info = fresco_info()
    _check(load().fresco_batch_get_info(batch, int(i), ctypes.byref(info)),
           "fresco_batch_get_info")
    return info.as_dict()


def fresco_batch_status_check(batch) -> int:
    return load().fresco_batch_status_check(batch)


def fresco_batch_profile(batch, enable: bool):
    _check(load().fresco_batch_profile(batch, 1 if enable else 0), "fresco_batch_profile")


def fresco_batch_profile_read(batch):
    """Per-stage device time since the last read: {stage: (ms, calls)}."""
    ms = (ctypes.c_double * FRESCO_N_STAGES)()
    cnt = (ctypes.c_int64 * FRESCO_N_STAGES)()
    _check(load().fresco_batch_profile_read(batch, ms, cnt), "fresco_batch_profile_read")
    return {STAGES[i]: (ms[i], cnt[i]) for i in range(FRESCO_N_STAGES)}


def fresco_batch_destroy(batch):
    _check(load().fresco_batch_destroy(batch), "fresco_batch_destroy")


def fresco_batch_lbfgs_create(batch, opts=None, max_iter=0):
    h = ctypes.c_void_p()
    _check(load().fresco_batch_lbfgs_create(ctypes.byref(h), batch,
                                            ctypes.byref(opts) if opts is not None else None,
                                            int(max_iter)), "fresco_batch_lbfgs_create")
    return h.value


def fresco_batch_lbfgs_start(solver, points):
    _check(load().fresco_batch_lbfgs_start(solver, _addr(points)), "fresco_batch_lbfgs_start")


def fresco_batch_lbfgs_step(solver, n_steps=1):
    _check(load().fresco_batch_lbfgs_step(solver, int(n_steps)), "fresco_batch_lbfgs_step")


def fresco_batch_lbfgs_read(solver, n_inst, points=None):
    """Returns (list of per-instance report dicts, instances still running)."""
    reps = (fresco_lbfgs_report * n_inst)()
    run = ctypes.c_int64()
    _check(load().fresco_batch_lbfgs_read(solver, _addr(points), reps, ctypes.byref(run)),
           "fresco_batch_lbfgs_read")
    return [r.as_dict() for r in reps], run.value


def fresco_batch_lbfgs_destroy(solver):
    _check(load().fresco_batch_lbfgs_destroy(solver), "fresco_batch_lbfgs_destroy")


class BatchLBFGS:
    """Per-instance L-BFGS over a Batch, all instances stepping together (fresco_batch_lbfgs_*
    in include/fresco.h). Steps after the first replay one CUDA graph each."""

    def __init__(self, batch, max_iter=0, history=10, max_step=0.0, c1=1e-4, max_backtrack=20,
                 gtol=0.0, ftol=0.0):
        o = fresco_lbfgs_opts_default()
        o.history, o.max_step, o.c1 = int(history), float(max_step), float(c1)
        o.max_backtrack, o.gtol, o.ftol = int(max_backtrack), float(gtol), float(ftol)
        self.batch = batch
        self.handle = fresco_batch_lbfgs_create(batch.handle, o, max_iter)

    def start(self, points):
        self.batch._check_points(points)
        self.batch.stream.wait_stream(self.batch._torch.cuda.current_stream())
        fresco_batch_lbfgs_start(self.handle, points)

    def step(self, n_steps=1):
        fresco_batch_lbfgs_step(self.handle, n_steps)

    def read(self, points=None):
        if points is not None:
            self.batch._check_points(points)
        return fresco_batch_lbfgs_read(self.handle, self.batch.n_inst, points)

    def run(self, points, max_steps, check_every=64):
        """Minimise every instance in place, for at most max_steps steps (evaluations); returns
        the per-instance reports."""
        self.start(points)
        done = 0
        while done < max_steps:
            n = min(check_every, max_steps - done)
            self.step(n)
            done += n
            _, running = self.read()
            if running == 0:
                break
        reps, _ = self.read(points)
        return reps

    def close(self):
        if getattr(self, "handle", None):
            fresco_batch_lbfgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fresco_uwu_plan(grid_shape, mask, S0, W, precision="f32", stream=None):
    """Plan for real weights on a uniform grid (grid_shape = (M_0, M_1[, M_2]), x first)."""
    lib = load()
    mask = np.ascontiguousarray(np.asarray(mask, dtype=np.int32))
    dim = mask.shape[1]
    grid = np.ascontiguousarray(np.asarray(grid_shape, dtype=np.int64).reshape(-1))
    if grid.size != dim:
        raise ValueError("one grid size per axis")
    S0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    h = ctypes.c_void_p()
    prec = parse_precision(precision)
    _check(lib.fresco_uwu_plan(ctypes.byref(h), dim, grid.ctypes.data, mask.ctypes.data,
                               mask.shape[0], S0.ctypes.data, W.ctypes.data, prec,
                               _stream_handle(stream)), "fresco_uwu_plan")
    return h.value


def fresco_uwu_loss_grad(plan, c, loss, grad=None):
    _check(load().fresco_uwu_loss_grad(plan, _addr(c), _addr(loss), _addr(grad)),
           "fresco_uwu_loss_grad")


def fresco_uwu_destroy(plan):
    _check(load().fresco_uwu_destroy(plan), "fresco_uwu_destroy")


class Uwu:
    """Weights on a uniform grid (fresco_uwu_* in include/fresco.h). Weights and gradients are
    CUDA tensors of shape grid_shape[::-1] (x the last, contiguous index) in the plan's dtype."""

    def __init__(self, grid_shape, mask, S0, W, precision="f32", stream=None):
        import torch
        self._torch = torch
        self.shape = tuple(int(x) for x in grid_shape)[::-1]
        self.dtype = _torch_dtype(parse_precision(precision))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = fresco_uwu_plan(grid_shape, mask, S0, W, precision, self.stream)

    def loss_grad(self, c, want_grad=True):
        t = self._torch
        if (not c.is_cuda or c.dtype != self.dtype or not c.is_contiguous()
                or tuple(c.shape) != self.shape):
            raise ValueError("weights must be a contiguous CUDA %s tensor %s" % (self.dtype,
                                                                                   self.shape))
        loss = t.empty((), dtype=t.float64, device=c.device)
        grad = t.empty_like(c) if want_grad else None
        fresco_uwu_loss_grad(self.handle, c, loss, grad)
        return loss, grad

    def close(self):
        if getattr(self, "handle", None):
            fresco_uwu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fresco_uwnu_plan(grid_shape, nu, S0, W, opts=None, stream=None):
    """Plan for real weights on a uniform grid with constraints at real frequencies nu [n_k, dim]
    (cycles per grid length; grid_shape = (M_0, M_1[, M_2]), x first)."""
    lib = load()
    nu = np.ascontiguousarray(np.asarray(nu, dtype=np.float64))
    dim = nu.shape[1]
    grid = np.ascontiguousarray(np.asarray(grid_shape, dtype=np.int64).reshape(-1))
    if grid.size != dim:
        raise ValueError("one grid size per axis")
    S0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    if S0.size != nu.shape[0] or W.size != nu.shape[0]:
        raise ValueError("one S0 and one W per constraint")
    h = ctypes.c_void_p()
    _check(lib.fresco_uwnu_plan(ctypes.byref(h), dim, grid.ctypes.data, nu.shape[0],
                                nu.ctypes.data, S0.ctypes.data, W.ctypes.data,
                                ctypes.byref(opts) if opts is not None else None,
                                _stream_handle(stream)), "fresco_uwnu_plan")
    return h.value


def fresco_uwnu_loss_grad(plan, c, loss, grad=None):
    _check(load().fresco_uwnu_loss_grad(plan, _addr(c), _addr(loss), _addr(grad)),
           "fresco_uwnu_loss_grad")


def fresco_uwnu_get_S(plan, S):
    _check(load().fresco_uwnu_get_S(plan, _addr(S)), "fresco_uwnu_get_S")


def fresco_uwnu_get_info(plan) -> dict:
    w = ctypes.c_int()
    beta = ctypes.c_double()
    nf = (ctypes.c_int * 3)()
    _check(load().fresco_uwnu_get_info(plan, ctypes.byref(w), ctypes.byref(beta), nf),
           "fresco_uwnu_get_info")
    return {"width": w.value, "beta": beta.value, "n_fine": list(nf)}


def fresco_uwnu_destroy(plan):
    _check(load().fresco_uwnu_destroy(plan), "fresco_uwnu_destroy")


def _uwnu_profile_read(fn, plan, name):
    ms = np.zeros(FRESCO_UWNU_N_STAGES)
    cnt = np.zeros(FRESCO_UWNU_N_STAGES, dtype=np.int64)
    _check(fn(plan, ms.ctypes.data, cnt.ctypes.data), name)
    return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(UWNU_STAGES)}


def fresco_uwnu_profile(plan, enable: bool):
    _check(load().fresco_uwnu_profile(plan, 1 if enable else 0), "fresco_uwnu_profile")


def fresco_uwnu_profile_read(plan):
    return _uwnu_profile_read(load().fresco_uwnu_profile_read, plan, "fresco_uwnu_profile_read")


def fresco_uwnu_launch_count(plan) -> int:
    return int(load().fresco_uwnu_launch_count(plan))


def fresco_nuwnu_profile(plan, enable: bool):
    _check(load().fresco_nuwnu_profile(plan, 1 if enable else 0), "fresco_nuwnu_profile")


def fresco_nuwnu_profile_read(plan):
    return _uwnu_profile_read(load().fresco_nuwnu_profile_read, plan, "fresco_nuwnu_profile_read")


class Uwnu:
    """Weights on a uniform grid with constraints at real frequencies (fresco_uwnu_* in
    include/fresco.h). Weights and gradients are CUDA tensors of shape grid_shape[::-1] (x the
    last, contiguous index) in the plan's dtype."""

    def __init__(self, grid_shape, nu, S0, W, precision="f32", tol=0.0, upsample=2.0,
                 stream=None):
        import torch
        self._torch = torch
        self.shape = tuple(int(x) for x in grid_shape)[::-1]
        self.n_k = int(np.asarray(nu).shape[0])
        self.dtype = _torch_dtype(parse_precision(precision))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opts = make_opts(precision=precision, tol=tol, upsample=upsample)
        self.handle = fresco_uwnu_plan(grid_shape, nu, S0, W, opts, self.stream)
        self.info = fresco_uwnu_get_info(self.handle)

    def loss_grad(self, c, want_grad=True):
        t = self._torch
        if (not c.is_cuda or c.dtype != self.dtype or not c.is_contiguous()
                or tuple(c.shape) != self.shape):
            raise ValueError("weights must be a contiguous CUDA %s tensor %s" % (self.dtype,
                                                                                   self.shape))
        loss = t.empty((), dtype=t.float64, device=c.device)
        grad = t.empty_like(c) if want_grad else None
        fresco_uwnu_loss_grad(self.handle, c, loss, grad)
        return loss, grad

    def S(self):
        t = self._torch
        out = t.empty(self.n_k, dtype=self.dtype, device="cuda")
        fresco_uwnu_get_S(self.handle, out)
        return out

    def profile(self, enable=True):
        fresco_uwnu_profile(self.handle, enable)

    def profile_read(self):
        return fresco_uwnu_profile_read(self.handle)

    def launch_count(self) -> int:
        return fresco_uwnu_launch_count(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fresco_uwnu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fresco_nuwnu_plan(box, kvec, S0, W, n_points, opts=None, stream=None):
    """Plan for points in [-L/2, L/2]^d with constraints at real wavevectors kvec [n_k, dim]
    (radians per unit length)."""
    lib = load()
    k = np.ascontiguousarray(np.asarray(kvec, dtype=np.float64))
    if k.ndim != 2:
        raise ValueError("kvec must be [n_k, dim]")
    dim = k.shape[1]
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (dim,)))
    S0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    if S0.size != k.shape[0] or W.size != k.shape[0]:
        raise ValueError("one S0 and one W per constraint")
    h = ctypes.c_void_p()
    _check(lib.fresco_nuwnu_plan(ctypes.byref(h), dim, b.ctypes.data, int(n_points), k.shape[0],
                                 k.ctypes.data, S0.ctypes.data, W.ctypes.data,
                                 ctypes.byref(opts) if opts is not None else None,
                                 _stream_handle(stream)), "fresco_nuwnu_plan")
    return h.value


def fresco_nuwnu_loss_grad(plan, points, loss, grad=None):
    _check(load().fresco_nuwnu_loss_grad(plan, _addr(points), _addr(loss), _addr(grad)),
           "fresco_nuwnu_loss_grad")


def fresco_nuwnu_get_S(plan, S):
    _check(load().fresco_nuwnu_get_S(plan, _addr(S)), "fresco_nuwnu_get_S")


def fresco_nuwnu_status_check(plan) -> int:
    return int(load().fresco_nuwnu_status_check(plan))


def fresco_nuwnu_get_info(plan) -> dict:
    w = ctypes.c_int()
    ng = (ctypes.c_int * 3)()
    nf = (ctypes.c_int * 3)()
    nl = ctypes.c_int64()
    _check(load().fresco_nuwnu_get_info(plan, ctypes.byref(w), ng, nf, ctypes.byref(nl)),
           "fresco_nuwnu_get_info")
    return {"width": w.value, "n_grid": list(ng), "n_fine": list(nf), "launches": nl.value}


def fresco_nuwnu_destroy(plan):
    _check(load().fresco_nuwnu_destroy(plan), "fresco_nuwnu_destroy")


class Nuwnu:
    """Points at free positions in [-L/2, L/2]^d with constraints at real wavevectors
    (fresco_nuwnu_* in include/fresco.h). Points and gradients are contiguous CUDA tensors
    [N, dim] in the plan's dtype, caller order."""

    def __init__(self, box, kvec, S0, W, n_points, precision="f32", tol=0.0, upsample=2.0,
                 stream=None):
        import torch
        self._torch = torch
        self.n_points = int(n_points)
        self.n_k = int(np.asarray(kvec).shape[0])
        self.dim = int(np.asarray(kvec).shape[1])
        self.dtype = _torch_dtype(parse_precision(precision))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opts = make_opts(precision=precision, tol=tol, upsample=upsample)
        self.handle = fresco_nuwnu_plan(box, kvec, S0, W, n_points, opts, self.stream)
        self.info = fresco_nuwnu_get_info(self.handle)

    def loss_grad(self, points, want_grad=True):
        t = self._torch
        if (not points.is_cuda or points.dtype != self.dtype or not points.is_contiguous()
                or tuple(points.shape) != (self.n_points, self.dim)):
            raise ValueError("points must be a contiguous CUDA %s tensor [%d, %d]"
                             % (self.dtype, self.n_points, self.dim))
        loss = t.empty((), dtype=t.float64, device=points.device)
        grad = t.empty_like(points) if want_grad else None
        fresco_nuwnu_loss_grad(self.handle, points, loss, grad)
        return loss, grad

    def S(self):
        out = self._torch.empty(self.n_k, dtype=self.dtype, device="cuda")
        fresco_nuwnu_get_S(self.handle, out)
        return out

    def profile(self, enable=True):
        fresco_nuwnu_profile(self.handle, enable)

    def profile_read(self):
        return fresco_nuwnu_profile_read(self.handle)

    def status(self) -> int:
        return fresco_nuwnu_status_check(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fresco_nuwnu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Ensemble of independent 2D problems evaluated together (fresco_batch_* in
    include/fresco.h). Points of all instances are one CUDA tensor [sum N, dim], instance after
    instance; losses come back as a float64 tensor [n_inst]. The batch runs on a stream of its
    own (needed for graph capture), ordered after and before torch's current stream."""

    def __init__(self, boxes, n_points, masks, S0s, Ws, precision="f32", tol=0.0, upsample=2.0,
                 width=0, tile=None, stream=None, grad_mode=FRESCO_GRAD_DIRECT):
        import torch
        self._torch = torch
        self.opts = make_opts(precision, tol, upsample, width, tile, grad_mode)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.n_points = [int(n) for n in n_points]
        self.first = np.concatenate([[0], np.cumsum(self.n_points)]).astype(np.int64)
        self.dim = np.asarray(masks[0]).shape[1]
        self.dtype = torch.float64 if self.opts.precision == FRESCO_F64 else torch.float32
        self.handle = fresco_batch_plan(boxes, n_points, masks, S0s, Ws, self.opts, self.stream)
        self.info = fresco_batch_info(self.handle)

    @property
    def n_inst(self):
        return len(self.n_points)

    def _check_points(self, points):
        if (not points.is_cuda or points.dtype != self.dtype or not points.is_contiguous()
                or tuple(points.shape) != (int(self.first[-1]), self.dim)):
            raise ValueError("points must be a contiguous CUDA %s tensor [%d, %d]"
                             % (self.dtype, int(self.first[-1]), self.dim))

    def loss_grad(self, points, losses=None, grad=None, want_grad=True):
        t = self._torch
        self._check_points(points)
        if losses is None:
            losses = t.empty(self.n_inst, dtype=t.float64, device=points.device)
        if grad is None and want_grad:
            grad = t.empty_like(points)
        cur = t.cuda.current_stream()
        self.stream.wait_stream(cur)
        fresco_batch_loss_grad(self.handle, points, losses, grad)
        cur.wait_stream(self.stream)
        return losses, grad

    def capture(self, points, losses, grad=None):
        """Record one evaluation on these tensors as a CUDA graph (replay with launch())."""
        self._check_points(points)
        t = self._torch
        self.stream.wait_stream(t.cuda.current_stream())
        fresco_batch_graph_capture(self.handle, points, losses, grad)
        self._graph_args = (points, losses, grad)   # keep the captured buffers alive

    def launch(self):
        t = self._torch
        self.stream.wait_stream(t.cuda.current_stream())
        fresco_batch_graph_launch(self.handle)
        t.cuda.current_stream().wait_stream(self.stream)

    def status(self) -> int:
        return fresco_batch_status_check(self.handle)

    def profile(self, enable=True):
        fresco_batch_profile(self.handle, enable)

    def profile_read(self):
        return fresco_batch_profile_read(self.handle)

    def split(self, x):
        """Per-instance views of a [sum N, ...] tensor."""
        return [x[self.first[i]:self.first[i + 1]] for i in range(self.n_inst)]

    def close(self):
        if getattr(self, "handle", None):
            fresco_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class PairTerm:
    """Repulsive pair term of the hybrid loss (Eq. 6) over torch CUDA tensors."""

    def __init__(self, box, dim, n_points, sigma, eps=1.0, alpha=2.0, precision="f32",
                 stream=None):
        import torch
        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.dim, self.n_points = int(dim), int(n_points)
        self.dtype = _torch_dtype(parse_precision(precision))
        self.handle = fresco_pair_plan(box, dim, n_points, sigma, eps, alpha, precision, stream)

    def energy_grad(self, points, energy=None, grad=None, accumulate=False):
        t = self._torch
        if energy is None:
            energy = t.zeros((), dtype=t.float64, device=points.device)
        if grad is None:
            grad = t.zeros_like(points)
        fresco_pair_energy_grad(self.handle, points, energy, grad, accumulate)
        return energy, grad

    def close(self):
        if getattr(self, "handle", None):
            fresco_pair_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class LBFGS:
    """Device-resident L-BFGS over a Plan (see fresco_lbfgs_* in include/fresco.h)."""

    def __init__(self, plan, history=10, max_step=0.0, c1=1e-4, max_backtrack=20, gtol=0.0,
                 ftol=0.0, tile_order=False):
        o = fresco_lbfgs_opts_default()
        o.history, o.max_step, o.c1 = int(history), float(max_step), float(c1)
        o.max_backtrack, o.gtol, o.ftol = int(max_backtrack), float(gtol), float(ftol)
        o.tile_order = 1 if tile_order else 0
        self.plan = plan
        self.handle = fresco_lbfgs_create(plan.handle, o)

    def set_pair(self, pair):
        """Minimise the hybrid loss of Eq. 6 (a PairTerm, or None to drop it)."""
        self.pair = pair
        fresco_lbfgs_set_pair(self.handle, pair.handle if pair is not None else None)

    def run(self, points, max_iter) -> dict:
        """Minimise in place (points: contiguous CUDA tensor [N, dim] of the plan's dtype)."""
        self.plan._check_points(points)
        return fresco_lbfgs_run(self.handle, points, max_iter)

    def reset(self):
        fresco_lbfgs_reset(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fresco_lbfgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience wrapper ------------------------------------------------------------------------

class Plan:
    """Owning wrapper around a plan handle, with torch-tensor helpers.

    Points and gradients are torch CUDA tensors of shape [N, dim] in the plan's dtype
    (float32 or float64); the loss is a CUDA float64 tensor of shape [] or [1].
    """

    def __init__(self, box, mask, S0, W, n_points, precision="f32", tol=0.0, upsample=2.0,
                 width=0, tile=None, stream=None, grad_mode=FRESCO_GRAD_DIRECT):
        import torch  # device memory and streams only
        self._torch = torch
        self.opts = make_opts(precision, tol, upsample, width, tile, grad_mode)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.handle = fresco_plan(box, mask, S0, W, n_points, self.opts, stream)
        self.info = fresco_get_info(self.handle)
        self.dim = self.info["dim"]
        self.n_points = int(n_points)
        self.n_k = int(np.asarray(mask).shape[0])
        self.dtype = torch.float64 if self.info["precision"] == FRESCO_F64 else torch.float32

    def _check_points(self, x):
        t = self._torch
        if not (isinstance(x, t.Tensor) and x.is_cuda and x.dtype == self.dtype
                and x.is_contiguous() and tuple(x.shape) == (self.n_points, self.dim)):
            raise ValueError("points must be a contiguous CUDA %s tensor of shape (%d, %d)"
                             % (self.dtype, self.n_points, self.dim))

    def loss_grad(self, points, want_grad=True):
        t = self._torch
        self._check_points(points)
        loss = t.empty((), dtype=t.float64, device=points.device)
        grad = t.empty_like(points) if want_grad else None
        fresco_loss_grad(self.handle, points, loss, grad)
        return loss, grad

    def forward(self, points):
        t = self._torch
        self._check_points(points)
        loss = t.empty((), dtype=t.float64, device=points.device)
        fresco_forward(self.handle, points, loss)
        return loss

    def backward(self, grad_out=None, out=None):
        t = self._torch
        dev = t.device("cuda", t.cuda.current_device())
        grad = out if out is not None else t.empty((self.n_points, self.dim), dtype=self.dtype,
                                                   device=dev)
        go = None
        if grad_out is not None:
            go = grad_out.to(dtype=t.float64).reshape(())
            if not go.is_contiguous():
                go = go.contiguous()
        fresco_backward(self.handle, go, grad)
        return grad

    def rho_S(self):
        t = self._torch
        dev = t.device("cuda", t.cuda.current_device())
        rho = t.empty((self.n_k, 2), dtype=self.dtype, device=dev)
        S = t.empty((self.n_k,), dtype=self.dtype, device=dev)
        fresco_get_rho_S(self.handle, rho, S)
        return rho, S

    def loss_grad_host(self, points: np.ndarray, grad: np.ndarray | None = None) -> float:
        return fresco_loss_grad_host(self.handle, points, grad)

    def status(self) -> int:
        return fresco_status_check(self.handle)

    def profile(self, enable=True):
        fresco_profile(self.handle, enable)

    def profile_read(self):
        return fresco_profile_read(self.handle)

    def launch_count(self) -> int:
        return fresco_launch_count(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fresco_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
