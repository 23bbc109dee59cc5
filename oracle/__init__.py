"""CPU FP64 oracle for the FReSCo loss and gradient (direct Fourier sums).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the bench's
CPU-baseline leg; never by the GPU library. It shares no code with the CUDA path. The C
source (fresco_oracle.c) writes the definitions of Eq. 1, Eq. 2 and Eq. 4 of arXiv
2305.15693 (and the pair term of the hybrid loss, Eq. 6) out as plain sums; this wrapper only
marshals numpy arrays.

Points stored in FP32 are promoted exactly to FP64, so both sides see identical inputs.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fresco_oracle.c")
_LIB = os.path.join(_HERE, "libfresco_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fresco_oracle.c with gcc -O2 -fopenmp into libfresco_oracle.so (in place)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_rho.argtypes = [ctypes.c_int, i64, p, p, i64, p, p, p]
            lib.oracle_rho.restype = ctypes.c_int
            lib.oracle_loss_grad.argtypes = [ctypes.c_int, i64, p, p, i64, p, p, p,
                                             p, p, p, p, i64, p, p]
            lib.oracle_loss_grad.restype = ctypes.c_int
            lib.oracle_pair_energy_grad.argtypes = [ctypes.c_int, i64, p, p, ctypes.c_double,
                                                    ctypes.c_double, ctypes.c_double, p, i64, p,
                                                    p]
            lib.oracle_pair_energy_grad.restype = ctypes.c_int
            lib.oracle_weight_loss_grad.argtypes = [ctypes.c_int, i64, p, p, p, i64, p, p, p,
                                                    p, p, p, p, p]
            lib.oracle_weight_loss_grad.restype = ctypes.c_int
            lib.oracle_weight_loss_grad_k.argtypes = [ctypes.c_int, i64, p, p, i64, p, p, p, p,
                                                      p, p, p, p]
            lib.oracle_weight_loss_grad_k.restype = ctypes.c_int
            lib.oracle_loss_grad_k.argtypes = [ctypes.c_int, i64, p, i64, p, p, p, p, p, p, p,
                                               p]
            lib.oracle_loss_grad_k.restype = ctypes.c_int
            lib.oracle_threads.argtypes = []
            lib.oracle_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(points, box, mask):
    r = np.ascontiguousarray(np.asarray(points).astype(np.float64))
    if r.ndim != 2:
        raise ValueError("points must be [N, dim]")
    dim = r.shape[1]
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (dim,)))
    m = np.ascontiguousarray(np.asarray(mask, dtype=np.int32).reshape(-1, dim))
    return r, dim, b, m


def threads() -> int:
    """OpenMP threads the oracle runs on."""
    return int(_load().oracle_threads())


def rho(points, mask, box=1.0) -> np.ndarray:
    """rho(n) = sum_j exp(-2 pi i n . r_j / L) for every row n of `mask` (complex128)."""
    r, dim, b, m = _prep(points, box, mask)
    re = np.empty(m.shape[0])
    im = np.empty(m.shape[0])
    rc = _load().oracle_rho(dim, r.shape[0], _ptr(r), _ptr(b), m.shape[0], _ptr(m),
                            _ptr(re), _ptr(im))
    if rc != 0:
        raise ValueError("oracle_rho failed (%d)" % rc)
    return re + 1j * im


def loss_grad(points, mask, S0, W, box=1.0, sel=None, want_grad=True):
    """Loss, gradient, S and rho by direct sums.

    Returns (loss, grad, S, rho); grad is [len(sel), dim] when `sel` (point indices) is
    given, [N, dim] otherwise, None when want_grad is False.
    """
    r, dim, b, m = _prep(points, box, mask)
    s0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    w = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    if s0.size != m.shape[0] or w.size != m.shape[0]:
        raise ValueError("S0 and W must have one entry per mask row")
    n_k = m.shape[0]
    loss = np.zeros(1)
    S = np.empty(n_k)
    re = np.empty(n_k)
    im = np.empty(n_k)
    grad = None
    sel_arr = None
    n_sel = 0
    if want_grad:
        if sel is not None:
            sel_arr = np.ascontiguousarray(np.asarray(sel, dtype=np.int64).reshape(-1))
            n_sel = sel_arr.size
            grad = np.empty((n_sel, dim))
        else:
            grad = np.empty((r.shape[0], dim))
    rc = _load().oracle_loss_grad(dim, r.shape[0], _ptr(r), _ptr(b), n_k, _ptr(m), _ptr(s0),
                                  _ptr(w), _ptr(loss), _ptr(S), _ptr(re), _ptr(im), n_sel,
                                  _ptr(sel_arr), _ptr(grad))
    if rc != 0:
        raise ValueError("oracle_loss_grad failed (%d)" % rc)
    return float(loss[0]), grad, S, re + 1j * im


def weight_loss_grad(points, weights, mask, S0, W, box=1.0, want_grad=True):
    """Weighted points (real weights c_j at positions r_j): rho = sum_j c_j e^{-ik.r_j},
    S = |rho|^2 / sum_j c_j^2. Returns (loss, dL/dc [N] or None, S, rho)."""
    r, dim, b, m = _prep(points, box, mask)
    c = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    if c.size != r.shape[0]:
        raise ValueError("one weight per point")
    s0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    w = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    n_k = m.shape[0]
    loss = np.zeros(1)
    S = np.empty(n_k)
    re = np.empty(n_k)
    im = np.empty(n_k)
    grad = np.empty(r.shape[0]) if want_grad else None
    rc = _load().oracle_weight_loss_grad(dim, r.shape[0], _ptr(r), _ptr(b), _ptr(c), n_k, _ptr(m),
                                         _ptr(s0), _ptr(w), _ptr(loss), _ptr(S), _ptr(re),
                                         _ptr(im), _ptr(grad))
    if rc != 0:
        raise ValueError("oracle_weight_loss_grad failed (%d)" % rc)
    return float(loss[0]), grad, S, re + 1j * im


def loss_grad_k(points, kvec, S0, W, want_grad=True):
    """Unit-weight points at arbitrary real wavevectors kvec [n_k, dim] (non-uniform constraints,
    free boundaries): rho = sum_j e^{-ik.r_j}, S = |rho|^2 / N.
    Returns (loss, dL/dr [N, dim] or None, S, rho)."""
    r = np.ascontiguousarray(np.asarray(points).astype(np.float64))
    dim = r.shape[1]
    k = np.ascontiguousarray(np.asarray(kvec, dtype=np.float64).reshape(-1, dim))
    s0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    w = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    n_k = k.shape[0]
    loss = np.zeros(1)
    S = np.empty(n_k)
    re = np.empty(n_k)
    im = np.empty(n_k)
    grad = np.empty_like(r) if want_grad else None
    rc = _load().oracle_loss_grad_k(dim, r.shape[0], _ptr(r), n_k, _ptr(k), _ptr(s0), _ptr(w),
                                    _ptr(loss), _ptr(S), _ptr(re), _ptr(im), _ptr(grad))
    if rc != 0:
        raise ValueError("oracle_loss_grad_k failed (%d)" % rc)
    return float(loss[0]), grad, S, re + 1j * im


def weight_loss_grad_k(points, weights, kvec, S0, W, want_grad=True):
    """Weighted points at arbitrary real wavevectors kvec [n_k, dim] (non-uniform constraints,
    free boundaries): rho = sum_j c_j e^{-ik.r_j}, S = |rho|^2 / sum_j c_j^2.
    Returns (loss, dL/dc [N] or None, S, rho)."""
    r = np.ascontiguousarray(np.asarray(points).astype(np.float64))
    dim = r.shape[1]
    k = np.ascontiguousarray(np.asarray(kvec, dtype=np.float64).reshape(-1, dim))
    c = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    if c.size != r.shape[0]:
        raise ValueError("one weight per point")
    s0 = np.ascontiguousarray(np.asarray(S0, dtype=np.float64).reshape(-1))
    w = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    n_k = k.shape[0]
    loss = np.zeros(1)
    S = np.empty(n_k)
    re = np.empty(n_k)
    im = np.empty(n_k)
    grad = np.empty(r.shape[0]) if want_grad else None
    rc = _load().oracle_weight_loss_grad_k(dim, r.shape[0], _ptr(r), _ptr(c), n_k, _ptr(k),
                                           _ptr(s0), _ptr(w), _ptr(loss), _ptr(S), _ptr(re),
                                           _ptr(im), _ptr(grad))
    if rc != 0:
        raise ValueError("oracle_weight_loss_grad_k failed (%d)" % rc)
    return float(loss[0]), grad, S, re + 1j * im


def grid_points(shape, box=1.0):
    """Positions of the cells of a uniform grid, row-major with the first axis fastest:
    cell (i_0, ..., i_{d-1}) at (i_a L_a / M_a)_a, flattened index i_0 + M_0 (i_1 + M_1 i_2)."""
    shape = tuple(int(x) for x in shape)
    dim = len(shape)
    b = np.broadcast_to(np.asarray(box, dtype=np.float64), (dim,))
    axes = [np.arange(m, dtype=np.float64) * (b[a] / m) for a, m in enumerate(shape)]
    mesh = np.meshgrid(*axes, indexing="ij")          # mesh[a][i_0, ..., i_{d-1}]
    pts = np.stack([g.transpose(tuple(range(dim))[::-1]).reshape(-1) for g in mesh], axis=1)
    return np.ascontiguousarray(pts)


def pair_energy_grad(points, sigma, eps=1.0, alpha=2.0, box=1.0, sel=None, want_grad=True,
                     want_energy=True):
    """Repulsive pair term of the hybrid loss (Eq. 6) by the direct double loop: returns
    (E, grad); grad is [len(sel), dim] when `sel` is given; E is None without want_energy."""
    r = np.ascontiguousarray(np.asarray(points).astype(np.float64))
    dim = r.shape[1]
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (dim,)))
    e = np.zeros(1)
    grad = None
    sel_arr = None
    n_sel = 0
    if want_grad:
        if sel is not None:
            sel_arr = np.ascontiguousarray(np.asarray(sel, dtype=np.int64).reshape(-1))
            n_sel = sel_arr.size
            grad = np.empty((n_sel, dim))
        else:
            grad = np.empty((r.shape[0], dim))
    rc = _load().oracle_pair_energy_grad(dim, r.shape[0], _ptr(r), _ptr(b), float(sigma),
                                         float(eps), float(alpha),
                                         _ptr(e) if want_energy else None, n_sel, _ptr(sel_arr),
                                         _ptr(grad))
    if rc != 0:
        raise ValueError("oracle_pair_energy_grad failed (%d)" % rc)
    return (float(e[0]) if want_energy else None), grad
