"""CPU-only checks of the C ABI: the library loads, exports every declared entry point, and its
host-side logic (parameter choice, mask folding, kernel transform, argument checks) is right.
No GPU call is made here."""

import math
import os
import re

import numpy as np
import pytest

from paper_2305_15693_gb300 import _build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fr():
    _build.build()
    from paper_2305_15693_gb300 import fresco
    fresco.load()
    return fresco


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "fresco.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fresco_[a-z_0-9A-Z]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(fr):
    declared = _declared_functions()
    assert len(declared) >= 15
    lib = fr.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(declared) == sorted(fr.EXPORTS)


def test_status_strings(fr):
    assert fr.status_string(0) == "ok"
    assert "argument" in fr.status_string(fr.FRESCO_ERR_ARG)
    assert fr.status_string(99) == "unknown status"


def _query(fr, mask, S0=None, W=None, n_points=1000, box=1.0, **kw):
    S0 = np.zeros(mask.shape[0]) if S0 is None else S0
    W = np.ones(mask.shape[0]) if W is None else W
    return fr.fresco_plan_query(box, mask, S0, W, n_points, fr.make_opts(**kw))


def test_parameters_of_the_named_workloads(fr):
    # 2D, K = 20, FP64 at eps = 1e-12: w = 13, n_f = 84 (smallest even 2-3-5-7-smooth >= 2*41)
    info = _query(fr, inputs.ball_mask(20, 2), precision="f64", tol=1e-12)
    assert info["width"] == 13 and info["n_fine"][:2] == [84, 84]
    assert info["beta"] == pytest.approx(2.30 * 13, rel=2e-3)
    assert info["n_rep"] == inputs.ball_count(20, 2) // 2
    # 2D, K = 757 at eps = 1e-6: w = 7, n_f = 3072
    info = _query(fr, inputs.ball_mask(757, 2), tol=1e-6)
    assert info["width"] == 7 and info["n_fine"][:2] == [3072, 3072]
    # 3D, K = 193: n_f = 784
    m3 = inputs.ball_mask(193, 3)[::97]
    m3 = np.vstack([m3, [[193, 0, 0], [0, 193, 0], [0, 0, -193]]]).astype(np.int32)
    info = _query(fr, m3, tol=1e-6)
    assert info["k_max"] == [193, 193, 193] and info["n_fine"] == [784, 784, 784]
    assert info["grad_mode"] == fr.FRESCO_GRAD_DIRECT
    info = _query(fr, m3, tol=1e-6, grad_mode="kderiv")
    assert info["grad_mode"] == fr.FRESCO_GRAD_KDERIV and info["n_fine"] == [784, 784, 784]


def _width_rule(eps, sigma):
    return max(2, math.ceil(math.log(1.0 / eps) / (math.pi * math.sqrt(1.0 - 1.0 / sigma))))


def test_fine_grid_is_smooth_and_large_enough(fr):
    """n_f is the smallest even 2-3-5-7-smooth size >= max(sigma (2K+1), 2 w_sigma, 2K+2), w_sigma
    the width rule at the requested sigma; the kernel then takes the width rule at the
    oversampling n_f / (2K+1) actually reached, which is never wider."""
    for K in (1, 2, 5, 13, 40, 101):
        for sigma in (1.25, 2.0, 2.5):
            info = _query(fr, inputs.ball_mask(K, 2), upsample=sigma)
            nf = info["n_fine"][0]
            w_sigma = _width_rule(1e-6, sigma)
            assert info["width"] == min(w_sigma, _width_rule(1e-6, nf / (2 * K + 1)))
            if info["width"] < w_sigma:
                reached = nf / (2 * K + 1)
                assert info["beta"] == pytest.approx(
                    0.976 * math.pi * (1 - 0.5 / reached) * info["width"], rel=1e-12)
            assert nf % 2 == 0 and nf >= sigma * (2 * K + 1) and nf >= 2 * w_sigma
            m = nf
            for p in (2, 3, 5, 7):
                while m % p == 0:
                    m //= p
            assert m == 1
            # smallest such: no smaller even smooth number qualifies
            for c in range(max(2, math.ceil(max(sigma * (2 * K + 1), 2 * w_sigma,
                                                2 * K + 2))), nf):
                if c % 2:
                    continue
                r = c
                for p in (2, 3, 5, 7):
                    while r % p == 0:
                        r //= p
                assert r != 1, (K, sigma, c, nf)


def test_tiles_cover_the_grid(fr):
    for K, tile in ((20, None), (20, (10, 7, 0)), (300, None), (37, (40, 40, 0))):
        info = _query(fr, inputs.ball_mask(K, 2), tile=tile)
        for a in range(2):
            nf, nb, tmax = info["n_fine"][a], info["n_tiles"][a], info["tile"][a]
            q, r = divmod(nf, nb)
            starts = [b * q + min(b, r) for b in range(nb + 1)]
            widths = np.diff(starts)
            assert starts[-1] == nf and widths.max() == tmax <= 255
            assert widths.min() >= (info["width"] + 1) // 2


def test_folding_counts_and_constant(fr):
    full = inputs.ball_mask(9, 2)
    half = full[inputs.half_space(full)]
    assert _query(fr, full)["n_rep"] == half.shape[0]
    assert _query(fr, half)["n_rep"] == half.shape[0]
    info = _query(fr, full, S0=np.full(full.shape[0], 3.5))
    assert info["loss_const"] == 0.0
    # one +-n pair with different targets and weights: W1 W2 (a - b)^2 / (W1 + W2)
    pair = np.array([[2, -1], [-2, 1]], dtype=np.int32)
    a, b, w1, w2 = 0.7, 2.9, 1.5, 0.25
    info = _query(fr, pair, S0=np.array([a, b]), W=np.array([w1, w2]))
    assert info["n_rep"] == 1
    assert info["loss_const"] == pytest.approx(w1 * w2 * (a - b) ** 2 / (w1 + w2), rel=1e-14)
    # duplicates add up; a zero-weight pair is dropped but keeps its constant
    dup = np.array([[1, 0], [1, 0], [0, 3], [0, -3]], dtype=np.int32)
    info = _query(fr, dup, S0=np.array([1.0, 3.0, 2.0, 2.0]), W=np.array([1.0, 1.0, 0.0, 0.0]))
    assert info["n_rep"] == 1
    assert info["loss_const"] == pytest.approx(2.0, rel=1e-14)   # 1 + 9 - 2 * 2^2


def test_kernel_transform_matches_adaptive_quadrature(fr):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    for w, nf in ((7, 3072), (13, 84), (4, 64)):
        beta = 2.30 * w

        def psi(u):
            z = 2.0 * u / w
            return math.exp(beta * (math.sqrt(max(0.0, 1.0 - z * z)) - 1.0))

        nus = [0, 1, nf // 8, nf // 4, nf // 2 - 1]
        got = fr.fresco_kernel_ft(w, beta, nf, nf // 2)
        for nu in nus:
            ref, _ = scipy_integrate.quad(lambda u: psi(u) * math.cos(2 * math.pi * nu * u / nf),
                                          -w / 2, w / 2, epsabs=1e-15, epsrel=1e-14, limit=400)
            assert got[nu] == pytest.approx(ref, rel=1e-12, abs=1e-15), (w, nf, nu)


def test_unreachable_tolerance_is_unsupported(fr):
    mask = inputs.ball_mask(3, 2)
    with pytest.raises(fr.FrescoError) as e:
        fr.fresco_plan_query(1.0, mask, np.zeros(mask.shape[0]), np.ones(mask.shape[0]), 10,
                             fr.make_opts("f64", tol=1e-12, upsample=1.25))
    assert e.value.status == fr.FRESCO_ERR_UNSUPPORTED


@pytest.mark.parametrize("bad", ["zero_n", "dim4", "neg_w", "nan_s0", "n0", "tol", "sigma",
                                 "grad_mode"])
def test_argument_errors(fr, bad):
    mask = inputs.ball_mask(3, 2)
    S0 = np.zeros(mask.shape[0])
    W = np.ones(mask.shape[0])
    kw = {}
    n = 100
    if bad == "zero_n":
        mask = np.vstack([mask, [[0, 0]]]).astype(np.int32)
        S0 = np.zeros(mask.shape[0])
        W = np.ones(mask.shape[0])
    elif bad == "dim4":
        mask = np.zeros((3, 4), dtype=np.int32) + 1
        S0 = np.zeros(3)
        W = np.ones(3)
    elif bad == "neg_w":
        W[3] = -1.0
    elif bad == "nan_s0":
        S0[0] = np.nan
    elif bad == "n0":
        n = 0
    elif bad == "tol":
        kw["tol"] = 2.0
    elif bad == "sigma":
        kw["upsample"] = 1.0
    elif bad == "grad_mode":
        kw["grad_mode"] = 2
    with pytest.raises(fr.FrescoError) as e:
        fr.fresco_plan_query(1.0, mask, S0, W, n, fr.make_opts(**kw))
    assert e.value.status == fr.FRESCO_ERR_ARG


@pytest.mark.parametrize("bad", ["grid_small", "grid_big", "dim4", "nan_nu", "huge_nu", "neg_w",
                                 "nan_s0", "n0", "tol", "sigma"])
def test_uwnu_argument_errors(fr, bad):
    """fresco_uwnu_plan rejects invalid arguments before it touches the device."""
    grid = (16, 12)
    nu = np.array([[0.5, -1.25], [3.0, 2.5], [-7.5, 0.0]])
    S0 = np.zeros(3)
    W = np.ones(3)
    kw = {}
    if bad == "grid_small":
        grid = (1, 12)
    elif bad == "grid_big":
        grid = (16, (1 << 20) + 2)
    elif bad == "dim4":
        grid = (4, 4, 4, 4)
        nu = np.ones((3, 4))
    elif bad == "nan_nu":
        nu[1, 0] = np.nan
    elif bad == "huge_nu":
        nu[2, 1] = 3e9
    elif bad == "neg_w":
        W[2] = -1.0
    elif bad == "nan_s0":
        S0[0] = np.inf
    elif bad == "n0":
        nu = np.zeros((0, 2))
        S0 = np.zeros(0)
        W = np.zeros(0)
    elif bad == "tol":
        kw["tol"] = 1.5
    elif bad == "sigma":
        kw["upsample"] = 3.5
    with pytest.raises(fr.FrescoError) as e:
        fr.fresco_uwnu_plan(grid, nu, S0, W, fr.make_opts(**kw))
    assert e.value.status == fr.FRESCO_ERR_ARG


def test_uwnu_unsupported_sizes(fr):
    nu = np.array([[0.5, 1.5]])
    for grid, kw in (((1 << 20, 1 << 20), {}),                        # fine grid > 4e9 cells
                     ((64, 64), {"precision": "f64", "tol": 1e-15, "upsample": 1.25})):   # w > 16
        with pytest.raises(fr.FrescoError) as e:
            fr.fresco_uwnu_plan(grid, nu, [0.0], [1.0], fr.make_opts(**kw))
        assert e.value.status == fr.FRESCO_ERR_UNSUPPORTED


def test_uwnu_profile_entry_points_reject_null_handles(fr):
    """The stage-timer and launch-count entry points of the weights-on-a-grid and type-3 plans
    answer a null handle without touching the device."""
    import ctypes
    lib = fr.load()
    ms = (ctypes.c_double * fr.FRESCO_UWNU_N_STAGES)()
    assert lib.fresco_uwnu_profile(None, 1) == fr.FRESCO_ERR_ARG
    assert lib.fresco_uwnu_profile_read(None, ms, None) == fr.FRESCO_ERR_ARG
    assert lib.fresco_nuwnu_profile(None, 1) == fr.FRESCO_ERR_ARG
    assert lib.fresco_nuwnu_profile_read(None, ms, None) == fr.FRESCO_ERR_ARG
    assert lib.fresco_uwnu_launch_count(None) == 0
    assert len(fr.UWNU_STAGES) == fr.FRESCO_UWNU_N_STAGES


def test_stage_counts_match_the_header(fr):
    src = open(os.path.join(ROOT, "include", "fresco.h")).read()
    assert int(re.search(r"#define FRESCO_UWNU_N_STAGES (\d+)", src).group(1)) == \
        fr.FRESCO_UWNU_N_STAGES
    assert int(re.search(r"#define FRESCO_N_STAGES (\d+)", src).group(1)) == fr.FRESCO_N_STAGES
