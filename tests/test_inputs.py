"""Host-side checks of the seeded workloads: mask sizes against the radii the paper prints."""

import math
import os

import numpy as np
import pytest

from paper_2305_15693_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_mask_sizes.txt")


def _paper_sizes():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            head = line.split("|")[0].split()
            rows.append((int(head[0]), int(head[1]), float(head[2]), int(head[3]),
                         float(head[4])))
    return rows


@pytest.mark.parametrize("N,dim,chi,K_paper,rtol", _paper_sizes())
def test_chi_rule_reproduces_paper_radii(N, dim, chi, K_paper, rtol):
    K = inputs.radius_for_chi(N, dim, chi)
    assert abs(K - K_paper) <= rtol * K_paper


def test_ball_count_matches_enumeration():
    for dim, K in [(2, 0), (2, 1), (2, 7), (3, 1), (3, 5)]:
        m = inputs.ball_mask(K, dim) if K > 0 else np.zeros((0, dim))
        assert m.shape[0] == inputs.ball_count(K, dim)
    assert inputs.ball_count(1, 2) == 4
    assert inputs.ball_count(1, 3) == 6
    # Gauss circle problem: N(K) -> pi K^2
    assert abs(inputs.ball_count(300, 2) / (math.pi * 300 ** 2) - 1) < 1e-3


def test_workload_sizes():
    assert inputs.workload("stealthy2d_n1e6_chi045_f32").K == 757
    assert inputs.workload("peaked2d_n1e8_chi03_f32").K == 6180
    assert inputs.workload("powerlaw3d_n2p24_chi03_f32").K == 193


def test_mask_is_symmetric_and_half_space_splits_it():
    for dim in (2, 3):
        m = inputs.ball_mask(6, dim)
        s = {tuple(r) for r in m}
        assert all(tuple(-np.asarray(r)) in s for r in m)
        h = inputs.half_space(m)
        assert h.sum() * 2 == m.shape[0]
        hs = {tuple(r) for r in m[h]}
        assert all(tuple(-np.asarray(r)) not in hs for r in m[h])


def test_seeded_points_are_reproducible():
    a = inputs.uniform_points(1000, 2, seed=0, dtype=np.float32)
    b = inputs.uniform_points(1000, 2, seed=0, dtype=np.float32)
    assert a.dtype == np.float32 and np.array_equal(a, b)
    assert a.min() >= 0 and a.max() < 1


def test_peaked_target_is_centrosymmetric():
    m = inputs.ball_mask(12, 2)
    s0 = inputs.peaked_target(m, 1000, 12)
    lut = {tuple(r): v for r, v in zip(m, s0)}
    for r, v in zip(m, s0):
        assert lut[tuple(-r)] == pytest.approx(v, rel=1e-12, abs=1e-300)
    assert s0.max() > 50


def test_variant_workloads_follow_their_recipes():
    """The NUwNU and UwNU bench workloads: seeded, sized and shaped as stated."""
    fw = inputs.free_workload("quasicrystal2d_n1e6_k1e6_f32")
    k = fw.wavevectors()
    assert k.shape == (10**6, 2) and np.abs(np.linalg.norm(k, axis=1)).max() <= fw.kmax * (1 + 1e-12)
    S0, W = fw.targets(k[:1000])
    assert (W == 1).all() and (S0 >= 0).all() and S0.max() <= fw.n_points / fw.n_peaks * 1.01
    np.testing.assert_array_equal(k[:5], fw.wavevectors()[:5])
    fld = inputs.field_workload("hexfield2d_m1024_k1e6_f32")
    c = fld.weights()
    assert c.shape == (1024, 1024) and c.dtype == np.float32 and 0 <= c.min() and c.max() < 1
    nu = fld.frequencies()
    assert nu.shape == (10**6, 2) and np.linalg.norm(nu, axis=1).max() <= fld.nu_max * (1 + 1e-12)
    # six peaks of height 10 on the ring |nu| = nu_max / 4, 60 degrees apart
    r = 0.25 * fld.nu_max
    ang = np.arange(6) * np.pi / 3
    centres = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
    S0, W = fld.targets(centres)
    assert (W == 1).all() and np.allclose(S0, 10.0, rtol=1e-6)
    S0_far, _ = fld.targets(np.array([[0.0, 0.0], [fld.nu_max, 0.0]]))
    assert S0_far.max() < 1e-100
    np.testing.assert_array_equal(nu[:5], fld.frequencies()[:5])
    with pytest.raises(KeyError):
        inputs.field_workload("nope")
