"""CPU checks of bench.py's host logic that shapes the reported numbers: the algorithmic bytes per
stage (the roofline numerators) at the bench workload's sizes, and the clock record's reduction
of nvidia-smi samples (median SM clock, throttle reasons seen)."""

import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _info(grad_mode, dim=2, nf=20736, kx=6180, n_rep=59_992_318):
    return {"dim": dim, "n_fine": [nf] * dim + [1] * (3 - dim), "k_max": [kx] * dim + [0] * (3 - dim),
            "n_rep": n_rep, "grad_mode": grad_mode}


def test_stage_bytes_per_unit_fp32_2d_kderiv():
    N, nf = 100_000_000, 20736
    cells = nf * nf
    b = bench.stage_bytes(_info(1), N, 4)
    assert b["sort"] == 20 * N                                   # 8 read + 8 packed + 4 index
    assert b["spread"] == 8 * N + 4 * cells
    assert b["mask"] == 32 * 59_992_318                          # n (8) + S0, W (8) + F (8) + E (8)
    assert b["interp"] == 4 * cells + 20 * N
    assert b["fft_fwd"] == 4 * cells + nf * (nf // 2 + 1) * 8    # real grid in, half spectrum out
    assert b["fft_inv"] == nf * (6180 + 1) * 8 + 4 * cells
    assert b["loss"] == 0


def test_stage_bytes_direct_mode_and_3d():
    N = 1 << 24
    b2 = bench.stage_bytes(_info(0, nf=4096, kx=1000, n_rep=10), N, 4)
    cells = 4096 * 4096
    assert b2["interp"] == cells * 8 + 20 * N                    # one complex grid (x + iy)
    assert b2["mask"] == 10 * (8 + 8 + 8 + 2 * 8)
    b3 = bench.stage_bytes(_info(1, dim=3, nf=648, kx=193, n_rep=15_055_467), N, 4)
    cells = 648 ** 3
    assert b3["sort"] == N * (12 + 16 + 4)
    assert b3["interp"] == 4 * cells + N * (16 + 4 + 12)
    b3f64 = bench.stage_bytes(_info(1, dim=3, nf=648, kx=193, n_rep=15_055_467), N, 8)
    assert b3f64["spread"] == 2 * b3["spread"]


def test_clock_record_reduction():
    c = bench.ClockSampler(None)
    c.proc = None
    assert c.stop() is None                                      # no sampler, no record

    class _P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.ClockSampler(None)
    c.proc = _P()
    c.rows = [["2070", "2070", "700", "0x0", "Not Active", "Not Active", "Not Active", "Active"],
              ["2055", "2070", "710", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["1980", "2070", "720", "0x8", "Active", "Not Active", "Not Active", "Not Active"],
              ["[N/A]", "2070", "0", "0x0", "", "", "", ""]]
    rec = c.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == pytest.approx(2055.0)
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_traffic_sources_exist_and_hash_is_stable():
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2305_15693_gb300", "csrc")
    names = bench.traffic_sources()
    assert "fresco_kernels.cuh" in names and "fresco_tiles.cuh" in names
    assert "fresco_host.cu" in names and "fresco_uwnu.cu" not in names
    for name in names:
        assert os.path.isfile(os.path.join(csrc, name)), name
    h = bench._kernel_source_hash()
    assert len(h) == 16 and h == bench._kernel_source_hash()


def test_rho_error_report_bins_and_row_maximum():
    import numpy as np
    K = 100
    rows = np.array([[10, 0], [0, 30], [60, 0], [0, 90], [70, 70]])   # |n|/K: .1 .3 .6 .9 .99
    want = np.array([3 + 4j, 5.0, 1j * 5, -5.0, 4 - 3j])              # every |rho| = 5
    got = want.copy()
    got[3] += 0.5                                                     # one row off by 0.1 |rho|
    rep = bench.rho_error_report(got, want, rows, K)
    assert rep["rows"] == 5
    assert rep["rel_l2"] == pytest.approx(0.5 / np.sqrt(5 * 25))
    assert rep["max_row_err_over_rms"] == pytest.approx(0.1)
    bins = {tuple(b["n_over_K"]): b for b in rep["by_n_over_K"]}
    assert bins[(0.0, 0.25)]["rows"] == 1 and bins[(0.0, 0.25)]["rel_l2"] == 0.0
    assert bins[(0.75, 1.0)]["rows"] == 2
    assert bins[(0.75, 1.0)]["rel_l2"] == pytest.approx(0.5 / np.sqrt(50))


def test_smem_roofline_counts_w_to_the_d_operations_per_point():
    stages = {"spread": {"ms": 2.0}, "interp": {"ms": 4.0}}
    out = bench.smem_rooflines(stages, 10**8, 2, 7, {"atomic_add": 9.8e12, "load": 9.8e12})
    assert out["spread"]["ops_per_launch"] == 49e8
    assert out["spread"]["achieved_ops_per_s"] == pytest.approx(49e8 / 2e-3)
    assert out["spread"]["frac"] == pytest.approx(49e8 / 2e-3 / 9.8e12, abs=1e-4)
    assert out["interp"]["frac"] == pytest.approx(49e8 / 4e-3 / 9.8e12, abs=1e-4)
    out3 = bench.smem_rooflines(stages, 1 << 24, 3, 7, {"atomic_add": 1.0, "load": 1.0})
    assert out3["spread"]["ops_per_launch"] == float((1 << 24) * 343)


def test_uwnu_traffic_sources_and_constraint_bytes():
    assert bench.traffic_sources("uwnu") == ["fresco_internal.h", "fresco_kernels.cuh",
                                             "fresco_uwnu.cu", "fresco_uwnu_tiles.h"]
    h = bench._kernel_source_hash("uwnu")
    assert len(h) == 16 and h != bench._kernel_source_hash()
    # 2D FP32, 10 constraints, a 4 x 4 fine grid: interp reads the grid once (128 B) and per
    # constraint cell + position (16 B), target and weight (8 B), caller index (4 B), writes the
    # strength and S (12 B); spread reads cell + position + strength (24 B) and writes the grid
    b = bench.constraint_side_bytes(2, 10, 16, 4, False)
    assert b == {"interp": 128 + 10 * 40, "spread": 10 * 24 + 128}
    assert bench.constraint_side_bytes(2, 10, 16, 4, True)["interp"] == 128 + 10 * 44
