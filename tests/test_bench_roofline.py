"""The benchmark's roofline arithmetic (CPU): algorithmic work per launch
from the per-cell figures (tensor-core Gram: N n_s bytes of samples in, its
4 N(N+1)/2 bytes of correlation export reported apart; eigensolver: the (4/3) N^3 flops of a
dense tridiagonal reduction; mask: 5 bytes per cell), achieved = work over
the launch time, frac = achieved over the peak, and the FP32 peak derived
from 152 SMs x 128 lanes x 2 flops x the maximum SM clock."""
import json
import os

import pytest

import bench


def test_fast_block_work_per_launch_and_fractions():
    cfg = bench.workload("fast_block", 0)[0]
    N, S, cells = cfg.n_beam, cfg.n_samp_sub, cfg.n_cells
    assert (N, S, cells) == (19, 1024, 819200)
    peaks = {"hbm_gbs": 6785.9, "source": "measured", "fp32_tflops": 80.54784}
    kt = {"gram_tc": (1, 4.5), "eig": (1, 1.5), "flag_clip": (1, 0.1)}
    r = bench.kernel_rooflines(cfg, kt, peaks)
    gram = cells * N * S                                  # samples in, read once
    assert gram == 15_938_355_200
    assert r["gram_tc"]["work_per_launch"] == gram
    assert r["gram_tc"]["achieved"] == pytest.approx(gram / 4.5e-3 / 1e9)
    assert r["gram_tc"]["frac"] == pytest.approx(gram / 4.5e-3 / 1e9 / 6785.9)
    export = cells * 4 * N * (N + 1) // 2                 # packed r, reported apart
    assert r["gram_tc"]["export_bytes"] == export
    assert r["gram_tc"]["frac_incl_export"] == pytest.approx(
        (gram + export) / 4.5e-3 / 1e9 / 6785.9)
    assert r["gram_tc"]["bound"] == "hbm" and r["gram_tc"]["unit"] == "GB/s"
    flops = cells * 4.0 * N ** 3 / 3.0
    assert r["eig"]["work_per_launch"] == pytest.approx(flops)
    assert r["eig"]["achieved"] == pytest.approx(flops / 1.5e-3 / 1e12)
    assert r["eig"]["frac"] == pytest.approx(flops / 1.5e-3 / 1e12 / 80.54784)
    assert r["eig"]["bound"] == "alu" and r["eig"]["unit"] == "TFLOP/s"
    assert r["flag_clip"]["work_per_launch"] == 5 * cells


def test_fp32_peak_is_derived_from_the_unit_counts():
    p = bench.measured_peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    mhz = 2070.0
    if os.path.exists(path) and p["source"] == "measured":
        with open(path) as f:
            d = json.load(f)
        assert p["hbm_gbs"] == float(d["hbm_gbs"])
        mhz = float(d.get("sm_max_mhz", 2070.0))
    assert p["fp32_tflops"] == pytest.approx(152 * 128 * 2 * mhz * 1e6 / 1e12)


def test_batched_fractions():
    import synth
    shapes = synth.BATCH_SHAPES
    peaks = {"hbm_gbs": 6785.9, "source": "measured", "fp32_tflops": 80.54784}
    f = bench.batched_fractions(shapes, 28.0, peaks)
    nbytes = sum(c.n_beam * c.n_sub * c.n_samp_sub * c.n_chan
                 + c.n_sub * c.n_chan * (5 + 8 * c.n_beam) for c in shapes)
    flops = sum(c.n_sub * c.n_chan * 4.0 * c.n_beam ** 3 / 3.0 for c in shapes)
    assert f["hbm"]["bytes_per_pass"] == nbytes
    assert f["hbm"]["frac"] == pytest.approx(nbytes / 28e-3 / 1e9 / 6785.9)
    assert f["alu"]["flops_per_pass"] == pytest.approx(flops)
    assert f["alu"]["frac"] == pytest.approx(flops / 28e-3 / 1e12 / 80.54784)
    assert [c.n_beam for c in shapes] == [13, 19, 36, 72]
