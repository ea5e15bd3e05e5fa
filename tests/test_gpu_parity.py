"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

Tolerances (tests/gpu_util.py): Gram sums bit-exact; correlation 2e-6;
eigenvalues 1e-4 of lambda_max per cell; q1 1e-3 where the oracle's relative
gap is >= 1e-2; flags identical except cells whose oracle statistic is
within 2e-4 s (+ the threshold difference) of the oracle threshold.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (all_cells, compare_eig, compare_flags, compare_q1, gpu_stages,
                      unpack_corr, unpack_sums, CORR_TOL, STAT_TOL)

pytestmark = pytest.mark.gpu


def oracle_all(data, n_samp_sub, n_threads=None):
    n_beam, n_time, n_chan = data.shape
    subs, chans = all_cells(n_time // n_samp_sub, n_chan)
    return oracle.cells(data, n_samp_sub, subs, chans, n_threads=n_threads or synth.default_threads())


def check_block(data, n_samp_sub, keep=None, check_flags=True, label=""):
    n_beam, n_time, n_chan = data.shape
    g = gpu_stages(data, n_samp_sub, keep=keep)
    o = oracle_all(data, n_samp_sub)
    # Eq. 1: exact sums
    np.testing.assert_array_equal(unpack_sums(g["sums"], n_beam), o["G"], err_msg=label)
    # correlation from the exact sums
    corr_g = unpack_corr(g["corr"], n_beam)
    worst = 0.0
    for i in range(0, o["G"].shape[0], max(1, o["G"].shape[0] // 512)):
        r, _ = oracle.corr_from_gram(o["G"][i])
        worst = max(worst, float(np.abs(corr_g[i] - r).max()))
    assert worst <= CORR_TOL, (label, worst)
    # Eq. 2
    emax, e99 = compare_eig(g["evals"], o["evals"], label)
    compare_q1(g["q1"], o["q1"], o["evals"])
    s_err = np.abs(g["stat"] - o["stat"]) / np.maximum(o["stat"], 1e-30)
    assert s_err.max() <= STAT_TOL, (label, s_err.max())
    # the fused run gives the same per-cell results as the stages
    np.testing.assert_array_equal(g["run"]["stat"], g["stat"])
    np.testing.assert_array_equal(g["run"]["evals"], g["evals"])
    if check_flags:
        f_o, i_o = oracle.flag(o["stat"], n_chan, keep)
        near, diff = compare_flags(g["flags"], f_o, o["stat"], g["info"], i_o, keep, n_chan)
        np.testing.assert_array_equal(g["run"]["flags"], g["flags"])
        assert g["info"]["iterations"] >= 1
    return g, o, (emax, e99)


def test_small_block_parity():
    """19 beams x 64 channels x 256 x 128 with narrowband, broadband and
    single-beam RFI: every cell against the oracle."""
    data = synth.generate(synth.SMALL)
    g, o, (emax, e99) = check_block(data, synth.SMALL.n_samp_sub, label="small")
    f_o, i_o = oracle.flag(o["stat"], synth.SMALL.n_chan)
    assert abs(g["info"]["thresh"] - i_o["thresh"]) < 1e-6
    assert g["info"]["converged"] == 1
    cells = synth.rfi_cells(synth.SMALL)
    F = g["flags"].reshape(synth.SMALL.n_sub, synth.SMALL.n_chan)
    assert all(F[k, c] for (k, c) in cells["narrow"] | cells["burst"])
    assert not any(F[k, c] for (k, c) in cells["spike"])


@pytest.mark.parametrize("n_beam,n_chan,n_samp_sub,n_sub", [
    (19, 37, 100, 3),    # ragged channels (byte staging) and a partial time chunk
    (19, 8, 1024, 4),    # FAST sub-integration length
    (2, 12, 64, 5),
    (3, 9, 33, 4),
    (4, 16, 96, 3),
    (13, 20, 512, 3),    # 13-beam receiver
    (5, 10, 48, 2),      # shared-memory Jacobi
    (36, 6, 256, 2),     # PAF-like
    (72, 3, 512, 2),     # PAF-like
])
def test_shapes_parity(n_beam, n_chan, n_samp_sub, n_sub):
    cfg = synth.SynthConfig(n_beam=n_beam, n_chan=n_chan, n_samp_sub=n_samp_sub, n_sub=n_sub,
                            seed=1000 + n_beam * 7 + n_chan, bandpass=1, n_narrow=1,
                            n_burst=1 if n_sub > 1 else 0, n_spike=1)
    data = synth.generate(cfg)
    check_block(data, n_samp_sub, check_flags=n_chan * n_sub >= 16, label=str(cfg))


@pytest.mark.parametrize("n_beam,n_chan,n_samp_sub,n_sub", [
    (19, 32, 1024, 3),   # FAST cell shape on the tensor-core Gram
    (13, 16, 512, 4),    # 13-beam receiver, one 16-channel box
    (2, 16, 64, 3),
    (15, 32, 128, 2),    # beams + ones = 16 rows: one MMA per group
    (16, 16, 192, 2),    # 17 rows: second MMA begins
    (23, 16, 64, 3),     # 24 rows: the largest tensor-core shape
])
def test_tensor_core_gram_shapes(n_beam, n_chan, n_samp_sub, n_sub):
    cfg = synth.SynthConfig(n_beam=n_beam, n_chan=n_chan, n_samp_sub=n_samp_sub, n_sub=n_sub,
                            seed=2000 + n_beam * 7 + n_chan, bandpass=1, n_narrow=1,
                            n_burst=1, n_spike=1)
    data = synth.generate(cfg)
    check_block(data, n_samp_sub, check_flags=n_chan * n_sub >= 32, label=str(cfg))


def test_long_subintegration_segments_exact():
    """n_s > 32768 exercises the int32 -> int64 segment flush."""
    rng = np.random.default_rng(5)
    data = rng.integers(200, 256, size=(3, 2 * 40000, 4), dtype=np.uint8)
    g = gpu_stages(data, 40000)
    o = oracle_all(data, 40000)
    np.testing.assert_array_equal(unpack_sums(g["sums"], 3), o["G"])


def test_extreme_and_zero_variance():
    rng = np.random.default_rng(6)
    data = rng.integers(0, 256, size=(19, 4 * 64, 8), dtype=np.uint8)
    data[:, :, 0] = 255                  # channel 0: every beam constant
    data[3, 64:128, 1] = 0               # beam 3 constant in cell (1, 1)
    data[:, 128:192, 2] = rng.integers(0, 2, size=(19, 64), dtype=np.uint8) * 255
    g = gpu_stages(data, 64)
    o = oracle_all(data, 64)
    np.testing.assert_array_equal(unpack_sums(g["sums"], 19), o["G"])
    compare_eig(g["evals"], o["evals"], "extreme")
    # constant channel: r = I, all eigenvalues one
    np.testing.assert_allclose(g["evals"][0], np.ones(19), atol=1e-6)
    assert g["run"]["info"]["n_degenerate"] == 4 * 19 + 1


def test_keep_channels_are_never_flagged():
    cfg = synth.SMALL
    data = synth.generate(cfg)
    keep = np.zeros(cfg.n_chan, dtype=np.uint8)
    ev = synth.events(cfg)
    keep[ev["narrow"][0][0]] = 1         # preserve one RFI channel (e.g. an HI line)
    keep[10] = 1
    check_block(data, cfg.n_samp_sub, keep=keep, label="keep")


def test_deterministic_and_host_path_matches():
    import torch
    import paper_2512_16278_gb300 as m
    cfg = synth.SMALL
    data = synth.generate(cfg)
    d = torch.from_numpy(data).cuda()
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        a = plan.run(d)
        b = plan.run(d)
        for k in ("evals", "q1", "stat", "flags"):
            assert torch.equal(a[k], b[k]), k
        h = torch.from_numpy(data).pin_memory()
        h_stat = torch.empty(cfg.n_cells, dtype=torch.float32, pin_memory=True)
        h_flags, info = plan.run_host(h, h_stat=h_stat)
        assert torch.equal(h_flags, a["flags"].cpu())
        assert torch.equal(h_stat, a["stat"].cpu())
        assert info["n_flagged"] == a["info"]["n_flagged"]


def test_invalid_calls_return_status():
    import torch
    import paper_2512_16278_gb300 as m
    with m.Plan(19, 8, 64, 2) as plan:
        with pytest.raises(m.MraidError) as e:
            m.mraid_ccm(plan.handle, None, None, None)
        assert e.value.status == 1
        with pytest.raises(m.MraidError):
            m.mraid_run(plan.handle, torch.empty(1, device="cuda"), None, None, None, None)
