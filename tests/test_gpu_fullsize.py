"""The FAST-shaped block at full size (19 beams x 4096 channels x 200
sub-integrations x 1024 samples, 819200 cells) through mraid_run, the
launch the benchmark times (needs a GPU and ~17 GB of device memory).

The oracle checks sampled cells one by one on the same host bytes; the
masking is checked through properties that hold at any size."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import Q1_GAP, STAT_TOL, compare_eig, compare_q1, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fast_block():
    import torch
    cfg = synth.FAST_BLOCK
    h = torch.empty(cfg.nbytes, dtype=torch.uint8, pin_memory=True)
    synth.generate(cfg, out_ptr=h.data_ptr())
    return cfg, h


def test_fast_block_sampled_parity_and_mask_properties(fast_block):
    import torch
    m = lib()
    cfg, h = fast_block
    d = h.to("cuda", non_blocking=False)
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        out = plan.run(d)
        torch.cuda.synchronize()
    stat = out["stat"].cpu().numpy()
    evals = out["evals"].cpu().numpy()
    q1 = out["q1"].cpu().numpy()
    flags = out["flags"].cpu().numpy().astype(bool)
    info = out["info"]
    del d
    torch.cuda.empty_cache()

    # sampled cells against the oracle on the same bytes
    rng = np.random.default_rng(2512)
    ev = synth.events(cfg)
    idx = set(rng.integers(0, cfg.n_cells, size=384).tolist())
    idx |= {k * cfg.n_chan + c for (_, c, k, _) in ev["spike"][:64]}
    idx |= {int(rng.integers(0, cfg.n_sub)) * cfg.n_chan + c for (c, _) in ev["narrow"][:32]}
    for (_, k) in ev["burst"]:
        idx |= {k * cfg.n_chan + int(c) for c in rng.integers(0, cfg.n_chan, size=16)}
    # every cell whose q1 took the FP64 step (relative gap below 2e-3 in the
    # FP32 eigenvalues): the count equals the report's, and their q1 is
    # checked at gaps down to Q1_GAP
    l1, l2 = evals[:, 0], evals[:, 1]
    with np.errstate(divide="ignore", invalid="ignore"):
        gap32 = (l1 - l2) / l1                       # float32, as on the device
    near = (l1 > 0) & (gap32 >= np.float32(1e-6)) & (gap32 < np.float32(2e-3))
    assert info["q1_refined"] == int(near.sum()), (info["q1_refined"], int(near.sum()))
    assert near.sum() > 100, int(near.sum())      # ~0.2 % of noise cells
    idx |= set(np.flatnonzero(near).tolist())
    idx = np.array(sorted(idx))
    subs, chans = (idx // cfg.n_chan).astype(np.int32), (idx % cfg.n_chan).astype(np.int32)
    o = oracle.cells(None, cfg.n_samp_sub, subs, chans, n_threads=synth.default_threads(),
                     data_ptr=h.data_ptr(), shape=(cfg.n_beam, cfg.n_time, cfg.n_chan))
    compare_eig(evals[idx], o["evals"], "fast block")
    n_q1, _ = compare_q1(q1[idx], o["q1"], o["evals"])
    gap = (o["evals"][:, 0] - o["evals"][:, 1]) / o["evals"][:, 0]
    assert np.sum((gap >= Q1_GAP) & (gap < 1e-3)) > 50   # the band the FP64 step serves
    s_err = np.abs(stat[idx] - o["stat"]) / o["stat"]
    assert s_err.max() <= STAT_TOL, s_err.max()

    # the oracle's own clip iteration on the device's 819 200 statistics:
    # identical flags away from the threshold and the same fit (the device
    # sums s and s^2 per thread in FP32 over ~10 cells, then in FP64, so its
    # mu and sigma carry ~1e-7 relative rounding; the FP64 oracle's far less)
    f_o, i_o = oracle.flag(stat.astype(np.float64), cfg.n_chan)
    for key in ("mu", "sigma", "thresh"):
        assert abs(info[key] - i_o[key]) <= 1e-6 * abs(i_o[key]), (key, info[key], i_o[key])
    assert info["iterations"] == i_o["iterations"]
    s64 = stat.astype(np.float64)
    band = STAT_TOL * s64 + abs(info["thresh"] - i_o["thresh"])
    at_thresh = np.abs(s64 - i_o["thresh"]) <= band
    diff = flags != f_o.astype(bool)
    assert not np.any(diff & ~at_thresh), (int((diff & ~at_thresh).sum()), int(diff.sum()))

    # masking properties: the reported fit is the fit of the unmasked cells,
    # every unmasked cell is at or below the final threshold, and the loop
    # converged
    assert info["converged"] == 1 and info["timed_out"] == 0
    un = stat[~flags].astype(np.float64)
    assert un.size == info["n_used"]
    assert abs(un.mean() - info["mu"]) <= 1e-9 * abs(info["mu"])
    assert abs(un.std() - info["sigma"]) <= 1e-6 * info["sigma"]
    assert np.all(un <= info["thresh"])
    assert abs(info["thresh"] - (info["mu"] + 3.0 * info["sigma"])) <= 1e-12
    assert flags.sum() == info["n_flagged"]

    # behaviour: beam-common RFI flagged, single-beam pulses not
    F = flags.reshape(cfg.n_sub, cfg.n_chan)
    for (c, _) in ev["narrow"]:
        assert F[:, c].all(), c
    for (_, k) in ev["burst"]:
        assert F[k].mean() > 0.99 and F[k + 1].mean() > 0.99
    spikes = [(k, c) for (_, c, k, _) in ev["spike"]]
    assert np.mean([F[k, c] for (k, c) in spikes]) < 0.05


def check_mask(stat, flags, info, k_sigma=3.0):
    """The reported fit is the fit of the unmasked cells and every unmasked
    cell is at or below the final threshold."""
    assert info["converged"] == 1 and info["timed_out"] == 0
    un = stat[~flags].astype(np.float64)
    assert un.size == info["n_used"]
    assert abs(un.mean() - info["mu"]) <= 1e-9 * abs(info["mu"])
    assert abs(un.std() - info["sigma"]) <= 1e-6 * info["sigma"]
    assert np.all(un <= info["thresh"])
    assert abs(info["thresh"] - (info["mu"] + k_sigma * info["sigma"])) <= 1e-12
    assert flags.sum() == info["n_flagged"]


def test_fast_block_seven_timescales(fast_block):
    """Table 1's seven sub-interval lengths (0.05 s to 10 s) in one
    mraid_multires call on the full block: sampled cells of every level
    against the oracle run at that level's sub-integration length, and the
    masking properties per level."""
    import torch
    m = lib()
    cfg, h = fast_block
    d = h.to("cuda", non_blocking=False)
    factors = [1, 4, 10, 20, 40, 100, 200]
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        levels = plan.multires(d, factors)
    del d
    torch.cuda.empty_cache()
    rng = np.random.default_rng(77)
    for lv in levels:
        f = lv["factor"]
        n_f = cfg.n_sub // f
        stat = lv["stat"].cpu().numpy()
        flags = lv["flags"].cpu().numpy().astype(bool)
        assert stat.shape == (n_f * cfg.n_chan,)
        check_mask(stat, flags, lv["info"])
        idx = np.unique(rng.integers(0, n_f * cfg.n_chan, size=24 if f <= 20 else 8))
        subs, chans = (idx // cfg.n_chan).astype(np.int32), (idx % cfg.n_chan).astype(np.int32)
        o = oracle.cells(None, f * cfg.n_samp_sub, subs, chans, n_threads=synth.default_threads(),
                         data_ptr=h.data_ptr(), shape=(cfg.n_beam, cfg.n_time, cfg.n_chan))
        s_err = np.abs(stat[idx] - o["stat"]) / o["stat"]
        assert s_err.max() <= STAT_TOL, (f, s_err.max())


def test_fast_block_bandpass_path(fast_block):
    """The bandpass-centred path on the full block with 1 s fit intervals:
    the baselines of two intervals (all 19 beams) against the oracle's ArPLS
    of the oracle's time-aggregated spectra, the statistic of sampled cells
    in those intervals from the oracle's CCM about the oracle's baselines,
    and the masking properties."""
    import torch
    m = lib()
    cfg, h = fast_block
    d = h.to("cuda", non_blocking=False)
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        out = plan.run_bandpass(d, evals=False)
    del d
    torch.cuda.empty_cache()
    bp = m.mraid_default_bandpass_params()
    band = out["bandpass"].cpu().numpy()
    stat = out["stat"].cpu().numpy()
    flags = out["flags"].cpu().numpy().astype(bool)
    check_mask(stat, flags, out["info"])
    data = h.numpy().reshape(cfg.n_beam, cfg.n_time, cfg.n_chan)
    rng = np.random.default_rng(78)
    for I in (0, 7):
        s0 = I * bp.interval
        z = np.empty((cfg.n_beam, cfg.n_chan))
        for a in range(cfg.n_beam):
            y = oracle.bandpass_input(data, cfg.n_samp_sub, s0, bp.interval, a)
            z[a], _ = oracle.arpls(y, bp.lam, bp.ratio, bp.itermax)
        np.testing.assert_allclose(band[I], z, rtol=2e-7)
        for _ in range(6):
            k = s0 + int(rng.integers(0, bp.interval))
            c = int(rng.integers(0, cfg.n_chan))
            C = oracle.cell_ccm_bandpass(data, cfg.n_samp_sub, k, c, z[:, c])
            so = oracle.stat(oracle.jacobi(C)[0])
            assert abs(stat[k * cfg.n_chan + c] - so) <= STAT_TOL * so, (I, k, c)


def test_fast_block_two_polarisations(fast_block):
    """Two recorded polarisations at full size (31.9 GB on the device): the
    block as polarisation 0 and the next seed's block as polarisation 1,
    through mraid_run_pol2 on the tensor cores, the launch the benchmark
    times. Sampled cells against the oracle's total-power path, the masking
    properties, the beam-common narrowband RFI of either polarisation
    flagged and single-beam pulses away from any other event not."""
    import torch
    m = lib()
    cfg, h = fast_block
    nb = cfg.nbytes
    cfg1 = cfg.replace(seed=cfg.seed + 1)
    h2 = torch.empty(2 * nb, dtype=torch.uint8, pin_memory=True)
    h2[:nb].copy_(h)
    synth.generate(cfg1, out_ptr=h2.data_ptr() + nb)
    d = h2.to("cuda", non_blocking=False)
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        m.mraid_profile_enable(plan.handle)
        out = plan.run_pol2(d)
        ran = m.mraid_profile_read(plan.handle)
    assert "gram_tc" in ran and "pol2_fold" not in ran, ran
    stat = out["stat"].cpu().numpy()
    evals = out["evals"].cpu().numpy()
    q1 = out["q1"].cpu().numpy()
    flags = out["flags"].cpu().numpy().astype(bool)
    del d
    torch.cuda.empty_cache()
    check_mask(stat, flags, out["info"])

    ev0, ev1 = synth.events(cfg), synth.events(cfg1)
    rng = np.random.default_rng(2513)
    idx = set(rng.integers(0, cfg.n_cells, size=192).tolist())
    for ev in (ev0, ev1):
        idx |= {k * cfg.n_chan + c for (_, c, k, _) in ev["spike"][:16]}
        idx |= {int(rng.integers(0, cfg.n_sub)) * cfg.n_chan + c for (c, _) in ev["narrow"][:16]}
    idx = np.array(sorted(idx))
    data = h2.numpy().reshape(2 * cfg.n_beam, cfg.n_time, cfg.n_chan)
    o = oracle.cells_pol2(data, cfg.n_samp_sub, (idx // cfg.n_chan).astype(np.int32),
                          (idx % cfg.n_chan).astype(np.int32), n_threads=synth.default_threads())
    compare_eig(evals[idx], o["evals"], "two polarisations, fast block")
    compare_q1(q1[idx], o["q1"], o["evals"])
    s_err = np.abs(stat[idx] - o["stat"]) / o["stat"]
    assert s_err.max() <= STAT_TOL, s_err.max()

    F = flags.reshape(cfg.n_sub, cfg.n_chan)
    for (c, _) in ev0["narrow"] + ev1["narrow"]:
        assert F[:, c].mean() > 0.9, c
    busy = set()
    for c_ in (cfg, cfg1):
        cells = synth.rfi_cells(c_)
        busy |= cells["narrow"] | cells["burst"]
    lone = [(k, c) for ev in (ev0, ev1) for (_, c, k, _) in ev["spike"] if (k, c) not in busy]
    assert len(lone) > 100
    assert np.mean([F[k, c] for (k, c) in lone]) < 0.05


def test_fast_block_float32_full_size(fast_block):
    """Float32 input (bit_depth 32) at its configured size, the size the
    benchmark times: all 200 sub-integrations (204 800 samples per beam and
    channel) of the block as (x - 128) / 20, 63.75 GB on the device, through
    mraid_run on the tensor cores; sampled cells against the oracle's FP64
    covariance path, and the masking properties."""
    import torch
    m = lib()
    cfg, h = fast_block
    N, C, S, K = cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub
    d = h.to("cuda", non_blocking=False)
    x = d.view(N, cfg.n_time, C)[:, :K * S, :].float().sub_(128.0).div_(20.0).contiguous()
    del d
    with m.Plan(N, C, S, K, bit_depth=32) as plan:
        m.mraid_profile_enable(plan.handle)
        out = plan.run(x)
        ran = m.mraid_profile_read(plan.handle)
    assert "gram_tc_f32" in ran, ran
    evals = out["evals"].cpu().numpy()
    stat = out["stat"].cpu().numpy()
    flags = out["flags"].cpu().numpy().astype(bool)
    check_mask(stat, flags, out["info"])
    rng = np.random.default_rng(2514)
    idx = np.unique(rng.integers(0, K * C, size=128))
    ev_o = np.zeros((idx.size, N))
    for j, i in enumerate(idx):
        k, c = int(i // C), int(i % C)
        cell = x[:, k * S:(k + 1) * S, c:c + 1].contiguous().cpu().numpy()
        r, _ = oracle.corr_from_cov(oracle.cell_cov_f32(cell, S, 0, 0))
        ev_o[j] = oracle.jacobi(r)[0]
    del x
    torch.cuda.empty_cache()
    compare_eig(evals[idx], ev_o, "float32, fast block")
    st_o = np.array([oracle.stat(e) for e in ev_o])
    s_err = np.abs(stat[idx] - st_o) / st_o
    assert s_err.max() <= STAT_TOL, s_err.max()
