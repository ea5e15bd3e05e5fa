"""Two recorded polarisations (Section 2): Eq. 1 of the total power, on the
GPU against the oracle through the C ABI (needs a GPU). The sums are exact
(bit for bit); eigenvalues, statistic and flags at the Pearson path's
tolerances."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import STAT_TOL, compare_eig, compare_flags, lib, unpack_sums

pytestmark = pytest.mark.gpu


def two_pol_block(n_beam, n_chan, n_s, n_sub, seed, n_burst=1):
    """Polarisation 0 and 1 of every beam: two independent synthetic blocks
    (each with its own RFI events), stacked polarisation-major."""
    cfg = synth.SMALL.replace(n_beam=n_beam, n_chan=n_chan, n_samp_sub=n_s, n_sub=n_sub,
                              seed=seed, n_burst=n_burst)
    p0 = synth.generate(cfg)
    p1 = synth.generate(cfg.replace(seed=seed + 1))
    return cfg, np.ascontiguousarray(np.concatenate([p0, p1], axis=0))


@pytest.mark.parametrize("n_beam,n_chan,n_s,n_sub,route", [
    (19, 48, 512, 3, "tc"),       # tensor cores add the polarisations; 2 pieces of 256
    (19, 48, 384, 2, "tc"),       # 2 pieces of 192 (the largest divisor within 256)
    (23, 16, 256, 4, "tc"),       # the most beams the tensor-core Gram takes
    (19, 32, 128, 6, "tc"),       # one piece
    (7, 40, 128, 6, "stacked"),   # 40 channels: the stacked 2N-block Gram on CUDA cores
    (30, 16, 64, 4, "stacked"),   # 30 beams: beyond the tensor-core kernel
])
def test_pol2_sums_exact(n_beam, n_chan, n_s, n_sub, route):
    import torch
    m = lib()
    cfg, data = two_pol_block(n_beam, n_chan, n_s, n_sub, 31 + n_beam)
    # extreme samples too: both polarisations 255 and 0 in places
    data[:, :n_s // 4, 0] = 255
    data[:, n_s // 4:n_s // 2, 1] = 0
    d = torch.from_numpy(data).cuda()
    with m.Plan(n_beam, n_chan, n_s, n_sub) as plan:
        m.mraid_profile_enable(plan.handle)
        sums, _ = plan.ccm_pol2(d, corr=False)
        plan.sync()
        ran = m.mraid_profile_read(plan.handle)
    assert ("pol2_fold" in ran) == (route == "stacked"), ran
    assert ("gram_tc" in ran) == (route == "tc"), ran
    G = unpack_sums(sums.cpu().numpy(), n_beam)
    for k in range(n_sub):
        for c in range(n_chan):
            np.testing.assert_array_equal(G[k * n_chan + c],
                                          oracle.cell_gram_pol2(data, n_s, k, c))


@pytest.mark.parametrize("S,C", [(256, 64), (128, 40)])   # tensor cores; stacked CUDA-core Gram
def test_pol2_run_matches_oracle(S, C):
    import torch
    m = lib()
    # no broadband bursts: in a block of 32 sub-integrations each burst
    # covers 2, and with the narrowband channels a fifth of the cells would
    # sit near s ~ 0.85, lifting mu + 3 sigma above 1 (nothing flagged)
    N, K = 19, 32
    cfg, data = two_pol_block(N, C, S, K, 101, n_burst=0)
    d = torch.from_numpy(data).cuda()
    with m.Plan(N, C, S, K) as plan:
        out = plan.run_pol2(d)
    subs = np.repeat(np.arange(K, dtype=np.int32), C)
    chans = np.tile(np.arange(C, dtype=np.int32), K)
    o = oracle.cells_pol2(data, S, subs, chans, n_threads=synth.default_threads())
    compare_eig(out["evals"].cpu().numpy(), o["evals"], "pol2")
    st = out["stat"].cpu().numpy()
    s_err = np.abs(st - o["stat"]) / np.maximum(o["stat"], 1e-30)
    assert s_err.max() <= STAT_TOL, s_err.max()
    f_o, i_o = oracle.flag(o["stat"], C)
    compare_flags(out["flags"].cpu().numpy(), f_o, o["stat"], out["info"], i_o)
    # the narrowband channels of either polarisation are flagged
    F = out["flags"].cpu().numpy().reshape(K, C).astype(bool)
    for (c, _) in synth.events(cfg)["narrow"] + synth.events(cfg.replace(seed=102))["narrow"]:
        assert F[:, c].mean() > 0.9, c


@pytest.mark.parametrize("S,C", [(256, 64), (128, 40)])
def test_pol2_with_silent_second_polarisation_equals_single(S, C):
    """Polarisation 1 all zero: the total power is polarisation 0, and the
    statistic and flags equal mraid_run's on polarisation 0 alone."""
    import torch
    m = lib()
    N, K = 19, 16
    cfg, data = two_pol_block(N, C, S, K, 7)
    data[N:] = 0
    d = torch.from_numpy(data).cuda()
    single = torch.from_numpy(np.ascontiguousarray(data[:N])).cuda()
    with m.Plan(N, C, S, K) as plan:
        a = plan.run_pol2(d, q1=False)
        b = plan.run(single, q1=False)
    np.testing.assert_array_equal(a["stat"].cpu().numpy(), b["stat"].cpu().numpy())
    np.testing.assert_array_equal(a["flags"].cpu().numpy(), b["flags"].cpu().numpy())


def test_pol2_rejects_unsupported_plans():
    import torch
    m = lib()
    code = {name: v for v, name in m.STATUS.items()}
    st = torch.empty(4 * 16, device="cuda")
    fl = torch.empty(4 * 16, dtype=torch.uint8, device="cuda")
    d = torch.zeros(2 * 65, 4 * 32, 16, dtype=torch.uint8, device="cuda")
    with m.Plan(65, 16, 32, 4) as plan:                     # 130 stacked blocks
        with pytest.raises(m.MraidError) as ei:
            m.mraid_run_pol2(plan.handle, d, None, None, st, fl)
        assert ei.value.status == code["MRAID_ERR_UNSUPPORTED"]
    x = torch.zeros(2 * 4, 4 * 32, 16, device="cuda")
    with m.Plan(4, 16, 32, 4, bit_depth=32) as plan:
        with pytest.raises(m.MraidError) as ei:
            m.mraid_run_pol2(plan.handle, x, None, None, st, fl)
        assert ei.value.status == code["MRAID_ERR_UNSUPPORTED"]
