"""Section 3.1 bandpass (ArPLS) and the bandpass-centred CCM on the GPU
against the FP64 oracle, through the C ABI (needs a GPU).

ArPLS runs in FP64 on both sides with the same steps, so baselines agree to
rounding and the solve counts are equal. The CCM about the bandpass is FP32
on the GPU from the exact integer covariance; eigenvalues, statistic and
flags are held to the tolerances of the Pearson path."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import STAT_TOL, compare_eig, compare_flags, lib

pytestmark = pytest.mark.gpu


def spectra(n_sys, n, seed):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    y = np.empty((n_sys, n))
    for i in range(n_sys):
        base = 110 + 30 * np.sin(2 + 3 * x * (1 + i % 3)) + 10 * x * x
        y[i] = base + rng.normal(scale=0.3 + 0.2 * (i % 4), size=n)
        k = max(1, n // 40)
        y[i, rng.choice(n, k, replace=False)] += rng.uniform(5, 50, size=k)
    return y


@pytest.mark.parametrize("n,lam,ratio,itermax", [
    (3, 10.0, 1e-3, 20),
    (64, 1e3, 1e-3, 50),
    (4096, 1e5, 1e-3, 50),     # FAST's channel count, arrays in shared memory
    (5000, 1e5, 1e-4, 30),     # too long for shared memory: global arrays
])
def test_arpls_matches_oracle(n, lam, ratio, itermax):
    import torch
    m = lib()
    y = spectra(12, n, n)
    d_y = torch.from_numpy(y).cuda()
    with m.Plan(2, 16, 16, 1) as plan:
        z, it = plan.arpls(d_y, lam=lam, ratio=ratio, itermax=itermax)
    z = z.cpu().numpy()
    it = it.cpu().numpy()
    for i in range(y.shape[0]):
        zo, io = oracle.arpls(y[i], lam, ratio, itermax)
        assert it[i] == io, (i, it[i], io)
        np.testing.assert_allclose(z[i], zo, rtol=0, atol=1e-9 * np.abs(y[i]).max())


@pytest.mark.parametrize("interval", [8, 7, 30])
def test_run_bandpass_matches_oracle(interval):
    """24 sub-integrations in fit intervals of 8 (three), 7 (the last one
    of 3) and 30 (one interval for the block)."""
    import torch
    m = lib()
    cfg = synth.SMALL.replace(n_sub=24)
    data = synth.generate(cfg)
    lam, ratio, itermax = 1e3, 1e-3, 50
    d = torch.from_numpy(data).cuda()
    with m.Plan(19, 64, 128, 24) as plan:
        g = plan.run_bandpass(d, lam=lam, ratio=ratio, itermax=itermax, interval=interval)
    o = oracle.block_bandpass(data, 128, interval, lam, ratio, itermax,
                              n_threads=synth.default_threads())
    bp = g["bandpass"].cpu().numpy()
    assert bp.shape == o["z"].shape
    np.testing.assert_allclose(bp, o["z"], rtol=2e-7, atol=0)
    compare_eig(g["evals"].cpu().numpy(), o["evals"], f"bandpass interval {interval}")
    st = g["stat"].cpu().numpy()
    s_err = np.abs(st - o["stat"]) / np.maximum(o["stat"], 1e-30)
    assert s_err.max() <= STAT_TOL, s_err.max()
    f_o, i_o = oracle.flag(o["stat"], 64)
    compare_flags(g["flags"].cpu().numpy(), f_o, o["stat"], g["info"], i_o)
    assert g["info"]["n_degenerate"] == 0


def test_bandpass_same_on_both_gram_kernels():
    """The tensor-core Gram (sums interleaved by 8 channels) and the
    CUDA-core Gram ([cell][P]) give the same exact sums, hence the same
    bandpass, CCM and statistic bit for bit."""
    import torch
    m = lib()
    cfg = synth.SMALL.replace(n_sub=16)
    d = torch.from_numpy(synth.generate(cfg)).cuda()
    outs = []
    for variant in (None, -1):
        with m.Plan(19, 64, 128, 16) as plan:
            if variant is not None:
                m.mraid_set_variant(plan.handle, variant)
            m.mraid_profile_enable(plan.handle)
            g = plan.run_bandpass(d, lam=1e3, interval=4)
            ran = m.mraid_profile_read(plan.handle)
        assert ("gram_tc" in ran) == (variant is None), ran
        outs.append({k: g[k].cpu().numpy() for k in ("bandpass", "stat", "flags")})
    for k in outs[0]:
        np.testing.assert_array_equal(outs[0][k], outs[1][k], err_msg=k)


def test_interval_beyond_the_block_is_one_interval():
    """Any interval at least as long as the block, up to the largest int32,
    fits the whole block once: outputs equal those of interval = n_sub."""
    import torch
    m = lib()
    cfg = synth.SMALL.replace(n_sub=16)
    d = torch.from_numpy(synth.generate(cfg)).cuda()
    with m.Plan(19, 64, 128, 16) as plan:
        a = plan.run_bandpass(d, lam=1e3, interval=16)
        b = plan.run_bandpass(d, lam=1e3, interval=2**31 - 1)
    for k in ("bandpass", "evals", "stat", "flags"):
        np.testing.assert_array_equal(a[k].cpu().numpy(), b[k].cpu().numpy(), err_msg=k)


def test_bandpass_rejects_bad_arguments():
    import torch
    m = lib()
    code = {name: v for v, name in m.STATUS.items()}
    d = torch.zeros(19, 4 * 128, 64, dtype=torch.uint8, device="cuda")
    st = torch.empty(4 * 64, device="cuda")
    fl = torch.empty(4 * 64, dtype=torch.uint8, device="cuda")
    with m.Plan(19, 64, 128, 4) as plan:
        for kw in ({"lam": 0.0}, {"ratio": -1.0}, {"itermax": 0}, {"itermax": 1001},
                   {"interval": 0}):
            bp = m.mraid_default_bandpass_params(**kw)
            with pytest.raises(m.MraidError) as ei:
                m.mraid_run_bandpass(plan.handle, d, bp, None, None, None, st, fl)
            assert ei.value.status == code["MRAID_ERR_INVALID_ARG"], kw
        y = torch.zeros(2, 2, dtype=torch.float64, device="cuda")
        with pytest.raises(m.MraidError):
            m.mraid_arpls(plan.handle, y, 2, 2, m.mraid_default_bandpass_params(), y)
    x = torch.zeros(19, 4 * 128, 64, device="cuda")
    with m.Plan(19, 64, 128, 4, bit_depth=32) as plan:
        with pytest.raises(m.MraidError) as ei:
            m.mraid_run_bandpass(plan.handle, x, m.mraid_default_bandpass_params(), None, None,
                                 None, st, fl)
        assert ei.value.status == code["MRAID_ERR_UNSUPPORTED"]
