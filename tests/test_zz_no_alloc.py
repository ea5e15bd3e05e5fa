"""mraid_ccm_noalloc: correlations for callers that cannot allocate device
memory (a pipeline that reserved the whole GPU for its own pool, or a loop
that must not make a possibly synchronising cudaMalloc). It must give the
same correlations as mraid_ccm, call after call, although every call reuses
the library's one fixed scratch array. Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import CORR_TOL, lib

pytestmark = pytest.mark.gpu


def test_noalloc_matches_mraid_ccm_twice():
    import torch
    m = lib()
    cfg = synth.SMALL.replace(n_sub=16)                 # 19 beams, 64 ch, 16 x 128
    data = synth.generate(cfg)
    d = torch.from_numpy(data).cuda()
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        _, ref = plan.ccm(d, sums=False)
        torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    np_ = cfg.n_beam * (cfg.n_beam + 1) // 2
    p = m.mraid_default_params(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        # two calls in a row, each over two ranges of sub-integrations
        out = torch.full((cfg.n_cells, np_), float("nan"), device="cuda")
        half = cfg.n_sub // 2
        m.mraid_ccm_noalloc(p, d, 0, half, out[: half * cfg.n_chan], stream)
        m.mraid_ccm_noalloc(p, d, half, cfg.n_sub - half, out[half * cfg.n_chan:], stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.abs(got - ref).max() <= CORR_TOL, (call, np.abs(got - ref).max())


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    m = lib()
    p = m.mraid_default_params(19, 4096, 1024, 8)       # 4 x 4096 cells > 4993
    d = torch.zeros(19 * 8 * 1024 * 4096, dtype=torch.uint8, device="cuda")
    out = torch.empty(4 * 4096, 190, device="cuda")
    with pytest.raises(m.MraidError) as e:
        m.mraid_ccm_noalloc(p, d, 0, 4, out)
    assert e.value.status == 1 and "scratch" in str(e.value)
    # one sub-integration (4096 cells) fits
    m.mraid_ccm_noalloc(p, d, 0, 1, out)
    torch.cuda.synchronize()
    assert torch.all(out[:4096, 0] == 1.0)              # r_00 = 1 (zero variance beams)


def test_noalloc_capacity_boundary():
    """The largest request the scratch holds is accepted and equals
    mraid_ccm; one cell more is refused. With one channel the limit
    (8 MiB - 256) / (8 * 210) = 4993 cells is a whole number of rows."""
    import torch
    m = lib()
    n_beam, n_chan, n_samp = 19, 1, 16
    psum = (n_beam + 1) * (n_beam + 2) // 2
    max_cells = ((8 << 20) - 256) // (8 * psum)
    assert max_cells == 4993
    n_sub = max_cells + 1
    rng = np.random.default_rng(7)
    data = rng.integers(0, 256, size=(n_beam, n_sub * n_samp, n_chan), dtype=np.uint8)
    d = torch.from_numpy(data).cuda()
    np_ = n_beam * (n_beam + 1) // 2
    with m.Plan(n_beam, n_chan, n_samp, n_sub) as plan:
        _, ref = plan.ccm(d, sums=False)
        torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    p = m.mraid_default_params(n_beam, n_chan, n_samp, n_sub)
    stream = torch.cuda.current_stream().cuda_stream
    for sub0 in (0, 1):
        out = torch.full((max_cells, np_), float("nan"), device="cuda")
        m.mraid_ccm_noalloc(p, d, sub0, max_cells, out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), sub0
        assert np.abs(got - ref[sub0: sub0 + max_cells]).max() <= CORR_TOL, sub0
    big = torch.empty((max_cells + 1, np_), device="cuda")
    with pytest.raises(m.MraidError) as e:
        m.mraid_ccm_noalloc(p, d, 0, max_cells + 1, big, stream)
    assert e.value.status == 1 and "scratch" in str(e.value)
