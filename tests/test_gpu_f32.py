"""Float32 samples (beamformer output, bit_depth 32) on the GPU against the
FP64 oracle (needs a GPU): N(0,1) noise plus beam-common RFI, and a large
common offset that a naive sum-of-products would cancel badly."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare_eig, compare_flags, lib

pytestmark = pytest.mark.gpu


def f32_block(n_beam, n_chan, n_s, n_sub, offset, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n_beam, n_sub * n_s, n_chan)).astype(np.float32)
    g = rng.uniform(0.5, 1.5, size=(n_beam, 1, 1)).astype(np.float32)
    t = np.arange(n_sub * n_s)
    x[:, :, 1] += 0.75 * g[:, :, 0] * np.sin(2 * np.pi * t / 16)[None, :]   # narrowband RFI
    x[:, n_s // 2: n_s // 2 + n_s, 8:12] += 2.0 * g[:, :, :1]                # a burst
    return np.ascontiguousarray(x + offset)


@pytest.mark.parametrize("offset", [0.0, 1000.0])
def test_f32_block_matches_oracle(offset):
    import torch
    m = lib()
    # RFI in 8 + 8 of 512 cells: few enough for the 3-sigma clip to isolate
    n_beam, n_chan, n_s, n_sub = 19, 64, 256, 8
    x = f32_block(n_beam, n_chan, n_s, n_sub, offset, 7)
    d = torch.from_numpy(x).cuda()
    with m.Plan(n_beam, n_chan, n_s, n_sub, bit_depth=32) as plan:
        _, corr = plan.ccm(d, sums=False)
        out = plan.run(d)
    corr = corr.cpu().numpy()
    iu = np.triu_indices(n_beam)
    ev_o = np.zeros((n_sub * n_chan, n_beam))
    st_o = np.zeros(n_sub * n_chan)
    worst = 0.0
    for k in range(n_sub):
        for c in range(n_chan):
            r, _ = oracle.corr_from_cov(oracle.cell_cov_f32(x, n_s, k, c))
            worst = max(worst, float(np.abs(corr[k * n_chan + c] - r[iu]).max()))
            ev_o[k * n_chan + c] = oracle.jacobi(r)[0]
            st_o[k * n_chan + c] = oracle.stat(ev_o[k * n_chan + c])
    # FP32 sums of shifted samples: |dr| stays ~1e-6 even with a 1000 offset
    assert worst <= 2e-5, worst
    compare_eig(out["evals"].cpu().numpy(), ev_o, f"f32 offset {offset}")
    flags_o, info_o = oracle.flag(st_o, n_chan)
    compare_flags(out["flags"].cpu().numpy(), flags_o, st_o, out["info"], info_o)
    F = flags_o.reshape(n_sub, n_chan).astype(bool)
    assert F[:, 1].all()                     # the narrowband channel
    assert F[0, 8:12].all() and F[1, 8:12].all()   # the burst's two sub-integrations
