"""The tensor-core Gram for 24..127 beams (one channel per MMA; Section 3.2,
Eq. 1) through the C ABI (needs a GPU).

Sub-integrations longer than 1024 samples are accumulated in exact pieces
of at most 1024 samples, so the saturated patterns (constant 0 or 255,
0/255 alternation: partial sums of 2^24 per piece) cross the FP32 edge in
every piece. The int64 sums must equal the oracle's bit for bit, the
correlation must match the oracle's to CORR_TOL, and the CUDA-core Gram
(variant -1) must give the same sums. The shapes cover one, two and four
passes over a 16-channel box (24, 36 and 72 beams), the three tile shapes
(four channels per MMA up to 31 beams, two up to 63, one from 64), 127 beams
(the largest that fits 128 rows with the row of ones), pieces of 768
samples (1536-sample sub-integrations) and more work items than SMs."""
import numpy as np
import pytest

import oracle
from gpu_util import CORR_TOL, edge_block, lib, unpack_corr

pytestmark = pytest.mark.gpu


def oracle_sums(data, n_s, n_sub, n_chan):
    n_beam = data.shape[0]
    M = n_beam + 1
    iu = np.triu_indices(M)
    G = np.zeros((n_sub * n_chan, M, M), dtype=np.int64)
    for k in range(n_sub):
        for c in range(n_chan):
            G[k * n_chan + c] = oracle.cell_gram(data, n_s, k, c)
    return G[:, iu[0], iu[1]], G


@pytest.mark.parametrize("n_beam,n_chan,n_s,n_sub", [
    (24, 32, 1024, 3),     # 16 channels per pass, one piece
    (36, 32, 2048, 2),     # 8 channels per pass, two pieces
    (72, 16, 4096, 2),     # 4 channels per pass, four pieces
    (127, 16, 512, 2),     # the largest beam count
    (40, 48, 1536, 2),     # pieces of 768 samples, three 16-channel boxes
    (63, 16, 1024, 2),     # N + 1 = 64: the largest two-channel tile
    (64, 16, 1024, 2),     # N + 1 = 65: one channel per tile
    (31, 16, 1024, 2),     # N + 1 = 32: the largest four-channel tile
])
def test_tcl_gram_exact(n_beam, n_chan, n_s, n_sub):
    import torch
    m = lib()
    data = edge_block(n_beam, n_chan, n_sub, seed=n_beam + n_s, n_s=n_s)
    want, G = oracle_sums(data, n_s, n_sub, n_chan)
    r_o = np.stack([oracle.corr_from_gram(G[i])[0] for i in range(G.shape[0])])
    d = torch.from_numpy(data).cuda()
    with m.Plan(n_beam, n_chan, n_s, n_sub) as plan:
        m.mraid_profile_enable(plan.handle)
        sums, corr = plan.ccm(d)
        plan.sync()
        ran = m.mraid_profile_read(plan.handle)
        assert "gram_tcl" in ran and "gram_u8" not in ran, ran
        got = sums.cpu().numpy()
        bad = np.flatnonzero(np.any(got != want, axis=1))
        assert bad.size == 0, (bad[:8], (bad % 8)[:8])
        r = unpack_corr(corr.cpu().numpy(), n_beam)
        assert np.abs(r - r_o).max() <= CORR_TOL, np.abs(r - r_o).max()
        # the CUDA-core Gram on the same data
        m.mraid_set_variant(plan.handle, -1)
        m.mraid_profile_enable(plan.handle)
        sums2, _ = plan.ccm(d, corr=False)
        plan.sync()
        assert "gram_u8" in m.mraid_profile_read(plan.handle)
        assert np.array_equal(sums2.cpu().numpy(), got)


def test_tcl_gram_noise_many_items():
    """Gaussian noise around 128 on a block with more work items than SMs
    (each CTA loops over items): every cell equal to the CUDA-core Gram,
    a sample of cells to the oracle."""
    import torch
    m = lib()
    n_beam, n_chan, n_s, n_sub = 36, 256, 1024, 12          # 12 x 16 x 2 = 384 items
    rng = np.random.default_rng(5)
    data = np.clip(np.rint(rng.normal(128, 20, size=(n_beam, n_sub * n_s, n_chan))), 0,
                   255).astype(np.uint8)
    d = torch.from_numpy(data).cuda()
    with m.Plan(n_beam, n_chan, n_s, n_sub) as plan:
        sums, _ = plan.ccm(d, corr=False)
        m.mraid_set_variant(plan.handle, -1)
        sums2, _ = plan.ccm(d, corr=False)
        plan.sync()
    got = sums.cpu().numpy()
    assert np.array_equal(got, sums2.cpu().numpy())
    iu = np.triu_indices(n_beam + 1)
    for cell in rng.choice(n_sub * n_chan, size=24, replace=False):
        k, c = divmod(int(cell), n_chan)
        assert np.array_equal(got[cell], oracle.cell_gram(data, n_s, k, c)[iu]), cell
