"""The tensor-core Gram at its exactness edge (Section 3.2, Eq. 1), through
the C ABI (needs a GPU).

The kernel forms the sums from centred samples x - 128 in f16 with FP32
accumulation in TMEM: exact while every partial sum stays within 2^24.
With 1024 samples per sub-integration, beams held at 0 (x - 128 = -128)
reach 1024 * 128^2 = 2^24 exactly, so constant-0 beams, constant-255
beams, 0/255 alternation (the largest variance) and saturated beams beside
noisy ones are the cells where an off-by-one in the centring or a lost bit
would show. Every tensor-core variant must give the oracle's int64 sums bit
for bit, and so must the two-polarisation instance (256-sample TMEM pieces,
total power 0..510) with both polarisations saturated."""
import numpy as np
import pytest

import oracle
from gpu_util import CORR_TOL, edge_block, lib, unpack_corr

pytestmark = pytest.mark.gpu

N_S = 1024


def oracle_packed(data, n_sub, n_chan, pol2=False):
    n_beam = data.shape[0] // (2 if pol2 else 1)
    M = n_beam + 1
    iu = np.triu_indices(M)
    G = np.zeros((n_sub * n_chan, M, M), dtype=np.int64)
    for k in range(n_sub):
        for c in range(n_chan):
            G[k * n_chan + c] = (oracle.cell_gram_pol2(data, N_S, k, c) if pol2
                                 else oracle.cell_gram(data, N_S, k, c))
    return G[:, iu[0], iu[1]], G


@pytest.mark.parametrize("n_beam,n_chan", [(19, 16), (19, 32), (23, 16), (4, 32)])
def test_tc_gram_exact_at_the_edge_every_variant(n_beam, n_chan):
    import torch
    m = lib()
    n_sub = 4
    data = edge_block(n_beam, n_chan, n_sub, seed=n_beam * 100 + n_chan)
    want, G = oracle_packed(data, n_sub, n_chan)
    # the oracle's correlation of each cell, for the fused epilogue
    r_o = np.stack([oracle.corr_from_gram(G[i])[0] for i in range(G.shape[0])])
    d = torch.from_numpy(data).cuda()
    with m.Plan(n_beam, n_chan, N_S, n_sub) as plan:
        for v in range(10):
            m.mraid_set_variant(plan.handle, v)
            m.mraid_profile_enable(plan.handle)
            sums, corr = plan.ccm(d)
            plan.sync()
            ran = m.mraid_profile_read(plan.handle)
            assert "gram_tc" in ran and "gram_u8" not in ran, (v, ran)
            got = sums.cpu().numpy()
            bad = np.flatnonzero(np.any(got != want, axis=1))
            assert bad.size == 0, (v, bad[:8], (bad % 8)[:8])
            r = unpack_corr(corr.cpu().numpy(), n_beam)
            assert np.abs(r - r_o).max() <= CORR_TOL, (v, np.abs(r - r_o).max())


@pytest.mark.parametrize("n_beam,n_chan", [(19, 16), (23, 32)])
def test_tc_gram_two_polarisations_saturated(n_beam, n_chan):
    import torch
    m = lib()
    n_sub = 4
    p0 = edge_block(n_beam, n_chan, n_sub, seed=7)
    p1 = edge_block(n_beam, n_chan, n_sub, seed=8)
    # both polarisations at the same extreme where the pattern is constant or
    # alternating: total power 0 or 510, or 0/510 alternation
    data = np.ascontiguousarray(np.concatenate([p0, p1], axis=0))
    want, _ = oracle_packed(data, n_sub, n_chan, pol2=True)
    d = torch.from_numpy(data).cuda()
    with m.Plan(n_beam, n_chan, N_S, n_sub) as plan:
        m.mraid_profile_enable(plan.handle)
        sums, _ = plan.ccm_pol2(d, corr=False)
        plan.sync()
        ran = m.mraid_profile_read(plan.handle)
    assert "gram_tc" in ran and "pol2_fold" not in ran, ran
    got = sums.cpu().numpy()
    bad = np.flatnonzero(np.any(got != want, axis=1))
    assert bad.size == 0, (bad[:8], (bad % 8)[:8])
