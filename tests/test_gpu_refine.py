"""Eigenvector refinement on the GPU (mraid_refine) against the oracle's,
each computed from its own q1 and flags (needs a GPU). Bits may differ only
where the oracle's |q1_b| lies within 1e-3 (+ the threshold difference) of
its beam threshold, or where the cell's eigenvalue flag itself differs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [synth.SMALL, synth.SMALL.replace(n_beam=36, n_chan=16, n_sub=64,
                                                                  seed=99)])
def test_refine_matches_oracle(cfg):
    import torch
    m = lib()
    data = synth.generate(cfg)
    d = torch.from_numpy(data).cuda()
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        out = plan.run(d)
        bits, ms = plan.refine(out["q1"], out["flags"])
    bits = bits.cpu().numpy().view(np.uint32)
    ms = ms.cpu().numpy()
    res = oracle.block(data, cfg.n_samp_sub, n_threads=synth.default_threads())
    f_o, _ = oracle.flag(res["stat"], cfg.n_chan)
    b_o, ms_o = oracle.beam_flags(res["q1"], f_o, cfg.n_chan, t=1.0)
    assert np.abs(ms - ms_o).max() < 1e-4
    W = bits.shape[1]
    same_flag = out["flags"].cpu().numpy() == f_o
    thr = ms_o[:, 0] + ms_o[:, 1]
    band = 1e-3 + np.abs((ms[:, 0] + ms[:, 1]) - thr)
    for b in range(cfg.n_beam):
        g = (bits[:, b // 32] >> (b % 32)) & 1
        o = (b_o[:, b // 32] >> (b % 32)) & 1
        near = np.abs(np.abs(res["q1"][:, b]) - thr[b]) <= band[b]
        bad = (g != o) & same_flag & ~near
        assert not bad.any(), (b, int(bad.sum()))
    assert W == (cfg.n_beam + 31) // 32
