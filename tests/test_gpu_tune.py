"""Autotuner (needs a GPU): every Gram variant it chooses among gives the same
exact correlations, and the tuning cache round-trips."""
import json

import numpy as np
import pytest

import synth
from gpu_util import lib

pytestmark = pytest.mark.gpu


def test_variants_agree_and_cache(tmp_path):
    import torch
    m = lib()
    cfg = synth.SMALL.replace(n_sub=32)
    d = torch.from_numpy(synth.generate(cfg)).cuda()
    outs = {}
    with m.Plan(cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub) as plan:
        for v in range(-1, 10):
            m.mraid_set_variant(plan.handle, v)
            s, c = plan.ccm(d)
            outs[v] = (s.cpu().numpy(), c.cpu().numpy())
        for v in range(10):
            np.testing.assert_array_equal(outs[v][0], outs[-1][0])
            assert np.abs(outs[v][1] - outs[-1][1]).max() <= 2e-6
        # every eigensolver variant gives the same eigenvalues to rounding
        evs = {}
        for v in (0, 1, 2, 3, 4, 5):
            m.mraid_set_eig_variant(plan.handle, v)
            evs[v] = plan.eig(c)[0].cpu().numpy()
        for v in (1, 2, 3, 4, 5):
            assert np.abs(evs[0] - evs[v]).max() <= 1e-5 * np.abs(evs[0]).max()
        cache = tmp_path / "tune.json"
        choice = m.tune(plan.handle, d, cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, str(cache), reps=2)
        assert -1 <= choice[0] < 10 and choice[1] in (0, 1, 2, 3, 4, 5)
        rec = json.loads(cache.read_text())
        key = f"{cfg.n_beam},{cfg.n_chan},{cfg.n_samp_sub},u8"
        assert (rec[key]["gram"], rec[key]["jacobi"]) == choice and len(rec[key]["ms"]) == 17
        # a second call reads the cache
        assert m.tune(plan.handle, d, cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, str(cache)) == choice
