"""Served form (mraid_serve_*), needs a GPU.

Blocks of several observations, cut at arbitrary sample counts (so
sub-integrations straddle block edges and are carried over), are submitted
interleaved. Every block's flags must equal those of the same whole
sub-integrations processed alone with mraid_run, and the cells must match
the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare_eig, lib

pytestmark = pytest.mark.gpu

# (n_beam, n_chan, n_samp_sub, block_samples)
STREAMS = [(13, 16, 512, 1300), (19, 32, 1024, 2500), (36, 6, 256, 700)]
N_BLOCKS = 6


def observation(i, shape):
    n_beam, n_chan, n_s, block = shape
    n_time = N_BLOCKS * block
    n_sub = n_time // n_s
    cfg = synth.SynthConfig(n_beam=n_beam, n_chan=n_chan, n_samp_sub=n_s, n_sub=n_sub,
                            seed=4000 + i, bandpass=1, n_narrow=1, n_burst=1, n_spike=1)
    data = synth.generate(cfg)                       # whole sub-integrations
    tail = np.random.default_rng(i).integers(0, 256, size=(n_beam, n_time - n_sub * n_s, n_chan),
                                             dtype=np.uint8)
    return np.ascontiguousarray(np.concatenate([data, tail], axis=1))


def test_served_blocks_equal_alone():
    import torch
    m = lib()
    obs = [observation(i, s) for i, s in enumerate(STREAMS)]
    blocks, flags_out = {}, {}
    with m.Server(STREAMS, max_inflight=4) as srv:
        # interleave the streams' blocks: the mix
        for k in range(N_BLOCKS):
            for i, (n_beam, n_chan, n_s, block) in enumerate(STREAMS):
                h = torch.from_numpy(np.ascontiguousarray(obs[i][:, k * block:(k + 1) * block, :]))
                h = h.pin_memory()
                f = torch.zeros(srv.flags_bytes(i), dtype=torch.uint8).pin_memory()
                blocks[(i, k)] = h
                flags_out[(i, k)] = f
                srv.submit(i, h, f, seq=k)
        srv.drain(120000)
        results = srv.poll(1024)
    assert len(results) == N_BLOCKS * len(STREAMS)
    for r in results:
        assert r["status"] == 0 and r["latency_ms"] > 0 and r["device_ms"] > 0
    # per stream: block k processed sub-integrations [s_k, s_k + n_sub_k)
    for i, (n_beam, n_chan, n_s, block) in enumerate(STREAMS):
        res = sorted([r for r in results if r["stream"] == i], key=lambda r: r["seq"])
        full = torch.from_numpy(obs[i]).cuda()
        n_time = obs[i].shape[1]
        s0 = 0
        for r in res:
            k, ns = r["seq"], r["n_sub"]
            assert ns == ((k + 1) * block) // n_s - (k * block) // n_s
            if ns == 0:
                continue
            # the same sub-integrations alone: a plan over a view of the
            # whole observation starting at sub-integration s0
            with m.Plan(n_beam, n_chan, n_s, ns, beam_stride=n_time * n_chan) as plan:
                alone = plan.run(full.view(-1)[s0 * n_s * n_chan:])
            got = flags_out[(i, k)][: ns * n_chan]
            assert torch.equal(got, alone["flags"].cpu()), (i, k)
            assert r["n_flagged"] == alone["info"]["n_flagged"]
            if i == 1 and k == 2:   # one block against the oracle
                subs = np.repeat(np.arange(s0, s0 + ns, dtype=np.int32), n_chan)
                chans = np.tile(np.arange(n_chan, dtype=np.int32), ns)
                orc = oracle.cells(obs[i], n_s, subs, chans, n_threads=synth.default_threads())
                compare_eig(alone["evals"].cpu().numpy(), orc["evals"], "served block")
            s0 += ns


def test_serve_rejects_bad_arguments():
    m = lib()
    with pytest.raises(m.MraidError):
        m.Server([(1, 16, 512, 100)])          # one beam
    with m.Server([(13, 16, 512, 1300)]) as srv:
        with pytest.raises(m.MraidError):
            srv.submit(5, 0, 0, 0)              # no such stream
