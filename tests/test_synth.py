"""The seeded input generator (synth/) against the recipe it implements (CPU).
Both the oracle and the CUDA path take their inputs from it, so its
properties are checked directly: determinism, the pointwise and block forms
agree, noise of mean 128 and sigma 20 DN, per-(beam, channel) bandpass
gains in U(0.7, 1.3), and the placement and shape of each injected event
(beam-common narrowband sines of period 16 samples, broadband boxcars one
sub-integration long that start inside a sub-integration, single-beam
16-sample pulses), at the rates of the FAST-shaped block."""
import numpy as np

import synth

CLEAN = synth.SMALL.replace(n_narrow=0, n_burst=0, n_spike=0)


def test_deterministic_and_seeded():
    a = synth.generate(synth.SMALL)
    assert np.array_equal(a, synth.generate(synth.SMALL))
    assert not np.array_equal(a, synth.generate(synth.SMALL.replace(seed=synth.SMALL.seed + 1)))
    assert a.shape == (19, synth.SMALL.n_time, 64) and a.dtype == np.uint8


def test_pointwise_sample_equals_block():
    cfg = synth.SMALL
    d = synth.generate(cfg)
    rng = np.random.default_rng(0)
    for b, t, c in zip(rng.integers(0, 19, 300), rng.integers(0, cfg.n_time, 300),
                       rng.integers(0, 64, 300)):
        assert synth.sample(cfg, int(b), int(t), int(c)) == d[b, t, c]


def test_noise_moments():
    x = synth.generate(CLEAN).astype(np.float64)
    n = x.size                                    # 40 M samples
    assert abs(x.mean() - 128.0) < 0.02           # standard error 20/sqrt(n) = 0.003
    assert abs(x.std() - 20.0) < 0.05
    assert abs(np.mean(np.abs(x - 128.0) <= 20.0) - 0.6827) < 0.01
    assert n == 19 * CLEAN.n_time * 64


def test_bandpass_gains_scale_the_noise_per_beam_and_channel():
    x = synth.generate(CLEAN.replace(bandpass=1)).astype(np.float64)
    g = x.std(axis=1) / 20.0                      # [beam][chan], 32768 samples each
    assert g.min() > 0.67 and g.max() < 1.33
    assert g.max() - g.min() > 0.4                # the gains do vary
    assert np.abs(x.mean(axis=1) - 128.0).max() < 1.0


def test_events_have_their_shape_and_place():
    cfg = synth.SMALL.replace(n_burst=0)
    x = synth.generate(cfg).astype(np.float64)
    ev = synth.events(cfg)
    assert len(ev["narrow"]) == cfg.n_narrow and len(ev["spike"]) == cfg.n_spike
    narrow = {c for (c, _) in ev["narrow"]}
    clean = [c for c in range(cfg.n_chan) if c not in narrow]
    for c in narrow:
        # beam-common: correlated across beams; period 16 samples
        assert np.corrcoef(x[0, :, c], x[1, :, c])[0, 1] > 0.05   # noise 0.0055
        f = np.abs(np.fft.rfft(x[:, :, c].mean(axis=0) - 128.0))
        assert np.argmax(f[1:]) + 1 == cfg.n_time // 16
    assert abs(np.corrcoef(x[0, :, clean[0]], x[1, :, clean[0]])[0, 1]) < 0.03
    for (b, c, k, off) in ev["spike"]:
        t = k * cfg.n_samp_sub + off
        assert 0 <= off <= cfg.n_samp_sub - 16
        assert x[b, t:t + 16, c].mean() > 128.0 + 60.0           # +80 DN on one beam
        others = np.delete(x[:, t:t + 16, c], b, axis=0)
        assert np.abs(others.mean(axis=1) - 128.0).max() < 25.0


def test_bursts_start_inside_a_sub_integration_and_span_two():
    cfg = synth.SMALL
    x = synth.generate(cfg).astype(np.float64)
    S = cfg.n_samp_sub
    for (t0, k) in synth.events(cfg)["burst"]:
        assert k * S < t0 < (k + 1) * S                          # never aligned
        assert x[:, t0:t0 + S, :].mean() > 128.0 + 15.0          # +40 DN x gain >= 0.5
        assert abs(x[:, t0 - S // 2:t0, :].mean() - 128.0) < 1.0
        cells = synth.rfi_cells(cfg)["burst"]
        assert (k, 0) in cells and (k + 1, 0) in cells


def test_fast_block_rates():
    F = synth.FAST_BLOCK
    assert (F.n_beam, F.n_chan, F.n_samp_sub, F.n_sub) == (19, 4096, 1024, 200)
    assert F.n_narrow == round(0.02 * F.n_chan)                  # 2 % of channels
    assert F.n_burst == round(0.01 * F.n_sub)                    # 1 % of sub-integrations
    assert F.n_spike == round(0.001 * F.n_chan * F.n_sub)        # 0.1 % of cells
    assert F.bandpass == 1
