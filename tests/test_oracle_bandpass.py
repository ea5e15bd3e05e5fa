"""Pins of the oracle's bandpass path (CPU): Section 3.1's ArPLS bandpass
(the method of Baek, Park, Ahn and Ahn 2015 that the paper names) and the
bandpass-centred reading of Eq. 1, C_ab = (1/N_s) sum_t (x_a - z_a)(x_b - z_b).

Each test checks the oracle against something other than itself: a dense
LAPACK solve of the same normal equations, exact properties of the
penalised fit (lines pass through unchanged, offsets carry over), numpy
brute force on the samples, an algebraic identity with the exact Gram sums,
and the behaviour the asymmetric weights exist for (positive RFI spikes do
not lift the baseline, negative dips pull it down)."""
import numpy as np
import pytest

import oracle
import synth


def second_difference(n):
    return np.diff(np.eye(n), 2, axis=0)


@pytest.mark.parametrize("n,lam", [(3, 1.0), (4, 0.0), (5, 7.5), (64, 1e3), (257, 1e5)])
def test_whittaker_matches_dense_solve(n, lam):
    rng = np.random.default_rng(n)
    y = rng.normal(size=n) * 10 + 100
    w = rng.uniform(0.05, 1.0, size=n)
    D = second_difference(n)
    dense = np.linalg.solve(np.diag(w) + lam * D.T @ D, w * y)
    z = oracle.whittaker(y, w, lam)
    np.testing.assert_allclose(z, dense, rtol=1e-9, atol=1e-9 * np.abs(y).max())


def test_whittaker_zero_penalty_returns_data():
    y = np.arange(10.0) ** 2
    np.testing.assert_allclose(oracle.whittaker(y, np.full(10, 0.3), 0.0), y, rtol=1e-14)


@pytest.mark.parametrize("lam", [1.0, 1e5])
def test_arpls_passes_lines_unchanged(lam):
    """D annihilates a line, so z = y solves the normal equations for any
    weights: the fit of a straight bandpass is the bandpass itself."""
    y = 80.0 + 0.37 * np.arange(300)
    z, it = oracle.arpls(y, lam, 1e-3, 50)
    np.testing.assert_allclose(z, y, rtol=1e-9)
    assert 1 <= it <= 50


def test_arpls_first_solve_is_unweighted():
    rng = np.random.default_rng(3)
    y = rng.normal(size=128) + 50
    z1, it = oracle.arpls(y, 1e2, 1e-3, 1)
    assert it == 1
    np.testing.assert_allclose(z1, oracle.whittaker(y, np.ones(128), 1e2), rtol=1e-14)


def test_arpls_offset_carries_over():
    """Adding c to every channel adds c to the baseline: D c = 0 and the
    residuals, hence the weights, are unchanged."""
    rng = np.random.default_rng(5)
    x = np.linspace(0, 1, 512)
    y = 100 + 30 * np.sin(4 * x) + rng.normal(scale=0.7, size=512)
    z0, i0 = oracle.arpls(y, 1e4, 1e-4, 60)
    z1, i1 = oracle.arpls(y + 37.0, 1e4, 1e-4, 60)
    assert i0 == i1
    np.testing.assert_allclose(z1 - 37.0, z0, atol=1e-8)


def test_arpls_ignores_positive_spikes_and_follows_dips():
    """What the asymmetric weights are for: RFI adds power, so channels far
    above the baseline lose their weight and do not lift it; an unweighted
    fit is lifted by the same spikes."""
    rng = np.random.default_rng(11)
    n = 1024
    x = np.linspace(0, 1, n)
    base = 120 + 25 * np.sin(3 * x) + 8 * x * x
    y = base + rng.normal(scale=0.5, size=n)
    spikes = rng.choice(np.arange(20, n - 20), 40, replace=False)
    y[spikes] += rng.uniform(20, 60, size=40)
    z, it = oracle.arpls(y, 1e4, 1e-4, 100)
    plain = oracle.whittaker(y, np.ones(n), 1e4)
    err_a = np.abs(z - base)
    err_p = np.abs(plain - base)
    assert err_a.max() < 1.0 and err_a.mean() < 0.5, (err_a.max(), err_a.mean())
    assert err_p.max() > 2 * err_a.max()
    # the baseline sits in the noise, below its centre line (asymmetry)
    assert np.median(y - z) > 0
    assert 2 <= it <= 100


def test_bandpass_input_is_the_time_mean():
    data = synth.generate(synth.SMALL.replace(n_sub=6))
    for beam, s0, ns in ((0, 0, 6), (7, 2, 3), (18, 5, 1)):
        y = oracle.bandpass_input(data, 128, s0, ns, beam)
        ref = data[beam, s0 * 128:(s0 + ns) * 128, :].astype(np.float64).mean(axis=0)
        np.testing.assert_allclose(y, ref, rtol=1e-15)


def test_ccm_bandpass_brute_force_and_gram_identity():
    """C from the samples equals numpy's (X - z)(X - z)^T / n, and equals
    cov / n^2 + (mu - z)(mu - z)^T with cov from the exact Gram sums."""
    data = synth.generate(synth.SMALL.replace(n_sub=8))
    rng = np.random.default_rng(2)
    for sub, chan in ((0, 0), (3, 17), (2, 63)):
        zc = 128 + rng.normal(scale=3, size=19)
        C = oracle.cell_ccm_bandpass(data, 128, sub, chan, zc)
        X = data[:, sub * 128:(sub + 1) * 128, chan].astype(np.float64) - zc[:, None]
        np.testing.assert_allclose(C, X @ X.T / 128, rtol=1e-12)
        G = oracle.cell_gram(data, 128, sub, chan)
        n = G[19, 19]
        S = G[:19, 19]
        cov = n * G[:19, :19] - np.outer(S, S)          # exact int64
        mu = S / n
        ident = cov / float(n) ** 2 + np.outer(mu - zc, mu - zc)
        np.testing.assert_allclose(C, ident, rtol=1e-12)


def test_block_bandpass_consistent_with_its_parts():
    cfg = synth.SMALL.replace(n_sub=10)
    data = synth.generate(cfg)
    out = oracle.block_bandpass(data, 128, 4, 1e3, 1e-3, 40, n_threads=4)
    assert out["z"].shape == (3, 19, 64)            # intervals of 4, 4 and 2
    for I, (s0, ns) in enumerate(((0, 4), (4, 4), (8, 2))):
        for beam in (0, 9, 18):
            y = oracle.bandpass_input(data, 128, s0, ns, beam)
            z, it = oracle.arpls(y, 1e3, 1e-3, 40)
            np.testing.assert_array_equal(out["z"][I, beam], z)
            assert out["iters"][I, beam] == it
    for sub, chan in ((0, 5), (9, 40)):
        C = oracle.cell_ccm_bandpass(data, 128, sub, chan, out["z"][sub // 4, :, chan])
        ev = oracle.jacobi(C)[0]
        i = sub * 64 + chan
        np.testing.assert_array_equal(out["evals"][i], ev)
        assert out["stat"][i] == oracle.stat(ev)


def test_single_beam_spike_separates_the_readings():
    """The synthetic block's single-beam spike is not flagged under the
    Pearson reading (it correlates with nothing) but is under the
    bandpass-centred one (it dominates C's diagonal); the beam-common
    narrowband RFI is flagged under both. No broadband bursts here: a burst
    that fills a sub-integration shifts every channel's mean, which the
    bandpass reading sees as s ~ 1 in all 64 channels, and with 16 % of the
    cells there the Gaussian fit's threshold exceeds 1 (nothing flagged)."""
    cfg = synth.SMALL.replace(n_sub=64, n_burst=0)
    data = synth.generate(cfg)
    cells = synth.rfi_cells(cfg)
    assert cells["spike"] and not cells["burst"]
    o = oracle.block(data, 128, n_threads=4, want_evals=False, want_q1=False)
    f_p, _ = oracle.flag(o["stat"], 64)
    b = oracle.block_bandpass(data, 128, 16, 1e3, 1e-3, 50, n_threads=4, want_evals=False)
    f_b, _ = oracle.flag(b["stat"], 64)
    for (k, c) in cells["spike"]:
        assert f_p[k * 64 + c] == 0
        assert f_b[k * 64 + c] == 1
    narrow = np.array([k * 64 + c for (k, c) in cells["narrow"]])
    assert f_p[narrow].mean() > 0.95 and f_b[narrow].mean() > 0.95
