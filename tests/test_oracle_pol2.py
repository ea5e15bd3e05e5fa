"""Pins of the oracle's two-polarisation input (CPU): the total power of a
beam is the sum of its two recorded polarisations (Section 2), and Eq. 1's
Gram is taken of that sum. Checked against numpy brute force on the summed
samples, the fold of the stacked 2N-beam Gram (the four polarisation
blocks add up exactly), and the single-polarisation path when the second
polarisation is zero."""
import numpy as np
import pytest

import oracle


def block(n_beam, n_time, n_chan, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(2 * n_beam, n_time, n_chan), dtype=np.uint8)


@pytest.mark.parametrize("n_beam,n_s,n_chan", [(2, 3, 2), (5, 16, 3), (19, 64, 4)])
def test_pol2_gram_brute_force(n_beam, n_s, n_chan):
    d = block(n_beam, 2 * n_s, n_chan, n_beam)
    for sub in (0, 1):
        for chan in range(n_chan):
            G = oracle.cell_gram_pol2(d, n_s, sub, chan)
            x = (d[:n_beam, sub * n_s:(sub + 1) * n_s, chan].astype(np.int64) +
                 d[n_beam:, sub * n_s:(sub + 1) * n_s, chan].astype(np.int64))
            xa = np.vstack([x, np.ones((1, n_s), dtype=np.int64)])
            np.testing.assert_array_equal(G, np.einsum("at,bt->ab", xa, xa))


def test_pol2_gram_is_the_fold_of_the_stacked_gram():
    N, n_s = 7, 40
    d = block(N, n_s, 3, 9)
    for chan in range(3):
        G2 = oracle.cell_gram(d, n_s, 0, chan)           # 2N stacked beams + ones
        G = oracle.cell_gram_pol2(d, n_s, 0, chan)
        A = G2[:2 * N, :2 * N]
        fold = A[:N, :N] + A[:N, N:] + A[N:, :N] + A[N:, N:]
        np.testing.assert_array_equal(G[:N, :N], fold)
        np.testing.assert_array_equal(G[:N, N], G2[:N, 2 * N] + G2[N:2 * N, 2 * N])
        assert G[N, N] == G2[2 * N, 2 * N] == n_s


def test_pol2_with_silent_second_polarisation_is_the_single_path():
    N, n_s = 19, 32
    d = block(N, 2 * n_s, 5, 4)
    d[N:] = 0
    single = np.ascontiguousarray(d[:N])
    subs = np.array([0, 1, 1], dtype=np.int32)
    chans = np.array([0, 2, 4], dtype=np.int32)
    a = oracle.cells_pol2(d, n_s, subs, chans)
    b = oracle.cells(single, n_s, subs, chans)
    np.testing.assert_array_equal(a["G"], b["G"])
    np.testing.assert_array_equal(a["evals"], b["evals"])
    np.testing.assert_array_equal(a["stat"], b["stat"])
