"""Pins of the oracle's float32-input functions (CPU): Eq. 1 for float32
samples (beamformer output), read as for 8-bit samples: the Pearson
correlation of a cell's N_s samples.

cell_cov_f32 is the population covariance, formed in FP64 by two passes
(beam means, then centred products); corr_from_cov normalises it. Each test
checks them against something other than themselves: numpy's cov and
corrcoef (different routines), the exact integer path of the 8-bit oracle on
integer-valued samples, the zero-variance rule, the invariance of r under a
positive affine map of a beam, and a noise-free common signal (r all ones,
s = 1)."""
import numpy as np
import pytest

import oracle
import synth


def f32_block(n_beam, n_time, n_chan, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n_beam, n_time, n_chan)) * 3.0 + 0.5
    return np.ascontiguousarray(x.astype(np.float32))


@pytest.mark.parametrize("n_beam,n_s,n_chan", [(2, 3, 1), (5, 16, 3), (19, 128, 4)])
def test_cov_and_corr_match_numpy(n_beam, n_s, n_chan):
    x = f32_block(n_beam, 3 * n_s, n_chan, 100 + n_beam)
    for sub in range(3):
        for chan in sorted({0, n_chan - 1}):
            X = x[:, sub * n_s:(sub + 1) * n_s, chan].astype(np.float64)
            C = oracle.cell_cov_f32(x, n_s, sub, chan)
            np.testing.assert_allclose(C, np.cov(X, bias=True), rtol=1e-12, atol=1e-13)
            r, deg = oracle.corr_from_cov(C)
            assert deg == 0
            np.testing.assert_allclose(r, np.corrcoef(X), rtol=0, atol=1e-12)


def test_integer_samples_agree_with_the_exact_integer_path():
    """On integer-valued samples the two-pass FP64 covariance and the exact
    int64 Gram give the same correlation (to rounding): two formulas for
    one quantity, sharing no step."""
    data = synth.generate(synth.SMALL.replace(n_sub=8))
    x = np.ascontiguousarray(data.astype(np.float32))
    for sub, chan in ((0, 0), (1, 17), (7, 63), (4, 40)):
        r_f, deg_f = oracle.corr_from_cov(oracle.cell_cov_f32(x, 128, sub, chan))
        r_i, deg_i = oracle.corr_from_gram(oracle.cell_gram(data, 128, sub, chan))
        assert deg_f == deg_i == 0
        np.testing.assert_allclose(r_f, r_i, rtol=0, atol=1e-12)


def test_zero_variance_beam_rule():
    x = f32_block(4, 64, 2, 7)
    x[2, :, 1] = 7.5                      # beam 2 constant in channel 1 only
    r, deg = oracle.corr_from_cov(oracle.cell_cov_f32(x, 32, 1, 1))
    assert deg == 1
    assert r[2, 2] == 1.0
    assert np.all(r[2, [0, 1, 3]] == 0.0) and np.all(r[[0, 1, 3], 2] == 0.0)
    r0, deg0 = oracle.corr_from_cov(oracle.cell_cov_f32(x, 32, 1, 0))
    assert deg0 == 0 and np.all(np.abs(r0[2, [0, 1, 3]]) > 0)


def test_positive_affine_map_of_a_beam_leaves_r_unchanged():
    """x_a -> 2 x_a + 1024 on integer-valued samples (exact in float32):
    the covariance row of beam a doubles and its variance quadruples, so r
    is unchanged; a negative scale flips the sign of r's row and column."""
    rng = np.random.default_rng(3)
    x = np.ascontiguousarray(rng.integers(-100, 101, size=(6, 256, 2)).astype(np.float32))
    r, _ = oracle.corr_from_cov(oracle.cell_cov_f32(x, 128, 1, 0))
    y = x.copy()
    y[4] = 2.0 * x[4] + 1024.0
    C = oracle.cell_cov_f32(x, 128, 1, 0)
    Cy = oracle.cell_cov_f32(y, 128, 1, 0)
    np.testing.assert_allclose(Cy[4, 4], 4.0 * C[4, 4], rtol=1e-13)
    np.testing.assert_allclose(Cy[4, [0, 1, 2, 3, 5]], 2.0 * C[4, [0, 1, 2, 3, 5]], rtol=1e-12,
                               atol=1e-12)
    np.testing.assert_allclose(oracle.corr_from_cov(Cy)[0], r, rtol=0, atol=1e-13)
    z = x.copy()
    z[1] = -x[1]
    rz, _ = oracle.corr_from_cov(oracle.cell_cov_f32(z, 128, 1, 0))
    sign = np.ones(6)
    sign[1] = -1.0
    np.testing.assert_allclose(rz, r * np.outer(sign, sign), rtol=0, atol=1e-13)


def test_common_signal_gives_all_ones_and_s_one():
    """x_b = g_b u(t) + c_b with g_b > 0 and no noise: r is the all-ones
    matrix (up to float32 rounding of the samples), its eigenvalues are
    N, 0, ..., 0 and s = 1."""
    rng = np.random.default_rng(11)
    N, n = 7, 256
    u = rng.normal(size=n)
    g = rng.uniform(0.5, 2.0, size=N)
    c = rng.uniform(-5.0, 5.0, size=N)
    x = np.ascontiguousarray((g[:, None] * u[None, :] + c[:, None]).astype(np.float32)[:, :, None])
    r, deg = oracle.corr_from_cov(oracle.cell_cov_f32(x, n, 0, 0))
    assert deg == 0
    np.testing.assert_allclose(r, np.ones((N, N)), rtol=0, atol=1e-6)
    ev = oracle.jacobi(r)[0]
    np.testing.assert_allclose(ev, [N] + [0.0] * (N - 1), rtol=0, atol=1e-5)
    assert abs(oracle.stat(ev) - 1.0) < 1e-9
