"""Pins of the CPU oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: brute force
with a different routine, closed forms, invariants, or distributional facts.
The method is mRAID (arXiv 2512.16278): Eq. 1 (CCM), Eq. 2 (eigen-
decomposition, normalised eigenvalues, Section 3.3), the iterative Gaussian-fit
threshold (Section 3.3 masking paragraph, k = 3 from Section 4.5) and preserved
ranges (Section 4.3).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def hadamard(n):
    H = np.array([[1]], dtype=np.int64)
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


def block_from_beams(x):
    """x: [beam][time] integer series -> uint8 block [beam][time][1 chan]."""
    x = np.asarray(x)
    assert x.min() >= 0 and x.max() <= 255
    return np.ascontiguousarray(x.astype(np.uint8)[:, :, None])


# ------------------------------------------------------------- Eq. 1 sums

@pytest.mark.parametrize("n_beam,n_s,n_chan", [(2, 1, 3), (3, 5, 4), (19, 128, 7), (13, 64, 2)])
def test_gram_matches_bruteforce_einsum(n_beam, n_s, n_chan):
    rng = np.random.default_rng(n_beam * 1000 + n_s)
    n_sub = 3
    d = rng.integers(0, 256, size=(n_beam, n_sub * n_s, n_chan), dtype=np.uint8)
    for sub in range(n_sub):
        for chan in range(n_chan):
            G = oracle.cell_gram(d, n_s, sub, chan)
            X = d[:, sub * n_s:(sub + 1) * n_s, chan].astype(np.int64)
            Xa = np.vstack([X, np.ones((1, n_s), dtype=np.int64)])
            np.testing.assert_array_equal(G, np.einsum("at,bt->ab", Xa, Xa))


def test_gram_is_additive_over_time():
    rng = np.random.default_rng(7)
    d = rng.integers(0, 256, size=(19, 4 * 96, 5), dtype=np.uint8)
    for k in (0, 2):
        for chan in range(5):
            g0 = oracle.cell_gram(d, 96, k, chan)
            g1 = oracle.cell_gram(d, 96, k + 1, chan)
            g01 = oracle.cell_gram(d, 192, k // 2, chan)
            np.testing.assert_array_equal(g0 + g1, g01)


def test_extreme_values_exact():
    d = np.full((19, 1024, 1), 255, dtype=np.uint8)
    d[::2, ::3, 0] = 0
    G = oracle.cell_gram(d, 1024, 0, 0)
    X = d[:, :, 0].astype(np.int64)
    np.testing.assert_array_equal(G[:19, :19], X @ X.T)
    assert G[19, 19] == 1024


# -------------------------------------------------- correlation (reading R1)

def test_corr_matches_numpy_corrcoef():
    rng = np.random.default_rng(11)
    d = rng.integers(0, 256, size=(19, 256, 3), dtype=np.uint8)
    for chan in range(3):
        G = oracle.cell_gram(d, 256, 0, chan)
        r, deg = oracle.corr_from_gram(G)
        assert deg == 0
        np.testing.assert_allclose(r, np.corrcoef(d[:, :, chan].astype(np.float64)),
                                   rtol=0, atol=1e-13)
        np.testing.assert_array_equal(np.diag(r), np.ones(19))


def test_zero_variance_beam_rule():
    rng = np.random.default_rng(12)
    x = rng.integers(60, 200, size=(5, 64))
    x[2, :] = 77                     # constant beam
    c = oracle.cell(block_from_beams(x), 64, 0, 0)
    assert c["n_degenerate"] == 1
    r = c["r"]
    assert r[2, 2] == 1.0
    assert np.all(r[2, [0, 1, 3, 4]] == 0.0) and np.all(r[[0, 1, 3, 4], 2] == 0.0)
    # the isolated beam contributes an eigenvalue of exactly one
    assert np.min(np.abs(c["evals"] - 1.0)) < 1e-13


def test_shift_invariance_is_exact():
    """A per-(beam, cell) constant offset (what subtracting a fitted bandpass
    does, Section 3.1) leaves the Pearson CCM bit-identical."""
    rng = np.random.default_rng(13)
    x = rng.integers(40, 200, size=(19, 128))
    offs = rng.integers(-40, 50, size=(19, 1))
    c0 = oracle.cell(block_from_beams(x), 128, 0, 0)
    c1 = oracle.cell(block_from_beams(x + offs), 128, 0, 0)
    np.testing.assert_array_equal(c0["r"], c1["r"])
    np.testing.assert_array_equal(c0["evals"], c1["evals"])


def test_negating_a_beam_keeps_eigenvalues():
    rng = np.random.default_rng(14)
    x = rng.integers(0, 256, size=(19, 128))
    y = x.copy()
    y[4] = 255 - y[4]
    c0 = oracle.cell(block_from_beams(x), 128, 0, 0)
    c1 = oracle.cell(block_from_beams(y), 128, 0, 0)
    np.testing.assert_allclose(c1["r"][4, :4], -c0["r"][4, :4], atol=1e-15)
    np.testing.assert_allclose(c0["evals"], c1["evals"], atol=1e-12)


def test_beam_permutation_invariance():
    rng = np.random.default_rng(15)
    x = rng.integers(0, 256, size=(19, 128))
    perm = rng.permutation(19)
    c0 = oracle.cell(block_from_beams(x), 128, 0, 0)
    c1 = oracle.cell(block_from_beams(x[perm]), 128, 0, 0)
    np.testing.assert_allclose(c0["evals"], c1["evals"], atol=1e-12)
    np.testing.assert_allclose(c1["q1"], c0["q1"][perm], atol=1e-9)


# --------------------------------------------------- Eq. 2 closed forms

@pytest.mark.parametrize("n_beam", [2, 3, 13, 19, 30])
def test_equicorrelation_closed_form(n_beam):
    """x_b = 128 + 9 w_1 + 12 w_(b+2) with orthogonal zero-mean Walsh rows:
    every pair has correlation 81/225 exactly, so the eigenvalues are
    1 + (N-1) rho (once) and 1 - rho (N-1 times)."""
    n_s = 64
    H = hadamard(n_s)
    x = np.array([128 + 9 * H[1] + 12 * H[b + 2] for b in range(n_beam)])
    c = oracle.cell(block_from_beams(x), n_s, 0, 0)
    rho = 81.0 / 225.0
    off = c["r"][~np.eye(n_beam, dtype=bool)]
    np.testing.assert_allclose(off, rho, rtol=0, atol=1e-15)
    want = np.array([1 + (n_beam - 1) * rho] + [1 - rho] * (n_beam - 1))
    np.testing.assert_allclose(c["evals"], want, rtol=0, atol=1e-12)
    # q1 of an equicorrelation matrix with rho > 0 is the uniform vector
    np.testing.assert_allclose(c["q1"], np.full(n_beam, 1 / math.sqrt(n_beam)), atol=1e-10)
    s_want = want[0] ** 2 / np.sum(want ** 2)
    assert abs(c["stat"] - s_want) < 1e-12


def test_common_signal_is_rank_one():
    """x_b = g_b u(t) + c_b with g_b > 0: r is all ones, lambda = (N, 0...),
    s = 1 (the beam-common RFI limit, Section 3.2)."""
    H = hadamard(128)
    g = [1, 2, 3, 4, 5, 6, 1, 2, 3, 4, 5, 6, 1, 2, 3, 4, 5, 6, 2]
    x = np.array([100 + g[b] * H[5] + b for b in range(19)])
    c = oracle.cell(block_from_beams(x), 128, 0, 0)
    np.testing.assert_allclose(c["r"], np.ones((19, 19)), atol=1e-15)
    np.testing.assert_allclose(c["evals"], [19.0] + [0.0] * 18, atol=1e-12)
    assert abs(c["stat"] - 1.0) < 1e-13


def test_two_beams_closed_form():
    rng = np.random.default_rng(21)
    for _ in range(20):
        x = rng.integers(0, 256, size=(2, 50))
        c = oracle.cell(block_from_beams(x), 50, 0, 0)
        r12 = np.corrcoef(x.astype(np.float64))[0, 1]
        np.testing.assert_allclose(c["evals"], [1 + abs(r12), 1 - abs(r12)], atol=1e-13)


def test_three_beams_characteristic_polynomial():
    """Roots of det(lambda I - r) for a unit-diagonal 3x3 matrix by the
    trigonometric solution of the depressed cubic."""
    rng = np.random.default_rng(22)
    for _ in range(50):
        base = rng.integers(0, 120, size=(1, 40))
        x = np.clip(base + rng.integers(0, 120, size=(3, 40)), 0, 255)
        c = oracle.cell(block_from_beams(x), 40, 0, 0)
        r = c["r"]
        a, b, d = r[0, 1], r[0, 2], r[1, 2]
        p1 = a * a + b * b + d * d
        p = math.sqrt(p1 / 3.0)
        half_det = (a * b * d) / p ** 3       # det(r - I) / (2 p^3)
        phi = math.acos(max(-1.0, min(1.0, half_det))) / 3.0
        l1 = 1 + 2 * p * math.cos(phi)
        l3 = 1 + 2 * p * math.cos(phi + 2 * math.pi / 3)
        l2 = 3 - l1 - l3
        np.testing.assert_allclose(c["evals"], [l1, l2, l3], atol=1e-12)


@pytest.mark.parametrize("n", [2, 7, 19, 36])
def test_jacobi_on_tridiagonal_toeplitz(n):
    """tridiag(-1, 2, -1): lambda_k = 2 - 2 cos(k pi / (n+1)); the top
    eigenvector is (-1)^j sin(j pi/(n+1)), j = 1..n."""
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    ev, q1, _ = oracle.jacobi(A)
    k = np.arange(n, 0, -1)
    np.testing.assert_allclose(ev, 2 - 2 * np.cos(k * np.pi / (n + 1)), atol=1e-13)
    j = np.arange(1, n + 1)
    v = (-1.0) ** (j + 1) * np.sin(j * np.pi / (n + 1))
    v /= np.linalg.norm(v)
    # same vector up to sign, and the sign rule: the largest-magnitude
    # element (lowest index among numerical ties) is positive
    np.testing.assert_allclose(abs(float(q1 @ v)), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.abs(q1), np.abs(v), atol=1e-12)
    top = np.flatnonzero(np.abs(q1) >= np.abs(q1).max() - 1e-12)
    assert q1[top[0]] > 0 or (len(top) > 1 and q1[top[1]] > 0)


def test_jacobi_diagonal_input_needs_no_sweep():
    ev, q1, sweeps = oracle.jacobi(np.diag([0.5, 3.0, 2.0]))
    assert sweeps == 0
    np.testing.assert_array_equal(ev, [3.0, 2.0, 0.5])
    np.testing.assert_array_equal(q1, [0.0, 1.0, 0.0])


def test_invariants_on_synthetic_block(small_block):
    """Unit diagonal, trace N, sum of squares = ||r||_F^2, PSD; eigenvalues
    equal LAPACK's (numpy eigvalsh) and q1 is a unit eigenvector."""
    d = small_block
    rng = np.random.default_rng(23)
    for _ in range(40):
        sub, chan = int(rng.integers(0, 256)), int(rng.integers(0, 64))
        c = oracle.cell(d, 128, sub, chan)
        r, ev, q1 = c["r"], c["evals"], c["q1"]
        assert np.all(np.diag(r) == 1.0)
        assert abs(ev.sum() - 19.0) < 1e-12
        assert abs(np.sum(ev ** 2) - np.sum(r * r)) < 1e-11
        assert ev.min() > -1e-12
        assert np.all(np.diff(ev) <= 0)
        np.testing.assert_allclose(ev, np.linalg.eigvalsh(r)[::-1], atol=1e-12)
        assert abs(np.linalg.norm(q1) - 1) < 1e-13
        np.testing.assert_allclose(r @ q1, ev[0] * q1, atol=1e-11)
        assert q1[np.argmax(np.abs(q1))] > 0



@pytest.mark.parametrize("n_threads,by_pointer", [(1, False), (4, False), (3, True)])
def test_cells_driver_matches_brute_force(small_block, n_threads, by_pointer):
    """The threaded selected-cells driver (the one the GPU parity tests call,
    also through a raw pointer) against numpy on the same bytes: Gram sums by
    einsum, eigenvalues by LAPACK of numpy's corrcoef, q1 an eigenvector of
    lambda_1 with the sign rule, s = lambda_1^2 / ||r||_F^2."""
    d = small_block
    rng = np.random.default_rng(29 + n_threads)
    subs = rng.integers(0, 256, size=23).astype(np.int32)
    chans = rng.integers(0, 64, size=23).astype(np.int32)
    if by_pointer:
        o = oracle.cells(None, 128, subs, chans, n_threads=n_threads,
                         data_ptr=d.ctypes.data, shape=d.shape)
    else:
        o = oracle.cells(d, 128, subs, chans, n_threads=n_threads)
    for i, (k, c) in enumerate(zip(subs, chans)):
        X = d[:, k * 128:(k + 1) * 128, c].astype(np.int64)
        Xa = np.vstack([X, np.ones((1, 128), dtype=np.int64)])
        np.testing.assert_array_equal(o["G"][i], np.einsum("at,bt->ab", Xa, Xa))
        r = np.corrcoef(X.astype(np.float64))
        ev = np.linalg.eigvalsh(r)[::-1]
        np.testing.assert_allclose(o["evals"][i], ev, rtol=0, atol=1e-12)
        q = o["q1"][i]
        np.testing.assert_allclose(r @ q, ev[0] * q, rtol=0, atol=1e-10)
        assert abs(np.linalg.norm(q) - 1.0) < 1e-12 and q[np.argmax(np.abs(q))] > 0
        assert abs(o["stat"][i] - ev[0] ** 2 / np.sum(r * r)) < 1e-12


# ------------------------------------------- noise statistics (Eq. 1-2)

def test_noise_only_second_moment_and_mp_edges():
    """Independent iid noise: E[r_ab^2] = 1/(n-1) exactly for exchangeable
    samples, so E[sum lambda^2] = N + N(N-1)/(n-1); eigenvalues pool inside
    the Marchenko-Pastur edges (1 +- sqrt(N/n))^2, widened by 0.2."""
    cfg = synth.SMALL.replace(n_narrow=0, n_burst=0, n_spike=0, seed=0x51)
    d = synth.generate(cfg)
    res = oracle.block(d, cfg.n_samp_sub, n_threads=synth.default_threads(), want_q1=False)
    ev = res["evals"]
    N, n = cfg.n_beam, cfg.n_samp_sub
    ss = np.sum(ev ** 2, axis=1)
    want = N + N * (N - 1) / (n - 1)
    se = ss.std(ddof=1) / math.sqrt(ss.shape[0])
    assert abs(ss.mean() - want) < 4 * se, (ss.mean(), want, se)
    # the 1/n alternative is many standard errors away: the pin has teeth
    assert abs(ss.mean() - (N + N * (N - 1) / n)) > 8 * se
    g = math.sqrt(N / n)
    lo, hi = (1 - g) ** 2 - 0.2, (1 + g) ** 2 + 0.2
    inside = np.mean((ev >= lo) & (ev <= hi))
    assert inside >= 0.99, inside
    # no RFI: the iterative 3-sigma clip flags only the upper tail
    flags, info = oracle.flag(res["stat"], cfg.n_chan)
    assert info["converged"] == 1
    assert flags.mean() < 0.03


# ------------------------------------------- masking rule (Section 3.3)

def test_flag_ramp_plus_outliers():
    """1000 cells on a narrow ramp around 0.1 plus 5 at 0.9: the first fit
    (mu ~0.104, sigma ~0.056) flags the five; the second (sigma = 0.01/sqrt 12)
    flags none of the ramp."""
    s = np.concatenate([0.1 + 0.01 * (np.arange(1000) / 999 - 0.5), np.full(5, 0.9)])
    flags, info = oracle.flag(s, 1)
    assert flags[:1000].sum() == 0 and flags[1000:].sum() == 5
    assert info["iterations"] == 2 and info["converged"] == 1
    ramp = s[:1000]
    assert abs(info["mu"] - ramp.mean()) < 1e-15
    assert abs(info["sigma"] - ramp.std()) < 1e-15
    assert abs(info["thresh"] - (ramp.mean() + 3 * ramp.std())) < 1e-15


def test_flag_single_outlier_closed_form():
    """n-1 zeros and a one: mu = 1/n, sigma = sqrt(n-1)/n; for n >= 11 the
    threshold is below one, the outlier goes, then sigma = 0 and nothing
    exceeds mu = 0."""
    for n in (11, 50, 1000):
        s = np.zeros(n)
        s[n // 2] = 1.0
        flags, info = oracle.flag(s, 1, max_iter=10)
        assert flags.sum() == 1 and flags[n // 2] == 1
        assert info["iterations"] == 2
        assert info["thresh"] == 0.0
    # n = 9: 1/9 + 3*sqrt(8)/9 = 1.054 > 1, nothing is flagged
    s = np.zeros(9)
    s[0] = 1.0
    flags, info = oracle.flag(s, 1)
    assert flags.sum() == 0 and info["iterations"] == 1
    assert abs(info["thresh"] - (1 / 9 + 3 * math.sqrt(8) / 9)) < 1e-15


def test_flag_keep_excludes_channel_from_stats_and_mask():
    rng = np.random.default_rng(31)
    n_chan = 16
    s = rng.normal(0.2, 0.01, size=(100, n_chan))
    s[:, 3] = 0.95                          # e.g. a line detected in all beams
    keep = np.zeros(n_chan, dtype=np.uint8)
    keep[3] = 1
    f_keep, i_keep = oracle.flag(s.ravel(), n_chan, keep)
    assert f_keep.reshape(100, n_chan)[:, 3].sum() == 0
    other = np.delete(s, 3, axis=1).ravel()
    f_ref, i_ref = oracle.flag(other, n_chan - 1)
    assert i_keep["n_flagged"] == i_ref["n_flagged"]
    assert abs(i_keep["mu"] - i_ref["mu"]) < 1e-12
    # without the keep mask the line channel is masked
    f_all, _ = oracle.flag(s.ravel(), n_chan)
    assert f_all.reshape(100, n_chan)[:, 3].sum() == 100


def test_flag_monotone_and_bounded():
    rng = np.random.default_rng(32)
    s = np.concatenate([rng.gamma(2.0, 0.05, size=5000), rng.uniform(0.5, 1.0, 50)])
    prev = np.zeros(s.shape[0], dtype=np.uint8)
    for it in range(1, 12):
        f, info = oracle.flag(s, 1, max_iter=it)
        assert np.all(f >= prev)            # the mask only grows
        assert info["iterations"] <= it
        prev = f
    f_full, info = oracle.flag(s, 1, max_iter=1000)
    assert info["converged"] == 1


def test_flag_cell_permutation_equivariance():
    rng = np.random.default_rng(33)
    s = np.concatenate([rng.normal(0.2, 0.02, 3000), rng.uniform(0.6, 0.9, 30)])
    perm = rng.permutation(s.shape[0])
    f0, i0 = oracle.flag(s, 1)
    f1, i1 = oracle.flag(s[perm], 1)
    np.testing.assert_array_equal(f1, f0[perm])
    assert i0["iterations"] == i1["iterations"]


# ------------------------------------ behaviour on injected RFI (Sec. 3.2)

def test_beam_common_rfi_flagged_single_beam_not(small_block):
    cfg = synth.SMALL
    res = oracle.block(small_block, cfg.n_samp_sub, n_threads=synth.default_threads(),
                       want_evals=False, want_q1=False)
    flags, info = oracle.flag(res["stat"], cfg.n_chan)
    F = flags.reshape(cfg.n_sub, cfg.n_chan)
    cells = synth.rfi_cells(cfg)
    assert all(F[k, c] for (k, c) in cells["narrow"])
    assert all(F[k, c] for (k, c) in cells["burst"])
    assert not any(F[k, c] for (k, c) in cells["spike"])
    S = res["stat"].reshape(cfg.n_sub, cfg.n_chan)
    # RFI cells have a near rank-one CCM
    assert min(S[k, c] for (k, c) in cells["burst"]) > 0.5
    assert info["converged"] == 1


# ------------------------------- eigenvector refinement (Sec. 3.3, 4.5)

def test_beam_flags_closed_form():
    """Unflagged cells with |q1_b| in {0.1, 0.3} equally often give mu_b = 0.2,
    sigma_b = 0.1 exactly; a flagged cell marks beam b iff |q1_b| > 0.2 + t 0.1."""
    n_beam, n_clean = 3, 100
    q = np.zeros((n_clean + 2, n_beam))
    q[:n_clean:2] = 0.1
    q[1:n_clean:2] = -0.3                  # magnitudes count, not signs
    flags = np.zeros(n_clean + 2, dtype=np.uint8)
    flags[n_clean:] = 1
    q[n_clean] = [0.35, 0.25, -0.31]        # t = 1: threshold 0.3
    q[n_clean + 1] = [0.29, 0.9, 0.0]
    bits, ms = oracle.beam_flags(q, flags, 1, t=1.0)
    np.testing.assert_allclose(ms[:, 0], 0.2, atol=1e-15)
    np.testing.assert_allclose(ms[:, 1], 0.1, atol=1e-15)
    assert bits[n_clean, 0] == 0b101 and bits[n_clean + 1, 0] == 0b010
    assert not bits[:n_clean].any()        # unflagged cells carry no beam bits
    bits2, _ = oracle.beam_flags(q, flags, 1, t=0.0)   # threshold 0.2
    assert bits2[n_clean, 0] == 0b111 and bits2[n_clean + 1, 0] == 0b011


def test_beam_flags_monotone_in_t_and_many_beams():
    rng = np.random.default_rng(41)
    n_cells, n_beam = 2000, 40                 # two words of bits
    q = rng.normal(0, 1, size=(n_cells, n_beam))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    flags = (rng.random(n_cells) < 0.1).astype(np.uint8)
    prev = None
    for t in (0.0, 1.0, 2.0, 3.0):
        bits, ms = oracle.beam_flags(q, flags, 1, t=t)
        assert bits.shape == (n_cells, 2)
        count = sum(bin(int(x)).count("1") for x in bits.ravel())
        if prev is not None:
            assert count <= prev
        prev = count
    # beam 35 lives in word 1, bit 3
    bits, ms = oracle.beam_flags(q, flags, 1, t=0.0)
    i = int(np.flatnonzero(flags)[0])
    assert ((bits[i, 1] >> 3) & 1) == (abs(q[i, 35]) > ms[35, 0])


def test_beam_flags_rfi_beams_on_small_block(small_block):
    """Beam-common narrowband RFI with per-beam gains (Sec. 3.3, Fig. 3): in
    its channel, the beams with larger eigenvector elements are the ones
    marked as affected; unflagged cells carry no beam bits."""
    cfg = synth.SMALL
    res = oracle.block(small_block, cfg.n_samp_sub, n_threads=synth.default_threads())
    flags, _ = oracle.flag(res["stat"], cfg.n_chan)
    bits, ms = oracle.beam_flags(res["q1"], flags, cfg.n_chan, t=1.0)
    assert not bits[flags == 0].any()
    ch = synth.events(cfg)["narrow"][0][0]
    b = bits.reshape(cfg.n_sub, cfg.n_chan, -1)[:, ch, 0]
    freq = np.array([np.mean((b >> k) & 1) for k in range(cfg.n_beam)])
    mag = np.abs(res["q1"].reshape(cfg.n_sub, cfg.n_chan, -1)[:, ch, :]).mean(axis=0)
    rank = lambda v: np.argsort(np.argsort(v))
    rho = np.corrcoef(rank(freq), rank(mag))[0, 1]      # Spearman
    assert rho > 0.6, rho
