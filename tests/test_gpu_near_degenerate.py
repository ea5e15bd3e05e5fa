"""q1 on near-degenerate spectra (Section 3.3, Eq. 2) through the C ABI.

Every cell carries two beam-common signals of nearly equal power: Walsh
sequences u, v (exactly orthogonal, equal power) with beam patterns
cos(theta_b) and (1 + eps_c) sin(theta_b), theta_b evenly spaced, plus
Gaussian noise. Without eps and noise r = a a^T + b b^T with lambda_1 =
lambda_2 = N / 2; eps_c (1e-5 .. 1e-1 over the channels) and the noise
spread the relative gap (lambda_1 - lambda_2) / lambda_1 from ~1e-6 to
~1e-1, so many cells fall where the FP32 solvers alone leave q1 mixed with
the second eigenvector and the FP64 final step decides it. q1 must match the
oracle to 1e-3 per element at every gap >= 1e-4, under every eigensolver
variant; the FP64 step's count in the report must equal the cells that the
FP32 eigenvalues select (relative gap below 2e-3, or below 1e-2 behind the
one-thread Jacobi variants)."""
import numpy as np
import pytest

import oracle
from gpu_util import EIG_TOL, Q1_GAP, compare_eig, compare_q1, lib

pytestmark = pytest.mark.gpu


def walsh(n, k):
    """Row k of the n x n Sylvester-Hadamard matrix (n a power of two)."""
    t = np.arange(n)
    bits = np.zeros(n, dtype=np.int64)
    kk = k
    b = 0
    while kk:
        if kk & 1:
            bits += (t >> b) & 1
        kk >>= 1
        b += 1
    return np.where(bits % 2 == 0, 1.0, -1.0)


def two_signal_block(n_beam, n_chan, n_sub, n_samp, seed):
    rng = np.random.default_rng(seed)
    theta = 2 * np.pi * np.arange(n_beam) / n_beam + 0.3
    eps = 10.0 ** np.linspace(-5, -1, n_chan)
    amp = 40.0
    x = np.empty((n_beam, n_sub * n_samp, n_chan))
    for k in range(n_sub):
        u = walsh(n_samp, 1 + 2 * k)
        v = walsh(n_samp, 2 + 2 * k)
        sig = amp * (np.cos(theta)[:, None, None] * u[None, :, None]
                     + (1 + eps)[None, None, :] * np.sin(theta)[:, None, None] * v[None, :, None])
        x[:, k * n_samp:(k + 1) * n_samp, :] = 128 + sig
    x += rng.normal(0.0, 2.0, size=x.shape)
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


@pytest.mark.parametrize("n_beam,n_chan,variants", [(19, 64, (0, 1, 2, 3, 4, 5)), (36, 32, (0, 3))])
def test_q1_near_degenerate_matches_oracle(n_beam, n_chan, variants):
    import torch
    m = lib()
    n_sub, n_samp = 24, 1024
    data = two_signal_block(n_beam, n_chan, n_sub, n_samp, seed=n_beam)
    subs = np.repeat(np.arange(n_sub, dtype=np.int32), n_chan)
    chans = np.tile(np.arange(n_chan, dtype=np.int32), n_sub)
    o = oracle.cells(data, n_samp, subs, chans, n_threads=4)
    gap = (o["evals"][:, 0] - o["evals"][:, 1]) / o["evals"][:, 0]
    # the construction covers the band the FP64 step serves
    assert np.sum((gap >= Q1_GAP) & (gap < 2e-3)) >= 100, np.sort(gap)[:20]
    d = torch.from_numpy(data).cuda()
    for variant in variants:
        with m.Plan(n_beam, n_chan, n_samp, n_sub) as plan:
            m.mraid_set_eig_variant(plan.handle, variant)
            out = plan.run(d)
            torch.cuda.synchronize()
        ev = out["evals"].cpu().numpy()
        q1 = out["q1"].cpu().numpy()
        compare_eig(ev, o["evals"], f"N={n_beam} variant={variant}")
        n_checked, err = compare_q1(q1, o["q1"], o["evals"])
        assert n_checked >= int(np.sum(gap >= Q1_GAP)), n_checked
        l1, l2 = ev[:, 0], ev[:, 1]
        g32 = (l1 - l2) / l1
        # the one-thread Jacobi solvers hand over below 1e-2, the others below 2e-3
        hi = 1e-2 if (variant < 2 and n_beam in (2, 3, 4, 13, 19)) else 2e-3
        sel = (l1 > 0) & (g32 >= np.float32(1e-6)) & (g32 < np.float32(hi))
        assert out["info"]["q1_refined"] == int(sel.sum()), (out["info"]["q1_refined"], int(sel.sum()))
        assert np.all(np.abs(np.linalg.norm(q1.astype(np.float64), axis=1) - 1) <= 1e-5)
    assert EIG_TOL > 0
