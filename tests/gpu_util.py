"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare it with the oracle at the tolerances the tests state."""
from __future__ import annotations

import numpy as np

# Eigenvalues: |d lambda| <= 1e-4 * lambda_max per cell (FP32 Jacobi vs FP64).
EIG_TOL = 1e-4
# Statistic s = lambda_1^2 / sum lambda^2: |d s| <= 2e-4 * s; the same band
# marks the cells whose flag may legitimately differ from the oracle's.
STAT_TOL = 2e-4
# q1 is compared where the oracle's relative gap (l1 - l2) / l1 >= 1e-4
# (below it q1 is "unpinned": the two leading eigenvectors mix). The FP32
# solvers leave an error of about 2.3e-7 / gap, so cells with a gap below
# 2e-3 take the FP64 final step (inverse iteration on the same FP32
# correlation); what remains is the FP32 rounding of r itself, ~1e-8 per
# element for noise correlations (|r| ~ 0.03), i.e. ~1e-8 N / gap.
Q1_GAP = 1e-4
Q1_TOL = 1e-3
CORR_TOL = 2e-6


def lib():
    from paper_2512_16278_gb300 import build
    build.build()
    import paper_2512_16278_gb300 as m
    m.load()
    return m


def unpack_sums(packed: np.ndarray, n_beam: int) -> np.ndarray:
    """[cells][P] upper-triangle rows of the (N+1)^2 Gram -> full [cells][N+1][N+1]."""
    M = n_beam + 1
    iu = np.triu_indices(M)
    out = np.zeros((packed.shape[0], M, M), dtype=np.int64)
    out[:, iu[0], iu[1]] = packed
    out[:, iu[1], iu[0]] = packed
    return out


def unpack_corr(packed: np.ndarray, n_beam: int) -> np.ndarray:
    iu = np.triu_indices(n_beam)
    out = np.zeros((packed.shape[0], n_beam, n_beam), dtype=np.float64)
    out[:, iu[0], iu[1]] = packed
    out[:, iu[1], iu[0]] = packed
    return out


def gpu_stages(data: np.ndarray, n_samp_sub: int, keep=None, eig_k: float = 3.0,
               max_clip_iter: int = 64):
    """ccm -> eig -> flag, and run, through the C ABI on cuda:0."""
    import torch
    m = lib()
    n_beam, n_time, n_chan = data.shape
    n_sub = n_time // n_samp_sub
    d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    with m.Plan(n_beam, n_chan, n_samp_sub, n_sub, keep=keep, eig_k=eig_k,
                max_clip_iter=max_clip_iter) as plan:
        sums, corr = plan.ccm(d)
        evals, q1, stat = plan.eig(corr)
        flags, info = plan.flag(stat)
        run = plan.run(d)
        torch.cuda.synchronize()
        out = {
            "sums": sums.cpu().numpy(), "corr": corr.cpu().numpy(),
            "evals": evals.cpu().numpy(), "q1": q1.cpu().numpy(), "stat": stat.cpu().numpy(),
            "flags": flags.cpu().numpy(), "info": info,
            "run": {k: (v.cpu().numpy() if hasattr(v, "cpu") else v)
                    for k, v in run.items() if not k.startswith("_")},
        }
    return out


def all_cells(n_sub: int, n_chan: int):
    subs = np.repeat(np.arange(n_sub, dtype=np.int32), n_chan)
    chans = np.tile(np.arange(n_chan, dtype=np.int32), n_sub)
    return subs, chans


def compare_eig(evals_gpu, evals_orc, what=""):
    lmax = np.abs(evals_orc).max(axis=1, keepdims=True)
    err = np.abs(evals_gpu.astype(np.float64) - evals_orc) / lmax
    per_cell = err.max(axis=1)
    assert np.all(np.isfinite(evals_gpu)), what
    assert per_cell.max() <= EIG_TOL, (what, per_cell.max(), np.percentile(per_cell, 99))
    return float(per_cell.max()), float(np.percentile(per_cell, 99))


def compare_q1(q1_gpu, q1_orc, evals_orc):
    """q1 where the spectral gap pins it. The sign rule (largest-magnitude
    element positive) is decided by rounding when the two largest
    magnitudes tie (always for N = 2), so such cells compare up to sign."""
    gap = (evals_orc[:, 0] - evals_orc[:, 1]) / evals_orc[:, 0]
    sel = gap >= Q1_GAP
    g = q1_gpu[sel].astype(np.float64)
    o = q1_orc[sel]
    err = np.abs(g - o).max(axis=1)
    mags = np.sort(np.abs(o), axis=1)
    tie = (mags[:, -1] - mags[:, -2]) <= Q1_TOL if o.shape[1] > 1 else np.zeros(len(o), bool)
    err_flip = np.abs(g + o).max(axis=1)
    err = np.where(tie, np.minimum(err, err_flip), err)
    assert err.size == 0 or err.max() <= Q1_TOL, (err.max(), int(sel.sum()))
    return int(sel.sum()), float(err.max()) if err.size else 0.0


def compare_flags(flags_gpu, flags_orc, stat_orc, info_gpu, info_orc, keep=None, n_chan=1):
    """Identical except cells within the tolerance band of the threshold."""
    t_orc, t_gpu = info_orc["thresh"], info_gpu["thresh"]
    band = STAT_TOL * stat_orc + (abs(t_gpu - t_orc) if np.isfinite(t_orc) else 0.0)
    near = np.abs(stat_orc - t_orc) <= band
    diff = flags_gpu.astype(bool) != flags_orc.astype(bool)
    assert not np.any(diff & ~near), (int((diff & ~near).sum()), int(diff.sum()))
    if keep is not None:
        kc = np.tile(np.asarray(keep, bool), flags_gpu.shape[0] // n_chan)
        assert not np.any(flags_gpu.astype(bool) & kc)
    return int(near.sum()), int(diff.sum())


def edge_block(n_beam, n_chan, n_sub, seed, n_s=1024):
    """uint8 block [beam][n_sub * n_s][chan] with one of eight saturated or
    extreme patterns per cell: every beam 0; every beam 255; 0/255
    alternation in phase; half the beams in anti-phase; one all-0 beam
    beside noise; 255 and 0 beams beside random 0/255; uniform bytes;
    random 0/255."""
    rng = np.random.default_rng(seed)
    x = np.empty((n_beam, n_sub * n_s, n_chan), dtype=np.uint8)
    alt = (np.arange(n_s) % 2).astype(np.uint8) * 255               # 0, 255, 0, ...
    for k in range(n_sub):
        for c in range(n_chan):
            t = slice(k * n_s, (k + 1) * n_s)
            kind = (k * n_chan + c) % 8
            if kind == 0:                                          # every beam 0
                x[:, t, c] = 0
            elif kind == 1:                                        # every beam 255
                x[:, t, c] = 255
            elif kind == 2:                                        # in-phase alternation
                x[:, t, c] = alt[None, :]
            elif kind == 3:                                        # half the beams anti-phase
                x[:, t, c] = alt[None, :]
                x[::2, t, c] = 255 - alt[None, :]
            elif kind == 4:                                        # one all-0 beam beside noise
                x[:, t, c] = rng.integers(0, 256, size=(n_beam, n_s), dtype=np.uint8)
                x[int(rng.integers(0, n_beam)), t, c] = 0
            elif kind == 5:                                        # 255 and 0 beams, random 0/255
                x[:, t, c] = rng.integers(0, 2, size=(n_beam, n_s), dtype=np.uint8) * 255
                x[0, t, c] = 255
                x[n_beam - 1, t, c] = 0
            elif kind == 6:                                        # uniform bytes
                x[:, t, c] = rng.integers(0, 256, size=(n_beam, n_s), dtype=np.uint8)
            else:                                                  # random 0/255
                x[:, t, c] = rng.integers(0, 2, size=(n_beam, n_s), dtype=np.uint8) * 255
    return x
