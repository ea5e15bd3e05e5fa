"""Every eigensolver variant of the register kernels (Jacobi with looped
rounds, Jacobi with the sweep unrolled, Householder + implicit QR) against
the FP64 oracle on the same FP32 correlations (needs a GPU), including the
structured spectra that stress deflation: rank one, the identity, a
block-diagonal (reducible) matrix and equicorrelation."""
import numpy as np
import pytest

import oracle
from gpu_util import STAT_TOL, compare_eig, compare_q1, lib

pytestmark = pytest.mark.gpu


def structured_corrs(N, n_cells, seed):
    rng = np.random.default_rng(seed)
    out = np.zeros((n_cells, N, N))
    for c in range(n_cells):
        kind = c % 8
        if kind == 0:                                   # rank one: all-ones
            r = np.ones((N, N))
        elif kind == 1:                                 # identity (zero-variance beams)
            r = np.eye(N)
        elif kind == 2:                                 # reducible: two uncorrelated groups
            k = max(1, N // 3)
            r = np.eye(N)
            r[:k, :k] = 0.9 + 0.1 * np.eye(k)
        elif kind == 3:                                 # equicorrelation
            rho = rng.uniform(-0.9 / max(N - 1, 1), 0.9)
            r = (1 - rho) * np.eye(N) + rho
        else:                                           # noise, some with common RFI
            n = int(rng.integers(2 * N, 64 * N))
            X = rng.standard_normal((N, n))
            if kind >= 6:
                X += np.outer(rng.uniform(0.5, 1.5, N), np.sin(np.arange(n) / 3.0)) * rng.uniform(0.05, 1.5)
            r = np.corrcoef(X)
        out[c] = r
    return out


@pytest.mark.parametrize("N", [2, 3, 4, 13, 19])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_eig_variant_matches_oracle(N, variant):
    import torch
    m = lib()
    n_chan, n_sub = 64, 6
    cells = n_chan * n_sub
    R = structured_corrs(N, cells, 100 + N)
    iu = np.triu_indices(N)
    packed = np.ascontiguousarray(R[:, iu[0], iu[1]], dtype=np.float32)
    # the oracle sees exactly the FP32 correlations the kernels see
    R32 = np.zeros_like(R)
    R32[:, iu[0], iu[1]] = packed
    R32[:, iu[1], iu[0]] = packed
    ev_o = np.zeros((cells, N))
    q1_o = np.zeros((cells, N))
    st_o = np.zeros(cells)
    for c in range(cells):
        ev_o[c], q1_o[c], _ = oracle.jacobi(R32[c])
        st_o[c] = oracle.stat(ev_o[c])
    with m.Plan(N, n_chan, 64, n_sub) as plan:
        m.mraid_set_eig_variant(plan.handle, variant)
        ev, q1, st = plan.eig(torch.from_numpy(packed).cuda())
        ev, q1, st = ev.cpu().numpy(), q1.cpu().numpy(), st.cpu().numpy()
    compare_eig(ev, ev_o, f"N={N} variant={variant}")
    compare_q1(q1, q1_o, ev_o)
    assert np.all(np.abs(st - st_o) <= STAT_TOL * st_o + 1e-7), np.abs(st - st_o).max()
    # closed forms: rank one gives (N, 0, ...), the identity all ones
    assert np.abs(ev[0::8, 0] - N).max() <= 1e-4 * N
    assert np.abs(ev[1::8] - 1.0).max() <= 1e-4


@pytest.mark.parametrize("N", [5, 8, 36, 72, 128])
@pytest.mark.parametrize("variant", [0, 3])
def test_large_beam_counts_match_oracle(N, variant):
    """Beam counts without a one-thread kernel: warp-per-matrix Jacobi
    (variant 0) and the tridiagonal solver (Householder by a warp, QR by a
    thread, back-transform by a warp; the default)."""
    import torch
    m = lib()
    n_chan, n_sub = 16, 6
    cells = n_chan * n_sub
    R = structured_corrs(N, cells, 300 + N)
    iu = np.triu_indices(N)
    packed = np.ascontiguousarray(R[:, iu[0], iu[1]], dtype=np.float32)
    R32 = np.zeros_like(R)
    R32[:, iu[0], iu[1]] = packed
    R32[:, iu[1], iu[0]] = packed
    ev_o = np.zeros((cells, N))
    q1_o = np.zeros((cells, N))
    st_o = np.zeros(cells)
    for c in range(cells):
        ev_o[c], q1_o[c], _ = oracle.jacobi(R32[c])
        st_o[c] = oracle.stat(ev_o[c])
    with m.Plan(N, n_chan, 64, n_sub) as plan:
        m.mraid_set_eig_variant(plan.handle, variant)
        ev, q1, st = plan.eig(torch.from_numpy(packed).cuda())
        ev, q1, st = ev.cpu().numpy(), q1.cpu().numpy(), st.cpu().numpy()
    compare_eig(ev, ev_o, f"N={N} variant={variant}")
    compare_q1(q1, q1_o, ev_o)
    assert np.all(np.abs(st - st_o) <= STAT_TOL * st_o + 1e-7), np.abs(st - st_o).max()
    assert np.abs(ev[0::8, 0] - N).max() <= 1e-4 * N
    assert np.abs(ev[1::8] - 1.0).max() <= 1e-4
