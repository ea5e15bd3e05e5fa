"""Float32 samples (beamformer output, bit_depth 32) on the GPU against the
FP64 oracle (needs a GPU): N(0,1) noise plus beam-common RFI, and a large
common offset that a naive sum-of-products would cancel badly."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare_eig, compare_flags, lib

pytestmark = pytest.mark.gpu


def f32_block(n_beam, n_chan, n_s, n_sub, offset, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n_beam, n_sub * n_s, n_chan)).astype(np.float32)
    g = rng.uniform(0.5, 1.5, size=(n_beam, 1, 1)).astype(np.float32)
    t = np.arange(n_sub * n_s)
    x[:, :, 1] += 0.75 * g[:, :, 0] * np.sin(2 * np.pi * t / 16)[None, :]   # narrowband RFI
    x[:, n_s // 2: n_s // 2 + n_s, 8:12] += 2.0 * g[:, :, :1]                # a burst
    return np.ascontiguousarray(x + offset)


# gram: None = the default (tensor cores, split-bf16 products, where the
# shape fits), -1 = the CUDA-core FP32 Gram
@pytest.mark.parametrize("gram", [None, -1])
@pytest.mark.parametrize("offset", [0.0, 1000.0])
def test_f32_block_matches_oracle(offset, gram):
    import torch
    m = lib()
    # RFI in 8 + 8 of 512 cells: few enough for the 3-sigma clip to isolate
    n_beam, n_chan, n_s, n_sub = 19, 64, 256, 8
    x = f32_block(n_beam, n_chan, n_s, n_sub, offset, 7)
    d = torch.from_numpy(x).cuda()
    with m.Plan(n_beam, n_chan, n_s, n_sub, bit_depth=32) as plan:
        if gram is not None:
            m.mraid_set_variant(plan.handle, gram)
        m.mraid_profile_enable(plan.handle)
        _, corr = plan.ccm(d, sums=False)
        out = plan.run(d)
        ran = m.mraid_profile_read(plan.handle)
    want = "gram_f32" if gram == -1 else "gram_tc_f32"
    assert ran.get(want, (0, 0.0))[0] == 2, ran
    corr = corr.cpu().numpy()
    iu = np.triu_indices(n_beam)
    ev_o = np.zeros((n_sub * n_chan, n_beam))
    st_o = np.zeros(n_sub * n_chan)
    worst = 0.0
    for k in range(n_sub):
        for c in range(n_chan):
            r, _ = oracle.corr_from_cov(oracle.cell_cov_f32(x, n_s, k, c))
            worst = max(worst, float(np.abs(corr[k * n_chan + c] - r[iu]).max()))
            ev_o[k * n_chan + c] = oracle.jacobi(r)[0]
            st_o[k * n_chan + c] = oracle.stat(ev_o[k * n_chan + c])
    # FP32 sums of shifted samples: |dr| stays ~1e-6 even with a 1000 offset
    assert worst <= 2e-5, worst
    compare_eig(out["evals"].cpu().numpy(), ev_o, f"f32 offset {offset}")
    flags_o, info_o = oracle.flag(st_o, n_chan)
    compare_flags(out["flags"].cpu().numpy(), flags_o, st_o, out["info"], info_o)
    F = flags_o.reshape(n_sub, n_chan).astype(bool)
    assert F[:, 1].all()                     # the narrowband channel
    assert F[0, 8:12].all() and F[1, 8:12].all()   # the burst's two sub-integrations


@pytest.mark.parametrize("n_beam,n_chan,n_s,n_sub", [
    (2, 32, 64, 6),      # smallest beam count, two 32-sample stages
    (13, 48, 32, 5),     # one stage per cell, three 16-channel boxes
    (16, 16, 96, 4),     # first count with the extra-slot MMA
    (23, 32, 128, 3),    # largest count on the tensor cores
    (19, 40, 64, 3),     # 40 channels: not a multiple of 16, CUDA cores
    (13, 32, 48, 4),     # 48 samples: not a multiple of 32, CUDA cores
    (24, 16, 64, 2),     # beyond 23 beams: CUDA cores
])
def test_f32_shapes_match_oracle(n_beam, n_chan, n_s, n_sub):
    """Correlations of float32 blocks of several shapes against the FP64
    oracle, through the tensor-core kernel where the shape fits it and the
    CUDA-core kernel elsewhere, with a constant beam in one channel (zero
    variance: r = 0 off the diagonal) and an offset of 300."""
    import torch
    m = lib()
    x = f32_block(n_beam, n_chan, n_s, n_sub, 300.0, 11 + n_beam)
    x[1, :, 3] = 42.5                         # beam 1 constant in channel 3
    d = torch.from_numpy(x).cuda()
    with m.Plan(n_beam, n_chan, n_s, n_sub, bit_depth=32) as plan:
        m.mraid_profile_enable(plan.handle)
        _, corr = plan.ccm(d, sums=False)
        plan.sync()
        ran = m.mraid_profile_read(plan.handle)
    tc = n_beam <= 23 and n_chan % 16 == 0 and n_s % 32 == 0
    assert ran.get("gram_tc_f32" if tc else "gram_f32", (0, 0.0))[0] == 1, ran
    corr = corr.cpu().numpy()
    iu = np.triu_indices(n_beam)
    worst = 0.0
    for k in range(n_sub):
        for c in range(n_chan):
            r, _ = oracle.corr_from_cov(oracle.cell_cov_f32(x, n_s, k, c))
            worst = max(worst, float(np.abs(corr[k * n_chan + c] - r[iu]).max()))
    assert worst <= 2e-5, worst
    row1 = corr[3::n_chan]                    # channel 3 of every sub-integration
    a = 1
    start = a * n_beam - a * (a - 1) // 2     # packed row of beam 1
    assert np.all(row1[:, start] == 1.0)
    assert np.all(row1[:, start + 1:start + n_beam - a] == 0.0)


def test_f32_autotune_times_both_gram_kernels():
    """For float32 samples the autotuner times the CUDA-core Gram (-1) and
    the one tensor-core kernel (0), nothing else, and keeps one of them."""
    import torch
    m = lib()
    x = f32_block(19, 64, 256, 4, 0.0, 5)
    d = torch.from_numpy(x).cuda()
    with m.Plan(19, 64, 256, 4, bit_depth=32) as plan:
        (g, e), times = m.mraid_autotune(plan.handle, d, reps=2)
    assert g in (-1, 0) and e in (0, 1, 2, 3, 4, 5)
    assert sorted(k for k in times if k.startswith("g")) == ["g-1", "g0"], times
