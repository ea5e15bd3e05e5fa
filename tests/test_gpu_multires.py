"""Several timescales in one pass (mraid_multires, Section 4.2 / Table 1)
against the oracle run directly at each longer sub-integration, and
against mraid_run on a plan with that sub-integration length (needs a GPU).

The longer levels' Gram sums are exact int64 sums of shorter ones, and the
correlation follows from the exact covariance with the same arithmetic on
every path, so each level's statistic, flags and report must equal
mraid_run's bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import STAT_TOL, compare_flags, lib

pytestmark = pytest.mark.gpu

N, C, S, K = 19, 64, 128, 48   # tensor-core Gram: sums interleaved by 8 channels
# unsorted; 5 leaves 3 sub-integrations out; 16 and 24 are formed from 8,
# 48 from 24, 6 from 3 (or 2): every source rule is exercised
FACTORS = [8, 1, 3, 5, 2, 48, 16, 24, 6]


@pytest.fixture(scope="module")
def block():
    cfg = synth.SMALL.replace(n_sub=K)
    return synth.generate(cfg)


def run_at(m, torch, d, f, keep=None):
    """mraid_run on the first (K // f) * f sub-integrations, f * S samples each."""
    n_f = K // f
    with m.Plan(N, C, f * S, n_f, beam_stride=K * S * C, keep=keep) as plan:
        out = plan.run(d, evals=False, q1=False)
        return out["stat"].cpu().numpy(), out["flags"].cpu().numpy(), out["info"]


def test_levels_equal_direct_runs_and_oracle(block):
    import torch
    m = lib()
    d = torch.from_numpy(block).cuda()
    with m.Plan(N, C, S, K) as plan:
        levels = plan.multires(d, FACTORS)
    assert [lv["factor"] for lv in levels] == FACTORS
    for lv in levels:
        f = lv["factor"]
        n_f = K // f
        st = lv["stat"].cpu().numpy()
        fl = lv["flags"].cpu().numpy()
        assert st.shape == (n_f * C,)
        # the same path at the longer sub-integration, bit for bit
        st_r, fl_r, info_r = run_at(m, torch, d, f)
        np.testing.assert_array_equal(st, st_r, err_msg=f"factor {f}")
        np.testing.assert_array_equal(fl, fl_r, err_msg=f"factor {f}")
        for key in ("mu", "sigma", "thresh", "iterations", "n_flagged", "n_used", "n_near",
                    "n_degenerate", "jacobi_sweeps"):
            assert lv["info"][key] == info_r[key], (f, key, lv["info"][key], info_r[key])
        # and the oracle run directly at f * S samples per sub-integration
        sub = np.ascontiguousarray(block[:, :n_f * f * S, :])
        o = oracle.block(sub, f * S, n_threads=synth.default_threads(),
                         want_evals=False, want_q1=False)
        s_err = np.abs(st - o["stat"]) / np.maximum(o["stat"], 1e-30)
        assert s_err.max() <= STAT_TOL, (f, s_err.max())
        f_o, i_o = oracle.flag(o["stat"], C)
        compare_flags(fl, f_o, o["stat"], lv["info"], i_o)
        assert lv["info"]["iterations"] >= 1 and lv["info"]["n_used"] > 0


def test_levels_with_preserved_channels_and_repeat_calls(block):
    """Preserved channels are never flagged at any level; a second call with
    another set of factors (the work buffers grow) and a third with the
    first set again give the same results as the first."""
    import torch
    m = lib()
    d = torch.from_numpy(block).cuda()
    keep = np.zeros(C, np.uint8)
    keep[1] = keep[40] = 1                    # channel 1 carries narrowband RFI
    with m.Plan(N, C, S, K, keep=keep) as plan:
        a = plan.multires(d, [4, 12])
        plan.multires(d, [1, 2, 3, 6, 48])
        b = plan.multires(d, [4, 12])
    for la, lb in zip(a, b):
        np.testing.assert_array_equal(la["stat"].cpu().numpy(), lb["stat"].cpu().numpy())
        np.testing.assert_array_equal(la["flags"].cpu().numpy(), lb["flags"].cpu().numpy())
        assert la["info"] == lb["info"]
        fl = la["flags"].cpu().numpy().reshape(-1, C)
        assert not fl[:, keep.astype(bool)].any()
        st_r, fl_r, _ = run_at(m, torch, d, la["factor"], keep=keep)
        np.testing.assert_array_equal(la["flags"].cpu().numpy(), fl_r)


def test_multires_rejects_bad_arguments(block):
    import torch
    m = lib()
    code = {name: v for v, name in m.STATUS.items()}
    d = torch.from_numpy(block).cuda()
    with m.Plan(N, C, S, K) as plan:
        st = torch.empty(K * C, device="cuda")
        fl = torch.empty(K * C, dtype=torch.uint8, device="cuda")
        for factors in ([0], [K + 1], [2, 2], [], list(range(1, 18))):
            n = len(factors)
            with pytest.raises(m.MraidError) as ei:
                m.mraid_multires(plan.handle, d, factors, [st] * n, [fl] * n)
            assert ei.value.status == code["MRAID_ERR_INVALID_ARG"], factors
        plan.sync()
    x = torch.zeros(N, K * S, C, device="cuda")
    with m.Plan(N, C, S, K, bit_depth=32) as plan:
        with pytest.raises(m.MraidError) as ei:
            m.mraid_multires(plan.handle, x, [2], [st], [fl])
        assert ei.value.status == code["MRAID_ERR_UNSUPPORTED"]


def test_levels_on_the_cuda_core_gram():
    """40 channels (not a multiple of 16), and 36 beams with the CUDA-core
    Gram selected: it writes the sums cell by cell; 36 beams by default:
    the tensor-core Gram for more than 23 beams writes them too. Every
    level still equals mraid_run at its longer sub-integration, bit for
    bit."""
    import torch
    m = lib()
    for (nb, nc, ns, nk, variant, gram) in ((13, 40, 64, 12, None, "gram_u8"),
                                            (36, 16, 64, 8, -1, "gram_u8"),
                                            (36, 16, 64, 8, None, "gram_tcl")):
        cfg = synth.SMALL.replace(n_beam=nb, n_chan=nc, n_samp_sub=ns, n_sub=nk, n_burst=1)
        data = synth.generate(cfg)
        d = torch.from_numpy(data).cuda()
        factors = [1, 2, 3, nk] if nk % 3 == 0 else [1, 2, 4, nk]
        with m.Plan(nb, nc, ns, nk) as plan:
            if variant is not None:
                m.mraid_set_variant(plan.handle, variant)
            m.mraid_profile_enable(plan.handle)
            levels = plan.multires(d, factors)
            ran = m.mraid_profile_read(plan.handle)
        assert "gram_tc" not in ran and gram in ran, ran
        for lv in levels:
            f = lv["factor"]
            n_f = nk // f
            with m.Plan(nb, nc, f * ns, n_f, beam_stride=nk * ns * nc) as p2:
                out = p2.run(d, evals=False, q1=False)
            np.testing.assert_array_equal(lv["stat"].cpu().numpy(), out["stat"].cpu().numpy())
            np.testing.assert_array_equal(lv["flags"].cpu().numpy(), out["flags"].cpu().numpy())
