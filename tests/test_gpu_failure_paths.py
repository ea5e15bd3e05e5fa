"""Failure detection through the C ABI (needs a GPU; nothing faults or hangs
the device).

A bounded wait that runs out: the host arms MRAID_FAULT_WITHHOLD_STAGE, so
the first CTA of the next tensor-core Gram launch (the block-diagonal kernel
at 19 beams, the large-beam kernel at 36) never issues one of its bulk
copies. Nothing is then in flight for that stage; the converter's wait
for it expires after the plan's wait limit (50 ms here), the kernel records
the error, every role returns, its own copies and MMAs are drained and its
tensor memory freed. mraid_sync must report MRAID_ERR_TIMEOUT with the
info's timed_out set, and the next, normal call on the same plan must give
the results of an undisturbed run.

An allocation failure: MRAID_FAULT_ALLOC makes the plan's next work-buffer
allocation fail as out of memory; the call returns MRAID_ERR_OOM and the
next call succeeds."""
import numpy as np
import pytest

from gpu_util import lib

pytestmark = pytest.mark.gpu

N_BEAM, N_CHAN, N_S, N_SUB = 19, 32, 1024, 4     # tensor-core Gram shape
SHAPES = [(19, 32, 1024, 4, "gram_tc"), (36, 32, 2048, 2, "gram_tcl")]
TIMEOUT, OOM = 5, 3


def block(seed, n_beam=N_BEAM, n_chan=N_CHAN, n_s=N_S, n_sub=N_SUB):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(n_beam, n_sub * n_s, n_chan), dtype=np.uint8)


def outputs(out):
    return {k: out[k].cpu().numpy() for k in ("evals", "q1", "stat", "flags")}


@pytest.mark.parametrize("n_beam,n_chan,n_s,n_sub,gram", SHAPES)
def test_expired_wait_is_reported_and_the_plan_recovers(n_beam, n_chan, n_s, n_sub, gram):
    import torch
    m = lib()
    d = torch.from_numpy(block(11, n_beam, n_chan, n_s, n_sub)).cuda()
    with m.Plan(n_beam, n_chan, n_s, n_sub) as plan:
        m.mraid_profile_enable(plan.handle)
        ref = outputs(plan.run(d))
        assert gram in m.mraid_profile_read(plan.handle)
        m.mraid_set_wait_limit(plan.handle, 50_000_000)
        for stage in (0, 5):
            m.mraid_inject_fault(plan.handle, m.FAULT_WITHHOLD_STAGE, stage)
            out = plan.run(d, sync=False)
            with pytest.raises(m.MraidError) as e:
                m.mraid_sync(plan.handle)
            assert e.value.status == TIMEOUT, e.value
            assert out["_info"].timed_out == 1
            # the injection is spent: the same plan runs normally again
            again = plan.run(d)
            assert again["info"]["timed_out"] == 0
            got = outputs(again)
            for k in ref:
                assert np.array_equal(got[k], ref[k]), (stage, k)


def test_withheld_stage_with_the_default_limit_is_not_armed_twice():
    """An armed fault that a sync clears does not touch the next launch."""
    import torch
    m = lib()
    d = torch.from_numpy(block(12)).cuda()
    with m.Plan(N_BEAM, N_CHAN, N_S, N_SUB) as plan:
        ref = outputs(plan.run(d))
        m.mraid_inject_fault(plan.handle, m.FAULT_WITHHOLD_STAGE, 2)
        m.mraid_inject_fault(plan.handle, m.FAULT_NONE)
        got = outputs(plan.run(d))
        for k in ref:
            assert np.array_equal(got[k], ref[k]), k
    with pytest.raises(m.MraidError):
        with m.Plan(N_BEAM, N_CHAN, N_S, N_SUB) as plan:
            m.mraid_set_wait_limit(plan.handle, 10)            # below 1 ms: refused
    with pytest.raises(m.MraidError):
        with m.Plan(N_BEAM, N_CHAN, N_S, N_SUB) as plan:
            m.mraid_inject_fault(plan.handle, 7)               # unknown kind


def test_injected_allocation_failure_is_out_of_memory():
    import torch
    m = lib()
    d = torch.from_numpy(block(13)).cuda()
    with m.Plan(N_BEAM, N_CHAN, N_S, N_SUB) as plan:
        ref = outputs(plan.run(d))
    with m.Plan(N_BEAM, N_CHAN, N_S, N_SUB) as plan:           # work buffers not yet made
        m.mraid_inject_fault(plan.handle, m.FAULT_ALLOC)
        with pytest.raises(m.MraidError) as e:
            plan.run(d)
        assert e.value.status == OOM, e.value
        got = outputs(plan.run(d))
        for k in ref:
            assert np.array_equal(got[k], ref[k]), k
