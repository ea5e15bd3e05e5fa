"""The values the paper prints (tests/golden/paper_values.txt, each with its
section) against the library's and the oracle's defaults, the synthetic
stand-in for the FAST observation, and the sub-interval lengths of the
multi-timescale pass (CPU only; the library is loaded but runs no kernel)."""
import inspect
import os

import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_values():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.split(";")[0].strip()
            if not line or line.startswith("#"):
                continue
            key, rhs = (s.strip() for s in line.split("=", 1))
            nums = [float(x) for x in rhs.split()]
            vals[key] = nums if len(nums) > 1 else nums[0]
    return vals


P = paper_values()


@pytest.fixture(scope="module")
def lib():
    from paper_2512_16278_gb300 import build
    build.build()
    import paper_2512_16278_gb300 as m
    return m.load()


def test_fixture_is_complete_and_self_consistent():
    for k in ("n_beam", "t_samp_us", "n_samp_sub", "n_chan", "bit_depth", "n_pol", "n_sub_file",
              "n_time_file", "eig_k", "vec_t", "timescales_s"):
        assert k in P, k
    # Sec. 2's sub-integrations of Sec. 2's length are Sec. 4.4's time samples
    assert P["n_sub_file"] * P["n_samp_sub"] == P["n_time_file"]


def test_library_defaults_are_the_papers(lib):
    import paper_2512_16278_gb300 as m
    p = m.mraid_default_params(int(P["n_beam"]), int(P["n_chan"]), int(P["n_samp_sub"]), 1)
    assert p.eig_k == P["eig_k"]
    assert p.vec_t == P["vec_t"]
    assert p.bit_depth == P["bit_depth"]


def test_oracle_defaults_are_the_papers():
    assert inspect.signature(oracle.flag).parameters["k_sigma"].default == P["eig_k"]
    assert inspect.signature(oracle.beam_flags).parameters["t"].default == P["vec_t"]


def test_fast_stand_in_has_the_observations_shape():
    cfg = synth.FAST_BLOCK
    assert (cfg.n_beam, cfg.n_chan, cfg.n_samp_sub) == (P["n_beam"], P["n_chan"], P["n_samp_sub"])
    assert cfg.n_sub <= P["n_sub_file"]
    # the block is Table 1's longest time resolution (10 s) to within 1 %
    block_s = cfg.n_sub * cfg.n_samp_sub * P["t_samp_us"] * 1e-6
    assert abs(block_s - P["timescales_s"][-1]) <= 0.01 * P["timescales_s"][-1]


def test_table1_time_resolutions_are_whole_sub_integrations():
    """Table 1's time resolutions are nominal multiples of its first entry,
    0.05 s, which is one sub-integration (1024 samples at 49.152 us =
    50.3 ms, rounded). The multi-timescale pass is measured with those
    multiples, each within 1 % of its time at the exact sub-integration
    length, and every level is a multiple of a shorter one, so it is
    formed from that level's sums."""
    import bench
    sub_s = P["n_samp_sub"] * P["t_samp_us"] * 1e-6
    T = P["timescales_s"]
    assert abs(sub_s - T[0]) <= 0.01 * T[0]
    factors = [round(t / T[0]) for t in T]
    assert tuple(factors) == tuple(bench.MULTIRES_FACTORS)
    for t, f in zip(T, factors):
        assert abs(f * sub_s - t) <= 0.01 * t, (t, f)
    for i, f in enumerate(factors[1:], 1):
        assert any(f % g == 0 for g in factors[:i]), f
