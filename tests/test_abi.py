"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/mraid.h declares, validates parameters on the host,
and refuses to run without a CUDA device (there is no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_16278_gb300 import build
    build.build()
    import paper_2512_16278_gb300 as m
    return m.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(mraid_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "mraid_run" in names and "mraid_plan" in names
    for n in names:
        assert hasattr(lib, n), n


def test_abi_version_and_status_strings(lib):
    import paper_2512_16278_gb300 as m
    assert m.mraid_abi_version() == 2
    for s, name in m.STATUS.items():
        assert m.mraid_status_string(s)
    assert m.mraid_status_string(999) == "unknown status"


def test_default_params_follow_the_paper(lib):
    import paper_2512_16278_gb300 as m
    p = m.mraid_default_params(19, 4096, 1024, 200)
    assert (p.n_beam, p.n_chan, p.n_samp_sub, p.n_sub) == (19, 4096, 1024, 200)
    assert p.eig_k == 3.0 and p.vec_t == 1.0          # Section 4.5
    assert p.bit_depth == 8 and p.beam_stride == 0 and p.max_clip_iter == 64
    assert m.mraid_validate(p) == 0


@pytest.mark.parametrize("field,value,status", [
    ("n_beam", 1, 1), ("n_beam", 129, 2), ("n_chan", 0, 1), ("n_sub", 0, 1),
    ("n_samp_sub", 1, 1), ("n_samp_sub", (1 << 20) + 1, 1), ("bit_depth", 16, 2),
    ("eig_k", 0.0, 1), ("eig_k", float("nan"), 1), ("vec_t", -1.0, 1),
    ("max_clip_iter", 0, 1), ("max_clip_iter", 1001, 1), ("beam_stride", 5, 1),
    ("reserved", 3, 1),
])
def test_validate_rejects(lib, field, value, status):
    import paper_2512_16278_gb300 as m
    p = m.mraid_default_params(19, 64, 128, 256)
    setattr(p, field, value)
    assert m.mraid_validate(p) == status
    assert m.mraid_last_error()


def test_validate_null(lib):
    assert lib.mraid_validate(None) == 1


def test_plan_without_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2512_16278_gb300 as m
    p = m.mraid_default_params(19, 64, 128, 256)
    out = ctypes.c_void_p()
    st = lib.mraid_plan(ctypes.byref(p), None, ctypes.byref(out))
    assert st == 4 and not out.value          # MRAID_ERR_CUDA, no plan
    assert m.mraid_last_error()


def test_null_plan_calls_are_rejected(lib):
    assert lib.mraid_ccm(None, None, None, None) == 1
    assert lib.mraid_sync(None) == 1
    lib.mraid_destroy(None)                    # no-op


def test_binding_rejects_non_contiguous_buffers():
    """A strided view would be read as if it were dense: refuse it."""
    import torch
    import paper_2512_16278_gb300 as m
    t = torch.zeros(6, 4)
    assert m._ptr(t) == t.data_ptr()
    assert m._ptr(None) is None and m._ptr(0x3abdac00) == 0x3abdac00
    with pytest.raises(ValueError):
        m._ptr(t.t())
    # a small integer (a count passed where a buffer belongs) is no address
    with pytest.raises(ValueError):
        m._ptr(4096)


def test_tuning_cache_key_separates_sample_types():
    import paper_2512_16278_gb300 as m
    assert m.tune_key(19, 4096, 1024) == "19,4096,1024,u8"
    assert m.tune_key(19, 4096, 1024, 32) == "19,4096,1024,f32"
    assert m.tune_key(19, 4096, 1024, 8) != m.tune_key(19, 4096, 1024, 32)
    with pytest.raises(ValueError):
        m.tune_key(19, 4096, 1024, 16)


def test_validate_rejects_too_many_cells_before_any_size_product(lib):
    """2^30 sub-integrations x 2^30 channels of 2^20 samples: the cell count
    is refused first, so no 64-bit block size is ever formed from it."""
    import paper_2512_16278_gb300 as m
    p = m.mraid_default_params(19, 1 << 30, 1 << 20, 1 << 30)
    p.beam_stride = 1
    assert m.mraid_validate(p) == 1
    assert "cells" in m.mraid_last_error()
