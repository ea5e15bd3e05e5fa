"""Python binding of libmraid (include/mraid.h): argument marshalling only.

Every step of the eigenvalue RFI flagger (mRAID, arXiv 2512.16278: Eq. 1
cross-correlation matrices, Eq. 2 eigendecomposition, Section 3.3 iterative
masking) runs in the CUDA kernels of libmraid.so. PyTorch supplies device
memory and streams. There is no CPU fallback: if the library or a CUDA
device is missing, the calls raise.

The functions mraid_* mirror the C ABI one to one and take raw pointers
(int) or torch tensors; `Plan` is a small convenience wrapper that
allocates the outputs as torch tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

__all__ = [
    "MraidError", "Params", "FlagInfo", "Plan", "load", "library_path",
    "mraid_default_params", "mraid_validate", "mraid_plan", "mraid_ccm", "mraid_eig",
    "mraid_flag", "mraid_run", "mraid_run_host", "mraid_sync", "mraid_query",
    "mraid_destroy", "mraid_status_string", "mraid_last_error", "mraid_abi_version",
    "mraid_profile_enable", "mraid_profile_read", "mraid_profile_reset", "mraid_ccm_noalloc",
    "mraid_batch_plan", "mraid_batch_run", "mraid_batch_sync", "mraid_batch_graph_stats",
    "mraid_batch_packing",
    "mraid_batch_destroy", "UnitIO", "Batch", "mraid_serve_open", "mraid_serve_submit",
    "mraid_serve_poll", "mraid_serve_drain", "mraid_serve_close", "StreamDesc", "BlockResult",
    "Server", "mraid_autotune", "mraid_set_variant", "mraid_set_eig_variant", "tune", "tune_key",
    "mraid_set_wait_limit", "mraid_inject_fault", "FAULT_NONE", "FAULT_WITHHOLD_STAGE",
    "FAULT_ALLOC",
    "mraid_refine", "mraid_multires", "BandpassParams", "mraid_default_bandpass_params",
    "mraid_arpls", "mraid_run_bandpass", "mraid_ccm_pol2", "mraid_run_pol2", "STATUS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))

STATUS = {0: "MRAID_OK", 1: "MRAID_ERR_INVALID_ARG", 2: "MRAID_ERR_UNSUPPORTED",
          3: "MRAID_ERR_OOM", 4: "MRAID_ERR_CUDA", 5: "MRAID_ERR_TIMEOUT",
          6: "MRAID_ERR_NOT_READY"}


class MraidError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


class BandpassParams(ctypes.Structure):
    """mraid_bandpass_params (Section 3.1 ArPLS bandpass; lam, ratio and
    itermax as Section 4.5 names them; interval in sub-integrations)."""
    _fields_ = [("lam", ctypes.c_double), ("ratio", ctypes.c_double),
                ("itermax", ctypes.c_int32), ("interval", ctypes.c_int32)]


class Params(ctypes.Structure):
    """mraid_params (Section 3.2 problem statement, Section 4.5 thresholds)."""
    _fields_ = [
        ("n_beam", ctypes.c_int32), ("n_chan", ctypes.c_int32),
        ("n_samp_sub", ctypes.c_int32), ("n_sub", ctypes.c_int32),
        ("bit_depth", ctypes.c_int32), ("beam_stride", ctypes.c_int64),
        ("eig_k", ctypes.c_double), ("vec_t", ctypes.c_double),
        ("max_clip_iter", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("keep", ctypes.c_void_p),
    ]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class FlagInfo(ctypes.Structure):
    """mraid_flag_info: result of the Section 3.3 masking."""
    _fields_ = [
        ("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("thresh", ctypes.c_double),
        ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
        ("n_flagged", ctypes.c_int64), ("n_used", ctypes.c_int64),
        ("n_near", ctypes.c_int64), ("n_degenerate", ctypes.c_int64),
        ("jacobi_sweeps", ctypes.c_int64), ("jacobi_warp_sweeps", ctypes.c_int64),
        ("timed_out", ctypes.c_int32), ("q1_refined", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class UnitIO(ctypes.Structure):
    """mraid_unit_io: one unit's device buffers in the batched form."""
    _fields_ = [("d_data", ctypes.c_void_p), ("d_evals", ctypes.c_void_p),
                ("d_q1", ctypes.c_void_p), ("d_stat", ctypes.c_void_p),
                ("d_flags", ctypes.c_void_p)]


class StreamDesc(ctypes.Structure):
    """mraid_stream_desc: one observation of the served form."""
    _fields_ = [("params", Params), ("block_samples", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class BlockResult(ctypes.Structure):
    """mraid_block_result: one finished block of the served form."""
    _fields_ = [("stream", ctypes.c_int32), ("n_sub", ctypes.c_int32), ("seq", ctypes.c_int64),
                ("n_cells", ctypes.c_int64), ("n_flagged", ctypes.c_int64),
                ("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("thresh", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


def library_path() -> str:
    return os.path.join(_HERE, "libmraid.so")


_lib = None
_P = ctypes.c_void_p


def load():
    """Load libmraid.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -m paper_2512_16278_gb300.build` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    i32, vp = ctypes.c_int32, ctypes.c_void_p
    sig = {
        "mraid_default_params": (None, [ctypes.POINTER(Params), i32, i32, i32, i32]),
        "mraid_validate": (ctypes.c_int, [ctypes.POINTER(Params)]),
        "mraid_plan": (ctypes.c_int, [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]),
        "mraid_ccm": (ctypes.c_int, [vp, vp, vp, vp]),
        "mraid_eig": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "mraid_flag": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(FlagInfo)]),
        "mraid_run": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.POINTER(FlagInfo)]),
        "mraid_run_host": (ctypes.c_int, [vp, vp, vp, vp, ctypes.POINTER(FlagInfo)]),
        "mraid_sync": (ctypes.c_int, [vp]),
        "mraid_query": (ctypes.c_int, [vp]),
        "mraid_destroy": (None, [vp]),
        "mraid_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "mraid_last_error": (ctypes.c_char_p, []),
        "mraid_abi_version": (ctypes.c_int32, []),
        "mraid_profile_enable": (ctypes.c_int, [vp, i32]),
        "mraid_profile_read": (ctypes.c_int, [vp, ctypes.POINTER(KernelTime), i32,
                                              ctypes.POINTER(i32)]),
        "mraid_profile_reset": (ctypes.c_int, [vp]),
        "mraid_ccm_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), vp, i32, i32, vp, vp]),
        "mraid_batch_plan": (ctypes.c_int, [ctypes.POINTER(Params), i32, vp, ctypes.POINTER(vp)]),
        "mraid_batch_run": (ctypes.c_int, [vp, ctypes.POINTER(UnitIO), ctypes.POINTER(FlagInfo)]),
        "mraid_batch_sync": (ctypes.c_int, [vp]),
        "mraid_batch_graph_stats": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "mraid_batch_packing": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_float)]),
        "mraid_batch_destroy": (None, [vp]),
        "mraid_serve_open": (ctypes.c_int, [ctypes.POINTER(StreamDesc), i32, ctypes.c_int64, i32,
                                            ctypes.POINTER(vp)]),
        "mraid_serve_submit": (ctypes.c_int, [vp, i32, vp, vp, ctypes.c_int64]),
        "mraid_serve_poll": (ctypes.c_int, [vp, ctypes.POINTER(BlockResult), i32,
                                            ctypes.POINTER(i32)]),
        "mraid_serve_drain": (ctypes.c_int, [vp, i32]),
        "mraid_serve_close": (None, [vp]),
        "mraid_autotune": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                          ctypes.c_char_p, i32]),
        "mraid_set_variant": (ctypes.c_int, [vp, i32]),
        "mraid_set_eig_variant": (ctypes.c_int, [vp, i32]),
        "mraid_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_int64]),
        "mraid_inject_fault": (ctypes.c_int, [vp, i32, ctypes.c_int64]),
        "mraid_refine": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "mraid_multires": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(vp),
                                          ctypes.POINTER(vp), ctypes.POINTER(FlagInfo)]),
        "mraid_default_bandpass_params": (None, [ctypes.POINTER(BandpassParams)]),
        "mraid_ccm_pol2": (ctypes.c_int, [vp, vp, vp, vp]),
        "mraid_run_pol2": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.POINTER(FlagInfo)]),
        "mraid_arpls": (ctypes.c_int, [vp, vp, i32, i32, ctypes.POINTER(BandpassParams), vp, vp]),
        "mraid_run_bandpass": (ctypes.c_int, [vp, vp, ctypes.POINTER(BandpassParams), vp, vp, vp,
                                              vp, vp, ctypes.POINTER(FlagInfo)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> Optional[int]:
    """Device/host address of a torch tensor, an int, or None. The C ABI
    takes dense row-major buffers, so a tensor with other strides is an
    error rather than a silently misread buffer."""
    if x is None:
        return None
    if isinstance(x, int):
        # 0 is NULL; no buffer lives elsewhere in the first 64 KiB of the
        # address space: a small count passed by mistake would otherwise
        # reach a kernel as a pointer
        if x == 0:
            return None
        if 0 < x < (1 << 16):
            raise ValueError(f"{x} is not a buffer address")
        return x
    if not x.is_contiguous():
        raise ValueError("mraid buffers must be contiguous (row-major) tensors")
    return x.data_ptr()


def _check(status: int, where: str):
    if status != 0:
        raise MraidError(status, where, mraid_last_error())


# ---------------------------------------------------------------- raw ABI

def mraid_default_params(n_beam: int, n_chan: int, n_samp_sub: int, n_sub: int) -> Params:
    p = Params()
    load().mraid_default_params(ctypes.byref(p), n_beam, n_chan, n_samp_sub, n_sub)
    return p


def mraid_validate(p: Params) -> int:
    return load().mraid_validate(ctypes.byref(p))


def mraid_plan(p: Params, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().mraid_plan(ctypes.byref(p), stream or None, ctypes.byref(out)), "mraid_plan")
    return out.value


def mraid_ccm(plan: int, d_data, d_sums=None, d_corr=None):
    _check(load().mraid_ccm(plan, _ptr(d_data), _ptr(d_sums), _ptr(d_corr)), "mraid_ccm")


def mraid_ccm_noalloc(p: Params, d_data, sub0: int, n_sub: int, d_corr, stream: int = 0):
    """Correlations of sub-integrations [sub0, sub0+n_sub) without any
    allocation: the library's fixed 8 MiB device array holds the Gram sums.
    For callers that cannot call cudaMalloc; calls must not overlap on the
    GPU (they share that array)."""
    _check(load().mraid_ccm_noalloc(ctypes.byref(p), _ptr(d_data), sub0, n_sub, _ptr(d_corr),
                                    stream or None), "mraid_ccm_noalloc")


def mraid_eig(plan: int, d_corr, d_evals=None, d_q1=None, d_stat=None):
    _check(load().mraid_eig(plan, _ptr(d_corr), _ptr(d_evals), _ptr(d_q1), _ptr(d_stat)),
           "mraid_eig")


def mraid_flag(plan: int, d_stat, d_flags, info: Optional[FlagInfo] = None):
    _check(load().mraid_flag(plan, _ptr(d_stat), _ptr(d_flags),
                             ctypes.byref(info) if info is not None else None), "mraid_flag")


def mraid_run(plan: int, d_data, d_evals, d_q1, d_stat, d_flags,
              info: Optional[FlagInfo] = None):
    _check(load().mraid_run(plan, _ptr(d_data), _ptr(d_evals), _ptr(d_q1), _ptr(d_stat),
                            _ptr(d_flags), ctypes.byref(info) if info is not None else None),
           "mraid_run")


def mraid_run_host(plan: int, h_data, h_stat, h_flags, info: Optional[FlagInfo] = None):
    _check(load().mraid_run_host(plan, _ptr(h_data), _ptr(h_stat), _ptr(h_flags),
                                 ctypes.byref(info) if info is not None else None),
           "mraid_run_host")


def mraid_multires(plan: int, d_data, factors, d_stats, d_flags, infos=None):
    """Several timescales in one pass: level i uses sub-intervals of
    factors[i] sub-integrations; d_stats[i] / d_flags[i] hold its
    (n_sub // factors[i]) * n_chan cells. infos, if given, is a ctypes array
    of len(factors) FlagInfo filled at mraid_sync (keep it alive until then)."""
    n = len(factors)
    if len(d_stats) != n or len(d_flags) != n or (infos is not None and len(infos) != n):
        raise ValueError("one stat, flag (and info) buffer per factor")
    f = (ctypes.c_int32 * n)(*factors)
    st = (ctypes.c_void_p * n)(*[_ptr(x) for x in d_stats])
    fl = (ctypes.c_void_p * n)(*[_ptr(x) for x in d_flags])
    _check(load().mraid_multires(plan, _ptr(d_data), n, f, st, fl, infos), "mraid_multires")


def mraid_default_bandpass_params(**kw) -> BandpassParams:
    bp = BandpassParams()
    load().mraid_default_bandpass_params(ctypes.byref(bp))
    for k, v in kw.items():
        setattr(bp, k, v)
    return bp


def mraid_arpls(plan: int, d_y, n_sys: int, n: int, bp: BandpassParams, d_z, d_iters=None):
    _check(load().mraid_arpls(plan, _ptr(d_y), n_sys, n, ctypes.byref(bp), _ptr(d_z),
                              _ptr(d_iters)), "mraid_arpls")


def mraid_run_bandpass(plan: int, d_data, bp: BandpassParams, d_bandpass, d_evals, d_q1, d_stat,
                       d_flags, info: Optional[FlagInfo] = None):
    _check(load().mraid_run_bandpass(plan, _ptr(d_data), ctypes.byref(bp), _ptr(d_bandpass),
                                     _ptr(d_evals), _ptr(d_q1), _ptr(d_stat), _ptr(d_flags),
                                     ctypes.byref(info) if info is not None else None),
           "mraid_run_bandpass")


def mraid_ccm_pol2(plan: int, d_data, d_sums=None, d_corr=None):
    _check(load().mraid_ccm_pol2(plan, _ptr(d_data), _ptr(d_sums), _ptr(d_corr)),
           "mraid_ccm_pol2")


def mraid_run_pol2(plan: int, d_data, d_evals, d_q1, d_stat, d_flags,
                   info: Optional[FlagInfo] = None):
    _check(load().mraid_run_pol2(plan, _ptr(d_data), _ptr(d_evals), _ptr(d_q1), _ptr(d_stat),
                                 _ptr(d_flags), ctypes.byref(info) if info is not None else None),
           "mraid_run_pol2")


def mraid_sync(plan: int):
    _check(load().mraid_sync(plan), "mraid_sync")


def mraid_query(plan: int) -> int:
    return load().mraid_query(plan)


def mraid_destroy(plan: int):
    load().mraid_destroy(plan)


def mraid_status_string(s: int) -> str:
    return load().mraid_status_string(s).decode()


def mraid_last_error() -> str:
    return load().mraid_last_error().decode()


def mraid_abi_version() -> int:
    return load().mraid_abi_version()


def mraid_profile_enable(plan: int, enable: bool = True):
    _check(load().mraid_profile_enable(plan, 1 if enable else 0), "mraid_profile_enable")


def mraid_profile_read(plan: int) -> dict:
    """{kernel name: (launches, total ms)} folded at the last mraid_sync."""
    arr = (KernelTime * 16)()
    n = ctypes.c_int32(0)
    _check(load().mraid_profile_read(plan, arr, 16, ctypes.byref(n)), "mraid_profile_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(n.value, 16))}


def mraid_profile_reset(plan: int):
    _check(load().mraid_profile_reset(plan), "mraid_profile_reset")


def mraid_batch_plan(params, stream: int = 0) -> int:
    arr = (Params * len(params))(*params)
    out = ctypes.c_void_p()
    _check(load().mraid_batch_plan(arr, len(params), stream or None, ctypes.byref(out)),
           "mraid_batch_plan")
    return out.value


def mraid_batch_run(batch: int, ios, infos=None):
    arr = (UnitIO * len(ios))(*ios)
    _check(load().mraid_batch_run(batch, arr, infos), "mraid_batch_run")


def mraid_batch_sync(batch: int):
    _check(load().mraid_batch_sync(batch), "mraid_batch_sync")


def mraid_batch_graph_stats(batch: int):
    a, b = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().mraid_batch_graph_stats(batch, ctypes.byref(a), ctypes.byref(b)),
           "mraid_batch_graph_stats")
    return a.value, b.value


def mraid_batch_packing(batch: int):
    """(packing, ms concurrent, ms chained): 0 = concurrent branches,
    1 = chained, -1 before the first run."""
    p = ctypes.c_int32(0)
    a, b = ctypes.c_float(0), ctypes.c_float(0)
    _check(load().mraid_batch_packing(batch, ctypes.byref(p), ctypes.byref(a), ctypes.byref(b)),
           "mraid_batch_packing")
    return p.value, a.value, b.value


def mraid_batch_destroy(batch: int):
    load().mraid_batch_destroy(batch)


def mraid_serve_open(descs, hbm_budget: int = 0, max_inflight: int = 8) -> int:
    arr = (StreamDesc * len(descs))(*descs)
    out = ctypes.c_void_p()
    _check(load().mraid_serve_open(arr, len(descs), hbm_budget, max_inflight, ctypes.byref(out)),
           "mraid_serve_open")
    return out.value


def mraid_serve_submit(srv: int, stream: int, h_block, h_flags, seq: int):
    _check(load().mraid_serve_submit(srv, stream, _ptr(h_block), _ptr(h_flags), seq),
           "mraid_serve_submit")


def mraid_serve_poll(srv: int, max_results: int = 256):
    arr = (BlockResult * max_results)()
    n = ctypes.c_int32(0)
    _check(load().mraid_serve_poll(srv, arr, max_results, ctypes.byref(n)), "mraid_serve_poll")
    return [arr[i].as_dict() for i in range(n.value)]


def mraid_serve_drain(srv: int, timeout_ms: int = 60000):
    _check(load().mraid_serve_drain(srv, timeout_ms), "mraid_serve_drain")


def mraid_serve_close(srv: int):
    load().mraid_serve_close(srv)


def mraid_autotune(plan: int, d_data, reps: int = 3):
    """((gram variant, jacobi variant), {"g<id>" / "e<id>": ms}) for the plan."""
    g, e = ctypes.c_int32(0), ctypes.c_int32(0)
    buf = ctypes.create_string_buffer(512)
    _check(load().mraid_autotune(plan, _ptr(d_data), reps, ctypes.byref(g), ctypes.byref(e),
                                 buf, 512), "mraid_autotune")
    times = {}
    for item in buf.value.decode().split(";"):
        if item:
            k, v = item.split(":")
            times[k] = float(v)
    return (g.value, e.value), times


def mraid_refine(plan: int, d_q1, d_flags, d_beam_bits, d_mu_sigma=None):
    _check(load().mraid_refine(plan, _ptr(d_q1), _ptr(d_flags), _ptr(d_beam_bits),
                               _ptr(d_mu_sigma)), "mraid_refine")


def mraid_set_variant(plan: int, variant: int):
    _check(load().mraid_set_variant(plan, variant), "mraid_set_variant")


def mraid_set_eig_variant(plan: int, variant: int):
    _check(load().mraid_set_eig_variant(plan, variant), "mraid_set_eig_variant")


FAULT_NONE, FAULT_WITHHOLD_STAGE, FAULT_ALLOC = 0, 1, 2


def mraid_set_wait_limit(plan: int, ns: int):
    """Bound (ns) of every wait inside the tensor-core kernels."""
    _check(load().mraid_set_wait_limit(plan, int(ns)), "mraid_set_wait_limit")


def mraid_inject_fault(plan: int, kind: int, arg: int = 0):
    """Arm a host-side fault for the next launch or allocation (tests of the
    failure paths; cleared by the next mraid_sync)."""
    _check(load().mraid_inject_fault(plan, kind, int(arg)), "mraid_inject_fault")


def tune_key(n_beam: int, n_chan: int, n_samp_sub: int, bit_depth: int = 8) -> str:
    """Key of a shape in the tuning cache: the variants of 8-bit and float32
    plans differ, so the sample type is part of it."""
    if bit_depth not in (8, 32):
        raise ValueError(f"bit_depth {bit_depth}: 8 or 32")
    return f"{n_beam},{n_chan},{n_samp_sub},{'u8' if bit_depth == 8 else 'f32'}"


def tune(plan: int, d_data, n_beam: int, n_chan: int, n_samp_sub: int,
         cache_path: Optional[str] = None, reps: int = 3, bit_depth: int = 8):
    """Pick the Gram and eigensolver variants for this shape: from the JSON
    tuning cache (keyed by beams, channels, samples per sub-integration and
    sample type, which must be the plan's bit_depth) if it holds the shape,
    else by mraid_autotune, recording the result.
    Returns (gram variant, eigensolver variant)."""
    import json
    key = tune_key(n_beam, n_chan, n_samp_sub, bit_depth)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        g, e = int(cache[key]["gram"]), int(cache[key]["jacobi"])
        mraid_set_variant(plan, g)
        mraid_set_eig_variant(plan, e)
        return g, e
    (g, e), times = mraid_autotune(plan, d_data, reps)
    if cache_path:
        cache[key] = {"gram": g, "jacobi": e, "ms": times}
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return g, e


# ------------------------------------------------------------ convenience

class Plan:
    """A plan bound to the current CUDA device and a torch stream; outputs
    are torch tensors on that device."""

    def __init__(self, n_beam: int, n_chan: int, n_samp_sub: int, n_sub: int, *,
                 eig_k: float = 3.0, vec_t: float = 1.0, max_clip_iter: int = 64,
                 keep=None, beam_stride: int = 0, stream=None, bit_depth: int = 8):
        import numpy as np
        import torch
        self.torch = torch
        self.p = mraid_default_params(n_beam, n_chan, n_samp_sub, n_sub)
        self.p.eig_k = eig_k
        self.p.vec_t = vec_t
        self.p.max_clip_iter = max_clip_iter
        self.p.beam_stride = beam_stride
        self.p.bit_depth = bit_depth
        self._keep = None
        if keep is not None:
            self._keep = np.ascontiguousarray(np.asarray(keep, dtype=np.uint8))
            if self._keep.shape != (n_chan,):
                raise ValueError("keep must have n_chan entries")
            self.p.keep = self._keep.ctypes.data
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle = mraid_plan(self.p, self.stream.cuda_stream)
        self.n_beam, self.n_chan, self.n_sub = n_beam, n_chan, n_sub
        self.n_cells = n_chan * n_sub

    def close(self):
        if getattr(self, "handle", None):
            mraid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _empty(self, *shape, dtype):
        return self.torch.empty(*shape, dtype=dtype, device=self.device)

    def ccm(self, data, sums: bool = True, corr: bool = True):
        N = self.n_beam
        s = self._empty(self.n_cells, (N + 1) * (N + 2) // 2, dtype=self.torch.int64) if sums else None
        c = self._empty(self.n_cells, N * (N + 1) // 2, dtype=self.torch.float32) if corr else None
        mraid_ccm(self.handle, data, s, c)
        return s, c

    def eig(self, corr, evals: bool = True, q1: bool = True):
        N = self.n_beam
        e = self._empty(self.n_cells, N, dtype=self.torch.float32) if evals else None
        q = self._empty(self.n_cells, N, dtype=self.torch.float32) if q1 else None
        st = self._empty(self.n_cells, dtype=self.torch.float32)
        mraid_eig(self.handle, corr, e, q, st)
        return e, q, st

    def flag(self, stat):
        f = self._empty(self.n_cells, dtype=self.torch.uint8)
        info = FlagInfo()
        mraid_flag(self.handle, stat, f, info)
        mraid_sync(self.handle)
        return f, info.as_dict()

    def run(self, data, evals: bool = True, q1: bool = True, sync: bool = True):
        N = self.n_beam
        out = {
            "evals": self._empty(self.n_cells, N, dtype=self.torch.float32) if evals else None,
            "q1": self._empty(self.n_cells, N, dtype=self.torch.float32) if q1 else None,
            "stat": self._empty(self.n_cells, dtype=self.torch.float32),
            "flags": self._empty(self.n_cells, dtype=self.torch.uint8),
        }
        info = FlagInfo()
        mraid_run(self.handle, data, out["evals"], out["q1"], out["stat"], out["flags"], info)
        out["_info"] = info
        if sync:
            mraid_sync(self.handle)
            out["info"] = info.as_dict()
        return out

    def refine(self, q1, flags):
        """(beam bits uint32 [cell][ceil(N/32)], (mu, sigma) [N][2]) of the
        eigenvector refinement."""
        t = self.torch
        W = (self.n_beam + 31) // 32
        bits = t.empty(self.n_cells, W, dtype=t.int32, device=self.device)
        ms = t.empty(self.n_beam, 2, dtype=t.float64, device=self.device)
        mraid_refine(self.handle, q1, flags, bits, ms)
        mraid_sync(self.handle)
        return bits, ms

    def run_host(self, h_data, h_stat=None, h_flags=None):
        """Whole path from a host block (pinned torch tensor or address)."""
        torch = self.torch
        if h_flags is None:
            h_flags = torch.empty(self.n_cells, dtype=torch.uint8, pin_memory=True)
        info = FlagInfo()
        mraid_run_host(self.handle, h_data, h_stat, h_flags, info)
        mraid_sync(self.handle)
        return h_flags, info.as_dict()

    def multires(self, data, factors):
        """Stat, flags and masking report per timescale: one dict per factor
        (sub-intervals of `factor` sub-integrations), in the given order."""
        t = self.torch
        stats = [self._empty((self.n_sub // f) * self.n_chan, dtype=t.float32) for f in factors]
        flags = [self._empty((self.n_sub // f) * self.n_chan, dtype=t.uint8) for f in factors]
        infos = (FlagInfo * len(factors))()
        mraid_multires(self.handle, data, list(factors), stats, flags, infos)
        mraid_sync(self.handle)
        return [{"factor": f, "stat": stats[i], "flags": flags[i], "info": infos[i].as_dict()}
                for i, f in enumerate(factors)]

    def ccm_pol2(self, data, sums: bool = True, corr: bool = True):
        """Gram sums / correlation of the total power of a two-polarisation
        block (2N blocks, polarisation-major)."""
        N = self.n_beam
        s = self._empty(self.n_cells, (N + 1) * (N + 2) // 2, dtype=self.torch.int64) if sums else None
        c = self._empty(self.n_cells, N * (N + 1) // 2, dtype=self.torch.float32) if corr else None
        mraid_ccm_pol2(self.handle, data, s, c)
        return s, c

    def run_pol2(self, data, evals: bool = True, q1: bool = True):
        """Whole path on the total power of a two-polarisation block."""
        N = self.n_beam
        t = self.torch
        out = {
            "evals": self._empty(self.n_cells, N, dtype=t.float32) if evals else None,
            "q1": self._empty(self.n_cells, N, dtype=t.float32) if q1 else None,
            "stat": self._empty(self.n_cells, dtype=t.float32),
            "flags": self._empty(self.n_cells, dtype=t.uint8),
        }
        info = FlagInfo()
        mraid_run_pol2(self.handle, data, out["evals"], out["q1"], out["stat"], out["flags"], info)
        mraid_sync(self.handle)
        out["info"] = info.as_dict()
        return out

    def arpls(self, y, **kw):
        """(z, solves) of the ArPLS baselines of the rows of y (float64
        [n_sys][n] on the device); keywords override lam, ratio, itermax."""
        t = self.torch
        bp = mraid_default_bandpass_params(**kw)
        z = t.empty_like(y)
        it = t.empty(y.shape[0], dtype=t.int32, device=self.device)
        mraid_arpls(self.handle, y, y.shape[0], y.shape[1], bp, z, it)
        mraid_sync(self.handle)
        return z, it

    def run_bandpass(self, data, evals: bool = True, q1: bool = False, **kw):
        """Whole path under the bandpass-centred reading; keywords override
        lam, ratio, itermax, interval."""
        t = self.torch
        bp = mraid_default_bandpass_params(**kw)
        n_int = (self.n_sub + bp.interval - 1) // bp.interval
        N = self.n_beam
        out = {
            "bandpass": self._empty(n_int, N, self.n_chan, dtype=t.float32),
            "evals": self._empty(self.n_cells, N, dtype=t.float32) if evals else None,
            "q1": self._empty(self.n_cells, N, dtype=t.float32) if q1 else None,
            "stat": self._empty(self.n_cells, dtype=t.float32),
            "flags": self._empty(self.n_cells, dtype=t.uint8),
        }
        info = FlagInfo()
        mraid_run_bandpass(self.handle, data, bp, out["bandpass"], out["evals"], out["q1"],
                           out["stat"], out["flags"], info)
        mraid_sync(self.handle)
        out["info"] = info.as_dict()
        return out

    def sync(self):
        mraid_sync(self.handle)


class Batch:
    """Batched form over units of uneven shapes (mraid_batch_*); outputs are
    torch tensors, one set per unit."""

    def __init__(self, shapes, stream=None, eig_k: float = 3.0, max_clip_iter: int = 64):
        import torch
        self.torch = torch
        self.params = []
        for (n_beam, n_chan, n_samp_sub, n_sub) in shapes:
            p = mraid_default_params(n_beam, n_chan, n_samp_sub, n_sub)
            p.eig_k = eig_k
            p.max_clip_iter = max_clip_iter
            self.params.append(p)
        self.shapes = list(shapes)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = mraid_batch_plan(self.params, self.stream.cuda_stream)

    def outputs(self):
        t = self.torch
        outs = []
        for (n_beam, n_chan, _, n_sub) in self.shapes:
            cells = n_chan * n_sub
            outs.append({
                "evals": t.empty(cells, n_beam, dtype=t.float32, device="cuda"),
                "q1": t.empty(cells, n_beam, dtype=t.float32, device="cuda"),
                "stat": t.empty(cells, dtype=t.float32, device="cuda"),
                "flags": t.empty(cells, dtype=t.uint8, device="cuda"),
            })
        return outs

    def run(self, datas, outs=None, sync: bool = True):
        outs = outs if outs is not None else self.outputs()
        ios = [UnitIO(_ptr(d), _ptr(o["evals"]), _ptr(o["q1"]), _ptr(o["stat"]), _ptr(o["flags"]))
               for d, o in zip(datas, outs)]
        infos = (FlagInfo * len(ios))()
        mraid_batch_run(self.handle, ios, infos)
        if sync:
            mraid_batch_sync(self.handle)
            for o, i in zip(outs, infos):
                o["info"] = i.as_dict()
        else:
            self._infos = infos
        return outs

    def graph_stats(self):
        return mraid_batch_graph_stats(self.handle)

    def packing(self):
        return mraid_batch_packing(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            mraid_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Served form (mraid_serve_*): streams = [(n_beam, n_chan, n_samp_sub,
    block_samples), ...]."""

    def __init__(self, streams, hbm_budget: int = 0, max_inflight: int = 8, eig_k: float = 3.0):
        self.descs = []
        for (n_beam, n_chan, n_samp_sub, block_samples) in streams:
            p = mraid_default_params(n_beam, n_chan, n_samp_sub, 1)
            p.eig_k = eig_k
            self.descs.append(StreamDesc(p, block_samples, 0))
        self.streams = list(streams)
        self.handle = mraid_serve_open(self.descs, hbm_budget, max_inflight)

    def flags_bytes(self, stream: int) -> int:
        n_beam, n_chan, n_s, block = self.streams[stream]
        return ((block + n_s) // n_s + 1) * n_chan

    def submit(self, stream: int, h_block, h_flags, seq: int):
        mraid_serve_submit(self.handle, stream, h_block, h_flags, seq)

    def poll(self, max_results: int = 256):
        return mraid_serve_poll(self.handle, max_results)

    def drain(self, timeout_ms: int = 60000):
        mraid_serve_drain(self.handle, timeout_ms)

    def close(self):
        if getattr(self, "handle", None):
            mraid_serve_close(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
