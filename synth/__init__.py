"""Seeded synthetic multi-beam filterbank data (ctypes wrapper of synth.c).

The generator draws noise and injects RFI; it contains none of the RFI
method's arithmetic, so both the CPU oracle and the CUDA path may take their
inputs from it. Layout of every block: uint8 [beam][time][chan].

Workload shapes follow the paper's data (Section 2: FAST 19-beam receiver,
49.152 us sampling, 4096 channels, 8-bit, 1024 samples per sub-integration)
and the PAF-like receivers named in Section 5.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libmraid_synth.so")


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("n_beam", ctypes.c_int32),
        ("n_chan", ctypes.c_int32),
        ("n_samp_sub", ctypes.c_int32),
        ("n_sub", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("mean_dn", ctypes.c_int32),
        ("sigma_dn", ctypes.c_int32),
        ("bandpass", ctypes.c_int32),
        ("n_narrow", ctypes.c_int32),
        ("narrow_amp_dn", ctypes.c_int32),
        ("n_burst", ctypes.c_int32),
        ("burst_amp_dn", ctypes.c_int32),
        ("n_spike", ctypes.c_int32),
        ("spike_amp_dn", ctypes.c_int32),
    ]


class _Narrow(ctypes.Structure):
    _fields_ = [("chan", ctypes.c_int32), ("phase", ctypes.c_int32)]


class _Burst(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int64), ("sub", ctypes.c_int32)]


class _Spike(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("chan", ctypes.c_int32),
                ("sub", ctypes.c_int32), ("off", ctypes.c_int32)]


@dataclasses.dataclass(frozen=True)
class SynthConfig:
    n_beam: int
    n_chan: int
    n_samp_sub: int
    n_sub: int
    seed: int
    mean_dn: int = 128
    sigma_dn: int = 20
    bandpass: int = 0
    n_narrow: int = 0
    narrow_amp_dn: int = 15
    n_burst: int = 0
    burst_amp_dn: int = 40
    n_spike: int = 0
    spike_amp_dn: int = 80

    @property
    def n_time(self) -> int:
        return self.n_sub * self.n_samp_sub

    @property
    def n_cells(self) -> int:
        return self.n_sub * self.n_chan

    @property
    def nbytes(self) -> int:
        return self.n_beam * self.n_time * self.n_chan

    def replace(self, **kw) -> "SynthConfig":
        return dataclasses.replace(self, **kw)

    def _c(self) -> _Cfg:
        return _Cfg(*[getattr(self, f[0]) for f in _Cfg._fields_])


def _rfi_scaled(n_beam, n_chan, n_samp_sub, n_sub, seed, bandpass=1):
    """Noise + RFI at the rates of the 19-beam block: 2 % of channels carry
    beam-common narrowband RFI, 1 % of sub-integrations a broadband burst and
    0.1 % of cells a single-beam pulse."""
    return SynthConfig(
        n_beam=n_beam, n_chan=n_chan, n_samp_sub=n_samp_sub, n_sub=n_sub,
        seed=seed, bandpass=bandpass,
        n_narrow=max(1, round(0.02 * n_chan)),
        n_burst=max(1, round(0.01 * n_sub)) if n_sub > 1 else 0,
        n_spike=max(1, round(0.001 * n_chan * n_sub)))


# 19 beams x 64 channels x 256 sub-integrations x 128 samples, noise N(128,20)
# without bandpass; 3 narrowband channels, 5 bursts, 1 single-beam spike.
SMALL = SynthConfig(n_beam=19, n_chan=64, n_samp_sub=128, n_sub=256,
                    seed=0x2512162781, n_narrow=3, n_burst=5, n_spike=1)

# FAST-shaped block: 19 beams x 4096 channels, 10.07 s at 49.152 us
# (204800 samples), 1024-sample sub-integrations -> 200 x 4096 cells.
FAST_BLOCK = _rfi_scaled(19, 4096, 1024, 200, 0x2512162782)

# Uneven receivers, 5 s blocks each (whole sub-integrations only).
BATCH_SHAPES = (
    _rfi_scaled(13, 1024, 512, 152, 0x2512162784),    # 64 us sampling
    _rfi_scaled(19, 4096, 1024, 99, 0x2512162785),    # 49.152 us
    _rfi_scaled(36, 2048, 2048, 38, 0x2512162786),    # PAF-like, 64 us
    _rfi_scaled(72, 1024, 4096, 19, 0x2512162787),    # PAF-like, 64 us
)


def build(force: bool = False) -> str:
    """Compile libmraid_synth.so in place (gcc, no GPU needed)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "synth.h"))):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-pthread", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.synth_generate.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_void_p, ctypes.c_int]
        lib.synth_generate.restype = ctypes.c_int
        lib.synth_events.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_events.restype = ctypes.c_int
        lib.synth_sample.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int32,
                                     ctypes.c_int64, ctypes.c_int32]
        lib.synth_sample.restype = ctypes.c_uint8
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def generate(cfg: SynthConfig, out_ptr: Optional[int] = None,
             n_threads: Optional[int] = None) -> Optional[np.ndarray]:
    """Generate the block. With out_ptr (host address of cfg.nbytes bytes,
    e.g. a pinned torch tensor) fill it and return None; otherwise return a
    new numpy array of shape (n_beam, n_time, n_chan)."""
    lib = _load()
    c = cfg._c()
    nt = n_threads or default_threads()
    if out_ptr is not None:
        rc = lib.synth_generate(ctypes.byref(c), ctypes.c_void_p(out_ptr), nt)
        if rc != 0:
            raise ValueError(f"synth_generate rejected {cfg}")
        return None
    arr = np.empty((cfg.n_beam, cfg.n_time, cfg.n_chan), dtype=np.uint8)
    rc = lib.synth_generate(ctypes.byref(c), arr.ctypes.data, nt)
    if rc != 0:
        raise ValueError(f"synth_generate rejected {cfg}")
    return arr


def events(cfg: SynthConfig) -> dict:
    """Injected events: narrowband channels (+phase), bursts (t0, sub) and
    spikes (beam, chan, sub, off)."""
    lib = _load()
    nb = (_Narrow * max(1, cfg.n_narrow))()
    bb = (_Burst * max(1, cfg.n_burst))()
    sp = (_Spike * max(1, cfg.n_spike))()
    c = cfg._c()
    if lib.synth_events(ctypes.byref(c), ctypes.addressof(nb), ctypes.addressof(bb),
                        ctypes.addressof(sp)) != 0:
        raise ValueError(f"synth_events rejected {cfg}")
    return {
        "narrow": [(nb[i].chan, nb[i].phase) for i in range(cfg.n_narrow)],
        "burst": [(bb[i].t0, bb[i].sub) for i in range(cfg.n_burst)],
        "spike": [(sp[i].beam, sp[i].chan, sp[i].sub, sp[i].off) for i in range(cfg.n_spike)],
    }


def sample(cfg: SynthConfig, beam: int, t: int, chan: int) -> int:
    """One generated byte (same value as generate() at [beam, t, chan])."""
    return int(_load().synth_sample(ctypes.byref(cfg._c()), beam, t, chan))


def rfi_cells(cfg: SynthConfig) -> dict:
    """Sets of (sub, chan) cells carrying each kind of injected event."""
    ev = events(cfg)
    narrow = {(k, c) for (c, _) in ev["narrow"] for k in range(cfg.n_sub)}
    burst = set()
    for (t0, k) in ev["burst"]:
        for kk in (k, k + 1):
            if kk < cfg.n_sub:
                burst.update((kk, c) for c in range(cfg.n_chan))
    spike = {(k, c) for (_, c, k, _) in ev["spike"]}
    return {"narrow": narrow, "burst": burst, "spike": spike}
