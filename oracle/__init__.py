"""ctypes binding of the plain C oracle (mraid_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg and reference arm (which time it) may import this; the
library's product path never does.

Method: mRAID (arXiv 2512.16278) Section 3.2 Eq. 1 (cross-correlation
matrix), Section 3.3 Eq. 2 (eigendecomposition, normalised eigenvalues),
Section 3.3 / 4.5 (iterative Gaussian-fit threshold, k = 3) and Section 4.3
(preserved frequency ranges).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libmraid_oracle.so")


class FlagInfo(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("sigma", ctypes.c_double),
                ("thresh", ctypes.c_double), ("iterations", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("n_flagged", ctypes.c_int64),
                ("n_used", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile libmraid_oracle.so in place (plain gcc, -O2, no fast-math and
    no FMA contraction, so results do not depend on the host's ISA)."""
    src = os.path.join(_HERE, "mraid_oracle.c")
    hdr = os.path.join(_HERE, "mraid_oracle.h")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(hdr)):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off",
                               "-fPIC", "-shared", "-pthread", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.orc_cell_gram_u8.argtypes = [_P, i32, i64, i32, i32, i32, i32, _P]
        lib.orc_cell_cov_f32.argtypes = [_P, i32, i64, i32, i32, i32, i32, _P]
        lib.orc_corr_from_gram.argtypes = [_P, i32, _P]
        lib.orc_corr_from_cov.argtypes = [_P, i32, _P]
        lib.orc_jacobi.argtypes = [_P, i32, _P, _P, _P]
        lib.orc_stat.argtypes = [_P, i32]
        lib.orc_stat.restype = dbl
        lib.orc_cell_u8.argtypes = [_P, i32, i64, i32, i32, i32, i32, _P, _P, _P, _P, _P]
        lib.orc_block_u8.argtypes = [_P, i32, i64, i32, i32, i32, i32, _P, _P, _P]
        lib.orc_cells_u8.argtypes = [_P, i32, i64, i32, i32, i64, _P, _P, i32, _P, _P, _P, _P]
        lib.orc_flag.argtypes = [_P, i64, i32, _P, dbl, i32, _P, ctypes.POINTER(FlagInfo)]
        lib.orc_beam_flags.argtypes = [_P, _P, i64, i32, _P, i32, dbl, _P, _P]
        lib.orc_cell_gram_pol2_u8.argtypes = [_P, i32, i64, i32, i32, i32, i32, _P]
        lib.orc_cells_pol2_u8.argtypes = [_P, i32, i64, i32, i32, i64, _P, _P, i32, _P, _P, _P,
                                          _P]
        lib.orc_whittaker.argtypes = [_P, _P, i32, dbl, _P]
        lib.orc_arpls.argtypes = [_P, i32, dbl, dbl, i32, _P]
        lib.orc_bandpass_input_u8.argtypes = [_P, i32, i64, i32, i32, i32, i32, i32, _P]
        lib.orc_cell_ccm_bandpass_u8.argtypes = [_P, i32, i64, i32, i32, i32, i32, _P, _P]
        lib.orc_block_bandpass_u8.argtypes = [_P, i32, i64, i32, i32, i32, i32, dbl, dbl, i32,
                                              i32, _P, _P, _P, _P]
        for f in ("orc_cell_gram_u8", "orc_cell_cov_f32", "orc_corr_from_gram",
                  "orc_corr_from_cov", "orc_jacobi", "orc_cell_u8", "orc_block_u8",
                  "orc_cells_u8", "orc_flag", "orc_beam_flags", "orc_whittaker", "orc_arpls",
                  "orc_bandpass_input_u8", "orc_cell_ccm_bandpass_u8",
                  "orc_block_bandpass_u8", "orc_cell_gram_pol2_u8", "orc_cells_pol2_u8"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed (rc={rc})")
    return rc


def _block_view(data: np.ndarray):
    if data.dtype not in (np.uint8, np.float32) or data.ndim != 3:
        raise ValueError("data must be [beam][time][chan] uint8 or float32")
    if not data.flags.c_contiguous:
        raise ValueError("data must be C-contiguous")
    n_beam, n_time, n_chan = data.shape
    return n_beam, n_time * n_chan, n_chan


def cell_gram(data: np.ndarray, n_samp_sub: int, sub: int, chan: int) -> np.ndarray:
    """Exact augmented Gram (N+1)x(N+1) int64 of one cell (Eq. 1 sums)."""
    n_beam, bstride, n_chan = _block_view(data)
    G = np.zeros((n_beam + 1, n_beam + 1), dtype=np.int64)
    _check(_load().orc_cell_gram_u8(_ptr(data), n_beam, bstride, n_chan, n_samp_sub,
                                    sub, chan, _ptr(G)), "gram")
    return G


def cell_cov_f32(data: np.ndarray, n_samp_sub: int, sub: int, chan: int) -> np.ndarray:
    """Population covariance N x N (FP64, two passes) of one cell of float32
    samples: Eq. 1 for float32 input, before the Pearson normalisation.
    Pinned by tests/test_oracle_f32.py."""
    n_beam, bstride, n_chan = _block_view(data)
    C = np.zeros((n_beam, n_beam), dtype=np.float64)
    _check(_load().orc_cell_cov_f32(_ptr(data), n_beam, bstride, n_chan, n_samp_sub,
                                    sub, chan, _ptr(C)), "cov_f32")
    return C


def corr_from_gram(G: np.ndarray):
    """(r, n_zero_variance_beams) from an augmented Gram."""
    G = np.ascontiguousarray(G, dtype=np.int64)
    n = G.shape[0] - 1
    r = np.zeros((n, n), dtype=np.float64)
    deg = _check(_load().orc_corr_from_gram(_ptr(G), n, _ptr(r)), "corr")
    return r, deg


def corr_from_cov(C: np.ndarray):
    """(r, n_zero_variance_beams) from a covariance: r_ab = C_ab /
    sqrt(C_aa C_bb), r_aa = 1, r_ab = 0 beside a zero-variance beam."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    n = C.shape[0]
    r = np.zeros((n, n), dtype=np.float64)
    deg = _check(_load().orc_corr_from_cov(_ptr(C), n, _ptr(r)), "corr_cov")
    return r, deg


def jacobi(A: np.ndarray):
    """(evals descending, q1, sweeps) of a symmetric matrix, FP64 Jacobi."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    ev = np.zeros(n)
    q1 = np.zeros(n)
    sw = ctypes.c_int32(0)
    _check(_load().orc_jacobi(_ptr(A), n, _ptr(ev), _ptr(q1), ctypes.addressof(sw)), "jacobi")
    return ev, q1, sw.value


def stat(evals: np.ndarray) -> float:
    evals = np.ascontiguousarray(evals, dtype=np.float64)
    return float(_load().orc_stat(_ptr(evals), evals.shape[0]))


def cell(data: np.ndarray, n_samp_sub: int, sub: int, chan: int) -> dict:
    """Whole path for one cell: G, r, evals, q1, stat, n_degenerate."""
    n_beam, bstride, n_chan = _block_view(data)
    if data.dtype != np.uint8:
        raise ValueError("cell() takes uint8 data")
    G = np.zeros((n_beam + 1, n_beam + 1), dtype=np.int64)
    r = np.zeros((n_beam, n_beam))
    ev = np.zeros(n_beam)
    q1 = np.zeros(n_beam)
    s = ctypes.c_double(0.0)
    deg = _check(_load().orc_cell_u8(_ptr(data), n_beam, bstride, n_chan, n_samp_sub,
                                     sub, chan, _ptr(G), _ptr(r), _ptr(ev), _ptr(q1),
                                     ctypes.addressof(s)), "cell")
    return {"G": G, "r": r, "evals": ev, "q1": q1, "stat": s.value, "n_degenerate": deg}


def block(data: np.ndarray, n_samp_sub: int, n_threads: int = 1,
          want_evals: bool = True, want_q1: bool = True) -> dict:
    """All cells [sub][chan] of a uint8 block."""
    n_beam, bstride, n_chan = _block_view(data)
    n_sub = data.shape[1] // n_samp_sub
    nc = n_sub * n_chan
    ev = np.zeros((nc, n_beam)) if want_evals else None
    q1 = np.zeros((nc, n_beam)) if want_q1 else None
    st = np.zeros(nc)
    _check(_load().orc_block_u8(_ptr(data), n_beam, bstride, n_chan, n_samp_sub, n_sub,
                                n_threads, _ptr(ev), _ptr(q1), _ptr(st)), "block")
    return {"evals": ev, "q1": q1, "stat": st}


def cells(data: np.ndarray, n_samp_sub: int, subs, chans, n_threads: int = 1,
          data_ptr: Optional[int] = None, shape=None) -> dict:
    """Selected cells; data may also be given as a raw host pointer + shape
    (n_beam, n_time, n_chan) for blocks held in pinned torch memory."""
    if data_ptr is None:
        n_beam, bstride, n_chan = _block_view(data)
        ptr = _ptr(data)
    else:
        n_beam, n_time, n_chan = shape
        bstride = n_time * n_chan
        ptr = data_ptr
    subs = np.ascontiguousarray(subs, dtype=np.int32)
    chans = np.ascontiguousarray(chans, dtype=np.int32)
    n = subs.shape[0]
    G = np.zeros((n, n_beam + 1, n_beam + 1), dtype=np.int64)
    ev = np.zeros((n, n_beam))
    q1 = np.zeros((n, n_beam))
    st = np.zeros(n)
    _check(_load().orc_cells_u8(ptr, n_beam, bstride, n_chan, n_samp_sub, n, _ptr(subs),
                                _ptr(chans), n_threads, _ptr(G), _ptr(ev), _ptr(q1),
                                _ptr(st)), "cells")
    return {"G": G, "evals": ev, "q1": q1, "stat": st}


def flag(stat_: np.ndarray, n_chan: int, keep: Optional[np.ndarray] = None,
         k_sigma: float = 3.0, max_iter: int = 64):
    """(flags uint8 [cells], info dict) of the iterative clip."""
    stat_ = np.ascontiguousarray(stat_, dtype=np.float64).ravel()
    flags = np.zeros(stat_.shape[0], dtype=np.uint8)
    kp = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    info = FlagInfo()
    _check(_load().orc_flag(_ptr(stat_), stat_.shape[0], n_chan, _ptr(kp), k_sigma,
                            max_iter, _ptr(flags), ctypes.byref(info)), "flag")
    return flags, info.as_dict()


def beam_flags(q1: np.ndarray, flags: np.ndarray, n_chan: int, keep: Optional[np.ndarray] = None,
               t: float = 1.0):
    """(bits uint32 [cells][ceil(N/32)], mu_sigma [N][2]) of the eigenvector
    refinement."""
    q1 = np.ascontiguousarray(q1, dtype=np.float64)
    n_cells, n_beam = q1.shape
    flags = np.ascontiguousarray(flags, dtype=np.uint8).ravel()
    W = (n_beam + 31) // 32
    bits = np.zeros((n_cells, W), dtype=np.uint32)
    ms = np.zeros((n_beam, 2))
    kp = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    _check(_load().orc_beam_flags(_ptr(q1), _ptr(flags), n_cells, n_chan, _ptr(kp), n_beam, t,
                                  _ptr(bits), _ptr(ms)), "beam_flags")
    return bits, ms


# ------------------------------------------------------------------ bandpass
# Section 3.1 (ArPLS bandpass; Baek, Park, Ahn and Ahn 2015) and the
# bandpass-centred reading of Eq. 1.

def whittaker(y: np.ndarray, w: np.ndarray, lam: float) -> np.ndarray:
    """z solving (W + lam D^T D) z = W y (D: second differences), FP64."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    z = np.zeros_like(y)
    _check(_load().orc_whittaker(_ptr(y), _ptr(w), y.shape[0], lam, _ptr(z)), "whittaker")
    return z


def arpls(y: np.ndarray, lam: float, ratio: float, itermax: int):
    """(baseline z, solves) of the ArPLS fit of y."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.zeros_like(y)
    it = _check(_load().orc_arpls(_ptr(y), y.shape[0], lam, ratio, itermax, _ptr(z)), "arpls")
    return z, it


def bandpass_input(data: np.ndarray, n_samp_sub: int, sub0: int, n_subs: int, beam: int):
    """Time-aggregated spectrum of one beam over [sub0, sub0 + n_subs)."""
    n_beam, bstride, n_chan = _block_view(data)
    y = np.zeros(n_chan)
    _check(_load().orc_bandpass_input_u8(_ptr(data), n_beam, bstride, n_chan, n_samp_sub,
                                         sub0, n_subs, beam, _ptr(y)), "bandpass_input")
    return y


def cell_ccm_bandpass(data: np.ndarray, n_samp_sub: int, sub: int, chan: int, zc) -> np.ndarray:
    """C (N x N) of one cell about the bandpass values zc[a] (FP64)."""
    n_beam, bstride, n_chan = _block_view(data)
    zc = np.ascontiguousarray(zc, dtype=np.float64)
    C = np.zeros((n_beam, n_beam))
    _check(_load().orc_cell_ccm_bandpass_u8(_ptr(data), n_beam, bstride, n_chan, n_samp_sub,
                                            sub, chan, _ptr(zc), _ptr(C)), "ccm_bandpass")
    return C


def block_bandpass(data: np.ndarray, n_samp_sub: int, interval: int, lam: float, ratio: float,
                   itermax: int, n_threads: int = 1, want_evals: bool = True) -> dict:
    """Whole block under the bandpass-centred reading: z [interval][beam][chan],
    iters [interval][beam], evals [cell][N], stat [cell]."""
    n_beam, bstride, n_chan = _block_view(data)
    n_sub = data.shape[1] // n_samp_sub
    n_int = (n_sub + interval - 1) // interval
    z = np.zeros((n_int, n_beam, n_chan))
    it = np.zeros((n_int, n_beam), dtype=np.int32)
    ev = np.zeros((n_sub * n_chan, n_beam)) if want_evals else None
    st = np.zeros(n_sub * n_chan)
    _check(_load().orc_block_bandpass_u8(_ptr(data), n_beam, bstride, n_chan, n_samp_sub, n_sub,
                                         interval, lam, ratio, itermax, n_threads, _ptr(z),
                                         _ptr(it), _ptr(ev), _ptr(st)), "block_bandpass")
    return {"z": z, "iters": it, "evals": ev, "stat": st}


# ---------------------------------------------------------- two polarisations
# Section 2 (two polarisations recorded): the total power of beam a is the
# sum of its two polarisations, blocks a and N + a of a 2N-block array.

def cell_gram_pol2(data: np.ndarray, n_samp_sub: int, sub: int, chan: int) -> np.ndarray:
    """Exact augmented Gram (N+1)x(N+1) of the total power; data has 2N blocks."""
    n_blocks, bstride, n_chan = _block_view(data)
    if n_blocks % 2:
        raise ValueError("two-polarisation data has an even number of blocks")
    N = n_blocks // 2
    G = np.zeros((N + 1, N + 1), dtype=np.int64)
    _check(_load().orc_cell_gram_pol2_u8(_ptr(data), N, bstride, n_chan, n_samp_sub, sub, chan,
                                         _ptr(G)), "gram_pol2")
    return G


def cells_pol2(data: np.ndarray, n_samp_sub: int, subs, chans, n_threads: int = 1) -> dict:
    """Selected cells of a two-polarisation block (G, evals, q1, stat)."""
    n_blocks, bstride, n_chan = _block_view(data)
    N = n_blocks // 2
    subs = np.ascontiguousarray(subs, dtype=np.int32)
    chans = np.ascontiguousarray(chans, dtype=np.int32)
    n = subs.shape[0]
    G = np.zeros((n, N + 1, N + 1), dtype=np.int64)
    ev = np.zeros((n, N))
    q1 = np.zeros((n, N))
    st = np.zeros(n)
    _check(_load().orc_cells_pol2_u8(_ptr(data), N, bstride, n_chan, n_samp_sub, n, _ptr(subs),
                                     _ptr(chans), n_threads, _ptr(G), _ptr(ev), _ptr(q1),
                                     _ptr(st)), "cells_pol2")
    return {"G": G, "evals": ev, "q1": q1, "stat": st}
