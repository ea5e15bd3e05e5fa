#!/usr/bin/env python3
"""Benchmark of the eigenvalue RFI flagger on a FAST-shaped block.

Workload (default): 19 beams x 4096 channels x 200 sub-integrations x 1024
samples of 8-bit data (a 10.07 s block at 49.152 us; 819200 cells of 19x19
correlation matrices), synthetic (seeded generator, noise + beam-common RFI
+ single-beam pulses). One step = mraid_run on the block resident in HBM:
Gram sums and correlation, all eigenvalues and q1 (Householder reduction and
implicit QR by default), the statistic and the iterative mask. Inputs (15.9 GB) are far larger than L2 (129 MB).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mraid|reference]

Under torchrun every rank processes its own block (different seed); there is
no data-path collective (weak scaling). Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("CCM+eig cells/s & HBM GB/s %peak (19-beam×4096-ch); "
          "served p50/p99 block latency")
UNIT = "cells/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mraid", "reference"], default="mraid")
    ap.add_argument("--workload", choices=["fast_block", "small", "paf13", "fast19", "paf36", "paf72"],
                    default="fast_block")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="budget of the oracle CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="oracle seconds of the reference arm over all its steps "
                         "(default: 60, and at least 2 per step)")
    ap.add_argument("--n-sub", type=int, default=0,
                    help="shrink the block to this many sub-integrations (profiling runs)")
    ap.add_argument("--f32-subs", type=int, default=200,
                    help="sub-integrations of the float32-input variant (0: skip)")
    ap.add_argument("--pol2-steps", type=int, default=3,
                    help="timed runs of the two-polarisation path (0: skip)")
    ap.add_argument("--bandpass-steps", type=int, default=3,
                    help="timed runs of the bandpass-centred path (0: skip)")
    ap.add_argument("--multires-steps", type=int, default=3,
                    help="timed calls of the seven-timescale pass (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=3,
                    help="timed passes of the batched form (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="seconds of Poisson arrivals per rate for the served form (0: skip)")
    return ap.parse_args()


RECEIVERS = {"paf13": 0, "fast19": 1, "paf36": 2, "paf72": 3}   # synth.BATCH_SHAPES index


def workload(name, rank, n_sub=0):
    import synth
    if name in RECEIVERS:       # one 5 s block of a receiver of the batched form
        base = synth.BATCH_SHAPES[RECEIVERS[name]]
        kind = f"{name} receiver block (5 s)"
    else:
        base = synth.FAST_BLOCK if name == "fast_block" else synth.SMALL
        kind = "FAST-shaped block" if name == "fast_block" else "small block"
    cfg = base.replace(seed=base.seed + 7919 * rank)
    if n_sub:
        cfg = cfg.replace(n_sub=n_sub, n_burst=min(cfg.n_burst, max(0, n_sub - 1)),
                          n_spike=min(cfg.n_spike, n_sub * cfg.n_chan // 1000 + 1))
    desc = (f"{kind}: {cfg.n_beam} beams x {cfg.n_chan} channels x {cfg.n_sub} "
            f"sub-integrations x {cfg.n_samp_sub} samples, uint8 ({cfg.n_cells} cells, "
            f"{cfg.nbytes / 1e9:.2f} GB)")
    return cfg, desc


def config_dict(cfg, desc, world):
    return {
        "workload": desc,
        "n_beam": cfg.n_beam, "n_chan": cfg.n_chan, "n_sub": cfg.n_sub,
        "n_samp_sub": cfg.n_samp_sub, "cells_per_gpu": cfg.n_cells,
        "bytes_per_gpu": cfg.nbytes, "rfi": {"narrowband_channels": cfg.n_narrow,
                                           "broadband_bursts": cfg.n_burst,
                                           "single_beam_pulses": cfg.n_spike},
        "l2": "inputs larger than L2 (no flush needed)",
        "parallelism": f"dp{world} (one independent block per GPU)",
    }


# ------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x for x in vis.split(",") if x.strip()]
        if local_rank < len(ids) and ids[local_rank].strip().isdigit():
            return int(ids[local_rank])
    return local_rank


# ------------------------------------------------------------- peaks

EIG_NAMES = {0: "jacobi (looped rounds)", 1: "jacobi (unrolled sweep)",
             2: "householder + implicit QR", 3: "householder + implicit QR (compact)",
             4: "householder + implicit QR, split (reduction and q1 / QR kernels)",
             5: "householder + root-free QR, split (reduction and q1 / QR kernels)"}
SMS, FP32_LANES = 152, 128          # GB300: SMs, FP32 lanes per SM


def measured_peaks():
    """HBM copy bandwidth (measured), and the FP32 ALU peak derived from the
    lane count at the maximum SM clock the same file records: 152 SMs x 128
    lanes x 2 flops per FMA x 2070 MHz = 80.5 TFLOP/s."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        mhz = float(d.get("sm_max_mhz", 2070.0))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured",
                "fp32_tflops": SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback",
                "fp32_tflops": SMS * FP32_LANES * 2 * 2070e6 / 1e12}


def kernel_traffic(name):
    """dram bytes per launch from a committed ncu summary, if it was taken
    on the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    rec = d.get(name)
    if not rec:
        return None
    src = os.path.join(ROOT, rec.get("source", ""))
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != rec.get("source_sha256_16"):
        return None
    return rec.get("bytes_per_launch_full_size")


# ------------------------------------------------------------- CPU oracle

def cpu_baseline(cfg, h_ptr, seconds):
    """The oracle as it stands, on the host's cores, on a random sample of
    the workload's cells (same bytes the GPU processed)."""
    import numpy as np
    import oracle
    import synth
    threads = synth.default_threads()
    rng = np.random.default_rng(12345)
    shape = (cfg.n_beam, cfg.n_time, cfg.n_chan)

    def run(n, n_threads=threads):
        idx = rng.integers(0, cfg.n_cells, size=n)
        subs = (idx // cfg.n_chan).astype(np.int32)
        chans = (idx % cfg.n_chan).astype(np.int32)
        t0 = time.perf_counter()
        res = oracle.cells(None, cfg.n_samp_sub, subs, chans, n_threads=n_threads,
                           data_ptr=h_ptr, shape=shape)
        return time.perf_counter() - t0, idx, res

    n = threads * 4
    t, _, _ = run(n)
    n2 = max(threads, int(n * max(seconds - t, 0.5) / max(t, 1e-6)))
    t2, idx, res = run(n2)
    # one thread on a quarter of the all-core sample's time: the per-core rate
    n1 = max(4, n2 // (4 * threads))
    t1, _, _ = run(n1, 1)
    return {"value": n2 / t2, "unit": UNIT, "cores": threads, "kind": "oracle",
            "single_thread_value": n1 / t1, "cpu_model": cpu_model(),
            "sample": f"{n2} random cells of the same block (per-cell Gram, FP64 Jacobi, "
                      f"statistic; {t2:.1f} s on {threads} threads; {n1} cells on one "
                      f"thread in {t1:.1f} s); the mask pass is excluded (it is O(cells) "
                      "and negligible)"}, (idx, res)


def cpu_model():
    """The host CPU's name as the kernel reports it (x86: model name; Arm:
    implementer and part numbers), else the machine type."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    if fields.get("CPU part"):
        return (f"{platform.machine()} (CPU implementer {fields.get('CPU implementer', '?')}, "
                f"part {fields['CPU part']})")
    return platform.machine() or "unknown"


def sampled_parity(sample, evals, q1, stat):
    """GPU outputs of the timed run against the outputs the cpu_baseline
    leg's oracle sample produced (no further oracle call), at the tests'
    tolerances: eigenvalues 1e-4 of lambda_max, s 2e-4 relative, q1 1e-3
    where the relative gap is at least 1e-4 (below it q1 is unpinned), with
    the q1 error also given per gap band."""
    import numpy as np
    idx, res = sample
    it = torch_index(idx)
    ev = evals.index_select(0, it.to(evals.device)).cpu().numpy().astype(np.float64)
    qv = q1.index_select(0, it.to(q1.device)).cpu().numpy().astype(np.float64)
    sv = stat.index_select(0, it.to(stat.device)).cpu().numpy().astype(np.float64)
    eo, qo, so = res["evals"], res["q1"], res["stat"]
    lmax = np.abs(eo).max(axis=1)
    e_err = (np.abs(ev - eo).max(axis=1) / lmax)
    s_err = np.abs(sv - so) / np.maximum(so, 1e-30)
    gap = (eo[:, 0] - eo[:, 1]) / eo[:, 0]
    # q1 error per cell; where the two largest magnitudes tie the sign rule
    # is decided by rounding, so those cells compare up to sign
    q_same = np.abs(qv - qo).max(axis=1)
    q_flip = np.abs(qv + qo).max(axis=1)
    mags = np.sort(np.abs(qo), axis=1)
    tie = (mags[:, -1] - mags[:, -2]) <= 1e-3
    q_err = np.where(tie, np.minimum(q_same, q_flip), q_same)
    sel = gap >= 1e-4
    bands = {}
    for name, lo, hi in (("gap>=1e-2", 1e-2, np.inf), ("1e-3<=gap<1e-2", 1e-3, 1e-2),
                         ("1e-4<=gap<1e-3", 1e-4, 1e-3)):
        b = (gap >= lo) & (gap < hi)
        bands[name] = {"cells": int(b.sum()),
                       "q1_err_max": float(q_err[b].max()) if b.any() else None}
    bands["gap<1e-4 (unpinned)"] = {"cells": int((gap < 1e-4).sum())}
    q_max = float(q_err[sel].max()) if sel.any() else 0.0
    return {"cells": int(len(idx)), "eig_err_rel_max": float(e_err.max()),
            "eig_err_rel_p99": float(np.percentile(e_err, 99)),
            "stat_err_rel_max": float(s_err.max()), "q1_err_max": q_max,
            "q1_cells": int(sel.sum()), "q1_by_gap": bands,
            "pass": bool(e_err.max() <= 1e-4 and s_err.max() <= 2e-4 and q_max <= 1e-3)}


def torch_index(idx):
    import torch
    return torch.from_numpy(idx.astype("int64"))


# ------------------------------------------------------------- main arms

def bench_f32(m, torch, d_u8, cfg, stream, n_sub, peaks):
    """Float32-input variant (beamformer output, bit_depth 32) on the first
    n_sub sub-integrations of the same block, converted on the device to
    (x - 128) / 20 (zero-mean, unit-variance noise with the same RFI): cells/s
    of the whole path with the tensor-core Gram (split-bf16 products) and
    with the CUDA-core FP32 Gram and the tensor-core kernel's HBM roofline.
    Its parity against the oracle is in the tests."""
    N, C, S = cfg.n_beam, cfg.n_chan, cfg.n_samp_sub
    n_sub = min(n_sub, cfg.n_sub)
    T = n_sub * S
    x = d_u8.view(N, cfg.n_time, C)[:, :T, :].float().sub_(128.0).div_(20.0).contiguous()
    # x is made on the current stream; the plan reads it on its own stream
    stream.wait_stream(torch.cuda.current_stream())
    cells = n_sub * C
    with torch.cuda.stream(stream):
        plan = m.Plan(N, C, S, n_sub, bit_depth=32, stream=stream)
        ev = torch.empty(cells, N, dtype=torch.float32, device="cuda")
        q = torch.empty(cells, N, dtype=torch.float32, device="cuda")
        st = torch.empty(cells, dtype=torch.float32, device="cuda")
        fl = torch.empty(cells, dtype=torch.uint8, device="cuda")
    info = m.FlagInfo()
    in_bytes = N * T * C * 4
    out = {"workload": f"float32 [{N}][{T}][{C}] ({n_sub} sub-integrations, "
                       f"{in_bytes / 1e9:.2f} GB)"}
    for gram, tag in ((0, "tensor_cores"), (-1, "cuda_cores")):
        m.mraid_set_variant(plan.handle, gram)
        for _ in range(3):
            m.mraid_run(plan.handle, x, ev, q, st, fl, info)
        m.mraid_sync(plan.handle)
        m.mraid_profile_reset(plan.handle)
        m.mraid_profile_enable(plan.handle, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            m.mraid_run(plan.handle, x, ev, q, st, fl, info)
        e1.record(stream)
        m.mraid_sync(plan.handle)
        m.mraid_profile_enable(plan.handle, False)
        prof = m.mraid_profile_read(plan.handle)
        ms = e0.elapsed_time(e1) / 5
        kern = "gram_tc_f32" if gram == 0 else "gram_f32"
        n_l, tot = prof.get(kern, (0, 0.0))
        res = {"ms_per_step": ms, "cells_per_s": cells / (ms / 1e3),
               "gbs": in_bytes / (ms / 1e3) / 1e9,
               "gram_kernel": kern, "gram_launches": n_l}
        if n_l > 0:
            kms = tot / n_l
            b = in_bytes                                        # samples in
            xb = cells * 4 * (N * (N + 1) // 2)                 # r out (reported apart)
            a = b / (kms / 1e3) / 1e9
            res["gram_roofline"] = {"bound": "hbm", "kernel": kern, "achieved": a,
                                    "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                    "frac": a / peaks["hbm_gbs"],
                                    "traffic": kernel_traffic(kern),
                                    "work_per_launch": b, "ms_per_launch": kms,
                                    "export_bytes": xb,
                                    "frac_incl_export": (b + xb) / (kms / 1e3) / 1e9
                                    / peaks["hbm_gbs"]}
        out[tag] = res
    out["path"] = ("Gram of per-beam shifted samples: tensor cores with bf16 hi/lo products "
                   "(four MMAs per 16 samples) or FP32 CUDA cores; FP32 eigensolver")
    plan.close()
    del x
    torch.cuda.empty_cache()
    return out


# sub-interval lengths of Table 1 (0.05 s to 10 s) in 1024-sample
# sub-integrations of 49.152 us: 0.05, 0.2, 0.5, 1, 2, 5, 10 s
MULTIRES_FACTORS = (1, 4, 10, 20, 40, 100, 200)


def bench_multires(m, torch, d, cfg, stream, steps, peaks):
    """All seven timescales of Table 1 in one mraid_multires call on the
    block (one pass over the samples), against mraid_run once per timescale
    (seven passes); per-level masking rate, and the aggregation kernel's HBM
    roofline."""
    N, C, S, K = cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub
    factors = [f for f in MULTIRES_FACTORS if f <= K]
    with torch.cuda.stream(stream):
        plan = m.Plan(N, C, S, K, stream=stream)
        stats = [torch.empty((K // f) * C, dtype=torch.float32, device="cuda") for f in factors]
        flags = [torch.empty((K // f) * C, dtype=torch.uint8, device="cuda") for f in factors]
    infos = (m.FlagInfo * len(factors))()
    m.mraid_multires(plan.handle, d, factors, stats, flags, infos)
    m.mraid_sync(plan.handle)
    m.mraid_profile_reset(plan.handle)
    m.mraid_profile_enable(plan.handle, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        m.mraid_multires(plan.handle, d, factors, stats, flags, infos)
    e1.record(stream)
    m.mraid_sync(plan.handle)
    m.mraid_profile_enable(plan.handle, False)
    prof = m.mraid_profile_read(plan.handle)
    ms = e0.elapsed_time(e1) / steps
    kt = {k: (n // steps, tot / steps) for k, (n, tot) in prof.items() if n > 0}
    levels = []
    for i, f in enumerate(factors):
        info = infos[i].as_dict()
        levels.append({"factor": f, "seconds": round(f * S * 49.152e-6, 3),
                       "cells": (K // f) * C, "masked_fraction": info["n_flagged"] / ((K // f) * C),
                       "iterations": info["iterations"], "threshold": info["thresh"]})
    plan.close()
    # one mraid_run per timescale, each a plan with the longer sub-integration
    sep = 0.0
    for f in factors:
        n_f = K // f
        with torch.cuda.stream(stream):
            p2 = m.Plan(N, C, f * S, n_f, beam_stride=cfg.n_time * C, stream=stream)
            st = torch.empty(n_f * C, dtype=torch.float32, device="cuda")
            fl = torch.empty(n_f * C, dtype=torch.uint8, device="cuda")
        m.mraid_run(p2.handle, d, None, None, st, fl)
        m.mraid_sync(p2.handle)
        e0.record(stream)
        m.mraid_run(p2.handle, d, None, None, st, fl)
        e1.record(stream)
        m.mraid_sync(p2.handle)
        sep += e0.elapsed_time(e1)
        p2.close()
    psum = (N + 1) * (N + 2) // 2
    agg = None
    if "gram_aggregate" in kt:
        n_l, tot = kt["gram_aggregate"]
        # bytes over all levels of one call: every level reads its source
        # sums once and writes its own (sources as chosen by the library)
        done, b = [1], 0
        for f in factors[1:]:
            g = max(x for x in done if f % x == 0)
            b += 8 * psum * C * ((K // f) * f // g + K // f)
            done.append(f)
        a = b / (tot / 1e3) / 1e9
        agg = {"bound": "hbm", "kernel": "gram_aggregate", "achieved": a, "peak": peaks["hbm_gbs"],
               "unit": "GB/s", "frac": a / peaks["hbm_gbs"], "launches": n_l,
               "work_per_call": b, "ms_per_call": tot}
    return {"workload": f"{cfg.n_beam} beams x {C} channels x {K} x {S} samples (uint8), "
                        f"timescales {factors} sub-integrations",
            "ms_per_call": ms, "ms_separate_runs": sep,
            "cells_per_s_all_levels": sum((K // f) * C for f in factors) / (ms / 1e3),
            "kernels_ms_per_call": {k: v[1] for k, v in kt.items()},
            "aggregate_roofline": agg, "levels": levels}


def bench_bandpass(m, torch, d, cfg, stream, steps):
    """The bandpass-centred path (Section 3.1 ArPLS bandpass, C about it) on
    the block with the default fit parameters (1 s intervals): time per
    step, kernel breakdown and mask. Its parity against the oracle, at this
    size too, is in the tests."""
    N, C, S, K = cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub
    bp = m.mraid_default_bandpass_params()
    n_int = (K + bp.interval - 1) // bp.interval
    with torch.cuda.stream(stream):
        plan = m.Plan(N, C, S, K, stream=stream)
        band = torch.empty(n_int, N, C, dtype=torch.float32, device="cuda")
        st = torch.empty(K * C, dtype=torch.float32, device="cuda")
        fl = torch.empty(K * C, dtype=torch.uint8, device="cuda")
    info = m.FlagInfo()
    m.mraid_run_bandpass(plan.handle, d, bp, band, None, None, st, fl, info)
    m.mraid_sync(plan.handle)
    m.mraid_profile_reset(plan.handle)
    m.mraid_profile_enable(plan.handle, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        m.mraid_run_bandpass(plan.handle, d, bp, band, None, None, st, fl, info)
    e1.record(stream)
    m.mraid_sync(plan.handle)
    m.mraid_profile_enable(plan.handle, False)
    prof = m.mraid_profile_read(plan.handle)
    ms = e0.elapsed_time(e1) / steps
    kt = {k: tot / steps for k, (n, tot) in prof.items() if n > 0}
    plan.close()
    return {"workload": f"{N} beams x {C} channels x {K} x {S} samples (uint8), "
                        f"fit intervals of {bp.interval} sub-integrations ({n_int} x {N} spectra)",
            "params": {"lam": bp.lam, "ratio": bp.ratio, "itermax": bp.itermax,
                       "interval": bp.interval},
            "ms_per_step": ms, "cells_per_s": K * C / (ms / 1e3),
            "kernels_ms_per_step": kt,
            "masked_fraction": info.n_flagged / (K * C), "mask_iterations": info.iterations}


def bench_pol2(m, torch, h, cfg, stream, steps, peaks):
    """Two recorded polarisations: the block as polarisation 0 and a second
    synthetic block (next seed, its own RFI) as polarisation 1, stacked in
    device memory; mraid_run_pol2 per step and the kernel breakdown. Its
    parity against the oracle, at this size too, is in the tests."""
    import synth
    N, C, S, K = cfg.n_beam, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub
    nb = cfg.nbytes
    h2 = torch.empty(2 * nb, dtype=torch.uint8, pin_memory=True)
    h2[:nb].copy_(h)
    synth.generate(cfg.replace(seed=cfg.seed + 1), out_ptr=h2.data_ptr() + nb)
    d2 = h2.to("cuda")
    cells = K * C
    with torch.cuda.stream(stream):
        plan = m.Plan(N, C, S, K, stream=stream)
        ev = torch.empty(cells, N, dtype=torch.float32, device="cuda")
        st = torch.empty(cells, dtype=torch.float32, device="cuda")
        fl = torch.empty(cells, dtype=torch.uint8, device="cuda")
    info = m.FlagInfo()
    m.mraid_run_pol2(plan.handle, d2, ev, None, st, fl, info)
    m.mraid_sync(plan.handle)
    m.mraid_profile_reset(plan.handle)
    m.mraid_profile_enable(plan.handle, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        m.mraid_run_pol2(plan.handle, d2, ev, None, st, fl, info)
    e1.record(stream)
    m.mraid_sync(plan.handle)
    m.mraid_profile_enable(plan.handle, False)
    prof = m.mraid_profile_read(plan.handle)
    ms = e0.elapsed_time(e1) / steps
    kt = {k: tot / steps for k, (n, tot) in prof.items() if n > 0}
    gram = None
    if "gram_tc" in kt:
        b = 2 * nb                                      # both polarisations in
        xb = cells * 4 * (N * (N + 1) // 2)             # r out (reported apart)
        a = b / (kt["gram_tc"] / 1e3) / 1e9
        gram = {"bound": "hbm", "kernel": "gram_tc (two polarisations)", "achieved": a,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
                "traffic": kernel_traffic("gram_tc_pol2"), "work_per_launch": b,
                "ms_per_launch": kt["gram_tc"], "export_bytes": xb,
                "frac_incl_export": (b + xb) / (kt["gram_tc"] / 1e3) / 1e9 / peaks["hbm_gbs"]}
    plan.close()
    del d2, h2
    torch.cuda.empty_cache()
    return {"workload": f"{N} beams x 2 polarisations x {C} channels x {K} x {S} samples "
                        f"(uint8, {2 * nb / 1e9:.1f} GB)",
            "ms_per_step": ms, "cells_per_s": cells / (ms / 1e3),
            "input_gbs": 2 * nb / (ms / 1e3) / 1e9,
            "kernels_ms_per_step": kt, "gram_roofline": gram,
            "masked_fraction": info.n_flagged / cells,
            "path": "tensor cores: polarisations added in the converter, TMEM pieces of 256 "
                    "samples added as integers in the epilogue, correlation fused; then the "
                    "eigensolver and mask"}


def batched_fractions(shapes, ms, peaks):
    """Whole-pass fractions of the batched form: the algorithmic bytes (every
    block's samples read once; s, flag, eigenvalues and q1 written) against
    the HBM peak, and the eigensolver's dense floor ((4/3) N^3 flops per
    cell) against the FP32 peak."""
    nbytes = sum(c.nbytes + c.n_cells * (5 + 8 * c.n_beam) for c in shapes)
    flops = sum(c.n_cells * 4.0 * c.n_beam ** 3 / 3.0 for c in shapes)
    gbs = nbytes / (ms / 1e3) / 1e9
    tflops = flops / (ms / 1e3) / 1e12
    return {"hbm": {"bytes_per_pass": nbytes, "achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
                    "frac": gbs / peaks["hbm_gbs"]},
            "alu": {"flops_per_pass": flops, "achieved_tflops": tflops,
                    "peak_tflops": peaks["fp32_tflops"], "frac": tflops / peaks["fp32_tflops"]}}


def bench_batched(m, torch, stream, steps, peaks=None):
    """Four receivers of 5 s each (13/19/36/72 beams) in one graph-captured
    pass, against the plain form (one mraid_run per block, one after the
    other on one stream) on the same data, with the pass's HBM and ALU
    fractions."""
    import synth
    shapes = synth.BATCH_SHAPES
    datas = []
    for cfg in shapes:
        h = torch.empty(cfg.nbytes, dtype=torch.uint8, pin_memory=True)
        synth.generate(cfg, out_ptr=h.data_ptr())
        datas.append(h.to("cuda"))
        del h
    cells = sum(c.n_cells for c in shapes)
    nbytes = sum(c.nbytes for c in shapes)
    dims = [(c.n_beam, c.n_chan, c.n_samp_sub, c.n_sub) for c in shapes]
    with torch.cuda.stream(stream):
        batch = m.Batch(dims, stream=stream)
        outs = batch.outputs()
        plans = [m.Plan(*d, stream=stream) for d in dims]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        batch.run(datas, outs, sync=True)
    e0.record(stream)
    for _ in range(steps):
        batch.run(datas, outs, sync=False)
    e1.record(stream)
    m.mraid_batch_sync(batch.handle)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / steps
    infos = [m.FlagInfo() for _ in plans]
    # the plain form writes the same outputs as the batch: evals, q1, stat, flags
    po = [{k: torch.empty_like(o[k]) for k in ("evals", "q1", "stat", "flags")} for o in outs]
    for _ in range(2):
        for plan, d, o, inf in zip(plans, datas, po, infos):
            m.mraid_run(plan.handle, d, o["evals"], o["q1"], o["stat"], o["flags"], inf)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for plan, d, o, inf in zip(plans, datas, po, infos):
            m.mraid_run(plan.handle, d, o["evals"], o["q1"], o["stat"], o["flags"], inf)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1) / steps
    inst, upd = batch.graph_stats()
    packing, ms_conc, ms_chain = batch.packing()
    for plan in plans:
        plan.close()
    batch.close()
    del datas, outs, po
    torch.cuda.empty_cache()
    return {"workload": "13b/1024ch/512, 19b/4096ch/1024, 36b/2048ch/2048, 72b/1024ch/4096; "
                        "5 s each, uint8", "cells": cells, "bytes": nbytes,
            "ms_per_pass": ms_b, "cells_per_s": cells / (ms_b / 1000.0),
            "plain_ms_per_pass": ms_p, "plain_cells_per_s": cells / (ms_p / 1000.0),
            "graph_instantiations": inst, "graph_updates": upd,
            "fractions": batched_fractions(shapes, ms_b, peaks) if peaks else None,
            "packing": {"chosen": "chained" if packing == 1 else "concurrent",
                        "ms_concurrent": ms_conc, "ms_chained": ms_chain},
            "note": "plain = one mraid_run per block, sequential on one stream, writing the same "
                    "outputs (evals, q1, stat, flags); default variants in both; the batch's "
                    "first run timed both packings"}


def bench_served(m, torch, seconds, rates=(1.0, 2.0, 4.0)):
    """8 observations (two of each receiver), 1 s blocks arriving as a
    Poisson process at 1x, 2x and 4x real time in aggregate; latency from
    submit (block complete in pinned host memory) to flags in host memory."""
    import numpy as np
    import synth
    recv = [(13, 1024, 512, 15625), (19, 4096, 1024, 20345), (36, 2048, 2048, 15625),
            (72, 1024, 4096, 15625)]   # (beams, channels, N_s, samples per 1 s block)
    streams = [r for r in recv for _ in range(2)]
    blocks = []
    for i, (nb, nc, ns, bs) in enumerate(streams):
        n_sub = -(-bs // ns)
        cfg = synth.SynthConfig(n_beam=nb, n_chan=nc, n_samp_sub=ns, n_sub=n_sub, seed=6000 + i,
                                bandpass=1, n_narrow=max(1, nc // 50), n_burst=0, n_spike=1)
        full = synth.generate(cfg)
        h = torch.from_numpy(np.ascontiguousarray(full[:, :bs, :])).pin_memory()
        blocks.append(h)
    out = {"streams": "2 x (13b/1024ch/512, 19b/4096ch/1024, 36b/2048ch/2048, 72b/1024ch/4096)",
           "block_s": 1.0, "rates": {}}
    rng = np.random.default_rng(77)
    with m.Server(streams, max_inflight=8) as srv:
        # warm-up: one block per stream
        for i in range(len(streams)):
            srv.submit(i, blocks[i], torch.empty(srv.flags_bytes(i), dtype=torch.uint8).pin_memory(), -1)
        srv.drain(120000)
        srv.poll(1024)
        for rate_x in rates:
            lam = rate_x * len(streams)   # blocks per second, aggregate
            n_blocks = max(8, int(lam * seconds))
            t_arr = np.cumsum(rng.exponential(1.0 / lam, size=n_blocks))
            keep = []
            t0 = time.perf_counter()
            for k, ta in enumerate(t_arr):
                while time.perf_counter() - t0 < ta:
                    time.sleep(min(0.0005, max(0.0, ta - (time.perf_counter() - t0))))
                i = k % len(streams)
                f = torch.empty(srv.flags_bytes(i), dtype=torch.uint8).pin_memory()
                keep.append(f)
                srv.submit(i, blocks[i], f, k)
            srv.drain(300000)
            wall = time.perf_counter() - t0
            res = [r for r in srv.poll(100000) if r["seq"] >= 0]
            lat = np.array([r["latency_ms"] for r in res])
            dev = np.array([r["device_ms"] for r in res])
            cells = sum(r["n_cells"] for r in res)
            out["rates"][f"{rate_x:g}x"] = {
                "blocks": len(res), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "device_p50_ms": float(np.percentile(dev, 50)),
                "device_p99_ms": float(np.percentile(dev, 99)), "cells_per_s": cells / wall,
                "offered_blocks_per_s": lam}
        # saturation: 16 s of every observation's blocks submitted at once;
        # the sustained rate is that work over the wall time to drain it
        n_sat = 16 * len(streams)
        keep = []
        t0 = time.perf_counter()
        for k in range(n_sat):
            i = k % len(streams)
            f = torch.empty(srv.flags_bytes(i), dtype=torch.uint8).pin_memory()
            keep.append(f)
            srv.submit(i, blocks[i], f, 1_000_000 + k)
        srv.drain(600000)
        wall = time.perf_counter() - t0
        res = [r for r in srv.poll(100000) if r["seq"] >= 1_000_000]
        lat = np.array([r["latency_ms"] for r in res])
        cells = sum(r["n_cells"] for r in res)
        out["saturation"] = {
            "blocks": len(res), "wall_s": wall, "blocks_per_s": len(res) / wall,
            "cells_per_s": cells / wall,
            "real_time_factor": len(res) / len(streams) / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "note": "all blocks queued at t=0; latency includes the queue"}
    # plain per-block launch on the same blocks: one block at a time, copy in,
    # mraid_run_host, flags back
    plain = []
    for i, (nb, nc, ns, bs) in enumerate(streams[::2]):
        n_sub = bs // ns
        with m.Plan(nb, nc, ns, n_sub, beam_stride=bs * nc) as plan:
            h = blocks[2 * i]
            fl = torch.empty(n_sub * nc, dtype=torch.uint8, pin_memory=True)
            plan.run_host(h, h_flags=fl)
            t0 = time.perf_counter()
            for _ in range(3):
                plan.run_host(h, h_flags=fl)
            plain.append((time.perf_counter() - t0) / 3 * 1000.0)
    out["plain_block_ms"] = {f"{s[0]}b": v for s, v in zip(recv, plain)}
    # the plain per-block launch's sustained rate on the same mix
    plain_cells = sum((bs // ns) * nc for (nb, nc, ns, bs) in recv)
    out["plain_cells_per_s"] = plain_cells / (sum(plain) / 1000.0)
    return out


def max_over_ranks(value, dist, device=None):
    """The largest value over all ranks (the step time the job is charged);
    value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device) if device else torch.tensor([float(value)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank, world, ms_max):
    """Whole-job cells/s: all ranks' cells over the slowest rank's time."""
    return world * cells_per_rank / (ms_max / 1000.0)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    import torch
    cfg, desc = workload(args.workload, 0, args.n_sub)
    import synth
    h = torch.empty(cfg.nbytes, dtype=torch.uint8)
    synth.generate(cfg, out_ptr=h.data_ptr())
    n_runs = max(1, args.steps + args.warmup)
    if args.ref_seconds is None:
        per_step = max(2.0, 60.0 / n_runs)
    else:
        per_step = max(0.1, args.ref_seconds / n_runs)
    vals = []
    for i in range(args.warmup + args.steps):
        r, _ = cpu_baseline(cfg, h.data_ptr(), per_step)
        if i >= args.warmup:
            vals.append(r["value"])
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * cfg.n_cells / v,
        "ms_per_step_note": ("extrapolated: the block's cells over the rate measured on "
                             "sampled cells; no step over the whole block was run"),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8->i64 Gram, f64 Jacobi", "data": "synthetic",
        "config": config_dict(cfg, desc, 1),
        "cpu_baseline": {"kind": "oracle", "cores": r["cores"], "sample": r["sample"],
                         "value": v, "unit": UNIT,
                         "single_thread_value": r["single_thread_value"],
                         "cpu_model": r["cpu_model"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def kernel_rooflines(cfg, kt, peaks):
    """Roofline of every timed kernel: algorithmic work per launch (bytes for
    the memory-bound kernels, flops for the eigensolver) over its average
    launch time, against the bound that limits it."""
    N, cells = cfg.n_beam, cfg.n_cells
    np_, psum = N * (N + 1) // 2, (N + 1) * (N + 2) // 2
    in_bytes = N * cfg.n_samp_sub * cells
    hbm = {  # bytes per launch: what the kernel must read and write once
        # the Gram reads every sample once (the per-cell input the path
        # counts); its correlation export, an intermediate the path would
        # keep on chip, is reported beside it, not as work
        "gram_tc": in_bytes,
        "gram_u8": in_bytes + cells * 8 * psum,                # samples in, sums out
        "corr_from_sums": cells * (8 * psum + 4 * np_),
        "flag_clip": cells * 5,                                # stat in, flag out
    }
    # eigensolver: the dense floor, (4/3) N^3 flops of a tridiagonal
    # reduction per cell (all N eigenvalues then cost O(N^2) more)
    eig_flops = cells * 4.0 * N ** 3 / 3.0
    out = {}
    for k, (n, ms) in kt.items():
        if k == "eig":
            a = eig_flops / (ms / 1e3) / 1e12
            out[k] = {"bound": "alu", "kernel": k, "achieved": a, "peak": peaks["fp32_tflops"],
                      "unit": "TFLOP/s", "frac": a / peaks["fp32_tflops"],
                      "traffic": kernel_traffic(k),
                      "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                      "work_per_launch": eig_flops, "ms_per_launch": ms}
        else:
            b = hbm.get(k, in_bytes)
            a = b / (ms / 1e3) / 1e9
            out[k] = {"bound": "hbm", "kernel": k, "achieved": a, "peak": peaks["hbm_gbs"],
                      "unit": "GB/s", "frac": a / peaks["hbm_gbs"], "traffic": kernel_traffic(k),
                      "peak_source": peaks["source"] + " (burst copy)",
                      "work_per_launch": b, "ms_per_launch": ms}
            if k == "gram_tc":
                x = cells * 4 * np_                               # packed r written
                out[k]["export_bytes"] = x
                out[k]["frac_incl_export"] = (b + x) / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]
    return out


def run_mraid(args):
    world, rank, local = dist_setup(args)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: a CUDA device is required (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2512_16278_gb300 as m
    from paper_2512_16278_gb300 import build as mbuild
    mbuild.build()
    import synth

    cfg, desc = workload(args.workload, rank, args.n_sub)
    h = torch.empty(cfg.nbytes, dtype=torch.uint8, pin_memory=True)
    synth.generate(cfg, out_ptr=h.data_ptr())
    d = h.to("cuda")
    stream = torch.cuda.Stream()
    N, cells = cfg.n_beam, cfg.n_cells
    with torch.cuda.stream(stream):
        plan = m.Plan(N, cfg.n_chan, cfg.n_samp_sub, cfg.n_sub, stream=stream)
        evals = torch.empty(cells, N, dtype=torch.float32, device="cuda")
        q1 = torch.empty(cells, N, dtype=torch.float32, device="cuda")
        stat = torch.empty(cells, dtype=torch.float32, device="cuda")
        flags = torch.empty(cells, dtype=torch.uint8, device="cuda")
    info = m.FlagInfo()
    # the plan's kernel variants, picked by the autotuner for this shape
    # (cached per shape; tuning runs before and outside the timed region)
    tune_cache = os.path.join(ROOT, "paper_2512_16278_gb300", "_build", "tune.json")
    variants = m.tune(plan.handle, d, N, cfg.n_chan, cfg.n_samp_sub, tune_cache)
    try:  # the tuner's per-variant times for this shape, as recorded in its cache
        with open(tune_cache) as f:
            tune_ms = json.load(f)[m.tune_key(N, cfg.n_chan, cfg.n_samp_sub)].get("ms")
    except (OSError, KeyError, ValueError):
        tune_ms = None

    def step():
        m.mraid_run(plan.handle, d, evals, q1, stat, flags, info)

    for _ in range(max(3, args.warmup)):
        step()
    m.mraid_sync(plan.handle)
    m.mraid_profile_reset(plan.handle)
    m.mraid_profile_enable(plan.handle, True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    m.mraid_sync(plan.handle)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    m.mraid_profile_enable(plan.handle, False)
    prof = m.mraid_profile_read(plan.handle)
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(cells, world, ms)

    # roofline of the dominant kernel (per-launch averages from the events
    # the plan recorded around each launch inside the timed region)
    kt = {k: (n, tot / n) for k, (n, tot) in prof.items() if n > 0}
    launches = sum(n for (n, _) in prof.values())
    dom = max(kt, key=lambda k: kt[k][0] * kt[k][1])
    peaks = measured_peaks()
    roofs = kernel_rooflines(cfg, kt, peaks)
    roof = roofs[dom]
    in_bytes = cfg.n_beam * cfg.n_samp_sub * cells          # samples read once
    out_bytes = cells * (4 + 1 + 8 * N)                     # stat, flag, evals, q1
    path_gbs = (in_bytes + out_bytes) / (ms / 1000.0) / 1e9

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if args.e2e_steps > 0:
        h_flags = torch.empty(cells, dtype=torch.uint8, pin_memory=True)
        h_stat = torch.empty(cells, dtype=torch.float32, pin_memory=True)
        hinfo = m.FlagInfo()
        m.mraid_run_host(plan.handle, h, h_stat, h_flags, hinfo)
        m.mraid_sync(plan.handle)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        steps_ms = []
        for _ in range(args.e2e_steps):
            ts = time.perf_counter()
            m.mraid_run_host(plan.handle, h, h_stat, h_flags, hinfo)
            m.mraid_sync(plan.handle)
            steps_ms.append((time.perf_counter() - ts) * 1000.0)
        te = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist, "cuda")
        # the box's plain host-to-device copy of the same pinned block, for
        # the copy/compute overlap of the host path
        dc = torch.empty_like(d)
        dc.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        tc0 = time.perf_counter()
        dc.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        tcopy = time.perf_counter() - tc0
        del dc
        torch.cuda.empty_cache()
        e2e = {"value": world * cells / te, "unit": UNIT, "h2d_bytes_per_step": cfg.nbytes,
               "d2h_bytes_per_step": cells * 5, "ms_per_step": te * 1000.0,
               "h2d_gbs_achieved": cfg.nbytes / te / 1e9,
               "copy_only_ms": tcopy * 1000.0, "copy_only_gbs": cfg.nbytes / tcopy / 1e9,
               "compute_hidden_frac": max(0.0, min(1.0, (tcopy * 1000.0 + ms - te * 1000.0) / ms)),
               "steps_ms": steps_ms, "steps_median_ms": statistics.median(steps_ms),
               "api": "mraid_run_host (pinned host input, stat + flags copied back)",
               "note": "bound by the host-to-device copy; its rate differs between boxes"}

    cpu = parity = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, sample = cpu_baseline(cfg, h.data_ptr(), args.cpu_seconds)
        parity = sampled_parity(sample, evals, q1, stat)

    # eigenvector refinement (per-beam bits) on the timed run's outputs
    refine = None
    if world == 1:
        W = (N + 31) // 32
        bits = torch.empty(cells, W, dtype=torch.int32, device="cuda")
        ms_b = torch.empty(N, 2, dtype=torch.float64, device="cuda")
        m.mraid_refine(plan.handle, q1, flags, bits, ms_b)
        m.mraid_sync(plan.handle)
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for _ in range(5):
            m.mraid_refine(plan.handle, q1, flags, bits, ms_b)
        r1.record(stream)
        m.mraid_sync(plan.handle)
        refine = {"ms": r0.elapsed_time(r1) / 5,
                  "beam_bits_set": int(sum(bin(int(x) & 0xffffffff).count("1")
                                           for x in bits.view(-1).cpu().tolist()))}
    pol2 = None
    if world == 1 and args.pol2_steps > 0:
        pol2 = bench_pol2(m, torch, h, cfg, stream, args.pol2_steps, peaks)
    bandpass = None
    if world == 1 and args.bandpass_steps > 0 and rank == 0:
        bandpass = bench_bandpass(m, torch, d, cfg, stream, args.bandpass_steps)
    multires = None
    if world == 1 and args.multires_steps > 0:
        multires = bench_multires(m, torch, d, cfg, stream, args.multires_steps, peaks)
    precision = None
    if world == 1 and args.f32_subs > 0:
        precision = bench_f32(m, torch, d, cfg, stream, args.f32_subs, peaks)
    plan.close()
    del d, h
    torch.cuda.empty_cache()
    batched = served = None
    if world == 1 and args.workload == "fast_block" and not args.n_sub:
        if args.batch_steps > 0:
            batched = bench_batched(m, torch, stream, args.batch_steps, peaks)
        if args.serve_seconds > 0:
            served = bench_served(m, torch, args.serve_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8 (exact Gram: f16 tensor cores, FP32 accumulate), f32 eigensolver",
            "data": "synthetic",
            "config": config_dict(cfg, desc, world),
            "hbm": {"path_bytes_per_step": in_bytes + out_bytes, "achieved_gbs": path_gbs,
                    "frac_of_measured": path_gbs / peaks["hbm_gbs"],
                    "frac_of_8tbs_nominal": path_gbs / 8000.0},
            "roofline": roof,
            "rooflines": roofs,
            "kernels_ms_per_launch": {k: v[1] for k, v in kt.items()},
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "sampled_parity": parity,
            "mask": {"flagged_fraction": info.n_flagged / cells, "iterations": info.iterations,
                     "threshold": info.thresh, "n_near": info.n_near},
            "q1_fp64_cells": info.q1_refined,
            "variants": {"gram": variants[0], "eig": variants[1],
                         "eig_name": EIG_NAMES.get(variants[1], "?"), "tune_ms": tune_ms},
            "eig_iterations": {"per_cell": info.jacobi_sweeps / cells,
                               "per_warp": info.jacobi_warp_sweeps / max(1, (cells + 31) // 32),
                               "unit": "QR steps" if variants[1] >= 2 else "Jacobi sweeps"},
            "refine": refine,
            "precision_f32": precision,
            "multires": multires,
            "bandpass": bandpass,
            "pol2": pol2,
            "batched": batched,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_mraid(args)


if __name__ == "__main__":
    sys.exit(main())
