#!/usr/bin/env python
"""Throughput of ball-harmonic subtomogram alignment on GB300: subtomograms aligned per second.

One step = the whole hot path over one batch of synthetic subtomograms already resident in HBM:
expansion of every subtomogram into ball-harmonic coefficients (bh_expand) + multi-start marching
gradient ascent over SO(3) with selection (bh_align_batch) + the FP64 re-score of the best starts
(bh_refine_fp64).  The template's coefficients are computed once before timing and stay resident.

Default workload (the precision form): 4096 distinct subtomograms of 64^3 (200-blob template, SNR 0.05,
+-60 deg missing wedge), l <= 32, lambda <= 32 pi, marching 4 -> 8 -> 16 -> 32, 32 starts, 30 steps per
band, BF16 hi/lo tensor-core expansion with FP32 accumulation, FP32 ascent, FP64 re-score of the 4 best
starts.  The plain FP32 form (FP32 expansion GEMM + FP32 ascent) is timed in the same run and reported
beside it with the median angle between the two forms' rotations.  Extra keys: the 1024 x 32^3 batch
(`batch32`, with the paper's Sec. III protocol and the missing-wedge constrained ascent), the mixed
batch in one CUDA graph (`mixed`) and the serving loop (`serving`, `serving_newton`).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
        (N > 1 is launched by torch.distributed.run: one independent replica per GPU, weak scaling.)
        python bench.py --profile-align ...   one kernel variant of the ascent alone, on a plan without the
                                              expansion table (small device footprint, for ncu captures)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "subtomograms aligned/s at <=1 deg median angle error vs plain FP32; p50/p99 latency"
UNIT = "subtomograms/s"
HEADLINE = "precision64"
L2_FLUSH_BYTES = 256 << 20
FMA_LANES = 128  # FP32 FMA lanes per SM (4 schedulers x 32)


def source_sha(text: str) -> str:
    """Hash of C++/CUDA source with its comments and blank lines removed (a comment edit keeps the hash)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()[:16]


def align_source_sha() -> str:
    """Hash of the alignment kernels' source: a stored ncu traffic figure is used only while it matches."""
    with open(os.path.join(ROOT, "paper_2509_01180_gb300", "csrc", "align.cu")) as f:
        return source_sha(f.read())


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the ascent kernel from an ncu
# capture, by (workload, lanes per start, starts per thread, orbit dealing): (bytes, subtomograms in the
# captured launch, source_sha of the align.cu it was taken on).  A capture of a smaller batch is scaled by
# the subtomogram count (the kernel reads each subtomogram's coefficients and starts once); the figure is
# used only while the hash matches.
ALIGN_TRAFFIC_BYTES = {
    ("precision64", 16, 2, 2): (194_948_352 + 3_172_352, 1024, "ef459484c605ecea"),
}


def describe(w) -> str:
    m = w.meta
    parts = [f"{w.B} x {w.N}^3 subtomograms", f"{m['blobs']}-blob template sigma {m['sigma']}"]
    if m["snr"] is not None:
        parts.append(f"SNR {m['snr']}")
    if m["wedge_deg"] is not None:
        parts.append(f"+-{m['wedge_deg']:.0f} deg wedge")
    parts += [f"l<={w.Lmax}", f"lambda<={w.N // 2}pi", "marching " + "-".join(map(str, w.stages)),
              f"{w.S} starts", f"{w.steps} steps"]
    return ", ".join(parts)


def orbit_steps(L: int) -> int:
    """Orbit-steps of one score+gradient evaluation at band L: sum_{m<=L} (2m+1)(L-m+1)."""
    return sum((2 * m + 1) * (L - m + 1) for m in range(L + 1))


# FP32 flop accounting of the alignment kernel (FMA = 2 flop), per score+gradient evaluation at band L:
#   each orbit-step (one l of one (m,n) orbit): t 2, g 4, e-recursion 3, e'-recursion 5, 8 accumulating
#   FMAs 16 -> 30 flop;  each orbit ((L+1)^2 of them): seed and derivative seed 10, phases and the four
#   sums 36 -> 46 flop.
FLOP_PER_ORBIT_STEP = 30
FLOP_PER_ORBIT = 46


def eval_flops(L: int) -> int:
    return FLOP_PER_ORBIT_STEP * orbit_steps(L) + FLOP_PER_ORBIT * (L + 1) ** 2


def align_flops(w) -> float:
    """FP32 flop of one ascent launch on the workload: every start runs (1 + steps) evaluations per stage."""
    per_start = sum((1 + w.steps) * eval_flops(L) for L in w.stages)
    return float(w.B) * w.S * per_start


def fp32_peak_tflops(device, peaks: dict) -> tuple[float, str]:
    """FP32 FMA peak from unit counts and the maximum SM clock: SMs x 128 lanes x 2 flop x clock."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = peaks.get("sm_max_mhz") or 2070.0
    return sms * FMA_LANES * 2 * mhz / 1e6, f"FP32 FMA: {sms} SMs x {FMA_LANES} lanes x 2 flop x {mhz:.0f} MHz"


class ClockSampler:
    """nvidia-smi samples (SM clock, reasons) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------------------------------------ CPU oracle
def _oracle_start(args):
    """One start's marching ascent in FP64 (oracle), for the process pool."""
    xi, q0, stages, steps = args
    from oracle import align
    return align.ascend(xi, q0, stages, steps).score


def _oracle_warm(_):
    from oracle import align  # noqa: F401
    return 0


def oracle_pool(n):
    import multiprocessing as mp
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    return mp.get_context("spawn").Pool(n)


def cpu_workers(cap: int = 1 << 30) -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    return max(1, min(n, cap))


def oracle_batch(pool, Bs, w, idx, t_hat) -> None:
    """The oracle's work for the subtomograms `idx`: one expansion call over their volumes (Sec. II-A), then for
    each of them every start's marching ascent (spread over the pool) and the selection."""
    import numpy as np
    from oracle import align, ball
    F = ball.expand(Bs, w.vols[list(idx)].astype(np.float64))
    for j, b in enumerate(idx):
        xi = align.build_xi(Bs, t_hat, F[j], max(w.stages))
        jobs = [(xi, w.starts[b, s].astype(np.float64), w.stages, w.steps) for s in range(w.S)]
        align.select_best(np.array(pool.map(_oracle_start, jobs)))


def cpu_baseline(w, n_particles: int) -> dict:
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the same workload: the first
    n_particles subtomograms (the template is expanded first, untimed, as on the GPU side)."""
    import numpy as np
    from oracle import ball
    Bs = ball.make_basis(w.Lmax, w.lam_max)
    workers = cpu_workers(w.S)
    with oracle_pool(workers) as pool:
        pool.map(_oracle_warm, range(workers))
        t_hat = ball.expand(Bs, w.template.astype(np.float64))[0]
        t0 = time.perf_counter()
        oracle_batch(pool, Bs, w, range(n_particles), t_hat)
        dt = time.perf_counter() - t0
    return {"value": n_particles / dt, "unit": UNIT, "cores": workers, "kind": "oracle", "seconds": dt,
            "sample": f"the first {n_particles} subtomograms of the workload ({w.N}^3, l<={w.Lmax}): one FP64 oracle "
                      f"expansion call over their volumes, then every subtomogram's {w.S} starts x marching "
                      f"{'-'.join(map(str, w.stages))} x {w.steps} steps over {workers} processes + selection; "
                      f"numpy/scipy FP64"}


# ------------------------------------------------------------------------------------------ arms
def run_reference(args, rank, world):
    """The oracle as the reference arm, on the host cores: W untimed warm-up subtomograms (ascents only), then
    the K timed ones -- one oracle expansion call over their volumes plus every start's ascent and the
    selection -- on the same workload, metric and unit as the GPU arm."""
    from paper_2509_01180_gb300 import synth
    if rank != 0:
        return None
    import numpy as np
    from oracle import align, ball
    K, W = args.steps, args.warmup
    w = synth.make_workload(args.workload, count=K + W, workers=cpu_workers(16))
    Bs = ball.make_basis(w.Lmax, w.lam_max)
    workers = cpu_workers(w.S)
    with oracle_pool(workers) as pool:
        pool.map(_oracle_warm, range(workers))
        t_hat = ball.expand(Bs, w.template.astype(np.float64))[0]
        xi_t = align.build_xi(Bs, t_hat, t_hat, max(w.stages))
        for b in range(W):  # warm-up: the ascents of the warm-up subtomograms' starts against the template
            pool.map(_oracle_start, [(xi_t, w.starts[b, s].astype(np.float64), w.stages, w.steps) for s in range(w.S)])
        t0 = time.perf_counter()
        oracle_batch(pool, Bs, w, range(W, W + K), t_hat)
        dt = time.perf_counter() - t0
    value = K / dt
    desc = describe(synth.make_workload(args.workload, count=1)).replace("1 x", f"per step 1 of the {K} timed")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * dt / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "parallelism": "host processes"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"{K} subtomograms: one FP64 oracle expansion call over their volumes, then "
                                       f"each one's {w.S} starts' ascents over {workers} processes + selection"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


_T0 = time.perf_counter()


def progress(msg: str) -> None:
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def make_workload(args, name: str, count: int, first: int = 0):
    """The workload's subtomograms (distinct unless --distinct asks for fewer, then tiled), rendered by a
    pool of spawned processes."""
    import numpy as np
    from paper_2509_01180_gb300 import synth
    distinct = args.distinct if (args.distinct and args.distinct < count) else 0
    w = synth.make_workload(name, count=distinct or count, first=first, workers=cpu_workers(16))
    if distinct:
        rep = np.arange(count) % distinct
        w.vols, w.q_true, w.starts = (np.ascontiguousarray(w.vols[rep]), w.q_true[rep],
                                      np.ascontiguousarray(w.starts[rep]))
    w.meta["distinct"] = distinct or count
    return w


def run_workload(args, w, rank, world, device, *, refine: int, sec3: bool, wedge: bool, sec3_starts: int):
    """Time the step on workload w in each requested form; returns {form: results}."""
    import numpy as np
    import torch

    from paper_2509_01180_gb300 import bh, replicas
    B = w.B
    forms = {"bf16split": bh.BH_MODE_BF16_SPLIT, "fp32": bh.BH_MODE_FP32}
    order = [args.form] if args.form != "both" else ["bf16split", "fp32"]
    stream = torch.cuda.current_stream(device)
    vols = torch.from_numpy(w.vols).to(device)
    starts = torch.from_numpy(w.starts).to(device)
    tvol = torch.from_numpy(w.template[None]).to(device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    steps, L_last = args.steps, w.stages[-1]
    results = {}
    for name in order:
        t0 = time.perf_counter()
        plan = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, forms[name], max_batch=min(B, 4096))
        plan_s = time.perf_counter() - t0
        progress(f"{w.name} {name}: plan {plan_s:.1f} s")
        if args.no_autotune:
            tune = {"align_group": args.group, "align_starts_per_thread": args.starts_per_thread, "gemm_bn": 128,
                    "align_dealing": args.dealing}
        else:
            tune = bh.bh_autotune(plan, B, w.S, w.stages, w.steps)  # picks kernel variants (untimed setup)
        grp = args.group if args.no_autotune else 0
        spt = args.starts_per_thread if args.no_autotune else 0
        dea = args.dealing if args.no_autotune else 0
        tmpl = bh.bh_expand(plan, tvol)[0].contiguous()
        coeffs = torch.empty((B, plan.Nb, 2), dtype=torch.float32, device=device)
        quat = torch.empty((B, 4), dtype=torch.float32, device=device)
        score = torch.empty((B,), dtype=torch.float32, device=device)
        sq = torch.empty((B, w.S, 4), dtype=torch.float32, device=device) if refine else None
        ss = torch.empty((B, w.S), dtype=torch.float32, device=device) if refine else None

        def ascend():
            if refine:  # per-start outputs feed the FP64 re-score of the best `refine` starts
                o = bh.AlignOpts()
                o.group, o.starts_per_thread, o.dealing = grp, spt, dea
                o.start_quat_out, o.start_score_out = sq.data_ptr(), ss.data_ptr()
                st = (bh.ctypes.c_int * len(w.stages))(*w.stages)
                bh._check(bh.lib().bh_align_batch(plan.handle, tmpl.data_ptr(), coeffs.data_ptr(), B,
                                                  starts.data_ptr(), w.S, st, len(w.stages), w.steps,
                                                  quat.data_ptr(), score.data_ptr(), bh.ctypes.byref(o),
                                                  stream.cuda_stream), "bh_align_batch")
            else:
                bh.bh_align_batch(plan, tmpl, coeffs, starts, w.stages, w.steps, quat_out=quat, score_out=score,
                                  stream=stream, group=grp, starts_per_thread=spt, dealing=dea)

        def rescore():
            if refine:
                bh.bh_refine_fp64(plan, tmpl, coeffs, sq, ss, L_last, refine, quat_out=quat, score_out=score,
                                  stream=stream)

        def step(v, ev=None):
            if ev:
                ev[0].record(stream)
            bh.bh_expand(plan, v, coeffs, stream=stream)
            if ev:
                ev[1].record(stream)
            ascend()
            if ev:
                ev[2].record(stream)
            rescore()
            if ev:
                ev[3].record(stream)

        for _ in range(args.warmup):
            step(vols)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        torch.cuda.synchronize(device)
        replicas.barrier()
        torch.cuda.synchronize(device)
        with ClockSampler(device.index if device.index is not None else 0) as clk:
            for k in range(steps):
                step(vols, ev[k])
                flush.zero_()  # evict L2 between timed steps (not timed)
            torch.cuda.synchronize(device)
        replicas.barrier()
        t_exp = sum(e[0].elapsed_time(e[1]) for e in ev)
        t_aln = sum(e[1].elapsed_time(e[2]) for e in ev)
        t_ref = sum(e[2].elapsed_time(e[3]) for e in ev)
        t_tot = t_exp + t_aln + t_ref
        t_tot, t_exp, t_aln, t_ref = replicas.max_over_ranks([t_tot, t_exp, t_aln, t_ref], device)
        q_res = quat.cpu().numpy().astype(np.float64)

        # end to end through the public API: every step copies its volumes from pinned host memory and
        # reads its rotations and scores back.  Three device input buffers: the copies of steps k+1 and
        # k+2 (copy stream) overlap the expansion and alignment of step k (compute stream), so that a host
        # copy slowed by other traffic on the host (measured: most 4.3 GB copies take 20 ms, a few up to
        # 190 ms) still finishes before its step; a buffer is refilled only after the expansion that read
        # it has finished.  Timed from the first timed copy to the last read-back.
        hv = torch.from_numpy(w.vols).pin_memory()
        hq = [torch.empty((B, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
        hs = [torch.empty((B,), dtype=torch.float32).pin_memory() for _ in range(2)]
        dv = [vols, torch.empty_like(vols), torch.empty_like(vols)]
        cstream = torch.cuda.Stream(device)
        copied = [torch.cuda.Event() for _ in range(3)]
        consumed = [None, None, None]
        t_first = torch.cuda.Event(enable_timing=True)
        t_last = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        for k in range(args.warmup + steps):
            j = k % 3
            if k == args.warmup:
                # the warm-up steps drain first, so that the timed window holds exactly the timed steps
                # (their first copy is then not overlapped: the pipeline fills inside the window)
                torch.cuda.synchronize(device)
                t_first.record(cstream)
            if consumed[j] is not None:
                cstream.wait_event(consumed[j])
            with torch.cuda.stream(cstream):
                dv[j].copy_(hv, non_blocking=True)
            copied[j].record(cstream)
            stream.wait_event(copied[j])
            bh.bh_expand(plan, dv[j], coeffs, stream=stream)
            consumed[j] = torch.cuda.Event()
            consumed[j].record(stream)
            ascend()
            rescore()
            hq[k % 2].copy_(quat, non_blocking=True)
            hs[k % 2].copy_(score, non_blocking=True)
        t_last.record(stream)
        torch.cuda.synchronize(device)
        e2e_ms = replicas.max_over_ranks([t_first.elapsed_time(t_last)], device)[0]
        del dv[1:]
        progress(f"{w.name} {name}: timed {t_tot / steps:.2f} ms/step, e2e {e2e_ms / steps:.2f} ms/step")
        sec3_res = sec3_leg(args, w, plan, tmpl, vols, coeffs, stream, flush, device, sec3_starts, refine) if (
            name == "bf16split" and sec3) else None
        wedge_res = wedge_leg(args, w, plan, tmpl, vols, coeffs, stream, flush, device) if (
            name == "bf16split" and wedge) else None
        band_res = band_leg(args, w, plan, tmpl, vols, coeffs, stream, flush, device, refine, tune) if (
            name == "bf16split" and args.band_leg) else None
        results[name] = {"refine": refine, "wedge": wedge_res, "sec3": sec3_res, "bands": band_res, "plan_s": plan_s, "tune": tune, "t_tot": t_tot,
                         "t_exp": t_exp, "t_aln": t_aln, "t_ref": t_ref, "q": q_res, "clocks": clk.summary(),
                         "e2e_ms": e2e_ms, "Nb": plan.Nb, "V": plan.V, "gemm_K": plan.gemm_K, "gemm_N": plan.gemm_N,
                         "passes": -(-B // plan.max_batch),
                         "h2d": int(hv.numel() * 4), "d2h": int(hq[0].numel() * 4 + hs[0].numel() * 4)}
        plan.destroy()
        del coeffs, hv
        torch.cuda.empty_cache()
    return results


def summarize(args, w, res, world, device) -> dict:
    """The JSON fields of one workload: throughput of the chosen form, its breakdown, the roofline of its
    dominant kernel (CUDA-event durations of that kernel's launches in the timed steps), end-to-end
    throughput, the plain FP32 form and accuracies."""
    import numpy as np
    steps = args.steps
    main_form = "bf16split" if "bf16split" in res else next(iter(res))
    r = res[main_form]
    B = w.B
    refine = r.get("refine", 0)
    peaks = measured_peaks()
    per = {"expand": r["t_exp"] / steps, "align": r["t_aln"] / steps, "rescore_fp64": r["t_ref"] / steps}
    fp32_pk, fp32_src = fp32_peak_tflops(device, peaks)
    # expansion: the octant-folded GEMM does 2 K Nb multiply-add flop per volume (K = fundamental voxels),
    # executed as three BF16 products over the padded shape (K x gemm_N) in the split form; the unfolded
    # dense contraction it replaces would be 2 V Nb
    mult = 3 if main_form == "bf16split" else 1
    t_exp = per["expand"] / 1e3
    fl_exp = 2.0 * B * r["gemm_K"] * r["Nb"]
    fl_exec = 2.0 * B * r["gemm_K"] * r["gemm_N"] * mult
    pk_exp = peaks.get("bf16_tflops", 1900.0) if mult == 3 else fp32_pk
    roof_exp = {"kernel": "bh_expand (octant projection + folded GEMM + complex)",
                "bound": "tensor" if mult == 3 else "alu",
                "achieved": fl_exp / t_exp / 1e12, "executed": fl_exec / t_exp / 1e12,
                "dense_equivalent": 2.0 * B * r["V"] * r["Nb"] / t_exp / 1e12, "unit": "TFLOP/s", "peak": pk_exp,
                "traffic": None,
                "peak_source": ("MEASURED_PEAKS bf16_tflops (burst), of measured" if mult == 3 else fp32_src)}
    roof_exp["frac"] = roof_exp["achieved"] / pk_exp
    roof_exp["frac_executed"] = roof_exp["executed"] / pk_exp
    tuned = (r["tune"]["align_group"], r["tune"]["align_starts_per_thread"], r["tune"].get("align_dealing", 1))
    ach = align_flops(w) / (per["align"] / 1e3) / 1e12
    tr = ALIGN_TRAFFIC_BYTES.get((w.name,) + tuned)
    traffic = None
    if tr is not None and tr[2] == align_source_sha():
        traffic = tr[0] * B / tr[1]
    kname = "k_align_flat" if tuned[2] == 2 else ("k_align_c" if tuned[1] == 2 else "k_align")
    roof_aln = {"kernel": f"{kname} (marching ascent, {tuned[0]} lanes x {tuned[1]} starts per thread, "
                          f"{'flat' if tuned[2] == 2 else 'row'} orbit dealing)",
                "bound": "alu", "achieved": ach, "peak": fp32_pk, "unit": "TFLOP/s", "frac": ach / fp32_pk,
                "traffic": traffic, "traffic_algorithmic": float(B) * r["Nb"] * 8 + float(B) * w.S * 16,
                "flop_per_launch": align_flops(w), "ms_per_launch": per["align"],
                "peak_source": fp32_src + " (nominal; no FP32 figure in MEASURED_PEAKS)"}
    roof = roof_aln if per["align"] >= per["expand"] else roof_exp
    line = {
        "value": world * B / (r["t_tot"] / steps / 1e3), "unit": UNIT, "ms_per_step": r["t_tot"] / steps,
        "dtype": ("bf16-split/fp32" if main_form == "bf16split" else "fp32") + ("+fp64-rescore" if refine else ""),
        "data": "synthetic" + (f" ({w.meta['distinct']} distinct phantoms tiled to {B})"
                               if w.meta.get("distinct", B) < B else f" ({B} distinct phantoms)"),
        "config": {"workload": describe(w), "form": main_form,
                   "expansion": "tcgen05 BF16 hi/lo split, FP32 accumulate" if main_form == "bf16split"
                   else "FP32 FFMA", "ascent": "FP32",
                   "fp64_rescore_top_k": refine,
                   "l2": "flushed between timed steps (256 MB write); inputs larger than L2",
                   "template": "expanded once before timing (resident)",
                   "autotuned": {"align_lanes_per_group": tuned[0], "align_starts_per_thread": tuned[1],
                                 "align_orbit_dealing": "flat" if tuned[2] == 2 else "row",
                                 "gemm_n_tile": r["tune"]["gemm_bn"]},
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "breakdown_ms_per_step": dict(per, plan_create_s=r["plan_s"]),
        "roofline": roof,
        "roofline_align": roof_aln,
        "roofline_expand": roof_exp,
        "clocks": r["clocks"],
        "e2e": {"value": world * B / (r["e2e_ms"] / steps / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": steps * (3 * r["passes"] + 1 + (1 if refine else 0)),
    }
    qt_inv = w.q_true * np.array([1, -1, -1, -1])
    ang = angle_deg(r["q"], qt_inv)
    acc = {"median_angle_vs_truth_deg": float(np.median(ang)), "frac_within_2deg_of_truth": float(np.mean(ang < 2.0))}
    if "fp32" in res and main_form != "fp32":
        f = res["fp32"]
        acc["median_angle_vs_fp32_deg"] = float(np.median(angle_deg(r["q"], f["q"])))
        acc["max_angle_vs_fp32_deg"] = float(np.max(angle_deg(r["q"], f["q"])))
        line["plain_fp32"] = {"value": world * B / (f["t_tot"] / steps / 1e3), "ms_per_step": f["t_tot"] / steps,
                              "breakdown_ms_per_step": {"expand": f["t_exp"] / steps, "align": f["t_aln"] / steps,
                                                        "rescore_fp64": f["t_ref"] / steps},
                              "median_angle_vs_truth_deg": float(np.median(angle_deg(f["q"], qt_inv)))}
    line["accuracy"] = acc
    if r.get("wedge"):
        wl = dict(r["wedge"])
        qw = wl.pop("q")
        if "fp32" in res:
            wl["median_angle_vs_fp32_deg"] = float(np.median(angle_deg(qw, res["fp32"]["q"])))
        line["wedge_constrained"] = wl
    if r.get("bands"):
        bl = dict(r["bands"])
        qb = bl.pop("q")
        if "fp32" in res:
            bl["median_angle_vs_fp32_deg"] = float(np.median(angle_deg(qb, res["fp32"]["q"])))
            bl["frac_within_1deg_of_fp32"] = float(np.mean(angle_deg(qb, res["fp32"]["q"]) < 1.0))
        line["band_choice"] = bl
    if r.get("sec3"):
        s3 = dict(r["sec3"])
        q3 = s3.pop("q")
        if "fp32" in res:
            s3["median_angle_vs_fp32_deg"] = float(np.median(angle_deg(q3, res["fp32"]["q"])))
        line["sec3_protocol"] = s3
    return line


def profile_align(args, device) -> dict:
    """Ascent (or Newton) variants alone on a plan without the expansion table, for sweeps and ncu captures:
    the subtomograms are expanded with a full plan that is destroyed before the matching launches, so the
    device holds only the coefficients and starts while they run."""
    import torch

    from paper_2509_01180_gb300 import bh
    w = make_workload(args, args.workload, args.count or 512)
    stream = torch.cuda.current_stream(device)
    plan = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_BF16_SPLIT, max_batch=min(w.B, 1024))
    vols = torch.from_numpy(w.vols).to(device)
    tmpl = bh.bh_expand(plan, torch.from_numpy(w.template[None]).to(device))[0].contiguous()
    coeffs = bh.bh_expand(plan, vols)
    torch.cuda.synchronize(device)
    plan.destroy()
    del vols
    torch.cuda.empty_cache()
    plan = bh.bh_plan_create(w.N, w.Lmax, w.lam_max, bh.BH_MODE_BF16_SPLIT, flags=bh.BH_PLAN_MATCH_ONLY)
    starts = torch.from_numpy(w.starts).to(device)
    quat = torch.empty((w.B, 4), dtype=torch.float32, device=device)
    score = torch.empty((w.B,), dtype=torch.float32, device=device)
    fl = align_flops(w)
    pk, src = fp32_peak_tflops(device, measured_peaks())
    def parse(v):  # "GxC" (row dealing) or "GxCf" (flat dealing); "nG" / "nGf": Newton steps, G lanes per start
        flat = v.endswith("f")
        v = v.rstrip("f")
        if v.startswith("n"):
            return int(v[1:]), 1, 2 if flat else 1, True
        G, C = (int(x) for x in v.split("x"))
        return G, C, 2 if flat else 1, False
    variants = [parse(v) for v in args.variants.split(",")] if args.variants else \
        [(args.group, args.starts_per_thread, args.dealing, False)]
    # Newton variants start from the first 8 of each subtomogram's starts, args.sec3_steps iterations per band
    # (the Sec. III leg's shape: 8 candidate starts at 64^3)
    nstarts = starts[:, :8].contiguous()
    out = []
    for G, C, D, newton in variants:
        try:
            def run():
                if newton:
                    bh.bh_align_batch(plan, tmpl, coeffs, nstarts, w.stages, args.sec3_steps, quat_out=quat,
                                      score_out=score, group=G, dealing=D, newton=True, stream=stream)
                    return
                bh.bh_align_batch(plan, tmpl, coeffs, starts, w.stages, w.steps, quat_out=quat, score_out=score,
                                  group=G, starts_per_thread=C, dealing=D, stream=stream)
            for _ in range(args.warmup):
                run()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            ev[0].record(stream)
            for k in range(args.steps):
                run()
                ev[k + 1].record(stream)
            torch.cuda.synchronize(device)
        except bh.BHError as e:
            out.append({"lanes": G, "starts_per_thread": C, "dealing": D, "newton": newton, "error": str(e)})
            continue
        ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        avg = sum(ms) / len(ms)
        rec = {"lanes": G, "starts_per_thread": C, "dealing": "flat" if D == 2 else "row", "ms_per_launch": ms}
        if newton:
            rec.update({"newton": True, "starts": 8, "steps_per_band": args.sec3_steps})
        else:
            rec.update({"achieved_tflops": fl / (avg / 1e3) / 1e12, "frac": fl / (avg / 1e3) / 1e12 / pk})
        out.append(rec)
    plan.destroy()
    return {"profile": "k_align", "workload": describe(w), "flop_per_launch": fl, "peak_tflops": pk,
            "peak_source": src, "align_src_sha": align_source_sha(), "variants": out}


def sec3_leg(args, w, plan, tmpl, vols, coeffs, stream, flush, device, S: int, refine: int) -> dict:
    """The paper's own protocol (Sec. III) on the same batch: expansion, candidate starts from the local maxima
    of the lowest marching band on a super-Fibonacci rotation grid, then damped Newton steps through the
    marching bands.  Timed with CUDA events like the main leg (L2 flushed between steps)."""
    import numpy as np
    import torch

    from paper_2509_01180_gb300 import bh, replicas, synth
    B = w.B
    n_grid, radius = args.sec3_grid, math.radians(args.sec3_radius)
    grid = bh.bh_grid_create(synth.super_fibonacci(n_grid), radius)
    tune = bh.bh_autotune_newton(plan, B, S, w.stages, args.sec3_steps) if not args.no_autotune else None
    cst = torch.empty((B, S, 4), dtype=torch.float32, device=device)
    quat = torch.empty((B, 4), dtype=torch.float32, device=device)
    score = torch.empty((B,), dtype=torch.float32, device=device)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        bh.bh_expand(plan, vols, coeffs, stream=stream)
        if ev:
            ev[1].record(stream)
        bh.bh_candidates(plan, grid, tmpl, coeffs, w.stages[0], S, starts_out=cst, stream=stream)
        if ev:
            ev[2].record(stream)
        bh.bh_align_batch(plan, tmpl, coeffs, cst, w.stages, args.sec3_steps, quat_out=quat, score_out=score,
                          stream=stream, newton=True, refine_fp64=min(refine, S))
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    steps = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    torch.cuda.synchronize(device)
    replicas.barrier()
    for k in range(steps):
        step(evs[k])
        flush.zero_()
    torch.cuda.synchronize(device)
    replicas.barrier()
    t = [sum(e[i].elapsed_time(e[i + 1]) for e in evs) for i in range(3)]
    t = replicas.max_over_ranks(t, device)
    q = quat.cpu().numpy().astype(np.float64)
    qt_inv = w.q_true * np.array([1, -1, -1, -1])
    ang = angle_deg(q, qt_inv)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    grid.destroy()
    return {"q": q, "value": world * B / (sum(t) / steps / 1e3), "unit": UNIT, "ms_per_step": sum(t) / steps,
            "breakdown_ms_per_step": {"expand": t[0] / steps, "candidates": t[1] / steps, "newton": t[2] / steps},
            "median_angle_vs_truth_deg": float(np.median(ang)), "frac_within_2deg": float(np.mean(ang < 2.0)),
            "config": {"grid": f"super-Fibonacci {n_grid} rotations, neighbour radius {args.sec3_radius:g} deg",
                       "candidate_band": w.stages[0], "candidates": S, "newton_steps_per_band": args.sec3_steps,
                       "bands": w.stages, "fp64_rescore_top_k": min(refine, S),
                       "newton_lanes_per_start": tune["newton_group"] if tune else "default",
                       "newton_orbit_dealing": ({1: "row", 2: "flat"}.get(tune["newton_dealing"]) if tune else "row")},
            "gpu_launches_per_step": 3 * math.ceil(B / min(B, 4096)) + 3 + 1 + (1 if min(refine, S) else 0)}


# energy-ratio thresholds of the band-choice leg, one per band of the fixed schedule (box edge -> thresholds):
# at these values the chosen first bands sit near the fixed schedule's first bands on the synthetic workloads,
# and the last band is where the cross-correlation energy left above it falls below the last threshold
BAND_THRESHOLDS = {32: (0.05, 0.01, 0.001), 64: (0.02, 0.01, 0.001, 0.0001)}


def band_leg(args, w, plan, tmpl, vols, coeffs, stream, flush, device, refine: int, tune) -> dict:
    """Marching bands chosen per subtomogram by the energy ratio (Fig. 1; Sec. III picks its L_set with it)
    instead of the fixed schedule: expansion + bh_choose_bands + the ascent on each subtomogram's own bands
    (+ the FP64 re-score at its own last band), timed like the main leg."""
    import numpy as np
    import torch

    from paper_2509_01180_gb300 import bh, replicas
    B = w.B
    thr = BAND_THRESHOLDS.get(w.N, (0.05, 0.01, 0.001))
    starts = torch.from_numpy(w.starts).to(device)
    quat = torch.empty((B, 4), dtype=torch.float32, device=device)
    score = torch.empty((B,), dtype=torch.float32, device=device)
    tab = torch.empty((B, bh.BH_STAGE_ROW), dtype=torch.int32, device=device)
    L_min = 2

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        bh.bh_expand(plan, vols, coeffs, stream=stream)
        if ev:
            ev[1].record(stream)
        bh.bh_choose_bands(plan, tmpl, coeffs, w.Lmax, thr, L_min=L_min, stage_table=tab, stream=stream)
        if ev:
            ev[2].record(stream)
        bh.bh_align_batch(plan, tmpl, coeffs, starts, w.stages, w.steps, quat_out=quat, score_out=score,
                          stream=stream, stage_table=tab, refine_fp64=refine)
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    steps = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    torch.cuda.synchronize(device)
    replicas.barrier()
    for k in range(steps):
        step(evs[k])
        flush.zero_()
    torch.cuda.synchronize(device)
    replicas.barrier()
    t = [sum(e[i].elapsed_time(e[i + 1]) for e in evs) for i in range(3)]
    t = replicas.max_over_ranks(t, device)
    q = quat.cpu().numpy().astype(np.float64)
    rows = bh.stage_rows(tab)
    hist = {}
    for r in rows:
        k = "-".join(map(str, r))
        hist[k] = hist.get(k, 0) + 1
    ang = angle_deg(q, w.q_true * np.array([1, -1, -1, -1]))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    top = sorted(hist.items(), key=lambda kv: -kv[1])[:6]
    return {"q": q, "value": world * B / (sum(t) / steps / 1e3), "unit": UNIT, "ms_per_step": sum(t) / steps,
            "breakdown_ms_per_step": {"expand": t[0] / steps, "choose_bands": t[1] / steps,
                                      "align" + ("+rescore_fp64" if refine else ""): t[2] / steps},
            "median_angle_vs_truth_deg": float(np.median(ang)), "frac_within_2deg": float(np.mean(ang < 2.0)),
            "config": {"thresholds": list(thr), "L_min": L_min, "degrees_counted": w.Lmax,
                       "fixed_schedule": w.stages, "schedules_most_common": dict(top),
                       "distinct_schedules": len(hist), "mean_last_band": float(np.mean([r[-1] for r in rows])),
                       "fp64_rescore_top_k": refine},
            "gpu_launches_per_step": 3 * math.ceil(B / plan.max_batch) + 2 + (1 if refine else 0)}


def wedge_leg(args, w, plan, tmpl, vols, coeffs, stream, flush, device) -> dict:
    """Missing-wedge constrained correlation (Sec. II-B) on the same batch: expansion + the constrained
    ascent (same starts, bands and steps as the main leg) with the data's own tilt half-angle."""
    import numpy as np
    import torch

    from paper_2509_01180_gb300 import bh, replicas
    B = w.B
    t0 = time.perf_counter()
    wd = bh.bh_wedge_create(plan, w.template, float(w.meta["wedge_deg"]), w.stages[-1])
    prep_s = time.perf_counter() - t0
    starts = torch.from_numpy(w.starts).to(device)
    quat = torch.empty((B, 4), dtype=torch.float32, device=device)
    score = torch.empty((B,), dtype=torch.float32, device=device)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        bh.bh_expand(plan, vols, coeffs, stream=stream)
        if ev:
            ev[1].record(stream)
        bh.bh_align_batch(plan, tmpl, coeffs, starts, w.stages, w.steps, quat_out=quat, score_out=score,
                          stream=stream, wedge=wd)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    steps = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    torch.cuda.synchronize(device)
    replicas.barrier()
    for k in range(steps):
        step(evs[k])
        flush.zero_()
    torch.cuda.synchronize(device)
    replicas.barrier()
    t = [sum(e[i].elapsed_time(e[i + 1]) for e in evs) for i in range(2)]
    t = replicas.max_over_ranks(t, device)
    q = quat.cpu().numpy().astype(np.float64)
    ang = angle_deg(q, w.q_true * np.array([1, -1, -1, -1]))
    wd.destroy()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return {"q": q, "value": world * B / (sum(t) / steps / 1e3), "unit": UNIT, "ms_per_step": sum(t) / steps,
            "breakdown_ms_per_step": {"expand": t[0] / steps, "constrained_align": t[1] / steps},
            "median_angle_vs_truth_deg": float(np.median(ang)), "frac_within_2deg": float(np.mean(ang < 2.0)),
            "config": {"wedge_half_angle_deg": float(w.meta["wedge_deg"]), "norm_band": w.stages[-1],
                       "norm_prepare_s": prep_s, "starts": w.S, "steps": w.steps, "bands": w.stages},
            "gpu_launches_per_step": 3 * math.ceil(B / min(B, 4096)) + 1}


def serving_leg(seconds: float, rate: float = 200.0, seed: int = 2509, newton: bool = False, piece: int = 0) -> dict:
    """Continuous-batching server under a Poisson stream of requests (mean `rate` req/s for `seconds`):
    1-512 subtomograms per request (log-uniform), box edge uniform over {24, 32, 48, 64}, one of 8 resident
    templates (2 per box), 16 starts, bands N/8 -> N/4 -> N/2, 30 steps; noise (SNR 0.1) and a +-60 deg
    wedge as in the batch workload.  Volumes come from a pool of 64 distinct phantoms per box (tiled to
    512) so that host memory stays bounded; the arithmetic per subtomogram is the same."""
    import numpy as np

    from paper_2509_01180_gb300 import bh, synth
    rng = np.random.default_rng(seed)
    boxes = [24, 32, 48, 64]
    t_setup = time.perf_counter()
    srv = bh.bh_serve_create(hbm_budget_bytes=48 << 30, max_inflight=4, max_batch=2048,
                             mode=bh.BH_MODE_BF16_SPLIT, steps=8 if newton else 30, newton=newton, piece=piece)
    tids, pools = {}, {}
    for N in boxes:
        tpls = [synth.blob_template(synth.rng_for(40 + N, t), 60, 1.5 * N / 32, 0.75 * N / 2) for t in range(2)]
        for t, tpl in enumerate(tpls):
            tids[(N, t)] = srv.add_template(synth.render(N, tpl).astype(np.float32))
        base = np.stack([synth.degrade(synth.render(N, tpls[j % 2], synth.uniform_quaternions(synth.rng_for(60 + N, j), 1)[0]),
                                       synth.rng_for(70 + N, j), 0.1, 60.0) for j in range(64)]).astype(np.float32)
        pools[N] = np.ascontiguousarray(np.tile(base, (8, 1, 1, 1)))
    for N in boxes:  # first use of every plan and kernel variant
        srv.wait(srv.submit(tids[(N, 0)], pools[N][:4], 16, seed=1), timeout_ms=600000)
    setup_s = time.perf_counter() - t_setup
    subm = []
    t0 = time.perf_counter()
    nxt = t0
    while nxt - t0 < seconds:
        now = time.perf_counter()
        if nxt > now:
            time.sleep(nxt - now)
        N = boxes[int(rng.integers(0, 4))]
        B = int(min(512, max(1, round(math.exp(rng.uniform(0.0, math.log(512.0)))))))
        off = int(rng.integers(0, 512 - B + 1))
        ts = time.perf_counter()
        tk = srv.submit(tids[(N, int(rng.integers(0, 2)))], pools[N][off:off + B], 16, seed=int(rng.integers(1 << 62)))
        subm.append((tk, B, N, ts))
        nxt += rng.exponential(1.0 / rate)
    lat, done_t = [], []
    for tk, B, N, ts in subm:
        l_ms = srv.wait(tk, timeout_ms=600000)[2]
        lat.append(l_ms)
        done_t.append(ts + l_ms / 1e3)
    total = sum(b for _, b, _, _ in subm)
    span = max(done_t) - t0
    st = srv.stats()
    srv.destroy()
    p50, p99 = (float(x) for x in np.percentile(lat, [50, 99]))
    return {"requests": len(subm), "subtomograms": total, "offered_req_per_s": rate, "seconds": seconds,
            "throughput": total / span, "unit": UNIT, "p50_ms": p50, "p99_ms": p99,
            "mean_subtomograms_per_request": total / max(1, len(subm)), "batches": int(st["batches"]),
            "volumes": ("read in place from host memory by the expansion (coherent C2C access)"
                        if st["in_place_batches"] == st["batches"] else "copied host to device per batch"),
            "setup_s": setup_s,
            "mix": "boxes 24/32/48/64 (l<=N/2, bands N/8-N/4-N/2), 1-512 subtomograms log-uniform, 16 starts, "
                   "8 resident templates, SNR 0.1, +-60 deg wedge, BF16-split expansion",
            "optimizer": "Newton steps, 8 per band" if newton else "gradient ascent, 30 steps per band",
            "piece": piece or 128, "p999_ms": float(np.percentile(lat, 99.9)),
            "p99_ms_small_requests": float(np.percentile([l for l, (_, B, _, _) in zip(lat, subm) if B <= 32], 99))}


def run_mixed(args, device, rank: int = 0, world: int = 1) -> dict:
    """Batched uneven form: the whole mixed batch (3 box classes, 4 templates each, 8/16/32 starts) is one
    CUDA-graph launch per step; value = subtomograms of the batch / graph time.  On several GPUs the one batch
    is split by a cost-balanced partition (strong scaling) and the time is the maximum over ranks."""
    import numpy as np
    import torch

    from paper_2509_01180_gb300 import mixed, replicas, synth
    classes = synth.make_mixed(scale=args.mixed_scale, distinct=args.distinct or None, workers=cpu_workers(16))
    n_all = sum(cw.B for cw in classes)
    if world > 1:
        classes, _ = mixed.shard_classes(classes, rank, world)
    mb = mixed.MixedBatch(classes, device)
    mb.capture()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    for _ in range(args.warmup):
        mb.replay()
    torch.cuda.synchronize(device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(device.index or 0) as clk:
        for e0, e1 in ev:
            e0.record(stream)
            mb.replay()
            e1.record(stream)
            flush.zero_()
        torch.cuda.synchronize(device)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms = replicas.max_over_ranks([ms], device)[0]
    res = mb.results()
    acc = []
    for cw, (q, _) in zip(classes, res):
        acc.append(float(np.median(angle_deg(q.astype(np.float64), cw.q_true * np.array([1, -1, -1, -1])))))
    total = n_all
    desc = "; ".join(f"{cw.B} x {cw.N}^3 l<={cw.Lmax} bands {'-'.join(map(str, cw.stages))} "
                     f"S groups {[g[2] for g in cw.groups()]}" for cw in classes)
    mb.destroy()
    return {"metric": METRIC, "value": total / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "bf16-split/fp32", "data": "synthetic", "gpu_launches": mb.launches_per_replay() * args.steps,
            "config": {"workload": f"mixed batch ({desc}), 4 templates (40-200 blobs) per class, SNR U[0.03,0.2], "
                                   f"wedge U[50,70] deg, 30 steps, one CUDA-graph launch per step",
                       "l2": "flushed between timed steps"},
            "accuracy": {"median_angle_vs_truth_deg_by_class": acc}, "clocks": clk.summary()}


def angle_deg(q1, q2):
    import numpy as np
    d = np.abs(np.sum(q1 * q2, axis=1) / (np.linalg.norm(q1, axis=1) * np.linalg.norm(q2, axis=1)))
    return np.degrees(2 * np.arccos(np.clip(d, 0, 1)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=HEADLINE, help="precision64 (default), batch32, pair16 or mixed")
    ap.add_argument("--count", type=int, default=None, help="subtomograms per GPU (default: the workload's)")
    ap.add_argument("--distinct", type=int, default=0, help="generate only this many distinct phantoms and tile them")
    ap.add_argument("--form", choices=["both", "bf16split", "fp32"], default="both")
    ap.add_argument("--refine", type=int, default=None,
                    help="FP64 re-score of the K best starts (default 4 for precision64, else 0)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="subtomograms in the oracle's timed sample (default 2 at 64^3, 8 at 32^3)")
    ap.add_argument("--extras", type=int, default=1,
                    help="also measure the 32^3 batch, the mixed batch and the serving loop (N = 1 only)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="serving leg duration, the 60 s window of the serving workload (0 = skip)")
    ap.add_argument("--serve-piece", type=int, default=0,
                    help="serving: admit requests in pieces of at most this many subtomograms (0 = the server's 128)")
    ap.add_argument("--serve-newton-seconds", type=float, default=20.0,
                    help="duration of the serving leg with Newton steps (0 = skip)")
    ap.add_argument("--mixed-scale", type=float, default=1.0, help="class-count multiplier of the mixed workload")
    ap.add_argument("--no-autotune", action="store_true", help="use --group/--starts-per-thread instead of tuning")
    ap.add_argument("--group", type=int, default=4, help="lanes per start (group) with --no-autotune")
    ap.add_argument("--starts-per-thread", type=int, default=2, help="starts per thread with --no-autotune")
    ap.add_argument("--dealing", type=int, default=1, help="orbit dealing with --no-autotune: 1 rows, 2 flat")
    ap.add_argument("--sec3", type=int, default=None,
                    help="also time the Sec. III protocol (candidates + Newton); default on for batch32 / precision64")
    ap.add_argument("--wedge-leg", type=int, default=None,
                    help="also time the missing-wedge constrained correlation; default on for batch32")
    ap.add_argument("--band-leg", type=int, default=1,
                    help="also time marching bands chosen per subtomogram by the energy ratio")
    ap.add_argument("--sec3-grid", type=int, default=4608, help="rotation grid size for the candidate starts")
    ap.add_argument("--sec3-radius", type=float, default=25.0, help="neighbour radius of the grid (degrees)")
    ap.add_argument("--sec3-steps", type=int, default=8, help="Newton steps per marching band")
    ap.add_argument("--variants", default="",
                    help="with --profile-align: lanes x starts-per-thread list, e.g. 4x2,8x1,16x2f (f: flat dealing); "
                         "nG / nGf: Newton steps with G lanes per start from 8 starts")
    ap.add_argument("--profile-align", action="store_true",
                    help="time one ascent variant (--group, --starts-per-thread) alone on a plan without the "
                         "expansion table; for ncu captures")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    from paper_2509_01180_gb300 import replicas, synth

    # host-side work before the first GPU call: the oracle's timed sample (its own spawn pool) and the
    # headline workload's volumes (rendered by a spawn pool)
    base = None
    headline = args.workload not in ("mixed",) and not args.profile_align
    if headline and rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = args.cpu_sample or (2 if synth.CONFIGS[args.workload][0] >= 64 else 8)
        base = cpu_baseline(synth.make_workload(args.workload, count=n), n)
        progress("cpu baseline done")
    w = None
    if headline:
        count = args.count or synth.CONFIGS[args.workload][-1]
        w = make_workload(args, args.workload, count, first=replicas.shard_first(rank, count))
        progress(f"{count} subtomograms synthesised")

    import torch
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=device)

    if args.profile_align:
        print(json.dumps(profile_align(args, device)), flush=True)
        return
    if args.workload == "mixed":
        line = run_mixed(args, device, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    refine = args.refine if args.refine is not None else (4 if args.workload == "precision64" else 0)
    sec3 = bool(args.sec3) if args.sec3 is not None else args.workload in ("batch32", "precision64")
    wedge = bool(args.wedge_leg) if args.wedge_leg is not None else args.workload == "batch32"
    res = run_workload(args, w, rank, world, device, refine=refine, sec3=sec3, wedge=wedge,
                       sec3_starts=8 if w.N >= 64 else 4)
    body = summarize(args, w, res, world, device)
    line = {"metric": METRIC, "value": body.pop("value"), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": body.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None}
    line.update(body)
    if base is not None:
        line["cpu_baseline"] = base
    del w, res
    torch.cuda.empty_cache()
    progress(f"headline done: {line['value']:.1f} {UNIT}")
    if rank == 0 and world == 1 and args.extras:
        def extra(key, fn):
            # an extra key that fails is reported in the line instead of taking the headline with it
            try:
                line[key] = fn()
            except Exception as e:  # noqa: BLE001
                line[key] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()
            progress(f"{key} done")

        def batch32():  # the 1024 x 32^3 plain-method batch, with its Sec. III, wedge and band-choice legs
            w32 = make_workload(args, "batch32", synth.CONFIGS["batch32"][-1])
            r32 = run_workload(args, w32, rank, world, device, refine=0, sec3=True, wedge=True, sec3_starts=4)
            b32 = summarize(args, w32, r32, world, device)
            b32["steps"] = args.steps
            return b32

        if args.workload != "batch32":
            extra("batch32", batch32)
        extra("mixed", lambda: run_mixed(args, device, rank, world))
        if args.serve_seconds > 0:
            extra("serving", lambda: serving_leg(args.serve_seconds, piece=args.serve_piece))
        if args.serve_newton_seconds > 0:
            extra("serving_newton", lambda: serving_leg(args.serve_newton_seconds, newton=True))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
