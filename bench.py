#!/usr/bin/env python
"""Throughput of the hierarchical 4D Gaussian rasterizer on one B300 (or N replicas).

Headline workload (the 300k-Gaussian hierarchical scene at 1920x1080): 300,000 Gaussians
in 6 nested layers of 50k (SH degree 3, 64 motion groups), 30 frames of cumulative group
motion, every frame rendered at every level L1..L6 on an orbit camera.  One step = those
180 renders through the library (motion, projection, depth sort, binning, tile sort,
blend), rendered per frame by the single-pass multi-level render (levels L1..L6 from one
list; every image equals its single-level render bit for bit), the step's 30 frames
replayed from one CUDA graph.  value = Mpixel/s of the forward step over all ranks;
fwd_bwd = the same with the backward of every frame.

Beside it, on the same GPU: the other workloads of the rasterizer - the tiny scene
(2,000 Gaussians, 128x128), the differentiation step (200k Gaussians, 1352x1014, forward,
L1 loss, backward), the 128-request batching workload (500k Gaussians, mixed levels and
resolutions), the precision workload (1M Gaussians at 3840x2160, FP32 against BF16/FP8
storage) - the batched and plain single-view forms of the headline step, per-stage times
and roofline fractions (L2 flushed before each stage, and warm), the end-to-end figure with
host buffers, and the FP64 oracle timed on the host cores.  The printed JSON line is a
summary; ``--detail PATH`` writes every figure.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--detail PATH]

Under torchrun each rank renders its own step on its own GPU (the requests are
independent, no data-path collective): weak scaling.  Timing: CUDA events on the
rendering stream, L2 flushed between steps (outside the events), max over ranks.
``--impl reference`` times the FP64 CPU oracle on the host.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Mpixel/s at 1920x1080, forward (fwd_bwd: forward + backward), layer levels L1-L6, "
          "300k-Gaussian hierarchical scene")
UNIT = "Mpixel/s"
WORKLOAD = ("hier1080: 300k Gaussians in 6 layers of 50k, SH degree 3, 64 motion groups, "
            "30 frames x levels L1..L6 = 180 renders of 1920x1080 per step")
FP32_LANES_PER_SM = 128
N_SMS = 148

# ---- algorithmic work per unit ----
# Blends (FP32 ALU).  Two FLOP units, both reported:
#  * per evaluated (pixel, entry) pair, 20 FLOPs forward, 50 reverse (2.5 x forward);
#  * the finer split: 14 FLOPs to evaluate a walked pair up to the 1/255 test, plus 10 per
#    blended (pair, level) forward or 51 reverse (FMA = 2 FLOPs).
REF_FWD_FLOPS_PER_PAIR = 20
REF_BWD_FLOPS_PER_PAIR = 50
EVAL_FLOPS_PER_PAIR = 14
FWD_BLEND_FLOPS_PER_PAIR = 10
BWD_BLEND_FLOPS_PER_PAIR = 51
REC_BYTES = 80          # projected record (five float4)
STAGES_HBM = ("preprocess", "depth_sort", "scan", "emit", "tile_sort", "ranges", "reduce",
              "preprocess_bwd", "group_reduce")


def attr_bytes(sh_degree: int, precision: str) -> int:
    """Bytes of one Gaussian's stored attributes (and group id)."""
    k = (sh_degree + 1) ** 2
    if precision == "bf16_fp8":
        return 2 * (3 + 3 + 4 + 1) + 3 * k + 4
    return 4 * (3 + 3 + 4 + 1 + 3 * k) + 4


def stage_work(stage: str, w: dict):
    """(amount, kind, amount at the implementation's own count or None) of one call of a
    stage; kind 'bytes' (HBM) or 'flops' (FP32).  w: n selected Gaussians, k list entries,
    tiles, attr bytes per Gaussian, and for the blends walked / blended pair counts."""
    n, k = w["n"], w["k"]
    if stage == "preprocess":          # attributes in; record, depth key, value, count out
        return n * (w["attr"] + REC_BYTES + 12), "bytes", None
    if stage == "depth_sort":          # one read + one write of 8 B (key, value) pairs;
        return n * 16, "bytes", n * (4 + 4 * 16)   # one-sweep: histogram read + 4 passes
    if stage == "scan":                # rank gather of record + count, scan of the counts
        return n * (4 + 2 * (REC_BYTES + 4) + 8), "bytes", None
    if stage == "emit":                # record read per Gaussian; 12 B per (tile, Gaussian) pair
        return n * (REC_BYTES + 8) + k * 12, "bytes", n * (REC_BYTES + 8) + k * 4  # one-word entries
    if stage == "tile_sort":           # 24 B per pair: one read + one write of a 12 B key-value pair;
        return k * 24, "bytes", k * 12  # one keys-only pass: histogram read 4 + read 4 + write 4
    if stage == "ranges":  # row-binned lists: two scanned digit counts read, one range written per tile
        return w["tiles"] * 16, "bytes", None
    if stage == "reduce":              # 36 B of partials per entry in, 36 B per Gaussian out
        return k * 36 + n * 44, "bytes", None
    if stage == "preprocess_bwd":      # attributes, 2D gradient and count in; gradients and
        return n * (w["attr"] + 40 + 236 + 28), "bytes", None   # motion terms out
    if stage == "group_reduce":
        return n * 32, "bytes", None
    if stage == "blend":
        return (REF_FWD_FLOPS_PER_PAIR * w["walked"], "flops",
                EVAL_FLOPS_PER_PAIR * w["walked"] + FWD_BLEND_FLOPS_PER_PAIR * w["blended"])
    if stage == "blend_bwd":
        return (REF_BWD_FLOPS_PER_PAIR * w["bwd_walked"], "flops",
                EVAL_FLOPS_PER_PAIR * w["bwd_walked"] + BWD_BLEND_FLOPS_PER_PAIR * w["blended"])
    return 0, "bytes", None


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def fp32_derived_peak(peaks) -> float:
    """FP32 FMA peak from the unit counts and the maximum SM clock, TFLOP/s."""
    return N_SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12


def measure_fp32_sgemm(dev, n=8192, iters=20):
    """cuBLAS SGEMM (TF32 off: plain FP32 FMAs) on n x n, TFLOP/s, after a warm-up; reported
    beside the derived FP32 peak."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = torch.randn((n, n), device=dev)
        b = torch.randn((n, n), device=dev)
        c = torch.empty((n, n), device=dev)
        for _ in range(3):
            torch.mm(a, b, out=c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(iters):
            torch.mm(a, b, out=c)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / iters
        del a, b, c
        torch.cuda.empty_cache()
        return 2.0 * n ** 3 / (ms / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
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


HEADLINE_TILE = (8, 32)  # tile shape (width x height) of the multi-level headline
# independent graph branches of the headline step (frame f on branch f mod n, each with its own
# saved state): one frame's sorts and binning run beside another frame's blend; measured on
# B300 over 1..4 branches, forward 14,414 / 17,232 / 17,990 / 18,318 Mpixel/s, forward +
# backward 5,565 / 6,466 / 6,485 / 6,463
HEADLINE_CHAINS = {"fwd": 4, "fwd_bwd": 3}
HOST_AHEAD_CYCLES = 200_000_000  # GPU spin before a stage-profiled step (about 0.1 s at 2 GHz)

# the source file that defines each profiled kernel; its hash covers that file and the kernel
# sources it includes (transitively).  A kernel not listed depends on every source file.
KERNEL_SOURCES = {"k_blend_levels_fwd": "gc_levels.cu", "k_blend_levels_bwd": "gc_levels.cu",
                  "k_blend_fwd": "gc_raster.cu", "k_emit": "gc_raster.cu", "k_radix_scatter": "gc_sort.cu",
                  "k_batch_blend_fwd": "gc_batch.cu", "k_batch_blend_bwd": "gc_batch.cu",
                  "k_batch_emit": "gc_batch.cu", "k_field_bwd": "gc_motion_field.cu",
                  "k_field_encode": "gc_motion_field.cu", "k_reduce_entries": "gc_backward.cu"}


def _include_closure(path: str) -> list:
    """`path` and every kernel source (same directory) reached through its #include "..."
    lines, sorted; the public C-ABI header (declarations) is not followed."""
    root = os.path.dirname(os.path.normpath(path))
    seen, todo = set(), [os.path.normpath(path)]
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(f) or os.path.dirname(f) != root:
            continue
        seen.add(f)
        with open(f, encoding="utf-8", errors="replace") as fh:
            for line in fh:
                m = re.match(r'\s*#\s*include\s+"([^"]+)"', line)
                if m:
                    todo.append(os.path.normpath(os.path.join(os.path.dirname(f), m.group(1))))
    return sorted(seen)


def kernel_source_hash(kernel: str | None = None) -> str:
    """First 16 hex digits of the sha256 over the sources that make up `kernel`: the file that
    defines it and its include closure (every csrc file when the kernel is not listed)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2509_17513_b300", "csrc")
    own = KERNEL_SOURCES.get(kernel)
    files = (_include_closure(os.path.join(d, own)) if own is not None
             else [os.path.join(d, n) for n in sorted(os.listdir(d))])
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.relpath(f, ROOT).encode() + fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, units_per_launch: int, tile: str | None = None):
    """DRAM bytes of one launch of `kernel` covering `units_per_launch` units (renders, or
    frames of a multi-level pass), from the committed ncu summary profiles/traffic.json
    (bytes per unit of a small capture), or None when the kernel's sources changed since it
    was taken, the capture used another tile shape, or the kernel was not captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get("kernels", {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    if e.get("tile") and tile and e["tile"] != tile:  # another template instance
        return None
    return int(e["dram_bytes_per_unit"] * units_per_launch)


def max_over_ranks(total: float, world: int, device) -> float:
    """The largest of every rank's value (the slowest replica decides the job's time)."""
    if world <= 1:
        return total
    import torch
    import torch.distributed as dist
    t = torch.tensor([total], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, total_ms: float) -> float:
    """Units processed by all ranks per second (weak scaling: every rank does a full step)."""
    return units_per_rank_step * steps * world / (total_ms / 1e3)


def psnr_db(a, b):
    """PSNR (peak 1.0) of two image tensors, over all pixels and channels."""
    mse = float(((a.double() - b.double()) ** 2).mean())
    return round(10 * math.log10(1.0 / mse), 2) if mse > 0 else None


class Timer:
    """K steps timed with CUDA events on the rendering stream, L2 flushed between steps
    (outside the events), clocks sampled during the region, max over ranks."""

    def __init__(self, r, stream, local, world, dev):
        import torch
        self.r, self.stream, self.local, self.world, self.dev = r, stream, local, world, dev
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def __call__(self, step, steps, profile=False, name="timed", host_ahead=False, flush_stages=False,
                 renderer=None):
        """profile: per-stage CUDA events of the library (flush_stages: L2 flushed before every
        stage, outside its events).  host_ahead: before each step the GPU spins for a bounded
        time (outside the events), so that the host queues the whole step before the GPU
        reaches it and the stage events measure the kernels rather than the host's launch rate."""
        import torch
        import torch.distributed as dist
        r = renderer or self.r
        clocks = ClockSampler(self.local)
        r.profile(profile, flush_l2=flush_stages)
        r.profile_read()
        if self.world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        total = 0.0
        torch.cuda.nvtx.range_push(name)  # lets a profiler select the kernels of this region
        for _ in range(steps):
            self.flush.fill_(1.0)
            if host_ahead:
                torch.cuda._sleep(HOST_AHEAD_CYCLES)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            step()
            e1.record(self.stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clk = clocks.stop()
        prof = r.profile_read()
        r.profile(False)
        total = max_over_ranks(total, self.world, self.dev)
        return total, prof, clk


def stage_summary(prof):
    st_ms, st_calls = prof["stage_ms"], prof["stage_calls"]
    tot = max(1e-9, sum(st_ms.values()))
    return ({k: round(v / max(1, st_calls[k]), 4) for k, v in st_ms.items() if v > 0},
            {k: round(v / tot, 4) for k, v in st_ms.items() if v > 0})


def stage_table(prof, work: dict, peaks: dict):
    """Per stage of one call: ms, achieved GB/s (HBM stages) or TFLOP/s (blends) on the
    algorithmic unit, and the fraction of the measured HBM copy bandwidth or of the derived
    FP32 peak; `impl_frac` the same on the implementation's own byte / FLOP count."""
    fp32 = fp32_derived_peak(peaks)
    out = {}
    for st, tot in prof["stage_ms"].items():
        calls = prof["stage_calls"][st]
        if calls <= 0 or tot <= 0:
            continue
        ms = tot / calls
        amount, kind, impl = stage_work(st, work)
        if amount <= 0:
            continue
        if kind == "flops":
            ach = amount / (ms / 1e3) / 1e12
            e = {"ms": round(ms, 4), "tflops": round(ach, 3), "frac": round(ach / fp32, 4)}
            if impl:
                e["impl_frac"] = round(impl / (ms / 1e3) / 1e12 / fp32, 4)
        else:
            ach = amount / (ms / 1e3) / 1e9
            e = {"ms": round(ms, 4), "gbs": round(ach, 1), "frac": round(ach / peaks["hbm_gbs"], 4)}
            if impl:
                e["impl_frac"] = round(impl / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 4)
        out[st] = e
    return out


def compact_stages(flushed: dict, warm: dict) -> dict:
    """stage -> [ms flushed, frac flushed, ms warm, frac warm], three decimals."""
    out = {}
    r3 = lambda x: None if x is None else round(x, 3)
    for st in flushed:
        f, w = flushed[st], warm.get(st, {})
        out[st] = [r3(f["ms"]), r3(f["frac"]), r3(w.get("ms")), r3(w.get("frac"))]
    return out


def blend_roofline(stage, per_launch_ms, work, peaks, sgemm, units_per_launch, tile):
    """Roofline object of a blend kernel on both FLOP units."""
    kern = {"blend": "k_blend_levels_fwd", "blend_bwd": "k_blend_levels_bwd"}[stage]
    fp32 = fp32_derived_peak(peaks)
    amount, _, impl = stage_work(stage, work)
    ach = amount / (per_launch_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp32, 2), "unit": "TFLOP/s",
            "frac": round(ach / fp32, 4), "traffic": load_traffic(kern, units_per_launch, tile),
            "kernel": kern, "launch_ms": round(per_launch_ms, 4),
            "flop_unit": f"{REF_FWD_FLOPS_PER_PAIR if stage == 'blend' else REF_BWD_FLOPS_PER_PAIR}"
                         " per evaluated pair",
            "frac_split": round(impl / (per_launch_ms / 1e3) / 1e12 / fp32, 4),
            "split_unit": f"14 per walked pair + {FWD_BLEND_FLOPS_PER_PAIR if stage == 'blend' else BWD_BLEND_FLOPS_PER_PAIR}"
                          " per blended (pair, level)",
            "frac_of_sgemm": round(ach / sgemm, 4),
            "peak_source": f"derived: {N_SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                           f"{peaks.get('sm_max_mhz', 2032.0)} MHz; cuBLAS SGEMM in this run {sgemm:.1f}"}


# --------------------------------------------------------------------------- GPU arm

def count_work(r, gs, frames, reqs, outs, tile, top_mask):
    """Walked / blended pairs and list entries of the requests' single-level renders at a
    tile shape (deterministic, outside the timed regions); *_top: of the top-level renders
    alone (what a multi-level pass walks)."""
    import torch
    r.set_options(tile=tile, key_capacity=0)
    c = {"walked": 0, "blended": 0, "bwd": 0, "keys": 0, "walked_top": 0, "bwd_top": 0, "kmax": 0,
         "keys_top": 0, "n_top": 0}
    for q, (cam, f, mask) in enumerate(reqs):
        r.forward(gs, frames[f] if frames is not None else None, mask, cam, out=outs[q])
        _, blended, walked, contrib = r.pixel_state(with_walked=True)
        wq = int(walked.sum(dtype=torch.int64).item())
        cq = int(contrib.sum(dtype=torch.int64).item())
        st = r.stats()
        c["walked"] += wq
        c["blended"] += int(blended.sum(dtype=torch.int64).item())
        c["bwd"] += cq
        if mask == top_mask:
            c["walked_top"] += wq
            c["bwd_top"] += cq
            c["keys_top"] += st["n_keys"]
            c["n_top"] += st["n_selected"]
        c["keys"] += st["n_keys"]
        c["kmax"] = max(c["kmax"], st["n_keys"])
    return c


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2509_17513_b300 as gc
    from synth import scenes

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    peaks, peak_kind = measured_peaks()
    peaks = dict(peaks)
    sgemm = round(measure_fp32_sgemm(dev), 2)
    fp32 = fp32_derived_peak(peaks)
    skip = {x.strip() for x in args.skip_forms.split(",") if x.strip()}
    detail = {"peaks": {"hbm_gbs": peaks["hbm_gbs"], "hbm_source": f"{peak_kind} (MEASURED_PEAKS.json)",
                        "fp32_derived_tflops": round(fp32, 2), "fp32_sgemm_tflops": sgemm}}

    w = scenes.hier1080(n_frames=args.frames)
    W, H = 1920, 1080
    order = [(f, lv) for f in range(args.frames) for lv in range(1, 7)]
    reqs = [(w.cameras[f], f, scenes.level_mask(lv)) for f, lv in order]
    n_req = len(reqs)
    pixels_per_step = n_req * W * H
    r = gc.Renderer(local)
    timer = Timer(r, stream, local, world, dev)
    gs = gc.GaussianSet.from_scene(w.scene, dev)
    frames = [gc.MotionFrame.from_motion(w.motion, f, dev) for f in range(args.frames)]
    outs = [torch.empty((3, H, W), device=dev) for _ in range(n_req)]
    upstream = (torch.randn((3, H, W), generator=torch.Generator().manual_seed(7)) * 1e-3).to(dev)
    dls = [upstream] * n_req

    def mpix(total_ms, steps, px=pixels_per_step):
        return round(whole_job_rate(px, steps, world, total_ms) / 1e6, 1)

    # ---- headline: single-pass multi-level form, per frame levels 1..6 from one list (the
    # same 180 images, bit for bit, as 180 single-level renders), fixed key capacity
    tile = HEADLINE_TILE
    work = count_work(r, gs, frames, reqs, outs, tile, scenes.level_mask(6))
    cap_levels = int(work["kmax"] * 1.05) + 4096  # the multi-level lists are the top level's
    r.set_options(key_capacity=cap_levels, tile=tile)
    lsaved = gc.Saved(r)
    lgrads = None

    def levels_fwd():
        for f in range(args.frames):
            r.levels_forward(gs, frames[f], 6, w.cameras[f], outs=outs[6 * f:6 * f + 6])

    def levels_fwd_bwd():
        nonlocal lgrads
        for f in range(args.frames):
            r.levels_forward(gs, frames[f], 6, w.cameras[f], lsaved, outs=outs[6 * f:6 * f + 6])
            lgrads = r.levels_backward(lsaved, gs, frames[f], dls[6 * f:6 * f + 6], lgrads)

    for _ in range(args.warmup):
        levels_fwd()
        levels_fwd_bwd()
    r.check()
    ef_lv_ms, efwd_prof, clk_e = timer(levels_fwd, args.steps, name="levels_fwd")
    efb_lv_ms, efb_lv_prof, clk_efb = timer(levels_fwd_bwd, args.steps, name="levels_fwd_bwd")
    # per-stage CUDA events with the host queued ahead of the GPU: kernel times, not launch
    # gaps; warm (stages in pipeline order) and with L2 flushed before every stage
    st_steps = max(1, min(args.steps, 3))
    _, fwd_prof, _ = timer(levels_fwd, st_steps, profile=True, name="levels_fwd_stages", host_ahead=True)
    _, fb_prof, _ = timer(levels_fwd_bwd, st_steps, profile=True, name="levels_fwd_bwd_stages", host_ahead=True)
    _, fb_prof_fl, _ = timer(levels_fwd_bwd, st_steps, profile=True, name="levels_fwd_bwd_stages_flushed",
                             host_ahead=True, flush_stages=True)
    r.check()
    # the headline value: the same steps replayed from one CUDA graph each (gc_levels_graph: no
    # host work, no launch gaps between the kernels of a frame, identical images)
    cams_step = w.cameras[:args.frames]
    lg_fwd = gc.LevelsGraph(r, gs, frames, cams_step, 6, outs=outs[:6 * args.frames],
                            chains=HEADLINE_CHAINS["fwd"])
    lg_fb = gc.LevelsGraph(r, gs, frames, cams_step, 6, outs=outs[:6 * args.frames],
                           dL_dimages=dls[:6 * args.frames], grads=[lgrads] * args.frames,
                           chains=HEADLINE_CHAINS["fwd_bwd"])
    for _ in range(args.warmup):
        lg_fwd.launch()
        lg_fb.launch()
    lg_fwd.check()
    lg_fb.check()
    fwd_ms, gfwd_prof, clk = timer(lg_fwd.launch, args.steps, name="levels_graph_fwd")
    fb_ms, gfb_prof, clk_fb = timer(lg_fb.launch, args.steps, name="levels_graph_fwd_bwd")
    lg_fwd.check()
    lg_fb.check()
    graph_nodes = {"fwd": lg_fwd.kernel_nodes, "fwd_bwd": lg_fb.kernel_nodes}
    lg_fwd.close()
    lg_fb.close()
    frame0_images = [o.clone() for o in outs[0:6]]   # checked against the oracle's sample
    del lsaved, lgrads
    r.set_options(key_capacity=0)

    nf = args.frames
    wk_frame = {"n": work["n_top"] / nf, "k": work["keys_top"] / nf, "tiles": 240 * 34,
                "attr": attr_bytes(3, "fp32"), "walked": work["walked_top"] / nf,
                "bwd_walked": work["bwd_top"] / nf, "blended": work["blended"] / nf}
    st_warm = stage_table(fb_prof, wk_frame, peaks)
    st_flushed = stage_table(fb_prof_fl, wk_frame, peaks)
    st_fwd = stage_table(fwd_prof, wk_frame, peaks)
    fwd_blend_ms = st_fwd["blend"]["ms"]
    bwd_blend_ms = st_warm["blend_bwd"]["ms"]
    headline = {
        "value": mpix(fwd_ms, args.steps), "ms_per_step": round(fwd_ms / args.steps, 3),
        "fps": round(n_req * args.steps * world / (fwd_ms / 1e3), 1),
        "gpu_launches": gfwd_prof["kernel_launches"], "clocks": clk,
        "roofline": blend_roofline("blend", fwd_blend_ms, wk_frame, peaks, sgemm, 1, f"{tile[0]}x{tile[1]}"),
        "fwd_bwd": {"value": mpix(fb_ms, args.steps), "ms_per_step": round(fb_ms / args.steps, 3),
                    "fps": round(n_req * args.steps * world / (fb_ms / 1e3), 1),
                    "gpu_launches": gfb_prof["kernel_launches"], "clocks": clk_fb,
                    "roofline": blend_roofline("blend_bwd", bwd_blend_ms, wk_frame, peaks, sgemm, 1,
                                               f"{tile[0]}x{tile[1]}")},
        "eager": {"fwd": mpix(ef_lv_ms, args.steps), "fwd_bwd": mpix(efb_lv_ms, args.steps),
                  "gpu_launches": {"fwd": efwd_prof["kernel_launches"], "fwd_bwd": efb_lv_prof["kernel_launches"]},
                  "graph_kernel_nodes": graph_nodes, "clocks": {"fwd": clk_e, "fwd_bwd": clk_efb}},
        "stages_per_frame": {"note": "one frame = one multi-level pass (six level images); warm: stages in "
                                     "pipeline order; flushed: L2 flushed before every stage",
                             "warm": st_warm, "flushed": st_flushed, "fwd_warm": st_fwd,
                             "share_fwd": stage_summary(fwd_prof)[1], "share_fwd_bwd": stage_summary(fb_prof)[1]},
        "work_per_frame": {k: (round(v) if isinstance(v, float) else v) for k, v in wk_frame.items()},
    }
    detail["headline"] = headline

    # ---- plain FP32 single-view form: one gc_render_forward (+ backward) per request
    if "single" not in skip:
        detail["single_view"] = run_single_view(args, r, timer, gs, frames, reqs, outs, upstream,
                                                W, H, world, mpix)
    # ---- batched form of the 180 renders: autotuned, CUDA graph; BF16/FP8 storage
    if "batched" not in skip:
        detail["batched"] = run_batched(args, r, timer, gs, w, frames, reqs, outs, dls, n_req, mpix)
    # ---- the headline step with the other inputs the paper's pipeline has
    if "planes" not in skip:
        detail["decoded_planes"] = run_planes(args, r, timer, w, frames, outs, n_req, tile, mpix, dev)
    if "field" not in skip:
        detail["motion_field"] = run_field(args, r, timer, w, gs, outs, tile, mpix, dev)
    if "kde" not in skip:
        detail["kde_rate"] = run_kde(args, r, timer, w, dev)
    if "residual" not in skip:
        detail["residual_deformation"] = run_residual(args, r, timer, w, gs, frames, outs, dls, tile, mpix, dev)
    del outs, dls
    torch.cuda.empty_cache()

    # ---- the other workloads of the rasterizer
    if "c1" not in skip:
        detail["c1_tiny"] = run_c1(args, r, timer, world)
    if "c3" not in skip:
        detail["c3_diff"] = run_c3(args, r, timer, world, peaks)
    if not args.no_batch128:
        detail["c4_batch128"] = run_batch128(args, r, timer, dev)
        torch.cuda.empty_cache()
    c5_state = None
    if "c5" not in skip:
        detail["c5_prec4k"], c5_state = run_c5(args, r, timer, world, peaks)
        torch.cuda.empty_cache()
    if not args.no_e2e:
        detail["e2e"] = run_e2e(args, r, w, reqs, cap_levels, tile, W, H, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        detail["cpu_baseline"] = cpu_baseline(w, frame0_images, c5_state)
    del c5_state

    line = summary_line(args, world, w, tile, cap_levels, headline, detail)
    if rank == 0:
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump({"line": line, "detail": detail}, f, indent=1)
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if world > 1:
        dist.destroy_process_group()


def summary_line(args, world, w, tile, cap_levels, hl, d):
    """The one JSON line: the contract's keys, the headline forward and forward + backward,
    then one short entry per other form and the per-stage fractions."""
    fb = hl["fwd_bwd"]
    rf = dict(hl["roofline"])
    for k in ("peak_source", "split_unit", "frac_of_sgemm"):
        rf.pop(k, None)
    rb = {k: fb["roofline"][k] for k in ("achieved", "frac", "frac_split", "traffic", "kernel", "launch_ms")}
    line = {"metric": METRIC, "value": hl["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hl["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic, seeded, shaped like the paper's scenes",
            "config": {"workload": "hier1080: 300k Gaussians, 6 layers, SH3, 64 groups; 30 frames x L1..L6 "
                                   "at 1920x1080", "tile": f"{tile[0]}x{tile[1]}",
                       "path": "multi-level pass per frame, CUDA graph of independent frame chains "
                               f"(fwd {HEADLINE_CHAINS['fwd']}, fwd_bwd {HEADLINE_CHAINS['fwd_bwd']})",
                       "l2": "flushed between steps", "parallelism": f"replicas x{world}"},
            "fps": hl["fps"], "gpu_launches": hl["gpu_launches"], "clocks": _clk(hl["clocks"]),
            "roofline": rf}
    if "e2e" in d:
        e = d["e2e"]
        line["e2e"] = {k: e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step",
                                          "all_images_on_host")}
    if "cpu_baseline" in d:
        c = d["cpu_baseline"]
        line["cpu_baseline"] = {k: c[k] for k in ("value", "unit", "cores", "kind", "sample_short")}
        line["cpu_baseline"]["sample"] = line["cpu_baseline"].pop("sample_short")
        line["parity_vs_oracle"] = c.get("parity_short")
    forms = {}
    if "single_view" in d:
        s = d["single_view"]
        forms["single_view"] = [s["fwd"], s["fwd_bwd"]]
    if "batched" in d:
        b = d["batched"]
        forms["batched_graph"] = [b["fwd"], b["fwd_bwd"]]
        forms["batched_bf16_fp8_fb"] = b["bf16_fp8"]["fwd_bwd"]
    for k in ("residual_deformation", "decoded_planes"):
        if k in d:
            forms[k] = [d[k].get("fwd"), d[k].get("fwd_bwd")]
    if "motion_field" in d:
        forms["motion_field_step"] = d["motion_field"]["step_fwd"]
    line["forms_mpix_fwd_fb"] = forms
    if "c1_tiny" in d:
        c = d["c1_tiny"]
        line["C1"] = {k: c[k] for k in ("fps_eager", "fps_graph", "fwd_bwd_fps")}
    if "c4_batch128" in d:
        c = d["c4_batch128"]
        line["C4"] = {"fb_batched_fp32_bf16_single": [c["batched_fp32"]["value"], c["batched_bf16_fp8"]["value"],
                                                      c["single_view_fp32"]["value"]]}
    if "c5_prec4k" in d:
        c = d["c5_prec4k"]
        line["C5"] = {"fp32": [c["fp32"]["fwd"], c["fp32"]["fwd_bwd"]],
                      "bf16_fp8": [c["bf16_fp8"]["fwd"], c["bf16_fp8"]["fwd_bwd"]],
                      "psnr_bf16_vs_fp32_db": c["psnr_bf16_fp8_vs_fp32_db"], "tile": c.get("tile"),
                      "stages_fb": compact_stages(c["stages"]["flushed"], c["stages"]["warm"])}
    if "c3_diff" in d:
        c = d["c3_diff"]
        line["C3"] = {k: c.get(k) for k in ("value", "fps", "ms_per_step", "tile")}
        line["C3"]["blend_bwd_frac"] = c["stages"]["blend_bwd"]["frac"]
    line["stages_fb"] = {"note": "per frame [ms,frac] L2 flushed, then warm; HBM or FP32 (20/50 FLOP/pair)",
                         **compact_stages(hl["stages_per_frame"]["flushed"], hl["stages_per_frame"]["warm"])}
    line["fwd_bwd"] = {"value": fb["value"], "ms_per_step": fb["ms_per_step"], "fps": fb["fps"],
                       "gpu_launches": fb["gpu_launches"], "roofline": rb}
    return line


def _clk(c):
    return {k: c.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")}


def run_single_view(args, r, timer, gs, frames, reqs, outs, upstream, W, H, world, mpix):
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes
    saved = gc.Saved(r)
    r.set_options(key_capacity=0, tile=(16, 16))
    kmax = 0
    for q, (cam, f, mask) in enumerate(reqs):
        r.forward(gs, frames[f], mask, cam, out=outs[q])
        kmax = max(kmax, r.stats()["n_keys"])
    r.set_options(key_capacity=int(kmax * 1.05) + 4096)
    grads1 = None

    def single_fwd():
        for q, (cam, f, mask) in enumerate(reqs):
            r.forward(gs, frames[f], mask, cam, out=outs[q])

    def single_fwd_bwd():
        nonlocal grads1
        for q, (cam, f, mask) in enumerate(reqs):
            r.forward(gs, frames[f], mask, cam, saved, out=outs[q])
            grads1 = r.backward(saved, gs, frames[f], upstream, grads1)

    for _ in range(args.warmup):
        single_fwd()
        single_fwd_bwd()
    r.check()
    s_steps = max(1, min(args.steps, 3))
    sf_ms, _, _ = timer(single_fwd, s_steps, name="single_fwd")
    sfb_ms, sfb_prof, _ = timer(single_fwd_bwd, s_steps, profile=True, name="single_fwd_bwd")
    per_level = {}
    for lv in range(1, 7):
        lv_reqs = [(cam, f, mask) for (cam, f, mask) in reqs if mask == scenes.level_mask(lv)]

        def level_fwd(lv_reqs=lv_reqs):
            for q, (cam, f, mask) in enumerate(lv_reqs):
                r.forward(gs, frames[f], mask, cam, out=outs[q])

        lv_ms, _, _ = timer(level_fwd, s_steps, name=f"single_level_{lv}")
        n_lv = len(lv_reqs) * s_steps
        per_level[f"L{lv}"] = {"fps": round(n_lv * world / (lv_ms / 1e3), 1),
                               "ms_per_render": round(lv_ms / n_lv, 4)}
    r.check()
    del saved, grads1
    r.set_options(key_capacity=0, tile=HEADLINE_TILE)
    torch.cuda.empty_cache()
    return {"form": "plain FP32, one gc_render_forward (+ gc_render_backward) per request, 16x16 tiles",
            "fwd": mpix(sf_ms, s_steps), "fwd_bwd": mpix(sfb_ms, s_steps), "unit": UNIT,
            "ms_per_step": {"fwd": round(sf_ms / s_steps, 2), "fwd_bwd": round(sfb_ms / s_steps, 2)},
            "per_level_fwd": per_level, "stage_ms_per_render": stage_summary(sfb_prof)[0], "steps": s_steps}


def run_batched(args, r, timer, gs, w, frames, reqs, outs, dls, n_req, mpix):
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes
    dev = outs[0].device
    tune = r.tune_batch(gs, frames, reqs, dL_dimages=dls, depths=(30, 60, 90, n_req), iters=2, outs=outs)
    depth, tile_b = tune["best"]["depth"], tuple(tune["best"]["tile"])
    r.set_options(tile=tile_b, key_capacity=0)
    grads = r.batch_grads(gs, frames)
    # the forward graph's own depth: smaller batches on parallel graph branches overlap one
    # batch's sorts with another's blend (the training step is tuned above, with its ordered
    # backwards); the faster of the two depths over two launches each
    fwd_depth, best_ms = depth, None
    for d in sorted({depth, 45}):
        g_try = gc.BatchGraph(r, gs, frames, reqs, d, outs=outs)
        g_try.launch()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(2):
            g_try.launch()
        ev[1].record()
        torch.cuda.synchronize()
        g_try.check()
        ms = ev[0].elapsed_time(ev[1])
        if best_ms is None or ms < best_ms:
            fwd_depth, best_ms = d, ms
        g_try.close()
        torch.cuda.empty_cache()
    g_fwd = gc.BatchGraph(r, gs, frames, reqs, fwd_depth, outs=outs)
    g_fb = gc.BatchGraph(r, gs, frames, reqs, depth, dL_dimages=dls, grads=grads, outs=outs)
    for _ in range(args.warmup):
        g_fwd.launch()
        g_fb.launch()
    g_fwd.check()
    g_fb.check()
    bf_ms, _, clk_bf = timer(g_fwd.launch, args.steps, name="graph_fwd")
    bfb_ms, _, clk_bfb = timer(g_fb.launch, args.steps, name="graph_fwd_bwd")
    g_fwd.check()
    g_fb.check()
    ref_imgs = [o.clone() for o in outs[:: max(1, n_req // 12)]]
    cap = g_fwd.key_capacity
    g_fwd.close()
    g_fb.close()
    del grads
    torch.cuda.empty_cache()
    # reduced-precision storage (BF16 geometry, FP8-E4M3 SH), the same batched graph
    gsq = gc.GaussianSet.from_quantized(scenes.quantize_scene(w.scene), w.scene, dev)
    gq = gc.BatchGraph(r, gsq, frames, reqs, depth, dL_dimages=dls, grads=r.batch_grads(gsq, frames), outs=outs)
    gqf = gc.BatchGraph(r, gsq, frames, reqs, depth, outs=outs)
    for _ in range(args.warmup):
        gq.launch()
        gqf.launch()
    gq.check()
    gqf.check()
    qf_ms, _, _ = timer(gqf.launch, args.steps, name="graph_bf16_fp8_fwd")
    q_ms, _, clk_q = timer(gq.launch, args.steps, name="graph_bf16_fp8_fwd_bwd")
    gq.check()
    q_imgs = outs[:: max(1, n_req // 12)]
    q_psnr = psnr_db(torch.stack(q_imgs), torch.stack(ref_imgs))
    gq.close()
    gqf.close()
    del gsq, ref_imgs
    r.set_options(key_capacity=0, tile=HEADLINE_TILE)
    torch.cuda.empty_cache()
    return {"form": "the 180 renders as batched requests replayed from one CUDA graph (autotuned tile "
                    "shape and batch depth)",
            "fwd": mpix(bf_ms, args.steps), "fwd_bwd": mpix(bfb_ms, args.steps), "unit": UNIT,
            "ms_per_step": {"fwd": round(bf_ms / args.steps, 3), "fwd_bwd": round(bfb_ms / args.steps, 3)},
            "tile": f"{tile_b[0]}x{tile_b[1]}", "batch_depth": {"fwd": fwd_depth, "fwd_bwd": depth},
            "key_capacity_per_batch": cap,
            "clocks": {"fwd": clk_bf, "fwd_bwd": clk_bfb}, "autotune": tune,
            "bf16_fp8": {"storage": "BF16 means/log-scales/quats/opacity, FP8-E4M3 SH, FP32 scales; FP32 math",
                         "fwd": mpix(qf_ms, args.steps), "fwd_bwd": mpix(q_ms, args.steps),
                         "psnr_vs_fp32_scene_db": q_psnr, "clocks": clk_q,
                         "bytes_per_gaussian": {"fp32": attr_bytes(3, "fp32"), "bf16_fp8": attr_bytes(3, "bf16_fp8")}}}


def run_planes(args, r, timer, w, frames, outs, n_req, tile, mpix, dev):
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes
    ref_imgs = [o.clone() for o in outs[:: max(1, n_req // 12)]]
    gpl = gc.GaussianSet.from_planes(scenes.quantize_planes(w.scene, plane_width=1024), w.scene, dev)
    r.set_options(key_capacity=0, tile=tile)
    kmax = 0
    for f in range(args.frames):
        r.levels_forward(gpl, frames[f], 6, w.cameras[f], outs=outs[6 * f:6 * f + 6])
        kmax = max(kmax, r.stats()["n_keys"])
    q_imgs = outs[:: max(1, n_req // 12)]
    ps = psnr_db(torch.stack(q_imgs), torch.stack(ref_imgs))
    r.set_options(key_capacity=int(kmax * 1.02) + 4096, tile=tile)

    def planes_fwd():
        for f in range(args.frames):
            r.levels_forward(gpl, frames[f], 6, w.cameras[f], outs=outs[6 * f:6 * f + 6])

    for _ in range(args.warmup):
        planes_fwd()
    r.check()
    pf_ms, pf_prof, clk_pf = timer(planes_fwd, args.steps, profile=True, name="planes_fwd")
    r.check()
    del gpl, ref_imgs
    r.set_options(key_capacity=0)
    torch.cuda.empty_cache()
    return {"form": "the headline multi-level forward step rendered from the decoded attribute planes "
                    "(uint16 positions, uint8 quaternion / log-scale / opacity / SH planes per layer, "
                    "per-layer per-channel min/max affine dequantisation in the preprocess)",
            "fwd": mpix(pf_ms, args.steps), "unit": UNIT, "ms_per_step": round(pf_ms / args.steps, 3),
            "bytes_per_gaussian": {"fp32": attr_bytes(3, "fp32"), "planes": 2 * 3 + 8 + 48},
            "preprocess_ms_per_call": stage_summary(pf_prof)[0].get("preprocess"),
            "psnr_vs_fp32_scene_db": ps, "clocks": clk_pf}


def run_field(args, r, timer, w, gs, outs, tile, mpix, dev):
    import numpy as np
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes
    fp = scenes.motion_field_params(np.random.default_rng(12), n_levels=16, log2_T=19, n_min=16, n_max=2048)
    field = gc.MotionField(fp, dev)
    means_d = gs.tensors["means"]
    fq, ft = r.motion_field_forward(field, means_d)
    r.set_options(key_capacity=0, tile=tile)
    r.levels_forward(gs, gc.MotionFrame(fq, ft, per_gaussian=True), 6, w.cameras[0], outs=outs[0:6])
    fcap = int(r.stats()["n_keys"] * 1.3) + 4096
    r.set_options(key_capacity=fcap, tile=tile)
    gq_up = torch.randn((w.scene.n, 4), generator=torch.Generator(device=dev).manual_seed(3), device=dev)
    gt_up = torch.randn((w.scene.n, 3), generator=torch.Generator(device=dev).manual_seed(4), device=dev)

    def field_fwd():
        for _ in range(args.frames):
            r.motion_field_forward(field, means_d)

    def field_bwd():
        for _ in range(args.frames):
            r.motion_field_backward(field, means_d, gq_up, gt_up)

    enc = torch.empty((w.scene.n, 32), device=dev)

    def field_train():  # the training form: the forward keeps the encodings for the backward
        for _ in range(args.frames):
            r.motion_field_forward(field, means_d, encodings=enc)
            r.motion_field_backward(field, means_d, gq_up, gt_up, encodings=enc)

    def field_step():
        for f in range(args.frames):
            q_, t_ = r.motion_field_forward(field, means_d)
            r.levels_forward(gs, gc.MotionFrame(q_, t_, per_gaussian=True), 6, w.cameras[f],
                             outs=outs[6 * f:6 * f + 6])

    for _ in range(args.warmup):
        field_fwd()
        field_bwd()
        field_train()
        field_step()
    r.check()
    mff_ms, _, _ = timer(field_fwd, args.steps, name="field_fwd")
    mfb_ms, _, _ = timer(field_bwd, args.steps, name="field_bwd")
    mft_ms, _, _ = timer(field_train, args.steps, name="field_train")
    mfs_ms, _, clk_fs = timer(field_step, args.steps, name="field_step")
    r.check()
    n_g = w.scene.n
    per_ms_f = mff_ms / args.steps / args.frames
    del field, fq, ft, gq_up, gt_up, enc
    r.set_options(key_capacity=0)
    torch.cuda.empty_cache()
    return {"form": "per-Gaussian motion source (Sec. 3.2): 16-level hash grid (2^19 entries x 2 features per "
                    "level, resolutions 16..2048) + translation and rotation MLPs (32-64-3, 32-64-4) for the "
                    "300k Gaussians of every frame, then the multi-level render with one rigid motion per Gaussian",
            "field_fwd_ms_per_frame": round(per_ms_f, 4),
            "field_bwd_ms_per_frame": round(mfb_ms / args.steps / args.frames, 4),
            "field_train_ms_per_frame": {
                "fwd_save_plus_bwd_saved": round(mft_ms / args.steps / args.frames, 4),
                "note": "forward keeping the hash-grid encodings, backward reading them (no second table gather)"},
            "field_fwd_gaussians_per_s": round(n_g / (per_ms_f / 1e3), 1),
            "field_fwd_tflops": round(n_g * 2 * (2 * 64 * 32 + 7 * 64) / (per_ms_f / 1e3) / 1e12, 3),
            "step_fwd": mpix(mfs_ms, args.steps), "unit": UNIT, "key_capacity": fcap, "clocks": clk_fs}


def run_kde(args, r, timer, w, dev):
    import numpy as np
    import torch

    from synth import scenes
    pq = scenes.quantize_planes(w.scene, plane_width=1024)
    W_p = 1024
    ys = []
    for l in range(w.scene.n_layers):
        n_l = int(w.scene.layer_offsets[l + 1] - w.scene.layer_offsets[l])
        u8 = pq["u8"][l]
        ys.append(torch.from_numpy(np.ascontiguousarray(
            u8[:, :, :W_p].reshape(u8.shape[0], -1)[:, :n_l].astype(np.float32))).to(dev))

    def kde_step():
        return [r.kde_rate(yl) for yl in ys]

    for _ in range(args.warmup):
        kde_step()
    k_ms, _, _ = timer(kde_step, args.steps, name="kde_rate")
    rates = torch.stack(kde_step()).cpu().numpy()
    gen = torch.Generator(device=dev).manual_seed(21)
    ys_noisy = [yl + (torch.rand(yl.shape, generator=gen, device=dev) - 0.5) for yl in ys]

    def kde_grad_step():
        return [r.kde_rate_grad(yl) for yl in ys_noisy]

    for _ in range(args.warmup):
        kde_grad_step()
    kg_ms, _, _ = timer(kde_grad_step, args.steps, name="kde_rate_grad")
    n_sym = sum(int(yl.numel()) for yl in ys)
    return {"form": "KDE rate estimate of the keyframe RD loss (Sec. 3.3): Silverman-bandwidth kernel density PMF "
                    "of the quantised symbols of each uint8 attribute channel of each layer (56 channels x 6 "
                    "layers of hier1080, 300k Gaussians)",
            "ms_per_step": round(k_ms / args.steps, 4), "channels": int(rates.size),
            "symbols_per_s": round(n_sym / (k_ms / args.steps / 1e3), 1),
            "mean_bits_per_symbol": round(float(np.nanmean(rates)), 4),
            "training_form": {"note": "noise-injected values, the symbols' density held fixed, rate and dR/dy of "
                                      "every value (gc_kde_rate_grad)",
                              "ms_per_step": round(kg_ms / args.steps, 4),
                              "values_per_s": round(n_sym / (kg_ms / args.steps / 1e3), 1)}}


def run_residual(args, r, timer, w, gs, frames, outs, dls, tile, mpix, dev):
    import numpy as np
    import torch

    import paper_2509_17513_b300 as gc
    gen = torch.Generator(device=dev).manual_seed(11)
    n = w.scene.n
    rframes = []
    for f in range(args.frames):
        sd = float(np.sqrt(f))
        rframes.append(gc.MotionFrame(frames[f].q, frames[f].t,
                                      torch.randn((n, 3), generator=gen, device=dev) * (0.01 * sd),
                                      torch.randn(n, generator=gen, device=dev) * (0.05 * sd),
                                      torch.randn((n, 16, 3), generator=gen, device=dev) * (0.01 * sd)))
    r.set_options(key_capacity=0, tile=tile)
    kmax = 0
    for f in range(args.frames):
        r.levels_forward(gs, rframes[f], 6, w.cameras[f], outs=outs[6 * f:6 * f + 6])
        kmax = max(kmax, r.stats()["n_keys"])
    r.set_options(key_capacity=int(kmax * 1.02) + 4096, tile=tile)
    rsaved = gc.Saved(r)
    rgrads = None

    def res_fwd():
        for f in range(args.frames):
            r.levels_forward(gs, rframes[f], 6, w.cameras[f], outs=outs[6 * f:6 * f + 6])

    def res_fwd_bwd():
        nonlocal rgrads
        for f in range(args.frames):
            r.levels_forward(gs, rframes[f], 6, w.cameras[f], rsaved, outs=outs[6 * f:6 * f + 6])
            rgrads = r.levels_backward(rsaved, gs, rframes[f], dls[6 * f:6 * f + 6], rgrads)

    for _ in range(args.warmup):
        res_fwd()
        res_fwd_bwd()
    r.check()
    rf_ms, _, clk_rf = timer(res_fwd, args.steps, name="residual_fwd")
    rfb_ms, _, clk_rfb = timer(res_fwd_bwd, args.steps, name="residual_fwd_bwd")
    r.check()
    del rsaved, rgrads, rframes
    r.set_options(key_capacity=0)
    torch.cuda.empty_cache()
    return {"form": "the headline multi-level step with per-frame residual deformation (Eq. 7): log-scale, "
                    "opacity-logit and SH residuals (208 B per Gaussian per frame) added inside the preprocess "
                    "and the chain rule",
            "fwd": mpix(rf_ms, args.steps), "fwd_bwd": mpix(rfb_ms, args.steps), "unit": UNIT,
            "ms_per_step": {"fwd": round(rf_ms / args.steps, 3), "fwd_bwd": round(rfb_ms / args.steps, 3)},
            "key_capacity": int(kmax * 1.02) + 4096, "clocks": {"fwd": clk_rf, "fwd_bwd": clk_rfb}}


def run_c1(args, r, timer, world):
    """The tiny scene (2,000 Gaussians, one layer, SH degree 0, 128x128, 16x16 tiles): a
    render is a few microseconds of GPU work, so the per-call latency decides; timed eagerly
    (one library call per render) and as 100 renders replayed from one CUDA graph."""
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes
    wt = scenes.tiny()
    cam = wt.cameras[0]
    rt = gc.Renderer(r.device, tile=(16, 16))
    gs = gc.GaussianSet.from_scene(wt.scene, f"cuda:{r.device}")
    out = torch.empty((3, cam.height, cam.width), device=f"cuda:{r.device}")
    up = torch.full_like(out, 1e-3)
    saved = gc.Saved(rt)
    n_per = 100
    rt.forward(gs, None, 1, cam, out=out)
    rt.set_options(key_capacity=int(rt.stats()["n_keys"] * 1.05) + 4096)
    grads = None

    def eager():
        for _ in range(n_per):
            rt.forward(gs, None, 1, cam, out=out)

    def eager_fb():
        nonlocal grads
        for _ in range(n_per):
            rt.forward(gs, None, 1, cam, saved, out=out)
            grads = rt.backward(saved, gs, None, up, grads)

    eager()
    eager_fb()
    steps = max(3, min(args.steps, 10))
    e_ms, _, _ = timer(eager, steps, name="c1_eager", renderer=rt)
    fb_ms, _, _ = timer(eager_fb, steps, name="c1_fwd_bwd", renderer=rt)
    g = gc.LevelsGraph(rt, gs, [None] * n_per, [cam] * n_per, 1)
    g.launch()
    g.check()
    g_ms, _, _ = timer(g.launch, steps, name="c1_graph", renderer=rt)
    g.check()
    g.close()
    rt.close()
    px = cam.width * cam.height
    n = n_per * steps * world
    return {"workload": "tiny: 2,000 Gaussians, one layer, SH degree 0, 128x128, 16x16 tiles",
            "fps_eager": round(n / (e_ms / 1e3), 1), "fps_graph": round(n / (g_ms / 1e3), 1),
            "fwd_bwd_fps": round(n / (fb_ms / 1e3), 1),
            "us_per_render": {"eager": round(e_ms * 1e3 / (n_per * steps), 2),
                              "graph": round(g_ms * 1e3 / (n_per * steps), 2),
                              "fwd_bwd_eager": round(fb_ms * 1e3 / (n_per * steps), 2)},
            "mpix_s_graph": round(n * px / (g_ms / 1e3) / 1e6, 1)}


def pick_tile(r, make_step, tiles=((16, 16), (8, 32), (32, 8)), reps=3):
    """Tile shape of a single-view form, chosen as the batched path's autotuner chooses its
    own: per shape, make_step() builds a step (with its own saved state), which runs twice to
    size its buffers and then `reps` times timed on the host around device synchronisations;
    the fastest shape is kept (key capacity back to grow-as-needed).
    Returns (tile, {"16x16": ms, ...})."""
    import torch
    ms = {}
    for tile in tiles:
        r.set_options(key_capacity=0, tile=tile)
        step = make_step()
        step()
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            step()
        torch.cuda.synchronize()
        ms[tile] = (time.perf_counter() - t0) * 1e3 / reps
    best = min(ms, key=ms.get)
    r.set_options(key_capacity=0, tile=best)
    return best, {f"{t[0]}x{t[1]}": round(v, 3) for t, v in ms.items()}


def run_c3(args, r, timer, world, peaks):
    """The differentiation step (200k Gaussians, SH 3, 32 groups, 1352x1014, FP32): forward
    of frame 1 at level L6, L1 loss against the target (the scene with perturbed means,
    rendered once outside the timing), backward to every attribute and group motion."""
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes
    wd = scenes.diff()
    cam = wd.cameras[0]
    dev = f"cuda:{r.device}"
    rd = gc.Renderer(r.device, tile=(16, 16))
    gs = gc.GaussianSet.from_scene(wd.scene, dev)
    mo = gc.MotionFrame.from_motion(wd.motion, 1, dev)
    tsc = wd.scene.subset(range(wd.scene.n))
    tsc.means = wd.extra["target_means"]
    tsc.layer_offsets = wd.scene.layer_offsets
    tgs = gc.GaussianSet.from_scene(tsc, dev)
    target = rd.forward(tgs, mo, 63, cam).clone()
    del tgs
    img = torch.empty_like(target)
    dl = torch.empty_like(target)
    loss = torch.empty(1, device=dev)

    def tune_step():
        s, g = gc.Saved(rd), [None]

        def step():
            rd.forward(gs, mo, 63, cam, s, out=img)
            rd.l1_loss(img, target, grad=dl, loss=loss)
            g[0] = rd.backward(s, gs, mo, dl, g[0])
        return step

    tile, tile_ms = pick_tile(rd, tune_step)
    rd.forward(gs, mo, 63, cam, out=img)
    st = rd.stats()
    rd.set_options(key_capacity=int(st["n_keys"] * 1.05) + 4096)
    saved = gc.Saved(rd)
    grads = None
    # walked pairs for the blend fractions (counted outside the timing)
    _, blended, walked, contrib = rd.pixel_state(with_walked=True)
    wk = {"n": st["n_selected"], "k": st["n_keys"], "tiles": st["n_tiles"], "attr": attr_bytes(3, "fp32"),
          "walked": int(walked.sum(dtype=torch.int64)), "bwd_walked": int(contrib.sum(dtype=torch.int64)),
          "blended": int(blended.sum(dtype=torch.int64))}

    def step():
        nonlocal grads
        rd.forward(gs, mo, 63, cam, saved, out=img)
        rd.l1_loss(img, target, grad=dl, loss=loss)
        grads = rd.backward(saved, gs, mo, dl, grads)

    for _ in range(args.warmup):
        step()
    rd.check()
    ms, _, clk = timer(step, args.steps, name="c3_fwd_loss_bwd", renderer=rd)
    _, prof, _ = timer(step, max(1, min(args.steps, 3)), profile=True, name="c3_stages", renderer=rd,
                       host_ahead=True)
    rd.check()
    lv = float(loss)
    rd.close()
    px = cam.width * cam.height
    return {"workload": "diff: 200k Gaussians, SH 3, 32 groups, 1352x1014, level L6; forward, L1 loss (gc_l1_loss) "
                        "against the perturbed-means target, backward",
            "value": round(whole_job_rate(px, args.steps, world, ms) / 1e6, 1), "unit": UNIT,
            "fps": round(args.steps * world / (ms / 1e3), 1), "ms_per_step": round(ms / args.steps, 4),
            "loss": round(lv, 6), "keys": st["n_keys"], "clocks": clk, "tile": f"{tile[0]}x{tile[1]}",
            "tile_sweep_ms": tile_ms, "stages": stage_table(prof, wk, peaks)}


def run_c5(args, r, timer, world, peaks):
    """The precision workload (1M Gaussians in 6 layers, SH 3, 256 groups, 3840x2160, frame 1,
    level L6): plain FP32 storage against BF16 geometry / FP8-E4M3 SH with per-channel FP32
    scales (FP32 math), forward and forward + backward, single view; per-stage fractions of
    the FP32 forward + backward with L2 flushed before each stage and warm (at this size the
    lists far exceed L2)."""
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes
    w5 = scenes.prec4k()
    cam = w5.cameras[0]
    dev = f"cuda:{r.device}"
    r5 = gc.Renderer(r.device, tile=(16, 16))
    q = scenes.quantize_scene(w5.scene)
    sets = {"fp32": gc.GaussianSet.from_scene(w5.scene, dev),
            "bf16_fp8": gc.GaussianSet.from_quantized(q, w5.scene, dev)}
    mo = gc.MotionFrame.from_motion(w5.motion, 1, dev)
    gen = torch.Generator(device=dev).manual_seed(13)
    up = torch.randn((3, cam.height, cam.width), generator=gen, device=dev) * 1e-3

    def tune_step():
        s, g = gc.Saved(r5), [None]
        o = torch.empty((3, cam.height, cam.width), device=dev)

        def step():
            r5.forward(sets["fp32"], mo, 63, cam, s, out=o)
            g[0] = r5.backward(s, sets["fp32"], mo, up, g[0])
        return step

    tile5, tile_ms = pick_tile(r5, tune_step)
    res, imgs, wk = {}, {}, None
    steps = max(2, min(args.steps, 10))
    for name, gset in sets.items():
        r5.set_options(key_capacity=0)
        img = r5.forward(gset, mo, 63, cam).clone()
        st = r5.stats()
        if name == "fp32":
            _, blended, walked, contrib = r5.pixel_state(with_walked=True)
            wk = {"n": st["n_selected"], "k": st["n_keys"], "tiles": st["n_tiles"], "attr": attr_bytes(3, name),
                  "walked": int(walked.sum(dtype=torch.int64)), "bwd_walked": int(contrib.sum(dtype=torch.int64)),
                  "blended": int(blended.sum(dtype=torch.int64))}
        imgs[name] = img
        r5.set_options(key_capacity=int(st["n_keys"] * 1.05) + 4096)
        saved = gc.Saved(r5)
        out = torch.empty_like(img)
        grads = None

        def fwd():
            r5.forward(gset, mo, 63, cam, out=out)

        def fwd_bwd():
            nonlocal grads
            r5.forward(gset, mo, 63, cam, saved, out=out)
            grads = r5.backward(saved, gset, mo, up, grads)

        for _ in range(args.warmup):
            fwd()
            fwd_bwd()
        r5.check()
        f_ms, _, clk = timer(fwd, steps, name=f"c5_{name}_fwd", renderer=r5)
        fb_ms, _, clk_fb = timer(fwd_bwd, steps, name=f"c5_{name}_fwd_bwd", renderer=r5)
        px = cam.width * cam.height
        res[name] = {"fwd": round(whole_job_rate(px, steps, world, f_ms) / 1e6, 1),
                     "fwd_bwd": round(whole_job_rate(px, steps, world, fb_ms) / 1e6, 1),
                     "ms": {"fwd": round(f_ms / steps, 3), "fwd_bwd": round(fb_ms / steps, 3)},
                     "keys": st["n_keys"], "bytes_per_gaussian": attr_bytes(3, name), "clocks": clk_fb}
        if name == "fp32":
            s_steps = max(1, min(args.steps, 3))
            _, prof_w, _ = timer(fwd_bwd, s_steps, profile=True, name="c5_stages_warm", renderer=r5,
                                 host_ahead=True)
            _, prof_f, _ = timer(fwd_bwd, s_steps, profile=True, name="c5_stages_flushed", renderer=r5,
                                 host_ahead=True, flush_stages=True)
            res["stages"] = {"warm": stage_table(prof_w, wk, peaks), "flushed": stage_table(prof_f, wk, peaks)}
        r5.check()
        del saved, grads, out
    res["psnr_bf16_fp8_vs_fp32_db"] = psnr_db(imgs["bf16_fp8"], imgs["fp32"])
    res["max_abs_bf16_fp8_vs_fp32"] = round(float((imgs["bf16_fp8"] - imgs["fp32"]).abs().max()), 5)
    res["workload"] = ("prec4k: 1M Gaussians, 6 layers, SH 3, 256 groups, 3840x2160, frame 1, level L6, "
                       f"single view, {tile5[0]}x{tile5[1]} tiles (the fastest of three in tile_sweep_ms)")
    res["tile"] = f"{tile5[0]}x{tile5[1]}"
    res["tile_sweep_ms"] = tile_ms
    res["unit"] = UNIT
    res["work"] = wk
    state = {"w": w5, "q": q, "cam": cam, "img_fp32": imgs["fp32"].cpu(), "img_bf16_fp8": imgs["bf16_fp8"].cpu(),
             "tile": tile5}
    r5.close()
    del sets
    return res, state


def run_batch128(args, r, timer, dev):
    """The 128-request batching workload: 500k Gaussians, 16 views x 8 frames, each at its
    own level and resolution; forward + backward, batched graph (autotuned) against the
    plain FP32 single-view loop, FP32 and BF16/FP8 storage."""
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes

    w = scenes.batch()
    gs = gc.GaussianSet.from_scene(w.scene, dev)
    gsq = gc.GaussianSet.from_quantized(scenes.quantize_scene(w.scene), w.scene, dev)
    frames = [gc.MotionFrame.from_motion(w.motion, f, dev) for f in range(w.motion.q.shape[0])]
    reqs = [(q.camera, q.frame, q.layer_mask) for q in w.requests]
    px = sum(q.camera.width * q.camera.height for q in w.requests)
    outs = [torch.empty((3, q.camera.height, q.camera.width), device=dev) for q in w.requests]
    gen = torch.Generator(device=dev).manual_seed(9)
    dls = [torch.randn(o.shape, generator=gen, device=dev) * 1e-3 for o in outs]
    steps = max(1, min(args.steps, 5))
    tune = r.tune_batch(gs, frames, reqs, dL_dimages=dls, depths=(16, 32, 64, 128), iters=2, outs=outs)
    best = tune["best"]
    res = {"workload": "500k Gaussians, SH degree 3, 128 motion groups; 16 views x 8 frames = 128 requests, "
                       "level ~ U{L1..L6}, resolution ~ U{960x540, 1280x720, 1920x1080}; forward + backward",
           "pixels_per_step": px, "unit": UNIT, "steps": steps,
           "tile": f"{best['tile'][0]}x{best['tile'][1]}", "batch_depth": best["depth"], "autotune": tune}
    for name, g_set in (("batched_fp32", gs), ("batched_bf16_fp8", gsq)):
        g = gc.BatchGraph(r, g_set, frames, reqs, best["depth"], dL_dimages=dls,
                          grads=r.batch_grads(g_set, frames), outs=outs)
        g.launch()
        g.check()
        ms, prof, clk = timer(g.launch, steps, name="b128_" + name)
        g.check()
        res[name] = {"value": round(px * steps / (ms / 1e3) / 1e6, 1), "ms_per_step": round(ms / steps, 2),
                     "gpu_launches": prof["kernel_launches"], "clocks": clk}
        g.close()
        torch.cuda.empty_cache()
    rs = gc.Renderer(r.device, tile=best["tile"])
    sv = gc.Saved(rs)
    grads = None

    def single():
        nonlocal grads
        for q, (cam, f, mask) in enumerate(reqs):
            rs.forward(gs, frames[f], mask, cam, sv, out=outs[q])
            grads = rs.backward(sv, gs, frames[f], dls[q], grads)

    single()
    ms, _, _ = timer(single, max(1, min(steps, 2)), name="b128_single_view")
    res["single_view_fp32"] = {"value": round(px * max(1, min(steps, 2)) / (ms / 1e3) / 1e6, 1),
                               "ms_per_step": round(ms / max(1, min(steps, 2)), 2)}
    del sv, grads
    rs.close()
    r.set_options(tile=HEADLINE_TILE, key_capacity=0)
    return res


def run_e2e(args, r, w, reqs, cap, tile, W, H, dev, stream):
    """Same metric through the public API with host buffers, on the headline path: every
    step copies the scene and motion tables from pinned host memory, renders levels 1..6
    of every frame in one pass each and copies every image to its own pinned host buffer
    (180 images per step); the copies of frame f's six images overlap the render of frame
    f + 1.  After the timed steps one sampled image on the host is compared with a fresh
    device render of the same request."""
    import numpy as np
    import torch

    import paper_2509_17513_b300 as gc

    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k), np.float32)).pin_memory()
            for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    host["group_id"] = torch.from_numpy(np.ascontiguousarray(w.scene.group_id, np.int32)).pin_memory()
    hq = torch.from_numpy(np.ascontiguousarray(w.motion.q[: args.frames])).pin_memory()
    ht = torch.from_numpy(np.ascontiguousarray(w.motion.t[: args.frames])).pin_memory()
    dev_t = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    dq = torch.empty_like(hq, device=dev)
    dt = torch.empty_like(ht, device=dev)
    gs = gc.GaussianSet(w.scene.layer_offsets, w.scene.sh_degree, 0, **dev_t)
    frames = [gc.MotionFrame(dq[f], dt[f]) for f in range(args.frames)]
    r.set_options(key_capacity=cap, tile=tile)
    nring = 2
    ring = [[torch.empty((3, H, W), device=dev) for _ in range(6)] for _ in range(nring)]
    n_img = 6 * args.frames
    out_host = torch.empty((n_img, 3, H, W), pin_memory=True)   # one pinned buffer per image
    copy_stream = torch.cuda.Stream(device=dev)
    rendered = [torch.cuda.Event() for _ in range(nring)]
    copied = [torch.cuda.Event() for _ in range(nring)]
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + hq.numel() * 4 + ht.numel() * 4
    d2h = n_img * 3 * H * W * 4

    def step():
        for k, v in host.items():
            dev_t[k].copy_(v, non_blocking=True)
        dq.copy_(hq, non_blocking=True)
        dt.copy_(ht, non_blocking=True)
        for f in range(args.frames):
            slot = f % nring
            if f >= nring:
                stream.wait_event(copied[slot])
            r.levels_forward(gs, frames[f], 6, w.cameras[f], outs=ring[slot])
            rendered[slot].record(stream)
            copy_stream.wait_event(rendered[slot])
            with torch.cuda.stream(copy_stream):
                for i in range(6):
                    out_host[6 * f + i].copy_(ring[slot][i], non_blocking=True)
                copied[slot].record(copy_stream)
        stream.wait_stream(copy_stream)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    steps = max(2, args.steps // 2)
    out_host.fill_(float("nan"))
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max(e0.elapsed_time(e1), 1e-6)
    wall = (time.perf_counter() - t0) * 1e3
    r.check()
    # every image of the step is on the host; a sampled one equals a fresh device render
    all_finite = bool(torch.isfinite(out_host).all())
    fs, ls = min(args.frames - 1, 17), 4
    chk = [torch.empty((3, H, W), device=dev) for _ in range(6)]
    r.levels_forward(gs, frames[fs], 6, w.cameras[fs], outs=chk)
    torch.cuda.synchronize()
    same = bool(torch.equal(chk[ls - 1].cpu(), out_host[6 * fs + ls - 1]))
    r.set_options(key_capacity=0)
    del out_host, ring, chk
    return {"value": round(n_img * W * H * steps / (ms / 1e3) / 1e6, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(ms / steps, 3), "wall_ms_per_step": round(wall / steps, 3),
            "all_images_on_host": all_finite and same,
            "check": f"all {n_img} host images finite; frame {fs} level L{ls} equals a fresh device render: {same}",
            "note": "pinned host scene + motion in, every image to its own pinned host buffer; one multi-level "
                    "pass per frame, the six images' copies on a second stream overlap the next frame"}


# --------------------------------------------------------------------------- oracle legs

def cpu_baseline(w=None, gpu_frame0=None, c5=None, n_pix=131072) -> dict:
    """The FP64 oracle as it stands, on the host cores, on a bounded sample: frame 0 of the
    workload at every level L1..L6, `n_pix` seeded pixels each (the timed part).  The same
    sampled pixels are then compared with the GPU's images of frame 0, and, when the
    precision workload ran, 2,048 sampled pixels of its frame with the GPU's FP32 and
    BF16/FP8 images (the latter on the dequantised scene and on the FP32 scene)."""
    import numpy as np

    import oracle
    from synth import scenes

    if w is None:
        w = scenes.hier1080(n_frames=1)
    cam = w.cameras[0]
    opts = oracle.default_options(tile=HEADLINE_TILE)
    t0 = time.perf_counter()
    px = 0
    refs = []
    for lv in range(1, 7):
        pix = scenes.sample_pixels(1000 + lv, cam.width, cam.height, n_pix)
        refs.append((pix, oracle.render(w.scene, w.motion, 0, cam, opts, scenes.level_mask(lv), pixels=pix)))
        px += len(pix)
    dt = time.perf_counter() - t0
    out = {"value": round(px / dt / 1e6, 4), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"frame 0 at levels L1..L6, {n_pix} seeded pixels each of 1920x1080 "
                     f"({6 * n_pix} pixels, per-render binning included), {dt:.1f} s",
           "sample_short": f"frame 0, L1..L6, {n_pix} px each, {dt:.1f} s"}
    parity = {}
    if gpu_frame0 is not None:
        worst, mse_sum, n_amb, n_tot = 0.0, 0.0, 0, 0
        for (pix, ref), img in zip(refs, gpu_frame0):
            g = img.cpu().numpy()[:, pix[:, 1], pix[:, 0]].T.astype(np.float64)
            want = np.asarray(ref["image"])          # (n, 3) at the sampled pixels
            amb = np.asarray(ref["ambiguous"]).reshape(-1)
            err = np.abs(g - want).max(axis=1)
            worst = max(worst, float(err[~amb].max()))
            mse_sum += float(((g - want) ** 2).mean()) * len(pix)
            n_amb += int(amb.sum())
            n_tot += len(pix)
        parity["hier1080_frame0"] = {"max_abs_err_non_ambiguous": worst,
                                     "psnr_db": round(10 * math.log10(1.0 / (mse_sum / n_tot)), 2)
                                     if mse_sum > 0 else None, "ambiguous": n_amb, "pixels": n_tot}
    if c5 is not None:
        w5, cam5 = c5["w"], c5["cam"]
        pix = scenes.sample_pixels(2024, cam5.width, cam5.height, 2048)
        o5 = oracle.default_options(tile=c5["tile"])
        deq = oracle.dequantize(c5["q"], w5.scene)
        for key, scene, img in (("c5_fp32", w5.scene, c5["img_fp32"]),
                                ("c5_bf16_fp8_vs_dequantised", deq, c5["img_bf16_fp8"]),
                                ("c5_bf16_fp8_vs_fp32_scene", w5.scene, c5["img_bf16_fp8"])):
            ref = oracle.render(scene, w5.motion, 1, cam5, o5, 63, pixels=pix)
            g = img.numpy()[:, pix[:, 1], pix[:, 0]].T.astype(np.float64)
            want = np.asarray(ref["image"])
            amb = np.asarray(ref["ambiguous"]).reshape(-1)
            mse = float(((g - want) ** 2).mean())
            parity[key] = {"max_abs_err_non_ambiguous": float(np.abs(g - want).max(axis=1)[~amb].max()),
                           "psnr_db": round(10 * math.log10(1.0 / mse), 2) if mse > 0 else None,
                           "ambiguous": int(amb.sum()), "pixels": len(pix)}
    out["parity"] = parity
    out["parity_short"] = {k: [round(v["max_abs_err_non_ambiguous"], 7), v["psnr_db"]] for k, v in parity.items()}
    return out


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    from synth import scenes

    w = scenes.hier1080(n_frames=min(args.frames, 30))
    opts = oracle.default_options()
    n_pix = 32768
    reqs = [(f, lv) for f in range(w.motion.n_frames) for lv in range(1, 7)]

    def one(i):
        f, lv = reqs[i % len(reqs)]
        cam = w.cameras[f]
        pix = scenes.sample_pixels(i, cam.width, cam.height, n_pix)
        oracle.render(w.scene, w.motion, f, cam, opts, scenes.level_mask(lv), pixels=pix)

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(args.warmup + i)
    dt = time.perf_counter() - t0
    value = n_pix * args.steps / dt / 1e6
    sample = (f"each step: one (frame, level) request of the workload cycling through the 180, "
              f"{n_pix} seeded pixels of 1920x1080, per-render binning included")
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scene shaped like the paper's workload; no dataset)",
            "config": {"workload": WORKLOAD, "n_gaussians": w.scene.n, "width": 1920,
                       "height": 1080, "parallelism": "host cores"},
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gc4d", choices=["gc4d", "reference"])
    ap.add_argument("--frames", type=int, default=30, help="frames of the workload (30 = full)")
    ap.add_argument("--detail", default=None, help="write every figure (JSON) to this path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch128", action="store_true", help="skip the 128-request batching workload")
    ap.add_argument("--skip-forms", default="",
                    help="comma list of forms to leave out: single, batched, residual, planes, field, kde, c1, c3, c5")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
