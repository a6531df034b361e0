#!/usr/bin/env python
"""Throughput of the hierarchical 4D Gaussian rasterizer on one B300 (or N replicas).

Workload (the 300k-Gaussian hierarchical scene at 1920x1080): 300,000 Gaussians in
6 nested layers of 50k (SH degree 3, 64 motion groups), 30 frames of cumulative
group motion, every frame rendered at every level L1..L6 on an orbit camera.  One
step = those 180 renders through the library (motion, projection, depth sort,
binning, tile sort, blend), rendered per frame by the single-pass multi-level render
(levels L1..L6 from one list; every image equals its single-level render bit for bit).
Value = Mpixel/s over all ranks.  The same line carries the forward + backward step,
the same 180 renders as batched requests replayed from one CUDA graph (tile shape and
batch depth autotuned), the plain FP32 single-view form (one call per render), the
BF16/FP8 storage form, the 128-request batching workload, the end-to-end figure with
host buffers, and the oracle timed on the host cores.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank renders its own 180-request step on its own GPU (the
requests are independent, no data-path collective): weak scaling.  Timing: CUDA
events on the rendering stream, L2 flushed between steps (outside the events),
max over ranks.  ``--impl reference`` times the FP64 CPU oracle on the host.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
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
# FP32 FLOPs (FMA = 2) of the compositing rule (Eq. 2): evaluating one (pixel, entry) pair up to
# the 1/255 test, and the extra work of a pair that is blended (forward / reverse step)
EVAL_FLOPS_PER_PAIR = 14
FWD_BLEND_FLOPS_PER_PAIR = 10
BWD_BLEND_FLOPS_PER_PAIR = 51
SORT_BYTES_PER_KEY_PASS = 20  # histogram read 4 B + scatter read 8 B + write 8 B


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def measure_fp32_peak(dev, n=8192, iters=20):
    """FP32 FMA throughput measured as cuBLAS SGEMM (TF32 off: plain FP32 FMAs) on n x n,
    TFLOP/s, after a warm-up; the denominator of the ALU-bound (blend) kernels."""
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


# the source file that defines each profiled kernel; its hash covers that file and the kernel
# sources it includes (transitively).  A kernel not listed depends on every source file.
HEADLINE_TILE = (8, 32)  # tile shape (width x height) of the multi-level headline
HOST_AHEAD_CYCLES = 200_000_000  # GPU spin before a stage-profiled step (about 0.1 s at 2 GHz)

KERNEL_SOURCES = {"k_blend_levels_fwd": "gc_levels.cu", "k_blend_levels_bwd": "gc_levels.cu",
                  "k_blend_fwd": "gc_raster.cu", "k_emit": "gc_raster.cu", "k_radix_scatter": "gc_sort.cu",
                  "k_batch_blend_fwd": "gc_batch.cu", "k_batch_blend_bwd": "gc_batch.cu",
                  "k_batch_emit": "gc_batch.cu", "k_field_bwd": "gc_motion_field.cu",
                  "k_field_encode": "gc_motion_field.cu"}


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


# --------------------------------------------------------------------------- GPU arm

def roofline_for(stage, per_launch_ms, work, peaks, peak_kind, batched=False, renders_per_launch=1, tile=None):
    """Roofline object of the dominant stage.  `work`: algorithmic FLOPs (ALU stages)
    or bytes (HBM stages) of one launch."""
    pre = "k_batch_" if batched else "k_"
    alu = {"blend": "k_batch_blend_fwd" if batched else "k_blend_levels_fwd",
           "blend_bwd": "k_batch_blend_bwd" if batched else "k_blend_levels_bwd"}
    hbm = {"tile_sort": "k_radix_scatter", "emit": pre + "emit", "reduce": pre + "reduce",
           "depth_sort": "k_radix_scatter"}
    if stage in alu:
        derived = N_SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        measured = peaks.get("fp32_sgemm_tflops")
        peak = measured if measured else derived
        achieved = work / (per_launch_ms / 1e3) / 1e12
        kern = alu[stage]
        src = (f"measured: cuBLAS FP32 SGEMM 8192^3 (TF32 off) in this run, {measured:.2f} TFLOP/s; derived "
               f"{N_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x {peaks.get('sm_max_mhz', 2032.0)} MHz = {derived:.2f}"
               if measured else
               f"derived, not measured: {N_SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
               f"x {peaks.get('sm_max_mhz', 2032.0)} MHz max SM clock ({peak_kind} file)")
        return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "frac_of_derived": round(achieved / derived, 4),
                "traffic": load_traffic(kern, renders_per_launch, tile), "kernel": kern,
                "launch_ms": round(per_launch_ms, 4), "peak_source": src}
    if stage in hbm:
        achieved = work / (per_launch_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": load_traffic(hbm[stage], renders_per_launch, tile),
                "kernel": hbm[stage], "launch_ms": round(per_launch_ms, 4),
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    return None


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


class Timer:
    """K steps timed with CUDA events on the rendering stream, L2 flushed between steps
    (outside the events), clocks sampled during the region, max over ranks."""

    def __init__(self, r, stream, local, world, dev):
        import torch
        self.r, self.stream, self.local, self.world, self.dev = r, stream, local, world, dev
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def __call__(self, step, steps, profile=False, name="timed", host_ahead=False):
        """host_ahead: before each step the GPU spins for a bounded time (outside the events),
        so that the host queues the whole step before the GPU reaches it and the stage events
        measure the kernels rather than the host's launch rate."""
        import torch
        import torch.distributed as dist
        clocks = ClockSampler(self.local)
        self.r.profile(profile)
        self.r.profile_read()
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
        prof = self.r.profile_read()
        self.r.profile(False)
        total = max_over_ranks(total, self.world, self.dev)
        return total, prof, clk


def stage_summary(prof):
    st_ms, st_calls = prof["stage_ms"], prof["stage_calls"]
    tot = max(1e-9, sum(st_ms.values()))
    return ({k: round(v / max(1, st_calls[k]), 4) for k, v in st_ms.items() if v > 0},
            {k: round(v / tot, 4) for k, v in st_ms.items() if v > 0})


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
    peaks["fp32_sgemm_tflops"] = round(measure_fp32_peak(dev), 2)
    skip = {x.strip() for x in args.skip_forms.split(",") if x.strip()}

    w = scenes.hier1080(n_frames=args.frames)
    W, H = 1920, 1080
    order = [(f, lv) for f in range(args.frames) for lv in range(1, 7)]
    reqs = [(w.cameras[f], f, scenes.level_mask(lv)) for f, lv in order]
    n_req = len(reqs)
    pixels_per_step = n_req * W * H
    r = gc.Renderer(local)
    timer = Timer(r, stream, local, world, dev)
    gs = gc.GaussianSet.from_scene(w.scene, dev)
    gsq = gc.GaussianSet.from_quantized(scenes.quantize_scene(w.scene), w.scene, dev)
    frames = [gc.MotionFrame.from_motion(w.motion, f, dev) for f in range(args.frames)]
    outs = [torch.empty((3, H, W), device=dev) for _ in range(n_req)]
    upstream = (torch.randn((3, H, W), generator=torch.Generator().manual_seed(7)) * 1e-3).to(dev)
    dls = [upstream] * n_req

    def mpix(total_ms, steps, px=pixels_per_step):
        return round(whole_job_rate(px, steps, world, total_ms) / 1e6, 1)

    # ---- plain FP32 single-view form: one gc_render_forward (+ backward) per request
    single_view = None
    s_steps = max(1, min(args.steps, 3))
    if "single" not in skip:
        saved = gc.Saved(r)
        kmax = 0
        for q, (cam, f, mask) in enumerate(reqs):
            r.forward(gs, frames[f], mask, cam, out=outs[q])
            kmax = max(kmax, r.stats()["n_keys"])
        cap_single = int(kmax * 1.05) + 4096
        r.set_options(key_capacity=cap_single)
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
        sf_ms, sf_prof, _ = timer(single_fwd, s_steps, profile=True, name="single_fwd")
        sfb_ms, sfb_prof, _ = timer(single_fwd_bwd, s_steps, profile=True, name="single_fwd_bwd")
        # per level: the frames of the step rendered at that level alone (forward), FPS and Mpixel/s
        per_level = {}
        for lv in range(1, 7):
            lv_reqs = [(cam, f, mask) for (cam, f, mask) in reqs if mask == scenes.level_mask(lv)]

            def level_fwd(lv_reqs=lv_reqs):
                for q, (cam, f, mask) in enumerate(lv_reqs):
                    r.forward(gs, frames[f], mask, cam, out=outs[q])

            lv_ms, _, _ = timer(level_fwd, s_steps, name=f"single_level_{lv}")
            n_lv = len(lv_reqs) * s_steps
            per_level[f"L{lv}"] = {"fps": round(n_lv * world / (lv_ms / 1e3), 1),
                                   "mpix_s": round(n_lv * W * H * world / (lv_ms / 1e3) / 1e6, 1),
                                   "ms_per_render": round(lv_ms / n_lv, 4)}
        r.check()
        single_view = {"form": "plain FP32, one gc_render_forward (+ gc_render_backward) per request",
                       "fwd": mpix(sf_ms, s_steps), "fwd_bwd": mpix(sfb_ms, s_steps), "unit": UNIT,
                       "ms_per_step": {"fwd": round(sf_ms / s_steps, 2), "fwd_bwd": round(sfb_ms / s_steps, 2)},
                       "per_level_fwd": per_level,
                       "stage_ms_per_render": stage_summary(sfb_prof)[0], "steps": s_steps}
        del saved, grads1
        r.set_options(key_capacity=0)

    # ---- batched form: autotuned tile shape x batch depth, CUDA graph of the whole step
    tune = None
    if "batched" not in skip:
        tune = r.tune_batch(gs, frames, reqs, dL_dimages=dls, depths=(30, 60, 90, n_req), iters=2, outs=outs)
        depth, tile_b = tune["best"]["depth"], tuple(tune["best"]["tile"])
    else:
        depth, tile_b = n_req, HEADLINE_TILE

    # algorithmic work of one step at a tile shape (deterministic, outside the timed regions):
    # walked / blended pairs per render, and of the top level alone (what a multi-level pass walks)
    def count_work(tl):
        r.set_options(tile=tl, key_capacity=0)
        c = {"walked": 0, "blended": 0, "bwd": 0, "keys": 0, "walked_top": 0, "bwd_top": 0, "kmax": 0}
        for q, (cam, f, mask) in enumerate(reqs):
            r.forward(gs, frames[f], mask, cam, out=outs[q])
            _, blended, walked, contrib = r.pixel_state(with_walked=True)
            wq = int(walked.sum(dtype=torch.int64).item())
            cq = int(contrib.sum(dtype=torch.int64).item())
            c["walked"] += wq
            c["blended"] += int(blended.sum(dtype=torch.int64).item())
            c["bwd"] += cq
            if mask == scenes.level_mask(6):
                c["walked_top"] += wq
                c["bwd_top"] += cq
            nk = r.stats()["n_keys"]
            c["keys"] += nk
            c["kmax"] = max(c["kmax"], nk)
        return c

    work_b = count_work(tile_b)
    r.set_options(tile=tile_b)

    def roof(prof, steps, batched, eval_pairs, bwd_eval_pairs, renders_per_step, work):
        st_ms, st_calls = prof["stage_ms"], prof["stage_calls"]
        dom = max(st_ms, key=lambda k: st_ms[k])
        launches = max(1, st_calls[dom])
        per_launch = st_ms[dom] / launches
        fwd_flops = EVAL_FLOPS_PER_PAIR * eval_pairs + FWD_BLEND_FLOPS_PER_PAIR * work["blended"]
        bwd_flops = EVAL_FLOPS_PER_PAIR * bwd_eval_pairs + BWD_BLEND_FLOPS_PER_PAIR * work["blended"]
        amount = {"blend": fwd_flops * steps / launches, "blend_bwd": bwd_flops * steps / launches,
                  "tile_sort": 2 * SORT_BYTES_PER_KEY_PASS * work["keys"] * steps / launches,
                  "emit": 8 * work["keys"] * steps / launches}.get(dom, 0.0)
        return roofline_for(dom, per_launch, amount, peaks, peak_kind, batched=batched,
                            renders_per_launch=renders_per_step * steps // launches,
                            tile=f"{r.options.tile_w}x{r.options.tile_h}")

    batched_obj = precision_obj = None
    if "batched" not in skip:
        grads = r.batch_grads(gs, frames)
        g_fwd = gc.BatchGraph(r, gs, frames, reqs, depth, outs=outs)
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

        # the same batched step, eager with per-stage CUDA events
        sv = [gc.Saved(r) for _ in range((n_req + depth - 1) // depth)]

        def eager(bwd):
            def step():
                for b, s in enumerate(sv):
                    r.batch_forward(gs, frames, reqs[b * depth:(b + 1) * depth], s,
                                    outs=outs[b * depth:(b + 1) * depth])
                if bwd:
                    for b, s in enumerate(sv):
                        r.batch_backward(s, gs, frames, dls[b * depth:(b + 1) * depth], grads=grads,
                                         accumulate=b > 0)
            return step

        r.set_options(key_capacity=cap)
        eager(True)()
        r.check()
        e_steps = max(1, min(args.steps, 3))
        ef_ms, ef_prof, _ = timer(eager(False), e_steps, profile=True, name="eager_fwd")
        efb_ms, efb_prof, _ = timer(eager(True), e_steps, profile=True, name="eager_fwd_bwd")
        r.check()
        del sv
        r.set_options(key_capacity=0)

        # ---- reduced-precision storage (BF16 geometry, FP8-E4M3 SH), same batched graph
        gq = gc.BatchGraph(r, gsq, frames, reqs, depth, dL_dimages=dls, grads=r.batch_grads(gsq, frames), outs=outs)
        for _ in range(args.warmup):
            gq.launch()
        gq.check()
        q_ms, _, clk_q = timer(gq.launch, args.steps, name="graph_bf16_fp8_fwd_bwd")
        gq.check()
        q_imgs = outs[:: max(1, n_req // 12)]
        mse = sum(float(((a - b) ** 2).mean()) for a, b in zip(q_imgs, ref_imgs)) / len(ref_imgs)
        q_psnr = round(10 * np.log10(1.0 / mse), 2) if mse > 0 else None
        gq.close()
        batched_obj = {"form": "the 180 renders as batched requests replayed from one CUDA graph "
                               "(autotuned tile shape and batch depth)",
                       "fwd": mpix(bf_ms, args.steps), "fwd_bwd": mpix(bfb_ms, args.steps), "unit": UNIT,
                       "ms_per_step": {"fwd": round(bf_ms / args.steps, 3), "fwd_bwd": round(bfb_ms / args.steps, 3)},
                       "tile": f"{tile_b[0]}x{tile_b[1]}", "batch_depth": depth, "key_capacity_per_batch": cap,
                       "clocks": {"fwd": clk_bf, "fwd_bwd": clk_bfb},
                       "roofline": {"fwd": roof(ef_prof, e_steps, True, work_b["walked"], work_b["bwd"], n_req, work_b),
                                    "fwd_bwd": roof(efb_prof, e_steps, True, work_b["walked"], work_b["bwd"], n_req,
                                                    work_b)},
                       "stage_ms_per_call": stage_summary(efb_prof)[0],
                       "stage_share_fwd": stage_summary(ef_prof)[1],
                       "stage_share_fwd_bwd": stage_summary(efb_prof)[1],
                       "eager_fwd": mpix(ef_ms, e_steps), "eager_fwd_bwd": mpix(efb_ms, e_steps)}
        precision_obj = {"storage": "BF16 means/log-scales/quats/opacity, FP8-E4M3 SH, FP32 scales; "
                                    "FP32 arithmetic; batched graph", "fwd_bwd": mpix(q_ms, args.steps),
                         "unit": UNIT, "ms_per_step": round(q_ms / args.steps, 3),
                         "psnr_vs_fp32_scene_db": q_psnr, "clocks": clk_q,
                         "bytes_per_gaussian": {"fp32": 4 * 59 + 4, "bf16_fp8": 2 * 11 + 48 + 4}}
        del ref_imgs, grads

    # ---- headline: single-pass multi-level form, per frame levels 1..6 from one list (the
    # same 180 images, bit for bit), fixed key capacity, per-stage CUDA events
    # the headline and the forms after it use 8x32 tiles, the shape the multi-level blend kernels
    # are profiled with; on this workload the batched autotuner finds 16x16 and 8x32 within a
    # fraction of a percent of each other
    tile = HEADLINE_TILE
    work = work_b if tuple(tile) == tuple(tile_b) else count_work(tile)
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
    # per-stage CUDA events with the host queued ahead of the GPU: kernel times, not launch gaps
    _, fwd_prof, _ = timer(levels_fwd, args.steps, profile=True, name="levels_fwd_stages", host_ahead=True)
    _, fb_prof, _ = timer(levels_fwd_bwd, args.steps, profile=True, name="levels_fwd_bwd_stages", host_ahead=True)
    r.check()
    # the headline value: the same steps replayed from one CUDA graph each (gc_levels_graph:
    # no host work, no launch gaps between the kernels of a frame, identical images); the
    # eager runs above give the per-stage split and the blend kernels' launch times
    cams_step = w.cameras[:args.frames]
    lg_fwd = gc.LevelsGraph(r, gs, frames, cams_step, 6, outs=outs[:6 * args.frames])
    lg_fb = gc.LevelsGraph(r, gs, frames, cams_step, 6, outs=outs[:6 * args.frames],
                           dL_dimages=dls[:6 * args.frames], grads=[lgrads] * args.frames)
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
    del lsaved, lgrads
    r.set_options(key_capacity=0)
    frames_per_step = args.frames

    # ---- the paper's decoded attribute planes (Sec. 3.4): the same multi-level step with the
    # scene stored as uint16 position planes and uint8 planes per layer (62 B per Gaussian)
    planes_obj = None
    if "planes" not in skip:
        ref_imgs = [o.clone() for o in outs[:: max(1, n_req // 12)]]
        gpl = gc.GaussianSet.from_planes(scenes.quantize_planes(w.scene, plane_width=1024), w.scene, dev)
        r.set_options(key_capacity=0, tile=tile)
        kmax = 0
        for f in range(args.frames):
            r.levels_forward(gpl, frames[f], 6, w.cameras[f], outs=outs[6 * f:6 * f + 6])
            kmax = max(kmax, r.stats()["n_keys"])
        q_imgs = outs[:: max(1, n_req // 12)]
        mse = sum(float(((a - b) ** 2).mean()) for a, b in zip(q_imgs, ref_imgs)) / len(ref_imgs)
        r.set_options(key_capacity=int(kmax * 1.02) + 4096, tile=tile)

        def planes_fwd():
            for f in range(args.frames):
                r.levels_forward(gpl, frames[f], 6, w.cameras[f], outs=outs[6 * f:6 * f + 6])

        for _ in range(args.warmup):
            planes_fwd()
        r.check()
        pf_ms, pf_prof, clk_pf = timer(planes_fwd, args.steps, profile=True, name="planes_fwd")
        r.check()
        planes_obj = {"form": "the headline multi-level forward step rendered from the decoded attribute planes "
                              "(uint16 positions, uint8 quaternion / log-scale / opacity / SH planes per layer, "
                              "per-layer per-channel min/max affine dequantisation in the preprocess)",
                      "fwd": mpix(pf_ms, args.steps), "unit": UNIT, "ms_per_step": round(pf_ms / args.steps, 3),
                      "bytes_per_gaussian": {"fp32": 4 * 59 + 4, "planes": 2 * 3 + 8 + 48},
                      "preprocess_ms_per_call": stage_summary(pf_prof)[0].get("preprocess"),
                      "psnr_vs_fp32_scene_db": round(10 * np.log10(1.0 / mse), 2) if mse > 0 else None,
                      "clocks": clk_pf}
        del gpl, ref_imgs
        r.set_options(key_capacity=0)
        torch.cuda.empty_cache()

    # ---- per-Gaussian motion source (Sec. 3.2): per frame the hash-grid + MLP motion of all
    # 300k Gaussians, then the multi-level render with one rigid motion per Gaussian
    field_obj = None
    if "field" not in skip:
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

        def field_step():
            for f in range(args.frames):
                q_, t_ = r.motion_field_forward(field, means_d)
                r.levels_forward(gs, gc.MotionFrame(q_, t_, per_gaussian=True), 6, w.cameras[f],
                                 outs=outs[6 * f:6 * f + 6])

        for _ in range(args.warmup):
            field_fwd()
            field_bwd()
            field_step()
        r.check()
        mff_ms, _, _ = timer(field_fwd, args.steps, name="field_fwd")
        mfb_ms, _, _ = timer(field_bwd, args.steps, name="field_bwd")
        mfs_ms, _, clk_fs = timer(field_step, args.steps, name="field_step")
        r.check()
        n_g = w.scene.n
        per_ms_f = mff_ms / args.steps / args.frames
        field_obj = {"form": "per-Gaussian motion source (Sec. 3.2): 16-level hash grid (2^19 entries x 2 features "
                             "per level, resolutions 16..2048) + translation and rotation MLPs (32-64-3, 32-64-4) "
                             "for the 300k Gaussians of every frame, then the multi-level render with one rigid "
                             "motion per Gaussian",
                     "field_fwd_ms_per_frame": round(per_ms_f, 4),
                     "field_bwd_ms_per_frame": round(mfb_ms / args.steps / args.frames, 4),
                     "field_fwd_gaussians_per_s": round(n_g / (per_ms_f / 1e3), 1),
                     "field_fwd_tflops": round(n_g * 2 * (2 * 64 * 32 + 7 * 64) / (per_ms_f / 1e3) / 1e12, 3),
                     "step_fwd": mpix(mfs_ms, args.steps), "unit": UNIT, "key_capacity": fcap,
                     "clocks": clk_fs}
        del field, fq, ft, gq_up, gt_up
        r.set_options(key_capacity=0)
        torch.cuda.empty_cache()

    # ---- KDE rate estimate (Sec. 3.3): bits per symbol of every uint8 attribute channel of every
    # layer of the quantised scene (the rate term of the layer-wise RD loss)
    kde_obj = None
    if "kde" not in skip:
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
            rates = kde_step()
        k_ms, _, _ = timer(kde_step, args.steps, name="kde_rate")
        rates = torch.stack(kde_step()).cpu().numpy()
        # training form: the same channels with injected uniform noise (device-generated), rate
        # and its gradient through the values, upstream gradient 1 per channel
        gen = torch.Generator(device=dev).manual_seed(21)
        ys_noisy = [yl + (torch.rand(yl.shape, generator=gen, device=dev) - 0.5) for yl in ys]

        def kde_grad_step():
            return [r.kde_rate_grad(yl) for yl in ys_noisy]

        for _ in range(args.warmup):
            kde_grad_step()
        kg_ms, _, _ = timer(kde_grad_step, args.steps, name="kde_rate_grad")
        n_sym = sum(int(yl.numel()) for yl in ys)
        kde_obj = {"form": "KDE rate estimate of the keyframe RD loss (Sec. 3.3): Silverman-bandwidth kernel "
                           "density PMF of the quantised symbols of each uint8 attribute channel of each layer "
                           "(56 channels x 6 layers of hier1080, 300k Gaussians)",
                   "ms_per_step": round(k_ms / args.steps, 4), "channels": int(rates.size),
                   "symbols_per_s": round(n_sym / (k_ms / args.steps / 1e3), 1),
                   "mean_bits_per_symbol": round(float(np.nanmean(rates)), 4),
                   "training_form": {"note": "noise-injected values, the symbols' density held fixed, rate and "
                                             "dR/dy of every value (gc_kde_rate_grad)",
                                     "ms_per_step": round(kg_ms / args.steps, 4),
                                     "values_per_s": round(n_sym / (kg_ms / args.steps / 1e3), 1)}}
        del ys, ys_noisy

    # ---- residual deformation (Eq. 7): the same multi-level step with per-frame log-scale,
    # logit and SH residuals fused into the preprocess (device-generated, N(0, f sigma^2))
    residual_obj = None
    if "residual" not in skip:
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
        residual_obj = {"form": "the headline multi-level step with per-frame residual deformation (Eq. 7): "
                                "log-scale, opacity-logit and SH residuals (208 B per Gaussian per frame) "
                                "added inside the preprocess and the chain rule",
                        "fwd": mpix(rf_ms, args.steps), "fwd_bwd": mpix(rfb_ms, args.steps), "unit": UNIT,
                        "ms_per_step": {"fwd": round(rf_ms / args.steps, 3), "fwd_bwd": round(rfb_ms / args.steps, 3)},
                        "key_capacity": int(kmax * 1.02) + 4096, "clocks": {"fwd": clk_rf, "fwd_bwd": clk_rfb}}
        del rsaved, rgrads, rframes
        r.set_options(key_capacity=0)
        torch.cuda.empty_cache()

    line = {"metric": METRIC, "value": mpix(fwd_ms, args.steps), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(fwd_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scene shaped like the paper's workload; no dataset)",
            "config": {"workload": WORKLOAD, "n_gaussians": w.scene.n, "width": W, "height": H,
                       "renders_per_step": n_req,
                       "path": "single-pass multi-level render: per frame one gc_render_levels_forward "
                               "(+ gc_render_levels_backward) renders levels L1..L6; the step's frames "
                               "replayed from one CUDA graph (gc_levels_graph)",
                       "tile": f"{tile[0]}x{tile[1]}", "key_capacity": cap_levels,
                       "l2": "flushed (256 MB write) between steps, outside the timed events",
                       "parallelism": f"replicas x{world}"},
            "fps": round(n_req * args.steps * world / (fwd_ms / 1e3), 1),
            "gpu_launches": gfwd_prof["kernel_launches"],
            "roofline": roof(fwd_prof, args.steps, False, work["walked_top"], work["bwd_top"], frames_per_step, work),
            "clocks": clk,
            "eager": {"note": "the same steps as eager calls (one library call per frame); stage_profile and "
                              "the roofline launch times come from per-stage CUDA events of further eager "
                              "steps, each queued whole by the host before the GPU starts it",
                      "fwd": mpix(ef_lv_ms, args.steps), "fwd_bwd": mpix(efb_lv_ms, args.steps), "unit": UNIT,
                      "gpu_launches": {"fwd": efwd_prof["kernel_launches"], "fwd_bwd": efb_lv_prof["kernel_launches"]},
                      "graph_kernel_nodes": graph_nodes, "clocks": {"fwd": clk_e, "fwd_bwd": clk_efb}},
            "fwd_bwd": {"metric": "Mpixel/s at 1920x1080, forward + backward (upstream dL/dimage given), "
                                  "gradients summed over the step's renders",
                        "value": mpix(fb_ms, args.steps), "unit": UNIT,
                        "ms_per_step": round(fb_ms / args.steps, 3),
                        "fps": round(n_req * args.steps * world / (fb_ms / 1e3), 1),
                        "gpu_launches": gfb_prof["kernel_launches"],
                        "roofline": roof(fb_prof, args.steps, False, work["walked_top"], work["bwd_top"],
                                         frames_per_step, work),
                        "clocks": clk_fb},
            "stage_profile": {"note": "ms per call of the headline path (one frame, six levels)",
                              "stage_ms_per_call_fwd_bwd": stage_summary(fb_prof)[0],
                              "stage_share_fwd": stage_summary(fwd_prof)[1],
                              "stage_share_fwd_bwd": stage_summary(fb_prof)[1]},
            "batched": batched_obj,
            "residual_deformation": residual_obj,
            "decoded_planes": planes_obj,
            "motion_field": field_obj,
            "kde_rate": kde_obj,
            "single_view": single_view,
            "reduced_precision": precision_obj,
            "autotune": tune,
            "work_per_step": {"blend_walked_pairs": work["walked"], "blended_pairs": work["blended"],
                              "blend_bwd_walked_pairs": work["bwd"], "top_level_walked_pairs": work["walked_top"],
                              "top_level_bwd_walked_pairs": work["bwd_top"],
                              "keys_per_render": round(work["keys"] / n_req),
                              "flops_per_pair": {"evaluate": EVAL_FLOPS_PER_PAIR,
                                                 "blend_fwd": FWD_BLEND_FLOPS_PER_PAIR,
                                                 "blend_bwd": BWD_BLEND_FLOPS_PER_PAIR}}}
    line = {k: v for k, v in line.items() if v is not None}
    del outs, dls
    torch.cuda.empty_cache()

    if not args.no_batch128:
        line["batch128"] = run_batch128(args, r, timer, dev)
        torch.cuda.empty_cache()
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, r, w, reqs, cap_levels, tile, W, H, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


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
           "tile": f"{best['tile'][0]}x{best['tile'][1]}", "batch_depth": best["depth"]}
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
    return res


def run_e2e(args, r, w, reqs, cap, tile, W, H, dev, stream):
    """Same metric through the public API with host buffers, on the headline path: every
    step copies the scene and motion tables from pinned host memory, renders levels 1..6
    of every frame in one pass each and reads every image back to pinned host memory;
    the copy of frame f's six images overlaps the render of frame f + 1."""
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
    out_host = [torch.empty((3, H, W)).pin_memory() for _ in range(6)]
    copy_stream = torch.cuda.Stream(device=dev)
    rendered = [torch.cuda.Event() for _ in range(nring)]
    copied = [torch.cuda.Event() for _ in range(nring)]
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + hq.numel() * 4 + ht.numel() * 4
    d2h = len(reqs) * 3 * H * W * 4

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
                    out_host[i].copy_(ring[slot][i], non_blocking=True)
                copied[slot].record(copy_stream)
        stream.wait_stream(copy_stream)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    steps = max(2, args.steps // 2)
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
    r.set_options(key_capacity=0)
    return {"value": round(len(reqs) * W * H * steps / (ms / 1e3) / 1e6, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(ms / steps, 3), "wall_ms_per_step": round(wall / steps, 3),
            "note": "pinned host scene + motion in, every image back to pinned host; one multi-level pass "
                    "per frame, the six images' copies on a second stream overlap the next frame"}


# --------------------------------------------------------------------------- oracle legs

def cpu_baseline(w=None, n_pix=131072) -> dict:
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    frame 0 of the workload at every level L1..L6, `n_pix` seeded pixels each."""
    import oracle
    from synth import scenes

    if w is None:
        w = scenes.hier1080(n_frames=1)
    cam = w.cameras[0]
    opts = oracle.default_options()
    t0 = time.perf_counter()
    px = 0
    for lv in range(1, 7):
        pix = scenes.sample_pixels(1000 + lv, cam.width, cam.height, n_pix)
        oracle.render(w.scene, w.motion, 0, cam, opts, scenes.level_mask(lv), pixels=pix)
        px += len(pix)
    dt = time.perf_counter() - t0
    return {"value": round(px / dt / 1e6, 4), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"frame 0 at levels L1..L6, {n_pix} seeded pixels each of 1920x1080 "
                      f"({6 * n_pix} pixels, per-render binning included), {dt:.1f} s"}


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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch128", action="store_true", help="skip the 128-request batching workload")
    ap.add_argument("--skip-forms", default="", help="comma list of side forms to leave out: single, batched, residual, planes, field, kde "
                    "(then 8x32 tiles are used and the BF16/FP8 form is left out too)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
