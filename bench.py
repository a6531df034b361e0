#!/usr/bin/env python
"""Throughput of the hierarchical 4D Gaussian rasterizer on one B300 (or N replicas).

Workload (the 300k-Gaussian hierarchical scene at 1920x1080): 300,000 Gaussians in
6 nested layers of 50k (SH degree 3, 64 motion groups), 30 frames of cumulative
group motion, every frame rendered at every level L1..L6 on an orbit camera.  One
step = those 180 renders through the library (motion, projection, depth sort,
binning, tile sort, blend).  Value = Mpixel/s over all ranks.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank renders its own 180-request step on its own GPU (the
requests are independent, no data-path collective): weak scaling.  Timing: CUDA
events on the rendering stream, L2 flushed between steps (outside the events),
max over ranks.  ``--impl reference`` times the FP64 CPU oracle on the host.
"""
from __future__ import annotations

import argparse
import hashlib
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
BLEND_FLOPS_PER_PAIR = 26  # FP32 ops of one compositing step (Eq. 2), see the design doc
BLEND_BWD_FLOPS_PER_PAIR = 48  # FP32 ops of one reverse compositing step incl. its share of the reduction
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


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2509_17513_b300", "csrc")
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if current."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- GPU arm

def roofline_for(stage, per_launch_ms, work, peaks, peak_kind):
    """Roofline object of the dominant stage.  `work`: algorithmic FLOPs (ALU stages)
    or bytes (HBM stages) of one launch."""
    alu = {"blend": ("k_blend_fwd", BLEND_FLOPS_PER_PAIR), "blend_bwd": ("k_blend_bwd", BLEND_BWD_FLOPS_PER_PAIR)}
    hbm = {"tile_sort": "k_radix_scatter", "emit": "k_emit", "reduce": "k_reduce_entries",
           "depth_sort": "k_radix_scatter"}
    if stage in alu:
        peak = N_SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        achieved = work / (per_launch_ms / 1e3) / 1e12
        kern = alu[stage][0]
        return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": load_traffic(kern), "kernel": kern,
                "launch_ms": round(per_launch_ms, 4),
                "peak_source": f"derived, not measured: {N_SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                               f"x {peaks.get('sm_max_mhz', 2032.0)} MHz max SM clock ({peak_kind} file)"}
    if stage in hbm:
        achieved = work / (per_launch_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": load_traffic(hbm[stage]),
                "kernel": hbm[stage], "launch_ms": round(per_launch_ms, 4),
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    return None


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

    w = scenes.hier1080(n_frames=args.frames)
    W, H = 1920, 1080
    reqs = [(f, lv) for f in range(args.frames) for lv in range(1, 7)]
    r = gc.Renderer(local)
    gs = gc.GaussianSet.from_scene(w.scene, dev)
    motions = [gc.MotionFrame.from_motion(w.motion, f, dev) for f in range(args.frames)]
    ring = [torch.empty((3, H, W), device=dev) for _ in range(4)]
    saved = gc.Saved(r)
    upstream = (torch.randn((3, H, W), generator=torch.Generator().manual_seed(7)) * 1e-3).to(dev)
    grads = None

    # capacity for the (tile, Gaussian) lists: the largest frame of the workload, plus slack
    kmax = 0
    for (f, lv) in reqs:
        r.forward(gs, motions[f], scenes.level_mask(lv), w.cameras[f], out=ring[0])
        kmax = max(kmax, r.stats()["n_keys"])
    cap = int(kmax * 1.05) + 4096
    r.set_options(key_capacity=cap)

    def step_fwd():
        for i, (f, lv) in enumerate(reqs):
            r.forward(gs, motions[f], scenes.level_mask(lv), w.cameras[f], out=ring[i % 4])

    def step_fwd_bwd():
        nonlocal grads
        for i, (f, lv) in enumerate(reqs):
            r.forward(gs, motions[f], scenes.level_mask(lv), w.cameras[f], saved, out=ring[i % 4])
            grads = r.backward(saved, gs, motions[f], upstream, grads)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step_fwd()
        step_fwd_bwd()
    r.check()
    torch.cuda.synchronize()

    # algorithmic work of one step (deterministic; measured outside the timed regions)
    walked_pairs = bwd_pairs = keys_total = 0
    for (f, lv) in reqs:
        r.forward(gs, motions[f], scenes.level_mask(lv), w.cameras[f], out=ring[0])
        _, _, walked, contrib = r.pixel_state(with_walked=True)
        walked_pairs += int(walked.sum(dtype=torch.int64).item())
        bwd_pairs += int(contrib.sum(dtype=torch.int64).item())
        keys_total += r.stats()["n_keys"]
    keys_mean = keys_total / len(reqs)
    torch.cuda.synchronize()

    def timed(step):
        """K steps, CUDA events on the rendering stream, L2 flushed between steps."""
        clocks = ClockSampler(local)
        r.profile(True)
        r.profile_read()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        total = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        clk = clocks.stop()
        prof = r.profile_read()
        r.profile(False)
        r.check()
        if world > 1:
            t = torch.tensor([total], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total = float(t.item())
        return total, prof, clk

    peaks, peak_kind = measured_peaks()
    pixels_per_step = len(reqs) * W * H

    def summary(total_ms, prof):
        st_ms, st_calls = prof["stage_ms"], prof["stage_calls"]
        dom = max(st_ms, key=lambda k: st_ms[k])
        per_launch = st_ms[dom] / max(1, st_calls[dom])
        work = {"blend": walked_pairs / len(reqs) * BLEND_FLOPS_PER_PAIR,
                "blend_bwd": bwd_pairs / len(reqs) * BLEND_BWD_FLOPS_PER_PAIR,
                "tile_sort": 2 * SORT_BYTES_PER_KEY_PASS * keys_mean,
                "emit": 8 * keys_mean, "reduce": 40 * keys_mean}.get(dom, 0.0)
        tot = max(1e-9, sum(st_ms.values()))
        return {"value": round(pixels_per_step * args.steps * world / (total_ms / 1e3) / 1e6, 1),
                "ms_per_step": round(total_ms / args.steps, 3),
                "fps": round(len(reqs) * args.steps * world / (total_ms / 1e3), 1),
                "stage_ms_per_render": {k: round(v / max(1, st_calls[k]), 4) for k, v in st_ms.items() if v > 0},
                "stage_share": {k: round(v / tot, 4) for k, v in st_ms.items() if v > 0},
                "gpu_launches": prof["kernel_launches"],
                "roofline": roofline_for(dom, per_launch, work, peaks, peak_kind)}

    fwd_ms, fwd_prof, clk = timed(step_fwd)
    fwd = summary(fwd_ms, fwd_prof)
    fb_ms, fb_prof, clk_fb = timed(step_fwd_bwd)
    fb = summary(fb_ms, fb_prof)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, r, w, reqs, W, H, dev, stream)

    line = {"metric": METRIC, "value": fwd["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": fwd["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scene shaped like the paper's workload; no dataset)",
            "config": {"workload": WORKLOAD, "n_gaussians": w.scene.n, "width": W, "height": H,
                       "renders_per_step": len(reqs), "tile": "16x16", "key_capacity": cap,
                       "l2": "flushed (256 MB write) between steps, outside the timed events",
                       "parallelism": f"replicas x{world}"},
            "fps": fwd["fps"],
            "stage_ms_per_render": fwd["stage_ms_per_render"], "stage_share": fwd["stage_share"],
            "gpu_launches": fwd["gpu_launches"],
            "roofline": fwd["roofline"], "clocks": clk, "e2e": e2e,
            "fwd_bwd": {"metric": "Mpixel/s at 1920x1080, forward + backward (upstream dL/dimage given)",
                        "value": fb["value"], "unit": UNIT, "ms_per_step": fb["ms_per_step"],
                        "fps": fb["fps"], "stage_ms_per_render": fb["stage_ms_per_render"],
                        "stage_share": fb["stage_share"], "gpu_launches": fb["gpu_launches"],
                        "roofline": fb["roofline"], "clocks": clk_fb},
            "work_per_step": {"blend_walked_pairs": walked_pairs, "blend_bwd_pairs": bwd_pairs,
                              "keys_per_render": round(keys_mean)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(args, r, w, reqs, W, H, dev, stream):
    """Same metric through the public API with host buffers: every step copies the
    scene and motion tables from pinned host memory and reads every image back."""
    import numpy as np
    import torch

    import paper_2509_17513_b300 as gc
    from synth import scenes

    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k), np.float32)).pin_memory()
            for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    host["group_id"] = torch.from_numpy(np.ascontiguousarray(w.scene.group_id, np.int32)).pin_memory()
    hq = torch.from_numpy(np.ascontiguousarray(w.motion.q[: args.frames])).pin_memory()
    ht = torch.from_numpy(np.ascontiguousarray(w.motion.t[: args.frames])).pin_memory()
    dev_t = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    dq = torch.empty_like(hq, device=dev)
    dt = torch.empty_like(ht, device=dev)
    gs = gc.GaussianSet(w.scene.layer_offsets, w.scene.sh_degree, 0, **dev_t)
    motions = [gc.MotionFrame(dq[f], dt[f]) for f in range(args.frames)]
    nring = 4
    ring = [torch.empty((3, H, W), device=dev) for _ in range(nring)]
    out_host = [torch.empty((3, H, W)).pin_memory() for _ in range(nring)]
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
        for i, (f, lv) in enumerate(reqs):
            slot = i % nring
            if i >= nring:
                stream.wait_event(copied[slot])
            r.forward(gs, motions[f], scenes.level_mask(lv), w.cameras[f], out=ring[slot])
            rendered[slot].record(stream)
            copy_stream.wait_event(rendered[slot])
            with torch.cuda.stream(copy_stream):
                out_host[slot].copy_(ring[slot], non_blocking=True)
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
    ms = e0.elapsed_time(e1)
    wall = (time.perf_counter() - t0) * 1e3
    r.check()
    ms = max(ms, 1e-6)
    return {"value": round(len(reqs) * W * H * steps / (ms / 1e3) / 1e6, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(ms / steps, 3), "wall_ms_per_step": round(wall / steps, 3),
            "note": "pinned host scene + motion in, every image back to pinned host; "
                    "copies on a second stream overlap rendering"}


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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
