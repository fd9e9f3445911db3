#!/usr/bin/env python
"""Benchmark of the instant-colorization hot path (Alg. 1 lines 1-6) on one GB300.

Headline workload ("segmentation", the large segmentation scene): 3,000,000 Gaussians from 40
anisotropic clusters in a radius-10 ball, 200 cameras on a radius-15 hemisphere at 1600x1060,
fov 55 deg; 16-class one-hot masks (a Voronoi partition of space with 16 seeds, each view's label
render arg-maxed, FP16), SH degree 0, lambda_0 = 1e-5. A step is one full icgs_colorize call over
the scene: projection, binning, depth sort, the blend-accumulate walk (the 16-channel contraction
on tcgen05 tensor cores in MIXED precision), and the per-Gaussian solve.

The same line carries, as extra keys, the other workloads measured the same way:
  segmentation_rgb  the RGB SH-degree-3 pass on the same scene and rig (FP32 targets rendered from
                    random degree-3 coefficients);
  relight           200,000 Gaussians, 100 cameras 800x800, L = 3 RGB (plus its adjoint and one
                    refinement step);
  features          1,000,000 Gaussians, 150 cameras 1000x750, 64 BF16 channels, L = 0.

Per workload:
  value / ms_per_scene  ms per colorized scene (device-resident targets, CUDA events), whole job
  e2e                   the same through icgs_colorize_host: pinned H2D of the targets and D2H of
                        the coefficients and status inside the timed region
  plain_fp32            the plain FP32 path on the same inputs, and MIXED's speedup over it
  roofline              the dominant (walk) kernel, timed live with CUDA events on its stream
  cpu_baseline          the FP64 oracle on the host cores, on a sample of cameras, scaled to a scene

`--impl reference` times the oracle (CPU) on the headline workload and prints the reference line.
Multi-GPU (torchrun): every rank colorizes its own replica of the scene (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_17155_gb300 import workloads as W  # noqa: E402

HEADLINE = "segmentation"
EXTRAS = ("segmentation_rgb", "relight", "features")
METRIC = "colorize ms/scene"
UNIT = "ms/scene"
FP32_LANES_PER_SM = 128

# scene (workload name in workloads.py), seed, SH degree, target kind of each benchmark workload
SPECS = {
    "segmentation": dict(scene="segmentation", seed=4000, L=0, target="masks"),
    "segmentation_rgb": dict(scene="segmentation", seed=4000, L=3, target="rgb"),
    "relight": dict(scene="relight", seed=2000, L=3, target="rgb"),
    "features": dict(scene="features", seed=3000, L=0, target="features"),
}

# DRAM bytes (read + write) of the walk kernel per scene, from one ncu capture each (the profiles
# directory holds the summaries and the commands). A figure is reported only while the kernel's
# source files hash to the value it was captured with; after any change it is null until
# re-captured.
KERNEL_SOURCES = {
    "cuda-core": ["blend.cu", "walk.cuh", "icgs_device.cuh", "icgs_internal.h"],
    "tensor-core": ["contract_tc.cu", "walk.cuh", "icgs_device.cuh", "icgs_internal.h"],
}
MEASURED_TRAFFIC = {
    # relight, 100 cameras: one full-size launch captured
    ("relight", "cuda-core"): {"bytes_per_scene": 2141550080 + 288479744, "source_sha": "6a638ba3bc449478"},
    # features: a 10-camera launch captured and scaled by 150/10 cameras (the targets, the per-camera
    # tile lists and the per-camera accumulator re-streaming all grow with the camera count)
    ("features", "tensor-core"): {"bytes_per_scene": 15 * (3270310656 + 1473606912), "source_sha": "912af52a3bb4b57b"},
    # segmentation masks: a 4-camera launch captured and scaled by 200/4 cameras (as above)
    ("segmentation", "tensor-core"): {"bytes_per_scene": 50 * (1781086720 + 501826560), "source_sha": "912af52a3bb4b57b"},
}


def kernel_source_sha(kind):
    """Hash of the kernel's source files with comments and blank space removed: a figure measured on
    one version stays valid across edits of comments only, and is dropped after any code change."""
    import hashlib
    import re
    m = hashlib.sha256()
    base = os.path.join(ROOT, "paper_2604_17155_gb300", "csrc")
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(base, f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        m.update("\n".join(line.strip() for line in src.splitlines() if line.strip()).encode())
    return m.hexdigest()[:16]


def measured_traffic(workload, kind, full_rig):
    t = MEASURED_TRAFFIC.get((workload, kind))
    if t is None or not full_rig or kernel_source_sha(kind) != t["source_sha"]:
        return None
    return t["bytes_per_scene"]


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="icgs", choices=["icgs", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "plain"])
    ap.add_argument("--workload", default=HEADLINE, choices=list(SPECS),
                    help="the workload of the headline value (default: the large segmentation masks)")
    ap.add_argument("--extras", default=",".join(EXTRAS),
                    help="comma-separated workloads measured as extra keys ('' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-cams", type=int, default=0,
                    help="cameras in each step's oracle sample of the reference arm (0: one per core, up to 16)")
    ap.add_argument("--cams", type=int, default=0, help="profiling only: use the first N cameras of each rig")
    ap.add_argument("--profile-step", action="store_true",
                    help="profiling only: the targets, W warm-up and K timed colorize calls of --workload, nothing else")
    return ap.parse_args(argv)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return dict(hbm_gbs=float(d["hbm_gbs"]), bf16_tflops=float(d["bf16_tflops"]),
                    bf16_tflops_sustained=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                    sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)), source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0,
                    source="fallback")


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
CLOCK_FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(CLOCK_FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < len(CLOCK_FIELDS):
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------
def make_workload(name, n_cams=0):
    sp = SPECS[name]
    scene = W.make_scene(sp["scene"], sp["seed"])
    cams = W.make_cameras(sp["scene"])
    if n_cams:
        cams = cams.subset(np.arange(min(n_cams, cams.n)))
    return scene, cams


def rgb_coefficients(name, scene):
    return W.sh_coefficients(scene.n, 3, 3, SPECS[name]["seed"] + 1)


def mask_labels(scene):
    return W.voronoi_labels(scene.means, 16, 4002, W.WORKLOADS["segmentation"]["radius"])


def device_fourier_fields(n_views, height, width, channels, seed, dev, n_modes=32, max_freq=4.0):
    """The smooth unit-variance field recipe of workloads.fourier_fields, evaluated on the device
    (the 64-channel feature targets are 14 GB): sqrt(2/n_modes) sum_q cos(2 pi (a x/W + b y/H) + phi)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    out = torch.empty((n_views, height, width, channels), dtype=torch.bfloat16, device=dev)
    xs = (torch.arange(width, device=dev, dtype=torch.float32) + 0.5) / width
    ys = (torch.arange(height, device=dev, dtype=torch.float32) + 0.5) / height
    amp = math.sqrt(2.0 / n_modes)
    for v in range(n_views):
        a = (torch.rand((channels, n_modes), generator=g) * 2 - 1) * max_freq
        b = (torch.rand((channels, n_modes), generator=g) * 2 - 1) * max_freq
        ph = torch.rand((channels, n_modes), generator=g) * 2 * math.pi
        a, b, ph = a.to(dev), b.to(dev), ph.to(dev)
        u = 2 * math.pi * a[:, :, None] * xs[None, None, :] + ph[:, :, None]       # [K,Q,W]
        w = 2 * math.pi * b[:, :, None] * ys[None, None, :]                        # [K,Q,H]
        f = torch.einsum("kqh,kqw->hwk", torch.cos(w), torch.cos(u)) - torch.einsum("kqh,kqw->hwk", torch.sin(w), torch.sin(u))
        out[v] = (amp * f).to(torch.bfloat16)
    return out


def make_targets(name, scene, cams, gs, gc, dev, icgs):
    """Device-resident targets of a workload (generated by the library's render or on the device)."""
    import torch
    kind = SPECS[name]["target"]
    if kind == "rgb":
        return icgs.render(gs, gc, torch.tensor(rgb_coefficients(name, scene), device=dev), 3)
    if kind == "features":
        return device_fourier_fields(cams.n, cams.height, cams.width, 64, 3002, dev)
    # masks: one-hot labels of a 16-cell Voronoi partition, rendered per view, arg-maxed -> FP16
    img = icgs.render(gs, gc, torch.tensor(W.one_hot_dc(mask_labels(scene), 16), device=dev), 0)
    t = torch.empty(img.shape, dtype=torch.float16, device=dev)
    for v in range(img.shape[0]):  # per view, to keep the int64 temporaries small
        t[v] = torch.nn.functional.one_hot(img[v].argmax(-1), 16).to(torch.float16)
    del img
    return t


def workload_config(name, n, n_cams, width, height, L, K, dtype_name, precision, world, target_bytes):
    """The `config` object of the JSON line; both arms describe the same workload with it."""
    return {"workload": f"{name}: {n} Gaussians, {n_cams} cameras {width}x{height}, L={L}, {K} channels {dtype_name}",
            "precision": precision, "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 ({target_bytes / 1e6:.0f} MB of targets per step)"}


# ------------------------------------------------------------------------------------------
# oracle baseline (host cores)
# ------------------------------------------------------------------------------------------
def strip_mask(cams, every):
    """Pixel mask [C,H,W] of every `every`-th strip of 16 image rows (the oracle builds its
    per-pixel lists strip by strip and skips strips without a selected pixel)."""
    m = np.zeros((cams.n, cams.height, cams.width), bool)
    for y0 in range(0, cams.height, 16 * every):
        m[:, y0:y0 + 16] = True
    return m


def oracle_sample(scene, cams, L, K, targets_host_fn, idx, threads, strip_every=1):
    """Times the oracle's colorize on the cameras idx (all Gaussians; all pixels, or every
    strip_every-th 16-row strip): the walk, then the fold and solve of every Gaussian. Returns
    (walk seconds, fold+solve seconds, contributing pairs)."""
    from oracle import oracle as O
    O.build()
    sub = cams.subset(idx)
    t_host = targets_host_fn(idx)
    mask = strip_mask(sub, strip_every) if strip_every > 1 else None
    t0 = time.perf_counter()
    V, S, _, _, pairs = O.accumulate(scene, sub, t_host, mask=mask, threads=threads)
    t1 = time.perf_counter()
    fs = oracle_fold_solve(scene, sub, V, S, L)
    return t1 - t0, fs, int(pairs.sum())


FOLD_SAMPLE = 200_000


def oracle_fold_solve(scene, cams, V, S, L):
    """Seconds the oracle's fold and solve (Eq. 12-14) take for every Gaussian: timed on the first
    FOLD_SAMPLE Gaussians and scaled by n / FOLD_SAMPLE (both are linear in the Gaussian count)."""
    from oracle import oracle as O
    m = min(scene.n, FOLD_SAMPLE)
    t0 = time.perf_counter()
    if L == 0:
        w = V[:, :m].sum(0)
        O.solve((w / (4 * math.pi))[:, None, None], S[:, :m].sum(0)[:, None, :] / math.sqrt(4 * math.pi), w,
                O.paper_lambda(0))
    else:
        G, b, w = O.fold(V[:, :m], S[:, :m], O.view_basis(scene.subset(np.arange(m)), cams, L))
        O.solve(G, b, w, O.paper_lambda(L))
    return (time.perf_counter() - t0) * scene.n / m


def cpu_baseline(name, scene, cams, L, K, targets_host_fn):
    """The oracle on all host cores (one camera per core, all pixels) and on one core (one camera,
    every 4th strip of rows), each extrapolated to the whole rig."""
    cores = os.cpu_count() or 1
    n_all = min(cores, 16, cams.n)
    idx = np.linspace(0, cams.n - 1, n_all).round().astype(int)
    walk, fold, pairs = oracle_sample(scene, cams, L, K, targets_host_fn, idx, cores)
    # cameras run in parallel, one per core: the walk of n_all cameras took `walk` seconds of wall time
    ms_all = 1e3 * (walk * cams.n / n_all + fold * cams.n / n_all)
    every = 4
    walk1, fold1, _ = oracle_sample(scene, cams, L, K, targets_host_fn, idx[:1], 1, strip_every=every)
    ms_one = 1e3 * (walk1 * every * cams.n + fold1 * cams.n)
    return {"value": ms_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_all} of {cams.n} cameras (all Gaussians and pixels), one per core; walk x {cams.n}/{n_all} "
                      f"and fold/solve (of {min(scene.n, FOLD_SAMPLE)} Gaussians x {scene.n}/{min(scene.n, FOLD_SAMPLE)})"
                      f" x {cams.n}/{n_all} (extrapolated)",
            "single_core": {"value": ms_one, "unit": UNIT, "cores": 1,
                            "sample": f"1 camera, every {every}th 16-row strip; walk x {every} x {cams.n} cameras, "
                                      f"fold/solve x {cams.n} (extrapolated)"},
            "pairs_oracle_sample": pairs}


# ------------------------------------------------------------------------------------------
# the reference arm: the oracle on the headline workload
# ------------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The oracle on the host cores, one bounded sample per step: one camera per core, every 8th
    16-row strip of pixels, extrapolated to the rig."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    name = args.workload
    sp = SPECS[name]
    scene, cams = make_workload(name, args.cams)
    cores = os.cpu_count() or 1
    n_sample = min(args.ref_cams or min(cores, 16), cams.n)
    every = 8
    idx = np.linspace(0, cams.n - 1, n_sample).round().astype(int)
    sub = cams.subset(idx)
    mask = strip_mask(sub, every)
    L = sp["L"]
    if sp["target"] == "masks":
        img = O.render(scene, sub, W.one_hot_dc(mask_labels(scene), 16), 0, mask=mask, threads=cores)
        targets = (np.eye(16, dtype=np.float32)[img.argmax(-1)] * mask[..., None]).astype(np.float32)
        del img
        K, dname = 16, "float16"
    elif sp["target"] == "rgb":
        targets = O.render(scene, sub, rgb_coefficients(name, scene), 3, mask=mask, threads=cores)
        K, dname = 3, "float32"
    else:
        targets = W.fourier_fields(sub.n, cams.height, cams.width, 64, 3002)
        K, dname = 64, "bfloat16"
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        V, S, _, _, pairs = O.accumulate(scene, sub, targets, mask=mask, threads=cores)
        t1 = time.perf_counter()
        fs = oracle_fold_solve(scene, sub, V, S, L)
        if step >= args.warmup:
            times.append(1e3 * ((t1 - t0) * every * cams.n / n_sample + fs * cams.n / n_sample))
    ms = float(np.mean(times))
    sample = (f"{n_sample} of {cams.n} cameras, one per core, every {every}th 16-row strip of pixels (all "
              f"{scene.n} Gaussians) per step; walk x {every} x {cams.n}/{n_sample}; fold/solve of "
              f"{min(scene.n, FOLD_SAMPLE)} Gaussians x {scene.n}/{min(scene.n, FOLD_SAMPLE)} x {cams.n}/{n_sample}")
    target_bytes = cams.n * cams.width * cams.height * K * (4 if dname == "float32" else 2)
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(name, scene.n, cams.n, cams.width, cams.height, L, K, dname, args.precision,
                                      world, target_bytes),
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# the library arm
# ------------------------------------------------------------------------------------------
def walk_roofline(name, kind, K, L, blend_ms, stats, target_bytes, n, n_cams, tiles, pk, sm_count, full_rig):
    """Roofline of the walk (blend-accumulate) kernel, from its CUDA-event time per scene.
    Algorithmic work (the method's own, per the survey's accounting):
      flops  contributing pairs x (15 FP32 ops + 1 exp for the weight + 2 (1 + K) for V and S),
      bytes  targets read once + 8 B list entry and 32 B Gaussian record per (Gaussian, tile)
             instance + the accumulator read-modify-write (1 + K floats per row and pass)."""
    pairs = stats["contrib_pairs"]
    inst = stats["instances"]
    sec = blend_ms * 1e-3
    flops = pairs * (15 + 2 * (1 + K))
    fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6
    acc_rows = n * (1 if L == 0 else n_cams)
    bytes_alg = target_bytes + inst * (8 + 32) + acc_rows * (1 + K) * 4 * 2
    hbm = {"algorithmic_bytes": bytes_alg, "achieved_gbs": bytes_alg / sec / 1e9, "peak_gbs": pk["hbm_gbs"],
           "frac": bytes_alg / sec / 1e9 / pk["hbm_gbs"], "peak_source": pk["source"]}
    alu = {"algorithmic_flops": flops, "achieved_tflops": flops / sec / 1e12, "peak_tflops": fp32_peak / 1e12,
           "frac": flops / sec / fp32_peak,
           "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {pk['sm_max_mhz']:.0f} MHz"}
    traffic = measured_traffic(name, kind, full_rig)
    if kind == "tensor-core":
        # a5 with 16-bit targets: bound by the target bytes (HBM) plus the tensor-core contraction
        # (survey 8(d)). The tensor view counts the dense MMA work issued: one
        # [64 x 256] x [256 x (K + 8)] product per batch of 64 Gaussians of a tile list.
        batches = inst / 64.0 + n_cams * tiles
        kpad = 16 if K <= 16 else (32 if K <= 32 else 64)
        mma_flops = batches * 2 * 64 * 256 * (kpad + 8)
        tensor = {"issued_mma_flops": mma_flops, "achieved_tflops": mma_flops / sec / 1e12,
                  "peak_tflops": pk["bf16_tflops"], "frac": mma_flops / sec / 1e12 / pk["bf16_tflops"],
                  "peak_source": f"{pk['source']} dense bf16 (fp16 has the same rate)"}
        kname = f"k_blend_accumulate_tc<{kpad}>"
        roof = {"kernel": kname, "bound": "hbm", "achieved": hbm["achieved_gbs"], "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": hbm["frac"], "traffic": traffic,
                "traffic_unit": "bytes per scene (DRAM read + write, ncu)", "peak_source": pk["source"],
                "tensor_view": tensor, "alu_view": alu}
    else:
        kname = f"k_blend_accumulate2<{K}>" if K <= 3 else f"k_blend_accumulate<{min(K, 16)}>"
        roof = {"kernel": kname, "bound": "alu", "achieved": alu["achieved_tflops"], "peak": alu["peak_tflops"],
                "unit": "TFLOP/s", "frac": alu["frac"], "traffic": traffic,
                "traffic_unit": "bytes per scene (DRAM read + write, ncu)", "peak_source": alu["peak_source"],
                "hbm_view": hbm}
    return roof


def measure(name, args, world, dev, icgs, with_e2e, with_cpu):
    """Times one workload: MIXED (or --precision) colorize on device-resident targets, the plain
    FP32 path, optionally the host-buffer call and the oracle. Returns the per-workload record."""
    import torch
    sp = SPECS[name]
    scene, cams = make_workload(name, args.cams)
    gs = icgs.Scene.from_workload(scene, dev)
    gc = icgs.Cameras.from_workload(cams)
    with torch.no_grad():
        targets = make_targets(name, scene, cams, gs, gc, dev, icgs)
    torch.cuda.synchronize(dev)
    L = sp["L"]
    K = int(targets.shape[-1])
    B = (L + 1) ** 2
    target_bytes = targets.numel() * targets.element_size()
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def timed(fn, n):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        barrier()
        t = torch.tensor([e0.elapsed_time(e1)], device=dev)
        if world > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def step():
        return icgs.colorize(gs, gc, targets, L, precision=args.precision)

    for _ in range(args.warmup):
        step()
    # ---- device-resident timed region (stage events on the same stream) ----
    icgs.set_stage_timing(True)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    stage_sum = {}

    def step_staged():
        step()
        for k, v in icgs.last_stage_ms().items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v

    elapsed = timed(step_staged, args.steps)
    clocks = sampler.stop()
    icgs.set_stage_timing(False)
    stats = icgs.last_stats()
    stage_ms = {k: v / args.steps for k, v in stage_sum.items() if v > 0}
    ms_scene = elapsed / args.steps
    rec = {"ms_per_scene": ms_scene, "stage_ms": stage_ms, "clocks": clocks,
           "gpu_launches": stats["launches"] * args.steps, "instances": stats["instances"],
           "contrib_pairs": stats["contrib_pairs"], "fp64_gaussians": stats["fp64"],
           "refolded_gaussians": stats["refold"],
           "blend_contribs_per_s": stats["contrib_pairs"] / (stage_ms.get("blend", float("nan")) * 1e-3)}
    tc = args.precision == "mixed" and K >= 16 and targets.dtype != torch.float32
    rec["walk"] = "tensor-core" if tc else "cuda-core"
    rec["dtype"] = "f16" if tc else "f32"
    rec["dtype_detail"] = ("weights FP32; the (Gaussian x pixel) x (pixel x channel) contraction on tcgen05 in FP16 "
                           "with FP32 accumulation (BF16 targets rescaled per tile by powers of two, exactly); fold "
                           "and solve FP32 / FP64" if tc else
                           "FP32 walk and fold; MIXED: compensated sums, float-float refinement, FP64 for flagged "
                           "Gaussians")
    rec["config"] = workload_config(name, scene.n, cams.n, cams.width, cams.height, L, K,
                                    str(targets.dtype).replace("torch.", ""), args.precision, world, target_bytes)
    props = torch.cuda.get_device_properties(dev)
    tiles = ((cams.width + 15) // 16) * ((cams.height + 15) // 16)
    full_rig = cams.n == W.make_cameras(sp["scene"]).n
    rec["roofline"] = walk_roofline(name, rec["walk"], K, L, stage_ms.get("blend", float("nan")), stats, target_bytes,
                                    scene.n, cams.n, tiles, peaks(), props.multi_processor_count, full_rig)
    rec["roofline"]["sm_count"] = props.multi_processor_count

    # ---- the plain FP32 path on the same inputs ----
    if args.precision == "mixed":
        n_plain = max(3, min(args.steps, 5))
        icgs.colorize(gs, gc, targets, L, precision="plain")
        plain_ms = timed(lambda: icgs.colorize(gs, gc, targets, L, precision="plain"), n_plain) / n_plain
        rec["plain_fp32"] = {"ms_per_scene": plain_ms, "mixed_speedup": plain_ms / ms_scene}

    # ---- end to end through the C ABI with host buffers (icgs_colorize_host) ----
    if with_e2e:
        old_cpus = bind_gpu_local_cpus(dev)
        local_cpus = host_cpus()
        host_t = torch.empty(targets.shape, dtype=targets.dtype, pin_memory=True)
        host_t.copy_(targets)
        host_c = torch.empty((scene.n, B, K), dtype=torch.float32, pin_memory=True)
        host_s = torch.empty((scene.n,), dtype=torch.uint8, pin_memory=True)

        def e2e_step():
            icgs.colorize_host(gs, gc, host_t, L, precision=args.precision, coeffs_out=host_c, status_out=host_s)

        e2e_step()
        e2e_ms = timed(e2e_step, args.steps) / args.steps
        # the pinned-to-device copy rate the end-to-end figure rests on (one plain copy of the targets)
        scratch = torch.empty_like(targets)
        scratch.copy_(host_t, non_blocking=True)
        copy_ms = timed(lambda: scratch.copy_(host_t, non_blocking=True), 2) / 2
        del scratch
        rec["e2e"] = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": target_bytes,
                      "d2h_bytes_per_step": scene.n * B * K * 4 + scene.n, "call": "icgs_colorize_host",
                      "h2d_copy_gbs": target_bytes / copy_ms / 1e6, "host_cpus": local_cpus}
        if old_cpus is not None:
            os.sched_setaffinity(0, old_cpus)
        del host_t, host_c, host_s

    # ---- relight extras: the adjoint (dL/dt, dL/do for L = sum r c^2) and refinement steps ----
    if name == "relight":
        c, st, chol = icgs.colorize(gs, gc, targets, L, precision=args.precision)
        r = torch.randn(c.shape, generator=torch.Generator(device=dev).manual_seed(5005), device=dev)
        gcoef = 2.0 * r * c
        icgs.colorize_backward(gs, gc, targets, L, c, chol, gcoef, precision=args.precision)
        n_adj = max(3, min(args.steps, 5))
        adj_ms = timed(lambda: icgs.colorize_backward(gs, gc, targets, L, c, chol, gcoef, precision=args.precision),
                       n_adj) / n_adj
        rec["adjoint"] = {"ms_per_scene": adj_ms,
                          "outputs": f"dL/dt [{cams.n},{cams.height},{cams.width},{K}] and dL/do [{scene.n}]",
                          "launches": icgs.last_stats()["launches"]}
        c_ref = c.clone()
        icgs.colorize_refine(gs, gc, targets, L, c_ref, chol, 1, precision=args.precision)  # warm-up
        n_ref, per_call = 3, 2

        def refine_call():
            c_ref.copy_(c)
            icgs.colorize_refine(gs, gc, targets, L, c_ref, chol, per_call, precision=args.precision)

        rec["refine"] = {"ms_per_step": timed(refine_call, n_ref) / (n_ref * per_call),
                         "step": "render + residual accumulate + fold of b + update, all cameras",
                         "launches_per_call": icgs.last_stats()["launches"]}

    # ---- the oracle on the host cores ----
    if with_cpu:
        def targets_host(idx):
            return targets[torch.as_tensor(idx, device=dev)].double().cpu().numpy()
        rec["cpu_baseline"] = cpu_baseline(name, scene, cams, L, K, targets_host)
    del targets
    torch.cuda.empty_cache()
    return rec


def bind_gpu_local_cpus(dev):
    """Runs this process on the host CPUs attached to the GPU (the PCI device's local_cpulist), so
    that pinned host memory allocated now lies next to it and host-to-device copies do not cross
    sockets. Returns the previous CPU set (to restore), or None where the system does not expose
    the list."""
    import torch
    try:
        old = os.sched_getaffinity(0)
        pr = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as fh:
            spec = fh.read().strip()
        cpus = set()
        for part in spec.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= old
        if cpus:
            os.sched_setaffinity(0, cpus)
            return old
    except (OSError, ValueError, AttributeError):
        pass
    return None


def host_cpus():
    try:
        return len(os.sched_getaffinity(0))
    except OSError:
        return None


def run_profile_step(args, dev, icgs):
    """Only the colorize calls of one workload (for launch lists and kernel captures)."""
    import torch
    sp = SPECS[args.workload]
    scene, cams = make_workload(args.workload, args.cams)
    gs = icgs.Scene.from_workload(scene, dev)
    gc = icgs.Cameras.from_workload(cams)
    with torch.no_grad():
        targets = make_targets(args.workload, scene, cams, gs, gc, dev, icgs)
    for _ in range(args.warmup + args.steps):
        icgs.colorize(gs, gc, targets, sp["L"], precision=args.precision)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_step": args.workload, "cams": cams.n, "calls": args.warmup + args.steps,
                      "stats": icgs.last_stats()}), flush=True)


def run_icgs(args, rank, world, local_rank):
    import torch

    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if args.profile_step:
        run_profile_step(args, dev, icgs)
        return
    with_cpu = world == 1 and not args.no_cpu_baseline
    head = measure(args.workload, args, world, dev, icgs, True, with_cpu)
    extras = {}
    for name in [x for x in args.extras.split(",") if x and x != args.workload]:
        extras[name] = measure(name, args, world, dev, icgs, name == "relight", with_cpu)
    if rank != 0:
        return
    launches = head["gpu_launches"]
    line = {
        "metric": METRIC, "value": head["ms_per_scene"] / world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_scene"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": head["dtype"], "dtype_detail": head["dtype_detail"], "data": "synthetic",
        "config": head["config"], "roofline": head["roofline"], "e2e": head["e2e"],
        "cpu_baseline": head.get("cpu_baseline"), "clocks": head["clocks"], "gpu_launches": launches,
        "walk": head["walk"], "blend_contribs_per_s": head["blend_contribs_per_s"], "stage_ms": head["stage_ms"],
        "instances": head["instances"], "contrib_pairs": head["contrib_pairs"],
        "fp64_gaussians": head["fp64_gaussians"], "refolded_gaussians": head["refolded_gaussians"],
        "plain_fp32": head.get("plain_fp32"),
        "extra_workloads": extras,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl != "reference":
        import torch
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_icgs(args, rank, world, local_rank)
    finally:
        if world > 1 and args.impl != "reference":
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
