#!/usr/bin/env python
"""Benchmark of the instant-colorization hot path (Alg. 1 lines 1-6) on one GB300.

Workload ("relight", the relighting-shaped scene): 200,000 Gaussians from 40 anisotropic clusters in
a radius-4 ball, 100 cameras on a radius-6 hemisphere at 800x800, fov 45 deg; RGB float32 targets
rendered from random degree-3 SH coefficients (DC ~ U(0,1), higher ~ N(0,0.1)); L = 3 with the
paper's per-band lambda. A step is one full icgs_colorize call: projection, binning, depth sort,
blend-accumulate, fold and the regularised solve for every Gaussian.

  value        ms per colorized scene (device-resident targets, CUDA events), whole job
  e2e          the same through icgs_colorize_host: pinned H2D of the targets and D2H of the
               coefficients inside the timed region
  roofline     the blend-accumulate kernel (dominant), timed live with CUDA events on its stream
  cpu_baseline the FP64 oracle on the host cores, on a sample of cameras, scaled to a scene

`--impl reference` times the oracle (CPU) on the same workload and prints the reference line.
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

WORKLOAD = "relight"
SEED = 2000
METRIC = "colorize ms/scene"
UNIT = "ms/scene"
SM_COUNT = 152
FP32_LANES_PER_SM = 128

# DRAM bytes (read + write) of the dominant kernel per scene, from one ncu capture each
# (profiles/ holds the summaries and the commands). A figure is reported only while the kernel's
# source files hash to the value it was captured with; after any change it is null until re-captured.
KERNEL_SOURCES = {
    "cuda-core": ["blend.cu", "walk.cuh", "icgs_device.cuh", "icgs_internal.h"],
    "tensor-core": ["contract_tc.cu", "walk.cuh", "icgs_device.cuh", "icgs_internal.h"],
}
MEASURED_TRAFFIC = {
    # relight, 100 cameras: one full-size launch captured (profiles/blend_accumulate_relight.md)
    ("relight", "cuda-core"): {"bytes_per_scene": 2148486912 + 288519424, "source_sha": "be1ccf7fce8493cc"},
    # features: a 10-camera launch captured and scaled by 150/10 cameras (the targets, the per-camera
    # tile lists and the per-camera accumulator re-streaming all grow with the camera count)
    ("features", "tensor-core"): {"bytes_per_scene": 15 * (3255527424 + 1463374848), "source_sha": "5d656c19d409fe9f"},
}


def kernel_source_sha(kind):
    """Hash of the kernel's source files with comments and blank space removed: a figure measured on
    one version stays valid across edits of comments only, and is dropped after any code change."""
    import hashlib
    import re
    m = hashlib.sha256()
    base = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2604_17155_gb300", "csrc")
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(base, f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        m.update("\n".join(line.strip() for line in src.splitlines() if line.strip()).encode())
    return m.hexdigest()[:16]


def measured_traffic(workload, kind, n_cams_full, n_cams):
    t = MEASURED_TRAFFIC.get((workload, kind))
    if t is None or n_cams != n_cams_full or kernel_source_sha(kind) != t["source_sha"]:
        return None
    return t["bytes_per_scene"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="icgs", choices=["icgs", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "plain"])
    ap.add_argument("--cpu-sample-cams", type=int, default=0, help="cameras in the oracle sample (0: host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cams", type=int, default=0, help="profiling only: use the first N cameras of the rig")
    ap.add_argument("--workload", default="relight", choices=["relight", "features", "segmentation", "segmentation_rgb"],
                    help="relight (the headline); the others document the feature / mask / large-RGB workloads")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)), source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


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
# oracle baseline (host cores)
# ------------------------------------------------------------------------------------------
def oracle_sample_ms_per_scene(scene, cams, targets_host_fn, n_sample, threads):
    """Times the oracle's colorize on n_sample cameras (all Gaussians, all pixels), scaled to the
    full rig: per-camera walk time x cameras + the fold and solve of every Gaussian."""
    from oracle import oracle as O
    O.build()
    idx = np.linspace(0, cams.n - 1, n_sample).round().astype(int)
    sub = cams.subset(idx)
    t_host = targets_host_fn(idx)
    t0 = time.perf_counter()
    V, S, _, _, pairs = O.accumulate(scene, sub, t_host, threads=threads)
    t1 = time.perf_counter()
    Y = O.view_basis(scene, sub, 3)
    G, b, w = O.fold(V, S, Y)
    O.solve(G, b, w, O.paper_lambda(3))
    t2 = time.perf_counter()
    walk_per_cam = (t1 - t0) / n_sample * min(threads, n_sample)  # wall time of one camera on one core
    fold_per_cam = (t2 - t1) / n_sample
    ms = 1e3 * (walk_per_cam * cams.n / threads + fold_per_cam * cams.n)
    return ms, int(pairs.sum()), idx, (t2 - t0)


# ------------------------------------------------------------------------------------------
def make_workload(n_cams=0, workload=WORKLOAD):
    name = {"relight": "relight", "features": "features", "segmentation": "segmentation",
            "segmentation_rgb": "segmentation"}[workload]
    seed = {"relight": SEED, "features": 3000, "segmentation": 4000, "segmentation_rgb": 4000}[workload]
    scene = W.make_scene(name, seed)
    cams = W.make_cameras(name)
    if n_cams:
        cams = cams.subset(np.arange(min(n_cams, cams.n)))
    coeffs = W.sh_coefficients(scene.n, 3, 3, seed + 1)
    return scene, cams, coeffs


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


def make_targets(workload, scene, cams, coeffs, gs, gc, dev, icgs):
    """Device-resident targets of each workload and its (L, lambda)."""
    import torch
    if workload in ("relight", "segmentation_rgb"):
        return icgs.render(gs, gc, torch.tensor(coeffs, device=dev), 3), 3
    if workload == "features":
        return device_fourier_fields(cams.n, cams.height, cams.width, 64, 3002, dev), 0
    # segmentation: one-hot labels of a 16-cell Voronoi partition, rendered per view, argmax -> FP16
    labels = W.voronoi_labels(scene.means, 16, 4002, W.WORKLOADS["segmentation"]["radius"])
    img = icgs.render(gs, gc, torch.tensor(W.one_hot_dc(labels, 16), device=dev), 0)
    t = torch.empty(img.shape, dtype=torch.float16, device=dev)
    for v in range(img.shape[0]):  # per view, to keep the int64 temporaries small
        t[v] = torch.nn.functional.one_hot(img[v].argmax(-1), 16).to(torch.float16)
    del img
    return t, 0


def workload_config(workload, n, n_cams, width, height, L, K, dtype_name, precision, world, target_bytes):
    """The `config` object of the JSON line; both arms describe the same workload with it."""
    return {"workload": f"{workload}: {n} Gaussians, {n_cams} cameras {width}x{height}, L={L}, {K} channels {dtype_name}",
            "precision": precision, "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 ({target_bytes / 1e6:.0f} MB of targets per step)"}


def run_reference(args, rank, world):
    """The oracle on the host cores, one bounded camera sample per step."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    scene, cams, coeffs = make_workload()
    cores = os.cpu_count() or 1
    n_sample = args.cpu_sample_cams or min(cores, 8)
    idx = np.linspace(0, cams.n - 1, n_sample).round().astype(int)
    sub = cams.subset(idx)
    targets = O.render(scene, sub, coeffs, 3, threads=cores)  # oracle-rendered targets of the sample
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        V, S, _, _, pairs = O.accumulate(scene, sub, targets, threads=cores)
        t1 = time.perf_counter()
        G, b, w = O.fold(V, S, O.view_basis(scene, sub, 3))
        O.solve(G, b, w, O.paper_lambda(3))
        t2 = time.perf_counter()
        if step >= args.warmup:
            walk = (t1 - t0) * min(cores, n_sample) / n_sample
            times.append(1e3 * (walk * cams.n / cores + (t2 - t1) / n_sample * cams.n))
    ms = float(np.mean(times))
    sample = f"{n_sample} of {cams.n} cameras (all 200,000 Gaussians, all 800x800 pixels) per step, scaled to {cams.n}"
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config("relight", scene.n, cams.n, cams.width, cams.height, 3, 3, "float32", args.precision,
                                      world, cams.n * cams.width * cams.height * 3 * 4),
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_icgs(args, rank, world, local_rank):
    import torch

    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    scene, cams, coeffs = make_workload(args.cams, args.workload)
    gs = icgs.Scene.from_workload(scene, dev)
    gc = icgs.Cameras.from_workload(cams)
    with torch.no_grad():
        targets, L = make_targets(args.workload, scene, cams, coeffs, gs, gc, dev, icgs)
    torch.cuda.synchronize(dev)
    K = int(targets.shape[-1])
    B = (L + 1) ** 2
    target_bytes = targets.numel() * targets.element_size()

    def step():
        return icgs.colorize(gs, gc, targets, L, precision=args.precision)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    stats_warm = icgs.last_stats()
    stream = torch.cuda.current_stream(dev)

    # ---- device-resident timed region (stage events on the same stream) ----
    icgs.set_stage_timing(True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    stage_sum = {}
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        for k, v in icgs.last_stage_ms().items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    icgs.set_stage_timing(False)
    elapsed = ev0.elapsed_time(ev1)
    stats = icgs.last_stats()
    t = torch.tensor([elapsed], device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    elapsed_max = float(t.item())
    stage_ms = {k: v / args.steps for k, v in stage_sum.items() if v > 0}

    # ---- end to end through the C ABI with host buffers (icgs_colorize_host): every step copies
    # the targets from pinned host memory (staged per camera chunk, overlapped with the walk) and
    # returns the coefficients and status to pinned host memory ----
    host_t = torch.empty(targets.shape, dtype=targets.dtype, pin_memory=True)
    host_t.copy_(targets)
    host_c = torch.empty((scene.n, B, K), dtype=torch.float32, pin_memory=True)
    host_s = torch.empty((scene.n,), dtype=torch.uint8, pin_memory=True)
    icgs.colorize_host(gs, gc, host_t, L, precision=args.precision, coeffs_out=host_c, status_out=host_s)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        icgs.colorize_host(gs, gc, host_t, L, precision=args.precision, coeffs_out=host_c, status_out=host_s)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    t = torch.tensor([e2e_ms], device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    e2e_max = float(t.item())

    # ---- the plain FP32 path on the same inputs ----
    plain = None
    if args.precision == "mixed":
        n_plain = max(3, min(args.steps, 5))
        icgs.colorize(gs, gc, targets, L, precision="plain")
        barrier()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(n_plain):
            icgs.colorize(gs, gc, targets, L, precision="plain")
        p1.record(stream)
        barrier()
        plain_ms = p0.elapsed_time(p1) / n_plain
        plain = {"ms_per_scene": plain_ms, "mixed_speedup": plain_ms / (elapsed_max / args.steps)}

    # ---- the adjoint (the differentiation workload: dL/dt and dL/d(opacity) for L = sum r c^2) ----
    adjoint = None
    if args.workload == "relight":
        c, st, chol = icgs.colorize(gs, gc, targets, L, precision=args.precision)
        r = torch.randn(c.shape, generator=torch.Generator(device=dev).manual_seed(5005), device=dev)
        gcoef = 2.0 * r * c
        icgs.colorize_backward(gs, gc, targets, L, c, chol, gcoef, precision=args.precision)
        n_adj = max(3, min(args.steps, 5))
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n_adj):
            icgs.colorize_backward(gs, gc, targets, L, c, chol, gcoef, precision=args.precision)
        a1.record(stream)
        barrier()
        adjoint = {"ms_per_scene": a0.elapsed_time(a1) / n_adj, "outputs": f"dL/dt [{cams.n},{cams.height},{cams.width},{K}] and dL/do [{scene.n}]",
                   "launches": icgs.last_stats()["launches"]}

    # ---- iterative refinement (Alg. 1 lines 7-10): render, accumulate the residual, update ----
    refine = None
    if args.workload == "relight":
        c, st, chol = icgs.colorize(gs, gc, targets, L, precision=args.precision)
        c_ref = c.clone()
        icgs.colorize_refine(gs, gc, targets, L, c_ref, chol, 1, precision=args.precision)  # warm-up
        n_ref, steps_per_call = 3, 2
        barrier()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for _ in range(n_ref):
            c_ref.copy_(c)
            icgs.colorize_refine(gs, gc, targets, L, c_ref, chol, steps_per_call, precision=args.precision)
        r1.record(stream)
        barrier()
        refine = {"ms_per_step": r0.elapsed_time(r1) / (n_ref * steps_per_call),
                  "step": "render + residual accumulate + fold of b + update, all cameras",
                  "launches_per_call": icgs.last_stats()["launches"]}

    if rank != 0:
        return
    pk = peaks()
    ms_scene = elapsed_max / (args.steps * world)
    blend_ms = stage_ms.get("blend", float("nan"))
    pairs = stats["contrib_pairs"]
    inst = stats["instances"]
    # algorithmic work of the blend-accumulate kernel per launch (one launch per scene here):
    # per contributing pair: weight (~15 FP32 ops + 1 exp) and accumulation 2(1+K)
    flops = pairs * (15 + 2 * (1 + K))
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6
    achieved_tflops = flops / (blend_ms * 1e-3) / 1e12
    acc_rows = scene.n * (1 if L == 0 else cams.n)
    bytes_alg = target_bytes + inst * (8 + 32) + acc_rows * (1 + K) * 4 * 2
    tc = args.precision == "mixed" and K >= 16 and targets.dtype != torch.float32
    if tc:
        kname = f"k_blend_accumulate_tc<{16 if K <= 16 else 32 if K <= 32 else 64}>"
    elif K <= 3:
        kname = f"k_blend_accumulate2<{K}>"  # two pixels per thread
    else:
        kname = f"k_blend_accumulate<{min(K, 16)}>"
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved_tflops,
            "peak": fp32_peak / 1e12, "unit": "TFLOP/s", "frac": achieved_tflops / (fp32_peak / 1e12),
            "traffic": measured_traffic(args.workload, "tensor-core" if tc else "cuda-core",
                                        W.make_cameras({"relight": "relight", "features": "features"}.get(
                                            args.workload, "segmentation")).n, cams.n),
            "traffic_unit": "bytes per scene (DRAM read + write, ncu)",
            "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {pk['sm_max_mhz']:.0f} MHz",
            "hbm_view": {"algorithmic_bytes": bytes_alg, "achieved_gbs": bytes_alg / (blend_ms * 1e-3) / 1e9,
                         "peak_gbs": pk["hbm_gbs"], "frac": bytes_alg / (blend_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                         "peak_source": pk["source"]}}
    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload == "relight":
        cores = os.cpu_count() or 1
        n_sample = args.cpu_sample_cams or min(cores, 16)

        def targets_host(idx):
            return targets[torch.as_tensor(idx, device=dev)].double().cpu().numpy()

        ms_cpu, opairs, idx, wall = oracle_sample_ms_per_scene(scene, cams, targets_host, n_sample, cores)
        # the GPU's contributing-pair count on the same camera sample, for the pair-count cross-check
        sub = icgs.Cameras.from_workload(cams.subset(idx))
        icgs.colorize(gs, sub, targets[torch.as_tensor(idx, device=dev)].contiguous(), L, precision=args.precision)
        gpairs = icgs.last_stats()["contrib_pairs"]
        cpu = {"value": ms_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_sample} of {cams.n} cameras, all Gaussians and pixels, walk x {cams.n}/{cores} cores "
                         f"+ fold/solve x {cams.n}/{n_sample}; {wall:.1f} s of CPU wall time",
               "pairs_oracle_sample": opairs, "pairs_gpu_sample": gpairs}
    line = {
        "metric": METRIC, "value": ms_scene, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_max / args.steps, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if targets.dtype == torch.float32 else ("f16" if tc else "f32"), "data": "synthetic",
        "config": workload_config(args.workload, scene.n, cams.n, cams.width, cams.height, L, K,
                                  str(targets.dtype).replace("torch.", ""), args.precision, world, target_bytes),
        "roofline": roof,
        "e2e": {"value": e2e_max / (args.steps * world), "unit": UNIT, "h2d_bytes_per_step": target_bytes,
                "d2h_bytes_per_step": scene.n * B * K * 4 + scene.n, "call": "icgs_colorize_host"},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": stats["launches"] * args.steps,
        "blend_contribs_per_s": pairs / (blend_ms * 1e-3),
        "stage_ms": stage_ms,
        "instances": inst, "contrib_pairs": pairs, "fp64_gaussians": stats["fp64"], "refolded_gaussians": stats["refold"],
        "plain_fp32": plain,
        "adjoint": adjoint,
        "refine": refine,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
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
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
