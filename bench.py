"""Benchmark of the column-density projection on the headline workload.

Workload (zel256_persp2048x128): a 256^3 particle lattice (100.7M
tetrahedra per snapshot), 8 Zel'dovich snapshots with maximum deformation
eigenvalue 0.5 .. 6, 16 perspective cameras on a sphere of radius 2 around
the box (60 degree field of view), 2048 x 2048 pixels: 128 frames per step,
rendered by one replay of a CUDA graph holding the project-and-bin pass and
the persistent tile raster. Inputs are synthetic and seeded; the positions
(2.1 GB) are larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0). `value` is fragments/s over the whole job: a
fragment is a (tetrahedron, pixel) pair with a positive chord, counted once
on the GPU for the workload (the counter is checked against the oracle in
the tests). `--impl reference` times the FP64 CPU oracle instead, on bounded
samples of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tet-pixel fragments/s and frames/s at 256^3 particles, 2048^2 px vs plain atomic form"
WORKLOAD = "zel256_persp2048x128"
# FP32 operations per fragment in the raster's inner loop (FFMA counted as 2):
# perspective: 4 edge FFMA + 3 min + 1 clamp + 2 depth-plane FFMA + 1 max +
# 1 FFMA + 1 FMUL + 1 reciprocal-multiply = 22
FLOPS_PER_FRAGMENT_PERSP = 22
FLOPS_PER_FRAGMENT_ORTHO = 12


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lt", choices=["lt", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--frames", type=int, default=0, help="override frame count (debug)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-atomic", action="store_true")
    ap.add_argument("--no-resample", action="store_true")
    ap.add_argument("--no-area", action="store_true")
    ap.add_argument("--one-frame", action="store_true",
                    help="profiling case: bin frame 0 of the workload (snapshot 0, camera 0) and render it three "
                         "times with --tile and --raster-threads; prints a summary instead of the JSON line")
    ap.add_argument("--tile", type=int, default=32)
    ap.add_argument("--raster-threads", type=int, default=256, help="raster CTA size of --one-frame")
    ap.add_argument("--area-only", action="store_true",
                    help="profiling case: the area-averaged pixel leg alone (128^3 lattice, orthographic 1024^2); "
                         "prints its summary instead of the JSON line")
    ap.add_argument("--cpu-sample-crop", type=int, default=384)
    ap.add_argument("--oracle-crop", type=int, default=256, help="crop edge of the atomic form's oracle check")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload


def make_workload(name: str, frames_override: int = 0):
    from lt_inputs import ZeldovichField, config, ortho_z, sphere_cameras

    c = config(name)
    N = c["N"]
    f = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"])
    lams = c["lams"]
    import numpy as np

    pos = np.empty((len(lams), N ** 3, 4), dtype=np.float32)
    for s, lam in enumerate(lams):
        pos[s] = f.positions(lam)
    if c["view"] == "sphere16":
        cams0 = sphere_cameras(16, c["W"], c["H"], radius=c["radius"], fov_y_deg=c["fov_y_deg"])
        cams, snaps = [], []
        for s in range(len(lams)):
            for cam in cams0:
                cams.append(cam)
                snaps.append(s)
    else:
        cams, snaps = [ortho_z(c["W"], c["H"])], [0]
    if frames_override:
        cams, snaps = cams[:frames_override], snaps[:frames_override]
    return c, pos, cams, snaps


# ---------------------------------------------------------------------------
# clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = os.path.join(tempfile.gettempdir(), f"lt_clocks_{os.getpid()}.csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm


def run_lt(args, rank: int, world: int):
    import numpy as np
    import torch

    from paper_1208_3206_gb300.render import Renderer

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    log("generating workload")
    c, pos_np, cams, snaps = make_workload(args.workload, args.frames)
    N = c["N"]
    F = len(cams)
    log(f"workload ready: N={N} frames={F}")
    W, H = cams[0]["W"], cams[0]["H"]
    persp = cams[0]["type"] == "persp"

    R = Renderer()
    pos = torch.from_numpy(pos_np).to(dev)
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record()
    R.build_tets(pos, N)  # volumes, densities and zero-volume masks of every snapshot
    q1.record()
    R.sync()
    build_ms = q0.elapsed_time(q1)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        # autotune the tile size and CTA shape on a subset of the frames
        tune_frames = list(range(0, F, max(1, F // 8)))
        best = R.autotune([cams[q] for q in tune_frames], [snaps[q] for q in tune_frames], reps=1)
        log(f"autotuned: {best}")
        R.project_bin(cams, snaps)
        frags = R.count_fragments()
        stats_bin = R.get_stats()
        img = torch.empty((F, H, W), dtype=torch.float32, device=dev)
        mass = torch.empty(F, dtype=torch.float64, device=dev)
        R.graph_build(cams, snaps, image=img, mass=mass, stream=stream)
        R.sync()
    total_frags = int(sum(frags))
    gstats = R.get_stats()
    log(f"graph built: {total_frags} fragments per step, {gstats['graph_kernels']} kernels")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            R.graph_launch(stream)
    stream.synchronize()
    exact_before = R.get_stats()["exact_fragments"]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            R.graph_launch(stream)
    e1.record(stream)
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    log(f"timed: {ms:.1f} ms per step")
    R.sync()
    tstats = R.get_stats()
    exact_per_step = (tstats["exact_fragments"] - exact_before) / args.steps

    # raster kernel alone (the dominant kernel), timed with events on its
    # stream; the project-and-bin pass before it is timed too (it includes one
    # host synchronisation, to size the lists)
    with torch.cuda.stream(stream):
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        R.project_bin(cams, snaps)
        p1.record(stream)
        R.render_tiles(image=img)
        stream.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        reps = max(2, min(args.steps, 5))
        r0.record(stream)
        for _ in range(reps):
            R.render_tiles(image=img)
        r1.record(stream)
        stream.synchronize()
    raster_ms = r0.elapsed_time(r1) / reps
    bin_ms = p0.elapsed_time(p1)
    R.sync()

    # end to end through the public API: pinned host positions in, images out,
    # pipelined per snapshot (see e2e_pipelined)
    host_pos = torch.from_numpy(pos_np).pin_memory()
    host_img = torch.empty((F, H, W), dtype=torch.float32).pin_memory()
    e2e_steps = max(2, min(args.steps, 3))
    e2e_ms = e2e_pipelined(pos, host_pos, img, host_img, N, cams, snaps, best, e2e_steps, barrier)
    log(f"end to end: {e2e_ms:.1f} ms per step")

    # plain one-cube-per-thread atomic form (same per-tetrahedron arithmetic and
    # the same exact path) on every 8th frame, against the tiled form on the
    # same frames
    atomic = None
    atomic_crops = []
    if not args.no_atomic:
        sub = list(range(0, F, 8))
        sub_cams, sub_snaps = [cams[q] for q in sub], [snaps[q] for q in sub]
        sub_frags = int(sum(frags[q] for q in sub))
        log(f"atomic form on {len(sub)} frames")
        with torch.cuda.stream(stream):
            a_img = torch.empty((len(sub), H, W), dtype=torch.float32, device=dev)
            t_img = torch.empty((len(sub), H, W), dtype=torch.float32, device=dev)
            R.render_atomic(sub_cams, sub_snaps, image=a_img)
            R.project_bin(sub_cams, sub_snaps)
            R.render_tiles(image=t_img)
            stream.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            R.render_atomic(sub_cams, sub_snaps, image=a_img)
            a1.record(stream)
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            R.project_bin(sub_cams, sub_snaps)
            R.render_tiles(image=t_img)
            b1.record(stream)
            stream.synchronize()
        a_ms, b_ms = a0.elapsed_time(a1), b0.elapsed_time(b1)
        nzmean = t_img[t_img > 0].mean().item()
        rel = ((a_img - t_img).abs() / torch.clamp(t_img, min=nzmean)).max().item()
        atomic = {"value": sub_frags / (a_ms * 1e-3), "unit": "fragments/s", "frames": len(sub),
                  "ms": a_ms, "tiled_ms_same_frames": b_ms, "speedup_tiled_over_atomic": a_ms / b_ms,
                  "max_rel_diff_vs_tiled": rel}
        # central crops of four of these frames from both forms, for the CPU
        # leg's comparison with the oracle
        for q in (0, 5, 10, 14):
            if q < len(sub):
                x0c, y0c, wc, hc = central_crop(cams[sub[q]], args.oracle_crop)
                atomic_crops.append((sub[q], a_img[q, y0c:y0c + hc, x0c:x0c + wc].cpu().numpy(),
                                     t_img[q, y0c:y0c + hc, x0c:x0c + wc].cpu().numpy()))
        del a_img, t_img
        R.sync()

    # resampling onto a periodic grid (the next row of the path): the 128^3
    # lattice onto 512^3 cells, density weighting
    resample = None if args.no_resample else bench_resample(dev)
    if resample is not None:
        log(f"resample: {resample['ms']:.1f} ms")
    # area-averaged pixels of the 128^3 lattice, orthographic 1024^2
    area = None if args.no_area else bench_area(dev)
    if area is not None:
        log(f"area-averaged pixels: {area['ms']:.2f} ms")

    # max over ranks
    if world > 1:
        ms, e2e_ms = max_over_ranks([ms, e2e_ms], dev)

    import torch.cuda as tc
    props = tc.get_device_properties(dev)
    sms = props.multi_processor_count
    flops_per_frag = FLOPS_PER_FRAGMENT_PERSP if persp else FLOPS_PER_FRAGMENT_ORTHO
    peak, peak_clock_mhz, clock_src = fp32_peak_tflops(sms)
    achieved = total_frags * flops_per_frag / (raster_ms * 1e-3) / 1e12

    value = world * total_frags / (ms * 1e-3)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "fragments/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": args.workload,
            "particles": N ** 3,
            "tets_per_snapshot": 6 * N ** 3,
            "snapshots": len(set(snaps)),
            "frames": F,
            "image": [W, H],
            "fragments_per_step": total_frags,
            "bin_entries": stats_bin["entries"],
            "tile": best.get("tile"),
            "raster_threads": best.get("raster_threads"),
            "l2": "inputs larger than L2 (positions %.2f GB)" % (pos.numel() * 4 / 1e9),
            "graph": "one CUDA graph replay per step (project-and-bin + persistent tile raster)",
        },
        "frames_per_s": world * F / (ms * 1e-3),
        "gpu_launches": int(gstats["graph_kernels"]) * args.steps,
        "clocks": clk,
        "roofline": {
            "bound": "alu",
            "kernel": "k_raster (persistent tile raster)",
            "achieved": achieved,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": raster_traffic(F),
            "traffic_from": RASTER_TRAFFIC["capture"] if raster_traffic(F) is not None else None,
            "counted": f"{flops_per_frag} FP32 flops per fragment",
            "peak_from": f"{sms} SMs x 128 FP32 lanes x 2 x {peak_clock_mhz:.0f} MHz ({clock_src})",
            "raster_ms": raster_ms,
        },
        "passes": {
            "build_ms": build_ms,
            "build": "lt_build_tets of all snapshots, once per set of positions (outside the step)",
            "bin_ms_per_step": bin_ms,
            "exact_fragments_per_step": exact_per_step,
            "exact_fragments": "fragments the per-fragment error test sent to the FP64 path, mean over the "
                               "timed steps",
            "raster_ms_per_step": raster_ms,
            "step_ms": ms,
        },
        "e2e": {
            "value": world * total_frags / (e2e_ms * 1e-3),
            "unit": "fragments/s",
            "ms_per_step": e2e_ms,
            "h2d_bytes_per_step": int(pos.numel() * 4),
            "d2h_bytes_per_step": int(img.numel() * 4),
        },
    }
    if atomic is not None:
        line["atomic"] = atomic
    if resample is not None:
        line["resample"] = resample
    if area is not None:
        line["area"] = area
    # the GPU's pixels of frame 0's central crop (from the last end-to-end
    # step's host copy), for the parity figure next to the CPU baseline
    x0c, y0c, wc, hc = central_crop(cams[0], args.cpu_sample_crop)
    gpu_crop = host_img[0, y0c:y0c + hc, x0c:x0c + wc].numpy().copy()
    return line, (c, pos_np, cams, snaps, gpu_crop, atomic_crops)


# FP64 operations the resampling counts (FMA as 2, division as 1): per
# (tetrahedron, line) interval, four face planes (two FMA and a division
# each) and four min/max; per piece of an interval in one slab, a max, a min,
# a subtraction and two multiplications.
RESAMPLE_FLOPS_PER_INTERVAL = 24
RESAMPLE_FLOPS_PER_PIECE = 5
# GB300 FP64 peak (nominal; there is no measured FP64 figure for this machine)
FP64_PEAK_TFLOPS = 1.25


def bench_resample(dev, n: int = 512, reps: int = 3):
    """Time lt_resample of the 128^3 workload (deformation eigenvalue 3) onto
    a periodic n^3 grid, density weighting, with CUDA events; report the
    (tetrahedron, line) intervals per second and the FP64 roofline."""
    import torch

    from lt_inputs import ZeldovichField, config
    from paper_1208_3206_gb300.render import Renderer

    c = config("zel128_ortho1024")
    N = c["N"]
    pos = torch.from_numpy(ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0]))
    R = Renderer()
    R.build_tets(pos.to(dev), N)
    grid = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    R.resample(n, "density", out=grid)  # warm-up (sizes the bins)
    R.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        R.resample(n, "density", out=grid)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    st = R.get_stats()
    # its bin pass alone (the same orthographic view of the grid's columns),
    # to time the resampling kernels without it
    from lt_inputs import ortho_z
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    for _ in range(reps):
        R.project_bin([ortho_z(n, n)])
    b1.record()
    torch.cuda.synchronize()
    bin_ms = b0.elapsed_time(b1) / reps
    R.close()
    kernel_ms = max(ms - bin_ms, 1e-6)
    iv, pc = st["resample_intervals"], st["resample_pieces"]
    flops = RESAMPLE_FLOPS_PER_INTERVAL * iv + RESAMPLE_FLOPS_PER_PIECE * pc
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    return {"workload": f"zel128 lattice (12.6M tetrahedra) onto {n}^3 cells, density weighting",
            "ms": ms, "value": iv / (ms * 1e-3), "unit": "intervals/s", "intervals": iv, "pieces": pc,
            "cells_per_s": n ** 3 / (ms * 1e-3), "bin_ms": bin_ms, "kernel_ms": kernel_ms,
            "timing": "ms: the whole call, with its bin pass (one host synchronisation); kernel_ms: ms - bin_ms",
            "roofline": {"bound": "alu", "kernel": "k_resample (FP64 clipping)", "achieved": achieved,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s (FP64)", "frac": achieved / FP64_PEAK_TFLOPS,
                         "counted": f"{RESAMPLE_FLOPS_PER_INTERVAL} FP64 flops per interval + "
                                    f"{RESAMPLE_FLOPS_PER_PIECE} per slab piece",
                         "peak_from": "GB300 nominal FP64 rate"}}


# FP32 operations lt_render_area counts per (tetrahedron, pixel) pair: the
# eight lines (four hull edges, four rays) evaluated at the pixel's corner in
# float-float (two error-free products, two two-sums and the small terms:
# 20 operations, FMA as 2), and per pyramid face the corner tests (8); the
# clip of partly covered squares is not counted.
AREA_FLOPS_PER_PAIR = 8 * 20 + 4 * 8


def bench_area(dev, reps: int = 5):
    """Time lt_render_area (area-averaged pixels) of the 128^3 workload
    (deformation eigenvalue 3) in the periodic orthographic 1024^2 view with
    CUDA events; report frames/s, (tetrahedron, pixel) pairs per second and
    the counted FP32 work against the FP32 peak."""
    import torch

    from lt_inputs import ZeldovichField, config, ortho_z
    from paper_1208_3206_gb300.render import Renderer

    c = config("zel128_ortho1024")
    N, W, H = c["N"], c["W"], c["H"]
    pos = torch.from_numpy(ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0]))
    R = Renderer()
    R.build_tets(pos.to(dev), N)
    cam = ortho_z(W, H)
    img = torch.empty((H, W), dtype=torch.float32, device=dev)
    for _ in range(3):
        R.render_area(cam, image=img)
    R.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        R.render_area(cam, image=img)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    st = R.get_stats()
    mass = img.double().sum().item() / (W * H)
    R.close()
    pairs, p64 = st["area_pairs"], st["area_fp64_pairs"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, mhz, src = fp32_peak_tflops(sms)
    achieved = AREA_FLOPS_PER_PAIR * pairs / (ms * 1e-3) / 1e12
    return {"workload": f"zel128 lattice (12.6M tetrahedra), orthographic {W}x{H} periodic window",
            "ms": ms, "value": 1e3 / ms, "unit": "frames/s", "pairs": pairs, "fp64_clip_pairs": p64,
            "pairs_per_s": pairs / (ms * 1e-3), "frame_mass": mass,
            "timing": "the whole call (frame upload, kernel, finalize, one host synchronisation)",
            "roofline": {"bound": "alu", "kernel": "k_area (float-float lines + FP32 clip)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "counted": f"{AREA_FLOPS_PER_PAIR} FP32 flops per (tetrahedron, pixel) pair",
                         "peak_from": f"{sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz ({src})"}}


def e2e_pipelined(pos, host_pos, img, host_img, N, cams, snaps, cfg, steps, barrier):
    """Milliseconds per step of the whole job through the public API with
    host buffers: every step copies all snapshots' positions in from pinned
    host memory and every frame's image out to it. One Renderer (context)
    and one graph per snapshot, over that snapshot's slice of the device
    positions and its frames' slice of the device images; three streams, so
    that the copy in of snapshot s + 1 and the copy out of snapshot s - 1 run
    under the render of snapshot s. A snapshot's copy in waits for its
    previous render (which reads the positions), and its render waits for
    its previous copy out (which reads the images)."""
    import torch

    from paper_1208_3206_gb300.render import Renderer

    groups = sorted(set(snaps))
    copy_in, compute, copy_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    parts = []
    for g in groups:
        fr = [q for q in range(len(cams)) if snaps[q] == g]
        lo, hi = fr[0], fr[-1] + 1
        assert fr == list(range(lo, hi)), "frames of a snapshot must be contiguous"
        Rg = Renderer(tile=cfg.get("tile", 0), raster_threads=cfg.get("raster_threads", 0))
        Rg.build_tets(pos[g], N)
        with torch.cuda.stream(compute):
            Rg.graph_build(cams[lo:hi], None, image=img[lo:hi], stream=compute)
            Rg.sync()
        ev = {k: torch.cuda.Event() for k in ("in", "done", "out")}
        parts.append((g, lo, hi, Rg, ev))
    torch.cuda.synchronize()

    def one_step():
        for g, lo, hi, Rg, ev in parts:
            copy_in.wait_event(ev["done"])
            with torch.cuda.stream(copy_in):
                pos[g].copy_(host_pos[g], non_blocking=True)
            ev["in"].record(copy_in)
            compute.wait_event(ev["in"])
            compute.wait_event(ev["out"])
            Rg.graph_launch(compute)
            ev["done"].record(compute)
            copy_out.wait_event(ev["done"])
            with torch.cuda.stream(copy_out):
                host_img[lo:hi].copy_(img[lo:hi], non_blocking=True)
            ev["out"].record(copy_out)

    one_step()  # warm-up
    torch.cuda.synchronize()
    barrier()
    x0 = torch.cuda.Event(enable_timing=True)
    x1 = torch.cuda.Event(enable_timing=True)
    x0.record(copy_in)
    for _ in range(steps):
        one_step()
    x1.record(copy_out)
    torch.cuda.synchronize()
    for _, _, _, Rg, _ in parts:
        Rg.sync()
        Rg.close()
    return x0.elapsed_time(x1) / steps


# ---------------------------------------------------------------------------
# CPU oracle


# DRAM bytes (read + write) of one k_tile launch per frame of the headline
# workload, from an ncu capture of the kernel built from the sources whose
# hash is recorded with it; None when the raster has changed since.
RASTER_TRAFFIC = {"bytes_per_frame": 432438784, "sources_sha16": "d73758b9859dd0d8",
                  "capture": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_tile launch, "
                             "python bench.py --one-frame --tile 64 --raster-threads 256 (frame 0), "
                             "scaled by the frames"}


def raster_sources_sha16() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("lt_tile.cu", "lt_common.cuh"):
        with open(os.path.join(ROOT, "paper_1208_3206_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def raster_traffic(frames: int):
    """Measured DRAM bytes of one raster launch over `frames` frames (the
    per-frame capture scaled by the frames), or None when the capture is
    missing or older than the raster's sources."""
    t = RASTER_TRAFFIC
    if not t["bytes_per_frame"] or t["sources_sha16"] != raster_sources_sha16():
        return None
    return t["bytes_per_frame"] * frames


def fp32_peak_tflops(sms: int):
    """FP32 peak for the ALU roofline: SMs x 128 lanes x 2 flops x the
    maximum SM clock, read from MEASURED_PEAKS.json when it is there (else
    GB300's 2070 MHz). Returns (TFLOP/s, MHz, where the clock came from)."""
    mhz, src = 2070.0, "GB300 maximum SM clock"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh).get("sm_max_mhz") or 0.0)
        if v > 0:
            mhz, src = v, "sm_max_mhz of MEASURED_PEAKS.json"
    except (OSError, ValueError):
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12, mhz, src


def central_crop(cam, crop: int):
    """(x0, y0, w, h) of the central crop x crop window of a frame."""
    W, H = cam["W"], cam["H"]
    crop = min(crop, W, H)
    return ((W - crop) // 2, (H - crop) // 2, crop, crop)


def oracle_sample(c, pos_np, cams, snaps, crop: int, frame: int = 0):
    """Time the FP64 oracle on the central crop of one frame; returns
    (fragments, seconds, crop image)."""
    import oracle

    N = c["N"]
    cam = cams[frame]
    s = snaps[frame]
    t = time.perf_counter()
    imgs, nf, _ = oracle.render_crops(pos_np[s], N, cam, [central_crop(cam, crop)])
    return nf, time.perf_counter() - t, imgs[0]


def crop_parity(ref, got, tol: float = 1e-4) -> dict:
    """Largest error of a GPU crop against the oracle's, relative to
    max(pixel, mean column density of the crop's nonzero oracle pixels)."""
    import numpy as np

    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    nz = ref[ref > 0]
    mean_cd = float(nz.mean()) if nz.size else 1.0
    err = float((np.abs(got - ref) / np.maximum(np.abs(ref), mean_cd)).max()) if ref.size else 0.0
    return {"max_rel_err": err, "tol": tol, "pass": err <= tol}


def cpu_baseline(c, pos_np, cams, snaps, crop: int, gpu_crop=None):
    """The oracle timed on the central crop of frame 0 (the CPU baseline);
    with the GPU's pixels of the same crop, also their parity."""
    nf, sec, ref = oracle_sample(c, pos_np, cams, snaps, crop)
    cores = os.cpu_count()
    x0, y0, w, h = central_crop(cams[0], crop)
    base = {"value": nf / sec, "unit": "fragments/s", "cores": cores, "kind": "oracle",
            "sample": f"frame 0, central {w}x{h} crop ({nf} fragments, {sec:.1f} s incl. the scan of all "
                      f"{6 * c['N'] ** 3} tetrahedra)"}
    parity = None
    if gpu_crop is not None:
        parity = dict(crop_parity(ref, gpu_crop), frame=0, crop=[x0, y0, w, h])
    return base, parity


def max_over_ranks(values, device):
    """Element-wise maximum of a list of floats over all ranks of the
    default process group (the slowest rank's times)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return None  # the CPU oracle runs on rank 0 only
    c, pos_np, cams, snaps = make_workload(args.workload, args.frames)
    # each step: one bounded sample of the same workload (a central crop of
    # one frame), rotating through the frames
    for w in range(args.warmup):
        oracle_sample(c, pos_np, cams, snaps, min(64, args.cpu_sample_crop), w % len(cams))
    tot_f, tot_s = 0, 0.0
    for st in range(args.steps):
        nf, sec, _ = oracle_sample(c, pos_np, cams, snaps, args.cpu_sample_crop, st % len(cams))
        tot_f += nf
        tot_s += sec
    value = tot_f / tot_s
    cores = os.cpu_count()
    sample = f"per step one central {args.cpu_sample_crop}^2 crop of one frame ({tot_f // max(1, args.steps)} fragments)"
    return {
        "metric": METRIC, "value": value, "unit": "fragments/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "particles": c["N"] ** 3, "frames": len(cams),
                   "image": [cams[0]["W"], cams[0]["H"]]},
        "cpu_baseline": {"value": value, "unit": "fragments/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "fragments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def one_frame(args):
    """A small case for profiler captures: the first frame of the workload
    (its snapshot alone on the device), binned once and rendered three
    times with a fixed tile and CTA size."""
    import torch

    from lt_inputs import ZeldovichField, config, ortho_z, sphere_cameras
    from paper_1208_3206_gb300.render import Renderer

    c = config(args.workload)
    N = c["N"]
    pos = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0])
    if c["view"] == "sphere16":
        cam = sphere_cameras(16, c["W"], c["H"], radius=c["radius"], fov_y_deg=c["fov_y_deg"])[0]
    else:
        cam = ortho_z(c["W"], c["H"])
    R = Renderer(tile=args.tile, raster_threads=args.raster_threads)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    R.project_bin([cam])
    img = R.render_tiles()
    for _ in range(2):
        R.render_tiles(image=img)
    R.sync()
    st = R.get_stats()
    print(f"one frame of {args.workload}: tile {args.tile}, {args.raster_threads} threads, {st['entries']} bin entries, "
          f"{st['exact_fragments']} exact fragments over 3 renders, image sum {float(img.double().sum()):.6f}")


def main():
    args = parse()
    if args.one_frame:
        one_frame(args)
        return
    if args.area_only:
        import torch
        print(json.dumps(bench_area(torch.device("cuda", 0))), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        # rank 0 alone times the oracle; the other ranks exit without work
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend="nccl")
    line, wl = run_lt(args, rank, world)
    if rank == 0 and not args.no_cpu_baseline:
        log("CPU oracle sample")
        c, pos_np, cams, snaps, gpu_crop, atomic_crops = wl
        line["cpu_baseline"], line["parity"] = cpu_baseline(c, pos_np, cams, snaps, args.cpu_sample_crop, gpu_crop)
        if atomic_crops and "atomic" in line:
            # both forms against the oracle on the same central crops
            a_err, t_err = 0.0, 0.0
            for fr, a_crop, t_crop in atomic_crops:
                _, _, ref = oracle_sample(c, pos_np, cams, snaps, args.oracle_crop, fr)
                a_err = max(a_err, crop_parity(ref, a_crop)["max_rel_err"])
                t_err = max(t_err, crop_parity(ref, t_crop)["max_rel_err"])
            line["atomic"]["err_vs_oracle"] = a_err
            line["atomic"]["tiled_err_vs_oracle"] = t_err
            line["atomic"]["err_sample"] = (f"central {args.oracle_crop}^2 crops of frames "
                                            f"{[fr for fr, _, _ in atomic_crops]}: max |GPU - oracle| / "
                                            f"max(pixel, mean of the crop), tolerance 1e-4")
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
