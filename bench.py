#!/usr/bin/env python3
"""Benchmark: Mpath-segments/s of the spectral DDM path tracer on one GB300.

Workload (one step = one full render, every step of the hot path): the
synthetic hotel room -- 6x4x3 m, ~200.5k triangles (40 boxes, 100 spheres of
2000 triangles, 20 of them metallic), two photochromic panes at s = 0.5 lit by
suns behind them, a ceiling lamp -- at 512x512 px, 16 spp, max depth 5, 41
wavelength bins, traced by domain decomposition over a 4x4x2 grid of
subdomains (or by the plain global-BVH megakernel with --method megakernel).

value   = (extension + shadow segments of all ranks) / (max over ranks of the
          summed device time of the K timed steps), inputs resident in HBM,
          L2 flushed between steps.
e2e     = the same metric through sddm_render_host: result image copied back
          to pinned host memory inside the timed region.
roofline: the trace kernel (k_trace_wave for DDM, k_megakernel for the plain
          path): algorithmic bytes = ray-record reads and writes + BVH node
          (64 B) and triangle (48 B) fetches counted per ray, divided by the
          kernel's own device time (CUDA events around each launch on the
          library's stream), against the measured HBM copy bandwidth.
--impl reference times the FP64 CPU oracle on a bounded pixel sample of the
same workload (there is no reference implementation to install).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpath-segments/s per GB300, DDM+MLP-BSDF vs plain, at image rel-RMSE<=1e-3"
UNIT = "Mpath-segments/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(method, width=512, height=512, spp=16, bsdf="exact"):
    from paper_1912_06474_gb300 import scenes
    scene = scenes.hotel_room(L=41, seed=0)
    spec = scenes.hotel_room_render(scene, width, height, spp, 5, seed=0)
    grid = (4, 4, 2) if method == "ddm" else (1, 1, 1)
    cfg = {"workload": f"hotel_room_{width}x{height}_{spp}spp_d5_L41", "triangles": scene.n_tris,
           "width": width, "height": height, "spp": spp, "max_depth": 5, "lambda_bins": 41, "method": method,
           "grid": list(grid), "bsdf": bsdf, "l2": "flushed between steps (256 MiB write)",
           "scaling_mode": "replicas"}
    return scene, spec, grid, cfg


def cpu_baseline(seconds_target=10.0, n_threads=0):
    """The FP64 oracle, as it stands, on a seeded pixel sample of the same workload."""
    import oracle
    from paper_1912_06474_gb300 import scenes
    scene, spec, _, _ = workload("ddm")
    orc = oracle.Oracle(scene)
    n_pix, done_pix, segs, t_total = 512, 0, 0, 0.0
    seed = 0
    while t_total < seconds_target and done_pix < spec.width * spec.height:
        pix = scenes.pixel_subset(spec.width, spec.height, n_pix, seed=seed)
        t0 = time.perf_counter()
        r = orc.render_pixels(spec, pix, n_threads=n_threads)
        dt = time.perf_counter() - t0
        t_total += dt
        segs += sum(r["segments"])
        done_pix += n_pix
        seed += 1
        n_pix = min(n_pix * 2, 8192)
    cores = n_threads if n_threads > 0 else (os.cpu_count() or 1)
    return {"value": segs / t_total / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done_pix} seeded pixels x 16 spp of the hotel-room workload ({segs} segments, "
                      f"{t_total:.1f} s wall)"}


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return
    _, _, _, cfg = workload(args.method, args.width, args.height, args.spp)
    times, vals = [], []
    base = None
    for k in range(args.warmup + args.steps):
        b = cpu_baseline(seconds_target=min(20.0, 60.0 / max(1, args.steps + args.warmup)))
        if k >= args.warmup:
            vals.append(b["value"])
            base = b
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run(args):
    import numpy as np
    import torch

    from paper_1912_06474_gb300 import sddm

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    scene, spec, grid, cfg = workload(args.method, args.width, args.height, args.spp, args.bsdf)
    spec.render_id = rank   # independent replicas: each rank renders its own stream of samples
    stream = torch.cuda.current_stream()
    ctx = sddm.Context(local, stream)
    ctx.set_scene(scene)
    t0 = time.perf_counter()
    ctx.build(grid=grid, blocks_per_sm=args.blocks_per_sm, paths_in_flight=args.paths_in_flight)
    build_s = time.perf_counter() - t0
    train = None
    if args.bsdf == "mlp":   # the surrogate is trained once, before and outside the timed steps
        train = ctx.mlp_train(scene.glass_materials()[0], seed=7)
        cfg["surrogate_training"] = {k: (round(v, 6) if isinstance(v, float) else v) for k, v in train.items()}
    out = torch.empty((spec.height, spec.width, 3), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # traversal counts of this exact workload (separately compiled counting kernel, untimed)
    ctx.set_profiling(count_traversal=True)
    cst = ctx.render_into([spec], [out], method=args.method, bsdf=args.bsdf)
    ctx.set_profiling(time_trace=True)
    for _ in range(args.warmup):
        ctx.render_into([spec], [out], method=args.method, bsdf=args.bsdf)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    segs, trace_ms, trace_launches, launches = 0, 0.0, 0, 0
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        st = ctx.render_into([spec], [out], method=args.method, bsdf=args.bsdf)
        ev[k][1].record(stream)
        segs += st["segments_ext"] + st["segments_shadow"]
        trace_ms += st["trace_ms"]
        trace_launches += st["trace_launches"]
        launches += st["kernel_launches"]
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    # the same steps replayed as a CUDA graph (the library's default launch path)
    ctx.set_profiling()
    for _ in range(3):
        ctx.render_into([spec], [out], method=args.method, bsdf=args.bsdf)
    gms, gsegs = 0.0, 0
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        st = ctx.render_into([spec], [out], method=args.method, bsdf=args.bsdf)
        ev[k][1].record(stream)
        gsegs += st["segments_ext"] + st["segments_shadow"]
    torch.cuda.synchronize()
    gms = sum(a.elapsed_time(b) for a, b in ev)
    # end to end through the host-buffer entry point
    host = torch.empty((spec.height, spec.width, 3), dtype=torch.float32).pin_memory()
    e2e_ms, e2e_segs = 0.0, 0
    for k in range(max(1, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.render_host([spec], [host], method=args.method, bsdf=args.bsdf)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_segs += st["segments_ext"] + st["segments_shadow"]
    clk = clocks.stop()

    if world > 1:
        t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        n = torch.tensor([segs, e2e_segs], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(n)
        total_ms, e2e_ms = float(t[0]), float(t[1])
        segs, e2e_segs = int(n[0]), int(n[1])
    if rank != 0:
        return
    value = segs / (total_ms / 1e3) / 1e6
    e2e = e2e_segs / (e2e_ms / 1e3) / 1e6
    # algorithmic bytes of the trace kernel per step, from the counting run
    visits, crossings = cst["ray_visits"], cst["crossings"]
    n_ext = cst["segments_ext"]
    bytes_step = (48 * visits + 48 * crossings + 32 * n_ext + 64 * cst["node_visits"] + 48 * cst["tri_tests"])
    trace_s = trace_ms / 1e3 / args.steps
    peak, peak_kind = _peaks()
    achieved = bytes_step / trace_s / 1e9 if trace_s > 0 else None
    traffic = None
    try:   # DRAM bytes per trace launch from an ncu capture, only while the kernel sources are unchanged
        import hashlib
        with open(os.path.join(ROOT, "profiles", "trace_traffic.json")) as f:
            tt = json.load(f)
        ent = tt.get(f"{args.method}:{cfg['workload']}")
        if ent and ent.get("valid", False):
            m = hashlib.sha256()
            for src in ent["sources"]:
                with open(os.path.join(ROOT, src), "rb") as f:
                    m.update(f.read())
            if m.hexdigest()[:16] == ent["source_sha256_16"]:
                traffic = ent["dram_bytes_per_launch"]
    except Exception:
        traffic = None
    h2d = 0   # render tables: a few hundred bytes, counted below from the descriptor layout
    h2d = 128 * 1 + 4 * len(scene.materials) + 3 * 8
    d2h = spec.width * spec.height * 3 * 4 + 64 + 16
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1) if achieved else None, "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
                     "traffic": traffic, "kernel": "k_trace_wave" if args.method == "ddm" else "k_megakernel",
                     "peak_kind": peak_kind, "bytes_per_step": bytes_step,
                     "trace_ms_per_step": round(trace_ms / args.steps, 4),
                     "trace_launches_per_step": trace_launches // args.steps,
                     "nodes_per_visit": round(cst["node_visits"] / max(visits, 1), 2),
                     "tris_per_visit": round(cst["tri_tests"] / max(visits, 1), 2)},
        "value_graph_replay": round(gsegs / (gms / 1e3) / 1e6, 3) if gms > 0 else None,
        "segments_per_step": segs // (args.steps * world), "build_s": round(build_s, 3), "clocks": clk,
        "mlp_fallback_batches_per_step": st.get("mlp_fallbacks", 0) if args.bsdf == "mlp" else None,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sddm", choices=["sddm", "reference"])
    ap.add_argument("--method", default="ddm", choices=["ddm", "megakernel"])
    ap.add_argument("--bsdf", default="exact", choices=["exact", "mlp"])
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--paths-in-flight", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--width", type=int, default=512)
    ap.add_argument("--height", type=int, default=512)
    ap.add_argument("--spp", type=int, default=16)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
