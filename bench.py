#!/usr/bin/env python
"""Benchmark of the 6D MCL sensor-update hot path on GB300.

One step = one pass of the whole path over one synthetic batch: scan packing,
pose matrices, transform + TSDF look-up + score + per-chunk sums (the sensor
kernel), log-weights, normalisation, systematic resampling with the particle
gather. Default workload: OS0-64-shaped scan (64 rings x 1,024 azimuths =
65,536 points) against a brick-sparse int16 TSDF of a 160 x 160 x 20 m
four-storey building at 5 cm, 1,000,000 particles uniform over free space.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on a bounded particle sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle×point evals/s (1M×65,536, int16 TSDF)"
UNIT = "evals/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=1_000_000)
    ap.add_argument("--azimuths", type=int, default=1024)
    ap.add_argument("--dtype", default="i16", choices=["f32", "f16", "i16"])
    ap.add_argument("--building", type=float, default=160.0, help="building edge (m)")
    ap.add_argument("--floors", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-gather", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target oracle CPU time for the cpu_baseline sample")
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--ppi", type=int, default=0)
    ap.add_argument("--unroll", type=int, default=0)
    ap.add_argument("--pipeline", type=int, default=0, help="0 auto, 1 off, 2 on")
    ap.add_argument("--order", type=int, default=0, help="particle order: 0 auto, 1 given, 2 spatial")
    ap.add_argument("--item-order", type=int, default=0,
                    help="work-item order: 0 auto, 1 chunk-major, 2 sweeps, 3 dynamic sweeps")
    ap.add_argument("--layout", type=int, default=0, help="brick layout: 0 linear, 1 4x4x4 blocks")
    ap.add_argument("--scan-rings", type=int, default=64,
                    help="rings of the OS0-64 scan given to the library (staging in 4 x 8 patches); 0: points as given")
    ap.add_argument("--trilinear", action="store_true",
                    help="the trilinear read (eight corners per evaluation) instead of the nearest voxel")
    ap.add_argument("--index", type=int, default=0, help="brick index: 0 auto, 1 hash, 2 cell grid")
    ap.add_argument("--mode", default="headline",
                    choices=["headline", "serving", "precision", "vlp16", "filter", "variants", "trilinear",
                             "batch"],
                    help="headline: 1M x 65,536 int16 step (+ serving probe); serving: 64 sessions over "
                         "8 maps; precision: f32/f16/i16 sweep with oracle weight error; vlp16: plain vs "
                         "batched graph-captured form on the VLP-16 tracking workload; filter: whole "
                         "filter steps (motion, sensor, estimate, resampling) as separate calls, as one "
                         "call and replayed from a CUDA graph; variants (or trilinear): the 1M x 65,536 "
                         "step with SUM on the TSDF, SUM on an FP16 score map and the trilinear read; "
                         "batch: the 1M x 65,536 update as one session and as a graph-captured batch of "
                         "--sessions sessions on the same map")
    ap.add_argument("--sessions", type=int, default=4, help="--mode batch: sessions of P / S particles")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving run of the headline")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the weight-error report and the storage/form comparison of the headline")
    ap.add_argument("--no-vlp16", action="store_true",
                    help="skip the VLP-16 tracking workload (dense hall) of the headline")
    ap.add_argument("--serving-seconds", type=float, default=8.0)
    ap.add_argument("--serving-batch", type=int, default=0,
                    help="sessions per batched serving step (0: the default policy)")
    ap.add_argument("--serving-scan-rings", action="store_true",
                    help="serving sessions given their scans' ring counts (4 x 8 patch staging)")
    ap.add_argument("--filter-workloads", default="room,hall",
                    help="--mode filter: comma list of room, hall")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(dist, value: float, device=None) -> float:
    """Largest value over all ranks (control plane only: one scalar)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self) -> dict:
        sm, smax, power, reasons = [], [], [], set()
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            try:
                power.append(float(f[2]))
            except ValueError:
                pass
            for name, val in zip(self.NAMES, f[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w": statistics.median(power) if power else None}


def energy(clocks: dict, ms_per_step: float, evals_per_step: float):
    """GPU board power during the timed region (median of the samples) and
    what it makes per step: the counterpart of the paper's run time and
    power figures (Table I)."""
    pw = clocks.get("power_w")
    if not pw:
        return None
    j = pw * ms_per_step / 1e3
    return {"power_w": pw, "joules_per_step": j, "evals_per_joule": evals_per_step / j}


# ------------------------------------------------------------------ workload
def make_workload(args, rank: int, with_f32: bool = False):
    """The building workload; with_f32 also voxelises FP32 values (the
    reference values of the weight-error report and the FP32 comparison)."""
    import scenes
    dt = {"f32": scenes.F32, "f16": scenes.F16, "i16": scenes.I16}[args.dtype]
    dts = tuple(sorted({dt, scenes.F32, scenes.F16})) if with_f32 else None
    return scenes.os064_building(P=args.particles, dtype=dt, seed=3, azimuths=args.azimuths,
                                 size=args.building, floors=args.floors, dtypes=dts)


def rank_particles(wl, rank: int):
    """Each rank localises its own robot session: same map, own particle cloud."""
    if rank == 0:
        return wl.particles
    import scenes
    return scenes.particles_free(wl.scene, len(wl.particles), 0.1, 10.0, 1000 + rank)


def algorithmic_bytes(P: int, N: int, elem: int, index_entry: int) -> int:
    """Bytes the sensor kernel must move per launch: one map element per
    (particle, point) evaluation plus one brick-index entry for a brick map
    (4 B in the cell grid, 8 B in the hash table); each pose record (48 B),
    scan point (16 B) and weight (4 B) once."""
    return P * N * (elem + index_entry) + P * 48 + N * 16 + P * 4


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
# Sessions per batched serving step: small batches complete sooner and cost
# no throughput on these workloads (64 sessions at the nominal rates: p50 778
# / 98 ms, p99 1.30 / 0.65 s for all pending sessions / 2 per step, 6.41e11
# / 6.31e11 evals/s).
SERVING_MAX_BATCH = 2


def kernel_source_digest() -> str:
    h = hashlib.sha256()
    for f in ("k_sensor.cu", "k_sensor_impl.cuh", "k_sensor_i16_grid.cu", "mcl_internal.h", "k_order.cu",
              "k_pose_scan.cu", "mcl_api.cpp"):
        with open(os.path.join(ROOT, "paper_2310_04172_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(P: int, N: int):
    """DRAM bytes (read + write) per sensor launch from the committed ncu
    summary, scaled by evaluations, if it was taken on the current kernel
    source; else None."""
    path = os.path.join(ROOT, "profiles", "sensor_dram_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("kernel_digest") != kernel_source_digest():
        return None
    per_eval = (rec["dram_bytes_read"] + rec.get("dram_bytes_write", 0.0)) / rec["evals"]
    return per_eval * P * N


def gather_source_digest() -> str:
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2310_04172_gb300", "csrc", "k_gather_bench.cu"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def gather_dram_bytes():
    """DRAM bytes one uniform-random gather moves (ncu, committed summary), or None."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "gather_dram_bytes.json")))
    except (OSError, ValueError):
        return None
    return rec["dram_bytes_per_gather"] if rec.get("kernel_digest") == gather_source_digest() else None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"], "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle timing
def time_oracle(wl, target_s: float, max_particles: int | None = None):
    """Oracle sensor update + normalise + resample on a particle sample sized
    to about target_s seconds of CPU work. Returns (evals/s, particles, seconds)."""
    import numpy as np
    import oracle
    om = oracle.Map.from_scene_map(wl.map)
    N = len(wl.scan)
    probe = 64
    t0 = time.perf_counter()
    L = oracle.sensor_update(om, wl.particles[:probe], wl.scan, wl.sigma_hit)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = int(min(len(wl.particles), max(probe, probe * target_s / dt)))
    if max_particles:
        n = min(n, max_particles)
    t0 = time.perf_counter()
    L = oracle.sensor_update(om, wl.particles[:n], wl.scan, wl.sigma_hit)
    w, *_ = oracle.normalise(L)
    oracle.resample(w.astype(np.float32), 0.5)
    dt = time.perf_counter() - t0
    return n * N / dt, n, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    import numpy as np
    import oracle
    wl = make_workload(args, 0)
    N = len(wl.scan)
    om = oracle.Map.from_scene_map(wl.map)
    total_budget = 150.0
    per_step = total_budget / max(1, args.steps + args.warmup)
    rate, _, _ = time_oracle(wl, min(per_step, 5.0))
    n = int(max(16, min(len(wl.particles), rate * per_step / N)))
    parts = wl.particles[:n]

    def step():
        L = oracle.sensor_update(om, parts, wl.scan, wl.sigma_hit)
        w, *_ = oracle.normalise(L)
        oracle.resample(w.astype(np.float32), 0.5)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = n * N * args.steps / dt
    cores = oracle.num_threads()
    sample = f"{n} of {len(wl.particles)} particles x {N} points per step (FP64 oracle, OpenMP)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args, wl),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(args, wl):
    m = wl.map
    return {
        "workload": wl.name, "particles": int(len(wl.particles)), "points": int(len(wl.scan)),
        "scan": f"64 rings (+-45 deg) x {args.azimuths} azimuths, sigma 0.02 m, ring-major"
                + (f", staged in 4 x 8 patches (scan_rings {args.scan_rings})" if args.scan_rings else ""),
        "map": {"kind": "brick16", "dtype": args.dtype,
                "layout": ["linear", "block4"][args.layout],
                "extent_m": [args.building, args.building, 5.0 * args.floors], "voxel_m": 0.05,
                "dims": list(m.dims), "bricks": int(len(m.coords)), "bytes": int(m.values.nbytes),
                "truncation_m": 0.3},
        "sigma_hit": wl.sigma_hit, "mode": "logprod",
        "read": "trilinear (8 corners)" if args.trilinear else "nearest voxel",
        "l2": "inputs larger than L2 (map %.2f GB, L2 129 MB)" % (m.values.nbytes / 1e9),
    }


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    from paper_2310_04172_gb300 import mcl
    mcl.lib()

    precision_on = rank == 0 and not args.no_precision
    wl = make_workload(args, rank, with_f32=precision_on)
    parts_np = rank_particles(wl, rank)
    P, N = len(parts_np), len(wl.scan)
    m = mcl.map_from_scene(wl.map, args.layout, args.index)
    elem = 4 if args.dtype == "f32" else 2
    stream = torch.cuda.Stream(device=dev)
    parts = torch.from_numpy(parts_np).to(dev)
    parts_next = torch.empty_like(parts)
    scan = torch.from_numpy(np.ascontiguousarray(wl.scan)).to(dev)
    logw = torch.empty(P, device=dev)
    w = torch.empty(P, device=dev)
    idx = torch.empty(P, dtype=torch.int32, device=dev)
    import scenes
    offsets = scenes.uniform(11 + rank, 200, args.steps + args.warmup + 64)
    prm = mcl.sensor_params(sigma_hit=wl.sigma_hit, points_per_chunk=args.chunk,
                            lanes_per_particle=args.lanes, particles_per_item=args.ppi,
                            unroll=args.unroll, pipeline=args.pipeline, particle_order=args.order,
                            item_order=args.item_order, scan_rings=args.scan_rings,
                            flags=mcl.MCL_TRILINEAR if args.trilinear else 0)
    plan = mcl.mcl_sensor_plan_get(m, P, N, prm)

    def step(k, s):
        mcl.mcl_sensor_update(m, parts, scan, prm, logw, w, s)
        mcl.mcl_resample(w, float(offsets[k % len(offsets)]), idx, parts, parts_next, s)

    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            step(k, stream)
    mcl.mcl_sync(stream)

    gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
    gpu_id = gpu_id if gpu_id.startswith("GPU-") else f"GPU-{gpu_id}"
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    with ClockSampler(gpu_id) as clocks:
        start.record(stream)
        mcl.mcl_profile_begin()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                step(args.warmup + k, stream)
        end.record(stream)
        torch.cuda.synchronize(dev)
        prof = mcl.mcl_profile_end()
    if dist is not None:
        dist.barrier()
    mcl.mcl_sync(stream)
    ms = start.elapsed_time(end)
    ms_max = max_over_ranks(dist, ms, dev)
    evals = float(P) * N * args.steps
    total_evals = sum_over_ranks(dist, evals, dev)
    value = total_evals / (ms_max / 1e3)
    launches = sum(v["launches"] for v in prof.values())

    # roofline of the dominant kernel, timed live in the region above
    sensor_ms = prof["sensor"]["ms"] / max(1, prof["sensor"]["launches"])
    index_entry = {1: 8, 2: 4}.get(m.info()["index"], 0)
    corners = 8 if args.trilinear else 1
    abytes = algorithmic_bytes(P, N, corners * elem, index_entry)
    achieved = abytes / (sensor_ms / 1e3) / 1e9
    peak, peak_src = peaks()
    traffic = None if args.trilinear else measured_traffic(P, N)  # the record is the nearest read's
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
            "kernel": "k_sensor", "kernel_ms": sensor_ms,
            "algorithmic_bytes_per_launch": abytes,
            "bytes_per_eval": corners * elem + index_entry}

    # gather roofline: uniform-random element reads over a buffer of the map's size
    gather = None
    if not args.no_gather:
        gather = gather_roofline(torch, mcl, dev, stream, int(wl.map.values.nbytes), elem, value)
        per_gather = gather_dram_bytes()
        if traffic is not None and per_gather is not None:
            # DRAM-traffic form: the sensor kernel's DRAM bytes/s against the DRAM
            # bytes/s that uniform-random gathers sustain at the map footprint
            sensor_gbs = traffic / (sensor_ms / 1e3) / 1e9
            gather_gbs = gather["map_footprint"]["gathers_per_s"] * per_gather / 1e9
            gather.update({"dram_bytes_per_gather": per_gather, "gather_dram_gbs": gather_gbs,
                           "sensor_dram_gbs": sensor_gbs, "frac_dram": sensor_gbs / gather_gbs,
                           # the sensor kernel's DRAM rate against the copy peak and
                           # against the part's nominal 7.9 TB/s
                           "sensor_dram_frac_of_copy_peak": sensor_gbs / peak,
                           "sensor_dram_frac_of_nominal": sensor_gbs / NOMINAL_HBM_GBS})
        # the absolute bound: every evaluation moving only its element bytes at
        # the copy peak
        gather["elem_bytes_bound_evals_per_s"] = peak * 1e9 / elem
        gather["frac_of_elem_bytes_bound"] = value / (peak * 1e9 / elem)

    # end to end through the C ABI with host buffers (pinned), copies in the region
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(torch, mcl, m, parts_np, wl.scan, prm, offsets, args, dev, dist)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        rate, n, dt = time_oracle(wl, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{n} of {P} particles x {N} points, sensor update + normalise + "
                         f"resample, {dt:.1f} s (FP64, OpenMP over particles)"}

    precision = forms = None
    if precision_on:
        try:
            precision, forms = precision_block(torch, mcl, wl, m, parts, scan, prm, sensor_ms, args)
        except Exception as e:  # the headline line is printed whatever happens here
            precision = {"error": f"{type(e).__name__}: {e}"}

    vlp16 = None
    if rank == 0 and not args.no_vlp16:
        try:
            vlp16 = vlp16_block(torch, mcl, max(args.steps, 20))
        except Exception as e:
            vlp16 = {"error": f"{type(e).__name__}: {e}"}

    serving = None
    if rank == 0 and not args.no_serving:
        try:
            serving = serving_block(mcl, args.serving_seconds, rings=args.serving_scan_rings)
        except Exception as e:
            serving = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        cfg = config_dict(args, wl)
        info = m.info()
        cfg["launch"] = dict(plan, brick_index={1: "hash", 2: "cell grid"}.get(info["index"], "none"),
                             brick_index_bytes=info["index_bytes"])
        if info["index"] == 2:  # cell-grid maps keep each brick rotated by its cell coordinates
            cfg["map"]["device_layout"] = "skewed per brick (value of voxel i at (ix + 16 iy + 256 iz) mod 4096)"
        cfg["parallelism"] = f"replicas{world}" if world > 1 else "single"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg, "roofline": roof, "gather_roofline": gather, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks.summary(),
            "precision": precision, "quantised_vs_plain_fp32": forms, "vlp16_tracking": vlp16,
            "serving": serving,
            "energy": energy(clocks.summary(), ms_max / args.steps, float(P) * N),
            "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items() if v["launches"]},
        }
        print(json.dumps(line), flush=True)
    m.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def gather_roofline(torch, mcl, dev, stream, nbytes, elem, evals_per_s):
    """Uniform-random gathers/s at the map footprint (HBM) and in L2 (64 MB)."""
    out = {}
    for label, size in (("map_footprint", nbytes), ("l2_resident_64MB", 64 << 20)):
        dt = torch.int16 if elem == 2 else torch.float32
        buf = torch.ones(max(1, size // elem), dtype=dt, device=dev)
        blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
        iters = 64
        with torch.cuda.stream(stream):
            mcl.mcl_gather_bench(buf, blocks, iters, 1, stream)
        best = None
        for rep in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with torch.cuda.stream(stream):
                n = mcl.mcl_gather_bench(buf, blocks, iters, 2 + rep, stream)
            b.record(stream)
            b.synchronize()
            rate = n / (a.elapsed_time(b) / 1e3)
            best = rate if best is None else max(best, rate)
        out[label] = {"bytes": int(buf.numel() * elem), "gathers_per_s": best}
        del buf
    out["frac_evals"] = evals_per_s / out["map_footprint"]["gathers_per_s"]
    out["elem_bytes"] = elem
    return out


def end_to_end(torch, mcl, m, parts_np, scan_np, prm, offsets, args, dev, dist):
    import numpy as np
    P, N = len(parts_np), len(scan_np)
    s = torch.cuda.Stream(device=dev)
    h_parts = torch.from_numpy(parts_np).pin_memory()
    h_scan = torch.from_numpy(np.ascontiguousarray(scan_np)).pin_memory()
    h_w = torch.empty(P, dtype=torch.float32).pin_memory()
    h_idx = torch.empty(P, dtype=torch.int32).pin_memory()
    d_parts = torch.empty((P, 6), device=dev)
    d_next = torch.empty_like(d_parts)
    d_scan = torch.empty((N, 3), device=dev)
    d_logw = torch.empty(P, device=dev)
    d_w = torch.empty(P, device=dev)
    d_idx = torch.empty(P, dtype=torch.int32, device=dev)

    def step(k):
        with torch.cuda.stream(s):
            d_parts.copy_(h_parts, non_blocking=True)
            d_scan.copy_(h_scan, non_blocking=True)
            mcl.mcl_sensor_update(m, d_parts, d_scan, prm, d_logw, d_w, s)
            mcl.mcl_resample(d_w, float(offsets[k % len(offsets)]), d_idx, d_parts, d_next, s)
            h_w.copy_(d_w, non_blocking=True)
            h_idx.copy_(d_idx, non_blocking=True)
        s.synchronize()

    step(0)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k + 1)
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dist, dt, dev)
    world = dist.get_world_size() if dist is not None else 1
    return {"value": world * float(P) * N * args.steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": int(h_parts.numel() * 4 + h_scan.numel() * 4),
            "d2h_bytes_per_step": int(h_w.numel() * 4 + h_idx.numel() * 4),
            "ms_per_step": 1e3 * dt / args.steps}


# ------------------------------------------------------------------ serving
def run_clients(mcl, srv, sessions, seconds, rate_scale, seed):
    """Poisson scan streams (one thread per session) for `seconds`; returns results."""
    import threading
    import numpy as np
    deadline = time.time() + seconds
    tickets, lock = [], threading.Lock()

    def client(k, sess, scan, rate):
        r = np.random.default_rng(seed + k)
        while True:
            time.sleep(r.exponential(1.0 / (rate * rate_scale)))
            if time.time() >= deadline:
                return
            t = sess.submit(scan)
            with lock:
                tickets.append(t)

    th = [threading.Thread(target=client, args=(k, s, sc, rt)) for k, (s, sc, rt) in enumerate(sessions)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    res = [srv.wait(t, 120_000) for t in tickets]
    return res


def serving_measure(mcl, srv, sessions, seconds, rate_scale, seed):
    import numpy as np
    srv.stats(reset=True)
    res = run_clients(mcl, srv, sessions, seconds, rate_scale, seed)
    st = srv.stats()
    lat = np.array([r["latency_ms"] for r in res if r["status"] == mcl.MCL_RESULT_DONE])
    offered = sum(rt * rate_scale * s.P * len(sc) for s, sc, rt in sessions)
    return {"offered_evals_per_s": offered, "achieved_evals_per_s": st["evals_per_s"],
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "max_ms": float(lat.max()) if len(lat) else None,
            "completed": int(st["completed"]), "superseded": int(st["superseded"]),
            "supersede_rate": st["superseded"] / max(1, len(res)),
            "mean_batch_sessions": st["mean_batch_sessions"], "seconds": seconds}


def serving_sessions(mcl, srv, maps, n, p_lo, p_hi, seed):
    """n sessions round-robin over (map, scene, scan) entries, P log-uniform, 10-20 Hz."""
    import numpy as np
    import scenes
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        m, sc, scan, rings = maps[k % len(maps)]
        P = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        parts = scenes.particles_free(sc, P, 0.1, 10.0, seed * 1000 + k)
        sess = srv.open(m, parts, len(scan), seed=seed * 1000 + k,
                        motion_sigma=(0.02, 0.02, 0.01, 0.002, 0.002, 0.01), scan_rings=rings)
        out.append((sess, scan, float(rng.uniform(10.0, 20.0))))
    return out


def vlp16_block(torch, mcl, reps: int):
    """The VLP-16 tracking workload: dense 512x512x128 FP32 hall (and the same
    hall as FP16), 50,000 Gaussian particles x 28,800 points; one step =
    sensor update + normalisation + resampling, plain calls against the
    batched, graph-captured form."""
    import scenes
    wl = scenes.vlp16_multiroom(P=50_000, dtype=scenes.F32)
    m = mcl.map_from_scene(wl.map)
    parts = torch.from_numpy(wl.particles).cuda()
    nxt = torch.empty_like(parts)
    scan = torch.from_numpy(wl.scan).cuda()
    P, N = parts.shape[0], scan.shape[0]
    logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    idx = torch.empty(P, dtype=torch.int32, device="cuda")
    prm = mcl.sensor_params(wl.sigma_hit)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(reps):
            fn()
        e.record()
        e.synchronize()
        return a.elapsed_time(e) / reps

    def plain(mm):
        mcl.mcl_sensor_update(mm, parts, scan, prm, logw, w)
        mcl.mcl_resample(w, 0.5, idx, parts, nxt)

    ms_plain = timed(lambda: plain(m))
    batch = mcl.Batch([{"map": m, "particles": parts, "scan": scan, "logw": logw, "w": w,
                        "resample_idx": idx, "particles_out": nxt}], use_graph=True)
    batch.set_offsets([0.5])
    ms_batch = timed(batch.run)
    kernels = batch.info()["kernels_per_run"]
    batch.close()
    m.close()
    wl16 = scenes.vlp16_multiroom(P=16, dtype=scenes.F16)
    m16 = mcl.map_from_scene(wl16.map)
    ms_f16 = timed(lambda: plain(m16))
    m16.close()
    ev = float(P) * N
    return {"workload": wl.name, "particles": P, "points": N,
            "plain": {"ms_per_step": ms_plain, "evals_per_s": ev / (ms_plain / 1e3)},
            "batched_graph": {"ms_per_step": ms_batch, "evals_per_s": ev / (ms_batch / 1e3),
                              "kernels_per_step": kernels},
            "plain_f16_map": {"ms_per_step": ms_f16, "evals_per_s": ev / (ms_f16 / 1e3)}}


def serving_block(mcl, seconds: float, max_batch: int = 0, rings: bool = False):
    """The 64-session serving workload: 64 robot sessions over 8 maps (4 dense
    512x512x128 FP16 halls, 4 brick int16 160x160x20 m buildings), P
    log-uniform in [1e3, 1e6], scans of 28,800 (halls, 16 rings) and 65,536
    (buildings, 64 rings) points, staged as given (`rings`: each session
    given its scan's ring count, staging in 4 x 8 patches, which costs more
    than it saves once a session's particles have converged), Poisson
    10-20 Hz per session:
    first at the nominal rates (offered load far above one GPU: the latest
    scan of a session wins), then scaled to 70 % of the achieved throughput.
    `seconds` of arrivals per load level."""
    import scenes
    maps = []
    for k in range(4):
        hall = scenes.vlp16_multiroom(P=16, dtype=scenes.F16, seed=11 + k)
        maps.append((mcl.map_from_scene(hall.map), hall.scene, hall.scan, 16 if rings else 0))
        bld = scenes.os064_building(P=16, dtype=scenes.I16, seed=15 + k)
        maps.append((mcl.map_from_scene(bld.map), bld.scene, bld.scan, 64 if rings else 0))
    max_batch = max_batch or SERVING_MAX_BATCH
    srv = mcl.Server(200 << 30, 64, max_in_flight=2, max_batch=max_batch)
    sess = serving_sessions(mcl, srv, maps, 64, 1e3, 1e6, 31)
    nominal = serving_measure(mcl, srv, sess, seconds, 1.0, 7)
    scale = 0.7 * nominal["achieved_evals_per_s"] / nominal["offered_evals_per_s"]
    scaled = serving_measure(mcl, srv, sess, seconds, scale, 9)
    out = {"sessions": len(sess), "maps": len(maps),
           "workload": "64 sessions over 4 dense FP16 halls + 4 int16 brick buildings",
           "policy": f"max_in_flight 2, max_batch {max_batch}, longest-waiting sessions first",
           "scan_staging": "4 x 8 patches (scan_rings 16 / 64)" if rings else "as given",
           "particles_total": int(sum(x.P for x, _, _ in sess)),
           "nominal_load": nominal, "scaled_load_70pct": dict(scaled, rate_scale=scale)}
    for x, _, _ in sess:
        x.close()
    srv.close()
    for mm, _, _, _ in maps:
        mm.close()
    return out


# ------------------------------------------------------------------ weight error against the oracle
def weight_report(Lg, wg, Lo) -> dict:
    """Errors of one GPU result (its log-weights Lg and its own normalised
    weights wg) against the FP64 oracle's log-weights Lo of the same particles
    (Eq. 3 per point, normalisation as in Sec. V-A)."""
    import numpy as np
    Lg = np.asarray(Lg, np.float64)
    wg = np.asarray(wg, np.float64)
    wo = np.exp(Lo - Lo.max())
    wo /= wo.sum()
    jo = int(np.argmax(Lo))
    near = np.flatnonzero(Lo >= Lo[jo] - 30.0)  # weights within e^-30 of the best
    ro = np.exp(Lo[near] - Lo[jo])
    with np.errstate(divide="ignore", invalid="ignore"):
        rg = wg[near] / wg[jo]
    k = min(100, len(Lo))
    top_o = set(np.argsort(-Lo, kind="stable")[:k].tolist())
    top_g = set(np.argsort(-Lg, kind="stable")[:k].tolist())
    big = wo >= 1e-6 * wo.max()  # weights within 1e-6 of the largest
    return {"max_rel_logw_err": float(np.max(np.abs(Lg - Lo) / np.maximum(1.0, np.abs(Lo)))),
            "max_abs_logw_err": float(np.max(np.abs(Lg - Lo))),
            "tv_distance": float(0.5 * np.abs(wg - wo).sum()),
            "particles_within_30_nats": int(len(near)),
            "max_rel_w_err_within_30_nats": float(np.max(np.abs(rg - ro) / ro)),
            "particles_w_above_1e-6_max": int(big.sum()),
            "max_rel_w_err_above_1e-6_max": float(np.max(np.abs(wg[big] - wo[big]) / wo[big])),
            "top100_agreement": len(top_o & top_g) / k,
            "argmax_agrees": bool(int(np.argmax(Lg)) == jo)}


def precision_block(torch, mcl, wl, m_head, parts, scan, prm, head_kernel_ms, args):
    """Weight error of the headline form (int16 map) and of the same step on
    FP16 and FP32 map values against the FP64 oracle (quality mode: FP64 throughout on
    the FP32 values) on two seeded 10,000-particle subsets: the headline's
    global-localisation cloud, and a tracking cloud Gaussian about the true
    pose (0.2 m, 2 deg), where more particles carry weight. Then the same
    1M x 65,536 update on the FP32 map, in the same kernel shape and in the
    plain per-session form (particles as given, chunk-major items, points as
    given), and the int16 map in a graph-captured batch of four
    250,000-particle sessions, each given the scan's ring count."""
    import numpy as np
    import oracle
    import scenes
    maps = wl.info["maps"]
    P, N = len(wl.particles), len(wl.scan)
    m32 = mcl.map_from_scene(maps[scenes.F32])
    m16 = mcl.map_from_scene(maps[scenes.F16])
    om = oracle.Map.from_scene_map(maps[scenes.F32])
    rng = np.random.default_rng(4)
    subsets = {"global_10000": wl.particles[np.sort(rng.choice(P, 10_000, replace=False))],
               "tracking_10000": scenes.particles_gaussian(wl.pose, 10_000, 0.2, 2.0, 41)}
    rep = {"reference": "FP64 oracle, quality mode (FP64 throughout on the FP32 map values)",
           "note": "LOGPROD: the weights of a 65,536-point scan concentrate on one particle "
                   "(the log-weights of neighbouring poses differ by thousands of nats), so "
                   "the weight error there is the argmax, top-100 and log-weight agreement; "
                   "SUM (Eq. 3 summed over points) spreads the weight over many particles "
                   "and gives a relative weight error",
           "subsets": {}}
    prm_sum = mcl.sensor_params(wl.sigma_hit, mode=mcl.MCL_SUM)
    for name, sub in subsets.items():
        dsub = torch.from_numpy(np.ascontiguousarray(sub)).to(parts.device)
        res = {}
        for mode, mprm, key in ((oracle.LOGPROD, prm, "logprod"), (oracle.SUM, prm_sum, "sum")):
            t0 = time.perf_counter()
            Lo = oracle.sensor_update(om, sub, wl.scan, wl.sigma_hit, mode=mode, parity=False)
            res[f"oracle_s_{key}"] = time.perf_counter() - t0
            for label, mm in (("i16", m_head), ("f16", m16), ("f32", m32)):
                lg = torch.empty(len(sub), device=parts.device)
                wg = torch.empty(len(sub), device=parts.device)
                mcl.mcl_sensor_update(mm, dsub, scan, mprm, lg, wg)
                mcl.mcl_sync()
                res[f"{label}_{key}"] = weight_report(lg.cpu().numpy(), wg.cpu().numpy(), Lo)
        rep["subsets"][name] = res

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(reps):
            fn()
        e.record()
        e.synchronize()
        return a.elapsed_time(e) / reps

    logw = torch.empty(P, device=parts.device)
    w = torch.empty(P, device=parts.device)
    plain = mcl.sensor_params(wl.sigma_hit, particle_order=1, item_order=1)
    ms_f32 = timed(lambda: mcl.mcl_sensor_update(m32, parts, scan, prm, logw, w))
    ms_f32_plain = timed(lambda: mcl.mcl_sensor_update(m32, parts, scan, plain, logw, w))
    ms_f16 = timed(lambda: mcl.mcl_sensor_update(m16, parts, scan, prm, logw, w))
    m16.close()
    S = 4
    per = P // S
    sess_parts = [parts[k * per:(k + 1) * per].contiguous() for k in range(S)]
    outs = [(torch.empty(per, device=parts.device), torch.empty(per, device=parts.device))
            for _ in range(S)]
    batch = mcl.Batch([{"map": m_head, "particles": sess_parts[k], "scan": scan,
                        "logw": outs[k][0], "w": outs[k][1], "scan_rings": args.scan_rings}
                       for k in range(S)], use_graph=True)
    ms_batch = timed(batch.run)
    kernels = batch.info()["kernels_per_run"]
    batch.close()
    m32.close()
    ev = float(P) * N

    def form(ms):
        return {"ms_per_update": ms, "evals_per_s": ev / (ms / 1e3)}

    err_i16 = rep["subsets"]["tracking_10000"]["i16_logprod"]
    err_f32 = rep["subsets"]["tracking_10000"]["f32_logprod"]
    sum_i16 = rep["subsets"]["tracking_10000"]["i16_sum"]
    sum_f32 = rep["subsets"]["tracking_10000"]["f32_sum"]
    forms = {
        "f32_same_shape": form(ms_f32),
        "f32_plain_per_session": dict(form(ms_f32_plain), shape="particles as given, chunk-major items"),
        "i16_single": form(head_kernel_ms),
        "f16_same_shape": form(ms_f16),
        "i16_batched_graph_4x250000": dict(form(ms_batch), kernels_per_run=kernels),
        "speedup_i16_batched_vs_f32_same_shape": ms_f32 / ms_batch,
        "speedup_i16_batched_vs_f32_plain": ms_f32_plain / ms_batch,
        "at_weight_error": {"subset": "tracking_10000",
                            "i16_tv_distance": err_i16["tv_distance"],
                            "f32_tv_distance": err_f32["tv_distance"],
                            "i16_max_rel_logw_err": err_i16["max_rel_logw_err"],
                            "f32_max_rel_logw_err": err_f32["max_rel_logw_err"],
                            "i16_top100_agreement": err_i16["top100_agreement"],
                            "f32_top100_agreement": err_f32["top100_agreement"],
                            "sum_mode_i16_max_rel_w_err": sum_i16["max_rel_w_err_above_1e-6_max"],
                            "sum_mode_f32_max_rel_w_err": sum_f32["max_rel_w_err_above_1e-6_max"],
                            "sum_mode_i16_tv_distance": sum_i16["tv_distance"],
                            "sum_mode_f32_tv_distance": sum_f32["tv_distance"]},
    }
    return rep, forms


def run_serving(args):
    """The 64-session serving workload alone (see serving_block), with twice
    the arrival time per load level."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_04172_gb300 import mcl
    torch.cuda.set_device(0)
    out = serving_block(mcl, args.serving_seconds * 2, args.serving_batch, rings=args.serving_scan_rings)
    line = {"mode": "serving", "metric": "serving p50/p99 update latency (64 sessions, 8 maps)",
            "value": out["scaled_load_70pct"]["p99_ms"], "unit": "ms (p99)", "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic", "dtype": "f32",
            "config": {k: out[k] for k in ("workload", "policy", "particles_total")},
            "nominal_load": out["nominal_load"], "scaled_load_70pct": out["scaled_load_70pct"]}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ precision sweep
def run_precision(args):
    """The building workload stored as FP32, FP16 and int16: update time for
    1M x 65,536 and the weight report (weight_report) of each against the FP64
    oracle (quality mode, FP32 values) on the two seeded 10,000-particle
    subsets of precision_block."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import scenes
    from paper_2310_04172_gb300 import mcl
    torch.cuda.set_device(0)
    wl = scenes.os064_building(P=args.particles, dtype=scenes.F32,
                               dtypes=(scenes.F32, scenes.F16, scenes.I16))
    maps = wl.info["maps"]
    P, N = len(wl.particles), len(wl.scan)
    parts = torch.from_numpy(wl.particles).cuda()
    scan = torch.from_numpy(wl.scan).cuda()
    rng = np.random.default_rng(4)
    subsets = {"global_10000": wl.particles[np.sort(rng.choice(P, 10_000, replace=False))],
               "tracking_10000": scenes.particles_gaussian(wl.pose, 10_000, 0.2, 2.0, 41)}
    om = oracle.Map.from_scene_map(maps[scenes.F32])
    modes = {"logprod": (oracle.LOGPROD, mcl.sensor_params(wl.sigma_hit)),
             "sum": (oracle.SUM, mcl.sensor_params(wl.sigma_hit, mode=mcl.MCL_SUM))}
    refs = {(k, mk): oracle.sensor_update(om, v, wl.scan, wl.sigma_hit, mode=mo, parity=False)
            for k, v in subsets.items() for mk, (mo, _) in modes.items()}
    prm = mcl.sensor_params(wl.sigma_hit)
    out = {}
    for dt, name in ((scenes.F32, "f32"), (scenes.F16, "f16"), (scenes.I16, "i16")):
        m = mcl.map_from_scene(maps[dt])
        logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
        mcl.mcl_sensor_update(m, parts, scan, prm, logw, w)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(args.steps):
            mcl.mcl_sensor_update(m, parts, scan, prm, logw, w)
        e.record()
        e.synchronize()
        ms = a.elapsed_time(e) / args.steps
        res = {"ms_per_update": ms, "evals_per_s": P * N / (ms / 1e3),
               "map_bytes": int(maps[dt].values.nbytes)}
        for k, sub in subsets.items():
            ds = torch.from_numpy(np.ascontiguousarray(sub)).cuda()
            for mk, (_, mprm) in modes.items():
                lg, wg = torch.empty(len(sub), device="cuda"), torch.empty(len(sub), device="cuda")
                mcl.mcl_sensor_update(m, ds, scan, mprm, lg, wg)
                mcl.mcl_sync()
                res[f"{k}_{mk}"] = weight_report(lg.cpu().numpy(), wg.cpu().numpy(), refs[(k, mk)])
        out[name] = res
        m.close()
    line = {"mode": "precision", "metric": METRIC, "value": out["i16"]["evals_per_s"], "unit": UNIT,
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic", "dtype": "f32",
            "config": {"workload": wl.name, "subsets": list(subsets),
                       "reference": "FP64 oracle, quality mode (FP64 throughout on the FP32 map values)"},
            "storage": out}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ VLP-16 tracking
def run_vlp16(args):
    """Dense 512x512x128 FP32 hall, 50,000 Gaussian particles x 28,800 points:
    the plain per-call form against the batched, graph-captured form."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import scenes
    from paper_2310_04172_gb300 import mcl
    torch.cuda.set_device(0)
    wl = scenes.vlp16_multiroom(P=50_000, dtype=scenes.F32)
    m = mcl.map_from_scene(wl.map)
    parts = torch.from_numpy(wl.particles).cuda()
    nxt = torch.empty_like(parts)
    scan = torch.from_numpy(wl.scan).cuda()
    P, N = parts.shape[0], scan.shape[0]
    logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    idx = torch.empty(P, dtype=torch.int32, device="cuda")
    prm = mcl.sensor_params(wl.sigma_hit)

    def plain():
        mcl.mcl_sensor_update(m, parts, scan, prm, logw, w)
        mcl.mcl_resample(w, 0.5, idx, parts, nxt)

    batch = mcl.Batch([{"map": m, "particles": parts, "scan": scan, "logw": logw, "w": w,
                        "resample_idx": idx, "particles_out": nxt}], use_graph=True)
    batch.set_offsets([0.5])

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(reps):
            fn()
        e.record()
        e.synchronize()
        return a.elapsed_time(e) / reps

    reps = max(args.steps, 20)
    ms_plain = timed(plain, reps)
    ms_batch = timed(batch.run, reps)
    # the same hall stored as FP16 (64 MB, the half-size form of this workload)
    wl16 = scenes.vlp16_multiroom(P=50_000, dtype=scenes.F16)
    m16 = mcl.map_from_scene(wl16.map)
    ms_f16 = timed(lambda: (mcl.mcl_sensor_update(m16, parts, scan, prm, logw, w),
                            mcl.mcl_resample(w, 0.5, idx, parts, nxt)), reps)
    m16.close()
    line = {"mode": "vlp16", "metric": "particle×point evals/s (50,000×28,800, FP32 dense TSDF)",
            "value": P * N / (ms_batch / 1e3), "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic", "dtype": "f32", "config": {"workload": wl.name},
            "plain": {"ms_per_step": ms_plain, "evals_per_s": P * N / (ms_plain / 1e3)},
            "batched_graph": {"ms_per_step": ms_batch, "evals_per_s": P * N / (ms_batch / 1e3),
                              "kernels_per_step": batch.info()["kernels_per_run"]},
            "plain_f16_map": {"ms_per_step": ms_f16, "evals_per_s": P * N / (ms_f16 / 1e3),
                              "map_bytes": int(wl16.map.values.nbytes)}}
    print(json.dumps(line), flush=True)
    batch.close()
    m.close()
    return 0


# ------------------------------------------------------------------ whole filter steps
def run_filter(args):
    """Whole filter steps on two tracking workloads: the 1,000-particle room
    (VLP-16 shape, 1,024 points: launch-bound) and the 50,000-particle hall
    (28,800 points). Three forms of the same step: separate C-ABI calls
    (motion, sensor update with estimate, resampling, copy back), one filter
    call per step, and the filter replayed from a CUDA graph."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import scenes
    from paper_2310_04172_gb300 import mcl
    torch.cuda.set_device(0)
    sigma_m = np.array([0.02, 0.02, 0.01, 0.005, 0.005, 0.01], np.float32)
    delta = np.array([0.05, 0.0, 0.0, 0.0, 0.0, 0.01], np.float32)
    reps = max(args.steps, 50)

    def timed(fn, n):
        for k in range(5):
            fn(k)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for k in range(n):
            fn(k)
        e.record()
        e.synchronize()
        return a.elapsed_time(e) / n

    out = {}
    cases = {"room": ("room_1000x1024", lambda: scenes.room_plain(P=1000)),
             "hall": ("hall_50000x28800", lambda: scenes.vlp16_multiroom(P=50_000, dtype=scenes.F32))}
    for key in args.filter_workloads.split(","):
        label, make = cases[key]
        wl = make()
        m = mcl.map_from_scene(wl.map)
        P, N = wl.particles.shape[0], wl.scan.shape[0]
        prm = mcl.sensor_params(wl.sigma_hit)
        scan = torch.from_numpy(wl.scan).cuda()
        parts = torch.from_numpy(wl.particles).cuda()
        nxt = torch.empty_like(parts)
        logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
        idx = torch.empty(P, dtype=torch.int32, device="cuda")
        est = mcl.estimate_buffer()

        def calls(k):
            mcl.mcl_motion_update(parts, delta, sigma_m, 7, k)
            mcl.mcl_sensor_update_estimate(m, parts, scan, prm, logw, w, est)
            mcl.mcl_resample(w, 0.5, idx, parts, nxt)
            parts.copy_(nxt)

        res = {"particles": P, "points": N}
        res["separate_calls_ms"] = timed(calls, reps)
        for name, graph in (("filter_call_ms", False), ("filter_graph_ms", True)):
            f = mcl.Filter(m, torch.from_numpy(wl.particles).cuda(), max_points=N, params=prm,
                           motion_sigma=sigma_m, seed=7, use_graph=graph)
            res[name] = timed(lambda k: f.step(scan, delta, est), reps)
            if not graph:  # where a step's device time goes (events around each phase)
                mcl.mcl_profile_begin()
                for k in range(10):
                    f.step(scan, delta, est)
                torch.cuda.synchronize()
                prof = mcl.mcl_profile_end()
                res["phases_ms_per_step"] = {k: v["ms"] / 10 for k, v in prof.items() if v["launches"]}
            f.close()
        # cost of the fused estimate: the sensor update with and without it
        res["sensor_update_ms"] = timed(lambda k: mcl.mcl_sensor_update(m, parts, scan, prm, logw, w), reps)
        res["sensor_update_estimate_ms"] = timed(
            lambda k: mcl.mcl_sensor_update_estimate(m, parts, scan, prm, logw, w, est), reps)
        res["graph_steps_per_s"] = 1e3 / res["filter_graph_ms"]
        res["graph_evals_per_s"] = P * N / (res["filter_graph_ms"] / 1e3)
        out[label] = res
        m.close()
    head = out.get("hall_50000x28800") or next(iter(out.values()))
    line = {"mode": "filter", "metric": "particle×point evals/s of whole filter steps (50,000×28,800)"
            if "hall_50000x28800" in out else "particle×point evals/s of whole filter steps (1,000×1,024)",
            "value": head["graph_evals_per_s"], "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic", "dtype": "f32", "steps": reps,
            "config": {"workload": ", ".join(label for label in out),
                       "step": "motion update, sensor update + pose estimate, systematic resampling"},
            "results": out}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ read and score variants
def run_variants(args):
    """The headline step size (1M x 65,536, int16 bricks) with each variant of
    the read and the score: nearest-voxel LOGPROD (the headline), SUM on the
    TSDF (exp per evaluation), SUM on an FP16 score map (the exponential
    precomputed per voxel), and the trilinear read (eight corner values per
    evaluation, one brick-index probe per distinct brick); the scan staged as
    the headline stages it (`--scan-rings`)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_04172_gb300 import mcl
    torch.cuda.set_device(0)
    wl = make_workload(args, 0)
    m = mcl.map_from_scene(wl.map)
    t0 = time.time()
    sc = mcl.mcl_map_create_score(m, wl.sigma_hit, mcl.MCL_F16)
    score_build_s = time.time() - t0
    P, N = wl.particles.shape[0], wl.scan.shape[0]
    parts = torch.from_numpy(wl.particles).cuda()
    scan = torch.from_numpy(np.ascontiguousarray(wl.scan)).cuda()
    logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    elem = 4 if args.dtype == "f32" else 2
    peak, peak_src = peaks()
    out = {}
    steps = max(1, min(args.steps, 5))
    variants = (("nearest_logprod", m, mcl.MCL_LOGPROD, 0, 1),
                ("nearest_sum_tsdf", m, mcl.MCL_SUM, 0, 1),
                ("nearest_sum_score_f16", sc, mcl.MCL_SUM, 0, 1),
                ("trilinear_logprod", m, mcl.MCL_LOGPROD, mcl.MCL_TRILINEAR, 8))
    for name, mm, mode, flags, corners in variants:
        prm = mcl.sensor_params(wl.sigma_hit, mode=mode, flags=flags, scan_rings=args.scan_rings)
        for _ in range(max(args.warmup, 3)):
            mcl.mcl_sensor_update(mm, parts, scan, prm, logw, w)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        mcl.mcl_profile_begin()
        a.record()
        for _ in range(steps):
            mcl.mcl_sensor_update(mm, parts, scan, prm, logw, w)
        e.record()
        e.synchronize()
        prof = mcl.mcl_profile_end()
        ms = a.elapsed_time(e) / steps
        kms = prof["sensor"]["ms"] / max(1, prof["sensor"]["launches"])
        per_eval = corners * elem + {1: 8, 2: 4}.get(mm.info()["index"], 0)
        abytes = P * N * per_eval + P * 52 + N * 16
        out[name] = {"ms_per_step": ms, "kernel_ms": kms, "evals_per_s": P * N / (ms / 1e3),
                     "roofline": {"bound": "hbm", "achieved": abytes / (kms / 1e3) / 1e9, "peak": peak,
                                  "unit": "GB/s", "frac": abytes / (kms / 1e3) / 1e9 / peak,
                                  "peak_source": peak_src, "bytes_per_eval": per_eval}}
    line = {"mode": "variants", "metric": "particle×point evals/s (1M×65,536, int16 TSDF, trilinear read)",
            "value": out["trilinear_logprod"]["evals_per_s"], "unit": UNIT, "higher_is_better": True,
            "n_gpus": 1, "data": "synthetic", "dtype": "f32", "steps": steps,
            "config": {"workload": config_dict(args, wl)["workload"],
                       "bytes_per_eval": "corner values x element bytes + one brick-index entry "
                                         "(4 B cell grid, 8 B hash)",
                       "scan": f"staged in 4 x 8 patches (scan_rings {args.scan_rings})"
                               if args.scan_rings else "points as given",
                       "score_map_build_s": score_build_s},
            "results": out}
    print(json.dumps(line), flush=True)
    sc.close()
    m.close()
    return 0


# ------------------------------------------------------------------ batched sessions on one map
def run_batch(args):
    """The headline update (int16 bricks, 1M uniform particles x 65,536
    points) as one sensor update and as a graph-captured batch of `--sessions`
    sessions of P / S particles on the same map (one persistent sensor launch,
    the sessions' work items interleaved sweep by sweep), each given the
    scan's ring count like the headline: milliseconds per update, evaluations
    per second and the kernels of a batched run."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_04172_gb300 import mcl
    torch.cuda.set_device(0)
    wl = make_workload(args, 0)
    m = mcl.map_from_scene(wl.map)
    parts = torch.from_numpy(wl.particles).cuda()
    scan = torch.from_numpy(np.ascontiguousarray(wl.scan)).cuda()
    P, N = parts.shape[0], scan.shape[0]
    S = max(1, args.sessions)
    per = P // S
    prm = mcl.sensor_params(wl.sigma_hit, scan_rings=args.scan_rings)
    logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    sessions = [{"map": m, "particles": parts[k * per:(k + 1) * per].contiguous(), "scan": scan,
                 "sigma_hit": wl.sigma_hit, "scan_rings": args.scan_rings,
                 "logw": torch.empty(per, device="cuda"), "w": torch.empty(per, device="cuda")}
                for k in range(S)]
    batch = mcl.Batch(sessions, use_graph=True)
    reps = max(1, args.steps)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(reps):
            fn()
        e.record()
        e.synchronize()
        return a.elapsed_time(e) / reps

    ms_single = timed(lambda: mcl.mcl_sensor_update(m, parts, scan, prm, logw, w))
    ms_batch = timed(batch.run)
    info = batch.info()
    batch.close()
    m.close()
    ev_batch = float(S * per) * N
    line = {"mode": "batch", "metric": "particle×point evals/s (1M×65,536, int16 TSDF, batched sessions)",
            "value": ev_batch / (ms_batch / 1e3), "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic", "dtype": "f32", "steps": reps,
            "config": {"workload": config_dict(args, wl)["workload"], "sessions": S,
                       "particles_per_session": per,
                       "scan": f"staged in 4 x 8 patches (scan_rings {args.scan_rings})"
                               if args.scan_rings else "points as given"},
            "results": {"single": {"particles": P, "ms_per_update": ms_single,
                                   "evals_per_s": float(P) * N / (ms_single / 1e3)},
                        "batched_graph": {"sessions": S, "ms_per_update": ms_batch,
                                          "evals_per_s": ev_batch / (ms_batch / 1e3),
                                          "groups": info["n_groups"], "items": info["n_items"],
                                          "kernels_per_run": info["kernels_per_run"]}}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "serving":
        return run_serving(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.mode == "vlp16":
        return run_vlp16(args)
    if args.mode == "filter":
        return run_filter(args)
    if args.mode in ("variants", "trilinear"):
        return run_variants(args)
    if args.mode == "batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
