"""Benchmark of the MARS path tracer on one GB300 (or N replicas).

Workload: the guided-room scene at 512 x 512 (64 seeded spheres, 70 % GGX,
four small ceiling lights), max depth 10, techniques BSDF + NEE + guided,
32^3 statistics grid.  A step is one fixed-point iteration: one sample per
pixel rendered with the MARS counts, the image statistics, and the count /
guide update.  The first W steps are the warm-up iterations (beta = 1).

Printed (one JSON line, rank 0):
  value      path vertices per second (closest-hit queries) over the K timed
             steps, device time from CUDA events on the rendering stream
  e2e        the same metric through the C ABI with the image returned to pinned
             host memory every step (host copies inside the timed region), on
             the same iterations: the cache is put back to its state before the
             timed steps (exact checkpoint / resume) and they are replayed
  roofline   the dominant kernel's algorithmic bytes per launch / its average
             launch time, against the measured HBM copy bandwidth
  efficiency equal-time efficiency 1 / (relMSE x seconds) of MARS (counts frozen
             after the timed steps) and of fixed-count MIS (beta = 1) on the
             same GPU, against a long fixed-count reference render
  cpu_baseline  the CPU oracle on a bounded pixel sample of the same workload

--impl reference runs the CPU oracle instead (the only reference arm: the paper
ships no GPU code) on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mars_workloads as W  # noqa: E402

METRIC = "efficiency 1/(relMSE·s) MARS vs fixed-count MIS; Mvertices/s; p50/p99 latency"
UNIT = "Mvertices/s"

# algorithmic bytes of the arena records (see the layout in csrc/internal.h)
RAY_BYTES = 80          # R0..R4: five float4 per ray
RAY_TRACE_BYTES = 32    # R0, R1: origin and direction
HIT_BYTES = 8           # H: (t, primitive), then (first child, first shadow ray)
V0_BYTES = 16           # V0 for every slot
VERT_EST_BYTES = 48     # V1..V3 for a vertex that runs the estimator
VERT_GUIDE_BYTES = 16   # V4 for a traced ray when the guided technique learns
SAMPLE_BYTES = 16       # S: one float4 per slot
EST_READ_BYTES = 16     # pixel estimate read per estimator vertex
SHADOW_VALUE_BYTES = 16  # SH2 per NEE sample
SHADOW_RAY_BYTES = 36   # SH0, SH1 and the work-list entry per traced shadow ray
SLOT_BYTES = RAY_BYTES + HIT_BYTES + V0_BYTES + VERT_EST_BYTES + VERT_GUIDE_BYTES + SAMPLE_BYTES


# Algorithmic bytes: the minimum traffic per unit of the path, whatever the
# record layout -- a ray 64 B (origin, direction, throughput, pixel/lineage),
# a hit 16 B, a vertex record 32 B, a shadow ray 32 B plus a 16 B result, a
# sample value 16 B; count reads and statistics atomics stay in L2.
ALG_RAY, ALG_RAY_TRACE, ALG_HIT, ALG_VERTEX, ALG_SHADOW, ALG_RESULT, ALG_VALUE = 64, 32, 16, 32, 32, 16, 16


def algorithmic_bytes(entries, pixels, shadow_traced):
    """Minimum HBM bytes each wave kernel must move for one step at the
    per-unit minima above (each record written once by its producer and read
    once by its consumer; camera rays are generated in registers, and an NEE
    sample of value zero needs no shadow ray and no result): trace reads a
    child ray's origin and direction and writes its hit; shade reads the ray
    and the hit, writes the vertex record, every child ray and every shadow
    ray; shadow reads the shadow rays and writes their results; reverse reads
    the vertex record, every child's value and every NEE result, and writes the
    slot's value."""
    children = entries - pixels
    return {
        "k_trace": ALG_RAY_TRACE * children + ALG_HIT * entries,
        "k_shade": (ALG_RAY * children + (ALG_HIT + ALG_VERTEX) * entries + ALG_RAY * children
                    + ALG_SHADOW * shadow_traced),
        "k_shadow": (ALG_SHADOW + ALG_RESULT) * shadow_traced,
        "k_reverse": (ALG_VERTEX + ALG_VALUE) * entries + ALG_VALUE * children + ALG_RESULT * shadow_traced,
    }


def kernel_bytes(entries, pixels, est_v, traced, shadows, shadow_traced, guided):
    """HBM bytes each wave kernel moves for one step with this design's arena
    records (csrc/internal.h: 80 B rays, 48 B estimator records, ...), inputs
    read once and outputs written once: the layout bytes, reported beside the
    algorithmic bytes."""
    children = entries - pixels
    guide = VERT_GUIDE_BYTES * (traced - pixels) if guided else 0
    return {
        "k_trace": RAY_TRACE_BYTES * children + HIT_BYTES * entries,
        "k_shade": (RAY_BYTES * children + HIT_BYTES * entries + V0_BYTES * entries
                    + (VERT_EST_BYTES + EST_READ_BYTES + HIT_BYTES) * est_v + RAY_BYTES * children
                    + SHADOW_VALUE_BYTES * shadows + SHADOW_RAY_BYTES * shadow_traced + guide),
        "k_shadow": SHADOW_RAY_BYTES * shadow_traced,
        "k_reverse": (V0_BYTES * entries + SAMPLE_BYTES * entries + (VERT_EST_BYTES + HIT_BYTES) * est_v
                      + SAMPLE_BYTES * children + SHADOW_VALUE_BYTES * shadows + guide),
    }


def workload(args):
    cfg = W.config_guided(args.width, args.height, seed=0)
    return cfg


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def sm_max_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    return 2070.0


# Algorithmic float32 operations of one traversal step, counted from the
# arithmetic of the intersection routines (every add, multiply, min, max,
# divide and square root is one operation; a fused multiply-add counts two):
# a BVH node visit tests two slab boxes (25 each); a quad test 67, a sphere
# test 25, a triangle test 45.
OPS_NODE, OPS_QUAD, OPS_SPHERE, OPS_TRI = 50, 67, 25, 45


KERNEL_SOURCES = ["paper_2410_20429_gb300/csrc/render.cu", "paper_2410_20429_gb300/csrc/device.cuh",
                  "paper_2410_20429_gb300/csrc/internal.h", "paper_2410_20429_gb300/build.py"]
TRAFFIC_FILE = "profiles/dram_traffic_wave_kernels_guided_room_256.txt"
SERVE_MULTIPLICITY = 16.0   # the server's path multiplicity cap for served jobs (csrc/server.cu)


BVH_KINDS = {"sah": 0, "lbvh": 1}   # MARS_BVH_SAH, MARS_BVH_LBVH
PATH_BYTES_PER_VERTEX = 330          # minimum DRAM traffic of one path vertex (ray, hit, vertex, shadow ray, ...)


def kernel_sources_sha():
    """sha256 of the wave kernels' sources: DRAM traffic measured on other
    sources does not describe these kernels."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes per unit of work (ray slot; traced shadow ray for k_shadow) of
    each wave kernel from the committed ncu summary, if it was taken on the
    current kernel sources and build flags; else {}."""
    p = os.path.join(ROOT, TRAFFIC_FILE)
    if not os.path.exists(p):
        return {}
    vals, sha = {}, None
    for line in open(p):
        parts = line.split()
        if line.startswith("#") or len(parts) < 2:
            continue
        if parts[0] == "sources_sha256":
            sha = parts[1]
        elif parts[0].startswith("k_"):
            vals[parts[0]] = float(parts[1])
    return vals if sha == kernel_sources_sha() else {}


def trace_ops(work):
    n, q, sp, t = work
    return OPS_NODE * n + OPS_QUAD * q + OPS_SPHERE * sp + OPS_TRI * t


def alu_peak_tflops(num_sms):
    """Float32 peak: SMs x 128 FP32 lanes x 2 operations (FMA) x max SM clock."""
    return num_sms * 128 * 2 * sm_max_mhz() * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle samples (every 20 ms, each with its
    timestamp); only samples taken between begin() and stop() -- the GPU under
    load -- enter the summary."""

    def __init__(self, gpu_index: int, out_path: str, interval_ms: int = 20):
        self.proc = None
        self.path = out_path
        self.t0 = None
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(out_path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", str(int(interval_ms))],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def begin(self) -> None:
        self.t0 = time.time()

    def stop(self, window: str = "") -> dict:
        import datetime
        t1 = time.time()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, total = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            total += 1
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, cmax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            if self.t0 is not None and not (self.t0 - 0.02 <= ts <= t1 + 0.02):
                continue
            sm.append(clk)
            smax.append(cmax)
            for k, nm in enumerate(names):
                if parts[6 + k].lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples under load"], "samples_total": total}
        return {"sm_mhz": float(np.median(sm)), "sm_min_mhz": float(min(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def rel_mse(img, ref, ref_var=None, eps=1e-2):
    """relMSE: mean over pixels and channels of (I - R)^2 / (R^2 + eps), eps =
    1e-2 by default, after dropping the 0.01 % largest per-pixel terms.  With
    ``ref_var`` (the variance of the reference's mean, per pixel and channel)
    each squared difference is reduced by it: E[(I - R)^2] = Var(I) + bias^2 +
    Var(R), so the estimate no longer charges the reference's own noise to the
    image."""
    d2 = (img - ref) ** 2
    if ref_var is not None:
        d2 = d2 - ref_var
    t = (d2 / (ref ** 2 + eps)).reshape(-1, 3).mean(axis=1)
    k = int(math.ceil(1e-4 * t.size))
    if k > 0:
        t = np.sort(t)[:-k]
    return float(t.mean())


def restore_state(cache, snap, iteration, stream):
    """Put a cache back to a checkpoint taken with get_state (exact resume)
    and return the iteration index to continue from."""
    extra = {k: snap[k] for k in ("oct_nodes", "oct_leaf_level") if snap.get(k) is not None}
    cache.set_state(q_rr=snap["q_rr"], q_s=snap["q_s"], valid=snap["valid"], stats=snap["stats"],
                    guide_hist=snap["guide_hist"], guide_cdf=snap["guide_cdf"], pixel_estimate=snap["pixel_estimate"],
                    run_sum=snap["run_sum"], n_iterations=snap["n_iterations"], has_estimate=snap["has_estimate"],
                    VI=snap["VI"], CI=snap["CI"], image_iterations=snap["image_iterations"], stream=stream, **extra)
    return iteration


def reduce_over_ranks(total_ms, units, world, device):
    """Whole-job aggregation across ranks: the slowest rank's time (MAX) and the
    units all ranks processed (SUM).  One rank: the inputs unchanged."""
    if world <= 1:
        return float(total_ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    v = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(v)
    return float(t.item()), float(v.item())


def run_mars(args):
    import torch
    import paper_2410_20429_gb300 as M
    from paper_2410_20429_gb300 import build as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    B.build()
    cfg = workload(args)
    sc = cfg.scene
    sc.bvh = BVH_KINDS[args.bvh]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        scene = M.Scene(sc, stream=stream)
        cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, arena_capacity=args.arena_capacity,
                        graphs=not args.no_graphs, lanes=args.lanes, stream=stream)
    if args.launch:
        parts = args.launch.split(":")
        regs = [int(x) for x in parts[2].split(",")] if len(parts) > 2 else [0, 0, 0, 0]
        cache.set_launch([int(x) for x in parts[0].split(",")], [int(x) for x in parts[1].split(",")], regs)
    npx = sc.n_pixels
    img = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    seed = 1000 + rank  # weak-scaling replicas: every rank renders its own job
    it = 0

    def step(i, mode, profile=False, image=img, collect=True):
        st = cache.render_iteration(image, seed=seed, iteration=i, mode=mode, collect=collect,
                                    update_estimate=True, profile=profile, stream=stream)
        cache.update_counts(stream=stream)
        return st

    curve = []
    for _ in range(args.warmup):
        curve.append(step(it, M.MARS_MODE_WARMUP))
        it += 1
    # launch shape of the wave kernels picked by the library's autotuner on a
    # MARS iteration with the counts learned so far (no state change)
    launch = cache.autotune(iteration=it, seed=seed, mode=M.MARS_MODE_MARS, repeats=2, stream=stream) \
        if not (args.no_autotune or args.launch) else cache.get_launch()
    torch.cuda.synchronize()
    clocks = ClockSampler(local, args.clocks_csv.replace("{rank}", str(rank)) if args.clocks_csv
                          else os.path.join(tempfile.gettempdir(), f"mars_clocks_{rank}.csv"))
    time.sleep(0.3)  # nvidia-smi starts sampling
    # the state after warm-up (the library's exact checkpoint): the profiled,
    # control and end-to-end loops below replay the timed iterations from it,
    # so every figure of the line is taken on the same iterations (MARS
    # converges over its iterations and later ones spawn fewer vertices)
    snap, it_snap = cache.get_state(stream=stream), it
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    captures0 = cache.info()["graph_captures"]
    timed = []
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    evs[0].record(stream)
    for k in range(args.steps):
        timed.append(step(it, M.MARS_MODE_MARS))
        it += 1
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = sum(per_step)
    verts = sum(s["vertices"] for s in timed)
    t_max, verts_all = reduce_over_ranks(total_ms, verts, world, "cuda")
    value = verts_all / (t_max * 1e-3) / 1e6
    captures = cache.info()["graph_captures"] - captures0

    # ---- as many MARS steps again with every launch between CUDA events
    # (direct launches, no graph replay): the per-kernel device times
    sts = []
    it = restore_state(cache, snap, it_snap, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        sts.append(step(it, M.MARS_MODE_MARS, profile=True))
        it += 1
    e1.record(stream)
    torch.cuda.synchronize()
    profiled_ms = e0.elapsed_time(e1) / args.steps
    verts_prof = sum(s["vertices"] for s in sts)

    # ---- dominant kernel roofline (live CUDA-event times of every launch)
    guided = bool(cfg.techniques & W.TECH_GUIDED)
    lb = kernel_bytes(sum(s["wave_entries"] for s in sts), npx * args.steps,
                      sum(s["estimator_vertices"] for s in sts), verts_prof, sum(s["shadow_entries"] for s in sts),
                      sum(s["shadow_traced"] for s in sts), guided)
    kb = algorithmic_bytes(sum(s["wave_entries"] for s in sts), npx * args.steps,
                           sum(s["shadow_traced"] for s in sts))
    kms = {k: sum(s[k[2:] + "_ms"] for s in sts) for k in kb}
    nlaunch = {k: sum(s["wave_launches"] for s in sts) for k in kb}
    nlaunch["k_shadow"] = sum(max(s["wave_launches"] - s["tiles"], 0) for s in sts)  # no shadow launch at d = D
    hbm, peak_kind = peaks()
    alu = alu_peak_tflops(torch.cuda.get_device_properties(local).multi_processor_count)
    # the traversal kernels are bound by float32 arithmetic and instruction issue,
    # the queue kernels by memory: each gets its own roofline
    ops = {"k_trace": sum(trace_ops(s["trace_work"][0]) for s in sts),
           "k_shadow": sum(trace_ops(s["trace_work"][1]) for s in sts)}
    per_kernel = {}
    for k in kb:
        ms_launch = kms[k] / max(nlaunch[k], 1)
        if k in ops:
            a = ops[k] / max(nlaunch[k], 1) / (ms_launch * 1e-3) / 1e12
            per_kernel[k] = {"bound": "alu", "achieved": round(a, 3), "peak": round(alu, 1), "unit": "TFLOP/s",
                             "frac": round(a / alu, 4), "per_launch": int(ops[k] / max(nlaunch[k], 1)),
                             "launch_ms": round(ms_launch, 4)}
        else:
            a = kb[k] / max(nlaunch[k], 1) / (ms_launch * 1e-3) / 1e9
            al = lb[k] / max(nlaunch[k], 1) / (ms_launch * 1e-3) / 1e9
            per_kernel[k] = {"bound": "hbm", "achieved": round(a, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(a / hbm, 4), "per_launch": int(kb[k] / max(nlaunch[k], 1)),
                             "launch_ms": round(ms_launch, 4),
                             "layout_bytes": {"per_launch": int(lb[k] / max(nlaunch[k], 1)),
                                              "achieved": round(al, 1), "frac": round(al / hbm, 4)}}
    tw = [[sum(s["trace_work"][k][q] for s in sts) for q in range(4)] for k in range(2)]
    n_closest = max(sum(s["wave_entries"] for s in sts), 1)
    n_shadow = max(sum(s["shadow_traced"] for s in sts), 1)
    per_kernel["k_trace"]["per_ray"] = {"nodes": round(tw[0][0] / n_closest, 2),
                                        "prim_tests": round(sum(tw[0][1:]) / n_closest, 2)}
    per_kernel["k_shadow"]["per_ray"] = {"nodes": round(tw[1][0] / n_shadow, 2),
                                         "prim_tests": round(sum(tw[1][1:]) / n_shadow, 2)}
    # dominant kernel: the longest of the kernels on the rendering stream (the
    # shadow kernel overlaps the next waves on the side stream, so its event
    # time is not time the iteration waits for)
    dom = max(("k_trace", "k_shade", "k_reverse"), key=kms.get)
    d0 = per_kernel[dom]
    # DRAM bytes per launch: the measured bytes per unit x this run's units per launch
    units = {"k_trace": sum(s["wave_entries"] for s in sts), "k_shade": sum(s["wave_entries"] for s in sts),
             "k_reverse": sum(s["wave_entries"] for s in sts), "k_shadow": sum(s["shadow_traced"] for s in sts)}
    per_unit = measured_traffic().get(dom)
    traffic = per_unit * units[dom] / max(nlaunch[dom], 1) if per_unit is not None else None
    roofline = {"kernel": dom, "bound": d0["bound"], "achieved": d0["achieved"], "peak": d0["peak"],
                "unit": d0["unit"], "frac": d0["frac"],
                "traffic": int(traffic) if traffic is not None else None,
                "traffic_note": "DRAM read + write bytes per launch: bytes per unit from one ncu pass over every "
                                "launch of one 256^2 iteration (cold L2), " + TRAFFIC_FILE + ", x this run's units "
                                "per launch",
                "overlapped": ["k_shadow"],
                "peak_kind": peak_kind if d0["bound"] == "hbm" else
                "derived: SMs x 128 FP32 lanes x 2 x max SM clock (measured)",
                "per_launch": d0["per_launch"], "launch_ms": d0["launch_ms"],
                "bytes_model": "algorithmic: per-unit minima (ray 64 B, hit 16, vertex record 32, shadow ray 32 "
                               "+ 16 result, sample value 16) x units; layout_bytes: this design's records",
                "layout_bytes": d0.get("layout_bytes"),
                "kernels": per_kernel,
                "kernel_ms_per_step": {k: round(v / args.steps, 4) for k, v in kms.items()}}
    roofline["kernel_ms_per_step"]["image"] = round(sum(s["image_ms"] for s in sts) / args.steps, 4)
    roofline["wave_rays_per_step"] = [int(sum(s["wave_rays"][d] for s in sts) / args.steps)
                                      for d in range(cfg.max_depth)]
    roofline["units_per_step"] = {"ray_slots": units["k_shade"] / args.steps,
                                  "shadow_traced": units["k_shadow"] / args.steps}
    roofline["wave_ms_per_step"] = {k: [round(sum(s["wave_ms"][ki][d] for s in sts) / args.steps, 4)
                                        for d in range(cfg.max_depth)]
                                    for ki, k in enumerate(["k_trace", "k_shade", "k_shadow", "k_reverse"])}
    entries = sum(s["wave_entries"] for s in sts)

    # ---- the same loop timed on the host clock with the image in device
    # memory (the control for the end-to-end figure below)
    it = restore_state(cache, snap, it_snap, stream)
    torch.cuda.synchronize()
    cap_ctl = cache.info()["graph_captures"]
    t0 = time.perf_counter()
    ctl_verts = 0
    for k in range(args.steps):
        ctl_verts += step(it, M.MARS_MODE_MARS)["vertices"]
        it += 1
    torch.cuda.synchronize()
    ctl_s = time.perf_counter() - t0
    cap_ctl = cache.info()["graph_captures"] - cap_ctl

    # ---- end to end through the C ABI with a pinned host image every step
    host_img = torch.empty(npx * 3, dtype=torch.float32, pin_memory=True).numpy()
    it = restore_state(cache, snap, it_snap, stream)
    torch.cuda.synchronize()
    cap_e2e = cache.info()["graph_captures"]
    t0 = time.perf_counter()
    e2e_verts = 0
    for k in range(args.steps):
        st = cache.render_iteration(host_img, seed=seed, iteration=it, mode=M.MARS_MODE_MARS, update_estimate=True,
                                    stream=stream)
        cache.update_counts(stream=stream)
        e2e_verts += st["vertices"]
        it += 1
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # clock samples under load: the timed steps and their three replays (the
    # same iterations), so that a short timed region still has several
    clk = clocks.stop("the timed steps and their three replays")
    e2e = {"value": round(e2e_verts / e2e_s / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": 48,
           "d2h_bytes_per_step": npx * 3 * 4 + 512,
           "host_clock_device_image": round(ctl_verts / ctl_s / 1e6, 3),
           "iterations": "the timed ones, replayed from the checkpoint taken before them",
           "graph_captures": {"device_image_loop": cap_ctl,
                              "host_image_loop": cache.info()["graph_captures"] - cap_e2e}}

    launches = sum(s["launches"] for s in timed) + args.steps * (2 if guided else 1)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "pixels": npx, "max_depth": cfg.max_depth, "grid": cfg.grid_n,
                   "techniques": "bsdf+nee+guided", "statistics_dtype": "f64", "bvh": args.bvh, "lanes": launch.get("lanes", args.lanes),
                   "l2": "working set > L2: queue arena %.0f MB per step" % (
                       entries / args.steps * SLOT_BYTES / 1e6),
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": round(float(np.percentile(per_step, 50)), 4),
                       "p99": round(float(np.percentile(per_step, 99)), 4)},
        "per_step": {"vertices": verts / args.steps, "rays": sum(s["rays"] for s in timed) / args.steps,
                     "mean_beta": [round(sum(s["mean_beta"][t] for s in timed) / args.steps, 4) for t in range(3)],
                     "tiles": sum(s["tiles"] for s in timed) / args.steps},
        # the timed steps replay a recorded CUDA graph per iteration shape; the
        # profiled steps (kernel times) launch every kernel directly
        "graphs": {"enabled": not args.no_graphs, "captures_in_timed_steps": captures,
                   "profiled_ms_per_step": round(profiled_ms, 4),
                   "profiled_mvertices_s": round(verts_prof / (profiled_ms * args.steps * 1e-3) / 1e6, 3)},
        "roofline": roofline, "e2e": e2e,
        # the whole path against HBM: at the minimum traffic of ~330 B per path
        # vertex (ray, hit, vertex record, shadow ray, count reads, statistics)
        # the copy bandwidth allows hbm / 330 B vertices per second
        "path_roofline": {"bytes_per_vertex": PATH_BYTES_PER_VERTEX,
                          "ceiling_mvertices_s": round(peaks()[0] * 1e9 / PATH_BYTES_PER_VERTEX / 1e6, 1),
                          "frac": round(value / (peaks()[0] * 1e9 / PATH_BYTES_PER_VERTEX / 1e6), 4)},
        "gpu_launches": int(launches), "clocks": clk,
        # Fig. convergence (E8): average allocation per technique and the image
        # efficiency estimate 1 / (V_I C_I) over the fixed-point iterations
        "convergence": {"mean_beta": [[round(b, 4) for b in s["mean_beta"]] for s in curve + timed + sts],
                        "efficiency_estimate": [round(1.0 / max(s["VI"] * s["CI"], 1e-30), 4)
                                                for s in curve + timed + sts]},
        "launch": {"kernels": ["trace", "shade", "shadow", "reverse"], **launch,
                   "autotuned": not (args.no_autotune or args.launch)},
    }

    if rank == 0 and not args.no_large:
        line["large_scene"] = large_scene(args, M, stream)
        line["largest_scene"] = largest_scene(args, M, stream)
    if rank == 0 and args.serve_requests > 0:
        line["serving"] = serving(args)
        if not args.no_efficiency:
            line["serving"]["efficiency"] = serving_efficiency(args, M, stream)
    if rank == 0 and not args.no_precision:
        line["precision"] = precision_study(cfg, cache, seed, it, stream)
    if rank == 0 and not args.no_efficiency:
        # the comparison's MARS arm learns as a job does: as many renders as the
        # bench cache saw, with the count update closing each training iteration
        eff_cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, arena_capacity=args.arena_capacity,
                            lanes=args.lanes, stream=stream)
        learn(M, eff_cache, img, seed, it, args.warmup, stream)
        line["efficiency"] = efficiency(args, M, cfg, scene, eff_cache, seed, it, stream)
        del eff_cache
        line["efficiency_box"] = box_efficiency(args, M, stream)
        # the same after 16 learning iterations: the counts of 3 one-sample MARS
        # iterations on a 64 x 64 image are still noisy
        line["efficiency_box_16"] = box_efficiency(args, M, stream, iterations=16)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, args.cpu_seconds, learn_iterations=args.warmup, warmup=args.warmup,
                                            iteration=it_snap)
    if world > 1:
        dist.barrier()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def bidirectional_scene(args, M, stream, cfg, seed, precision_study_too, unaware=False):
    """A bidirectional workload (Sec. 5: BSDF sampling, NEE and connections to
    light subpaths, each with its own budget; whole-path budget-aware balance
    weights) with the adaptive octree cache (starting as the 32^3 grid, at most
    64k leaves) and the application's image-level rules (Sec. 5.1: V_I without
    the 10 brightest pixels, iterations combined with weights 1 / V_I):
    hierarchy build time, the workload's warm-up iterations, then its MARS
    iterations timed (the whole job: `cfg.iterations` renders in all, the count
    update closing each training iteration of the library's schedule), then 3
    more renders with every launch timed, the equal-time efficiency against fixed-count MIS on the
    same GPU, and optionally the float32 versus float64 statistics comparison
    at this size."""
    import torch
    cfg.scene.bvh = BVH_KINDS[args.bvh]
    t0 = time.perf_counter()
    scene = M.Scene(cfg.scene, stream=stream)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    npx = cfg.scene.n_pixels
    cap = 2 * npx * cfg.max_depth
    kw = dict(octree=True, max_leaves=65536, split_samples=4096.0, arena_capacity=cap)
    cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream, **kw)
    img = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    it = 0
    for k in range(cfg.warmup):
        cache.render_iteration(img, seed=seed, iteration=it, mode=M.MARS_MODE_WARMUP, update_estimate=True,
                               vi_drop_brightest=10, stream=stream)
        cache.update_counts(stream=stream)
        it += 1
    launch = cache.autotune(iteration=it, seed=seed, mode=M.MARS_MODE_MARS, repeats=1, stream=stream)
    timed_iters = cfg.iterations - cfg.warmup
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sts = []
    torch.cuda.synchronize()
    e0.record(stream)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(timed_iters + 1)]
    evs[0] = e0
    for k in range(timed_iters):
        sts.append(cache.render_iteration(img, seed=seed, iteration=it, mode=M.MARS_MODE_MARS, update_estimate=True,
                                          vi_drop_brightest=10, combine=2 if k == 0 else 1, stream=stream))
        if M.training_step_ends(it, cfg.warmup, cfg.iterations):
            cache.update_counts(stream=stream)
        it += 1
        if k + 1 < timed_iters:
            evs[k + 1].record(stream)
    e1.record(stream)
    evs[timed_iters] = e1
    torch.cuda.synchronize()
    sts_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(timed_iters)]
    ms = e0.elapsed_time(e1) / timed_iters
    verts = sum(s["vertices"] for s in sts) / timed_iters
    timed = sts
    # kernel times: 3 renders more with the job's final counts (no update), every
    # launch between events
    sts = []
    for k in range(3):
        sts.append(cache.render_iteration(img, seed=seed, iteration=it, mode=M.MARS_MODE_MARS, update_estimate=True,
                                          profile=True, vi_drop_brightest=10, combine=1, stream=stream))
        it += 1
    tw = [sum(s["trace_work"][0][q] for s in sts) for q in range(4)]
    n = max(sum(s["wave_entries"] for s in sts), 1)
    k_n = len(sts)
    out = {"workload": cfg.name, "primitives": int(len(cfg.scene.tris) + len(cfg.scene.spheres) + len(cfg.scene.quads)),
           "techniques": "bsdf+nee+light_connection", "bvh_build_s": round(build_s, 3), "ms_per_step": round(ms, 3),
           "mvertices_s": round(verts / (ms * 1e-3) / 1e6, 1), "vertices_per_step": int(verts),
           "timed_iterations": timed_iters, "warmup_iterations": cfg.warmup,
           "training_schedule": M.training_schedule(cfg.iterations, cfg.warmup),
           "ms_per_step_first_last": [round(sts_ms[0], 3), round(sts_ms[-1], 3)],
           "vertices_note": "closest-hit queries of camera paths and light subpaths",
           "light_subpath_rays_per_step": int(sum(s["light_rays"] for s in timed) / timed_iters),
           "connection_rays_per_step": int(sum(s["connection_rays"] for s in timed) / timed_iters),
           "light_samples_per_step": int(sum(s["light_samples"] for s in timed) / timed_iters),
           "kernel_ms_per_step": {k: round(sum(s[k + "_ms"] for s in sts) / k_n, 4)
                                  for k in ("trace", "shade", "shadow", "light", "reverse", "image")},
           "closest_hit_per_ray": {"nodes": round(tw[0] / n, 2), "prim_tests": round(sum(tw[1:]) / n, 2)},
           "mean_beta": {"bsdf": round(sum(s["mean_beta"][0] for s in sts) / k_n, 4),
                         "nee": round(sum(s["mean_beta"][1] for s in sts) / k_n, 4),
                         "light_connection": round(sum(s["mean_beta"][2] for s in sts) / k_n, 4)},
           "octree_leaves": int(cache.info()["oct_n_leaves"]), "launch": launch,
           "tiles": [s["tiles"] for s in timed], "arena_slots": cap,
           "device_gb": round(cache.info()["device_bytes"] / 1e9, 2),
           "progressive": {"vi_drop_brightest": 10, "combined_iterations": timed_iters + 3,
                           "combined_weight": round(cache.combined_image(stream=stream)[1], 4),
                           "VI": [round(s["VI"], 5) for s in timed + sts]}}
    if not args.no_efficiency:
        out["efficiency"] = efficiency(args, M, cfg, scene, cache, seed, cfg.iterations, stream,
                                       ref_spp=args.large_ref_spp,
                                       cache_kw=kw, unaware=unaware, vi_drop=10)
    if precision_study_too and not args.no_precision:
        # float32 versus float64 statistics at this size (the large bidirectional
        # workload's precision comparison), on the learned state and tree
        from paper_2410_20429_gb300 import precision
        g = cache.get_state(stream=stream)
        del cache
        torch.cuda.synchronize()
        rep = precision.compare(cfg.scene, cfg.grid_n, cfg.techniques, cfg.max_depth, g["q_rr"], g["q_s"],
                                g["valid"], g["pixel_estimate"], g["run_sum"], g["n_iterations"], iteration=it,
                                seed=seed, stream=stream, cache_kw=kw,
                                tree=(g["oct_nodes"], g["oct_leaf_level"]), guide_cdf=g.get("guide_cdf"))
        out["precision"] = {k: [float("%.3g" % rep[k]["max"]), float("%.3g" % rep[k]["median"])]
                            for k in precision.STATISTICS}
        out["precision"]["entries"] = rep["cells_compared"]
        out["precision"]["images_equal"] = rep["images_equal"]
    else:
        del cache
    del scene
    return out


def large_scene(args, M, stream):
    """The bidirectional workload: heightfield of 256 x 256 quads (131k
    triangles) + 200 spheres with one small emitter hidden between two
    spheres, 1024 x 1024, D = 10, light subpaths of at most 6 vertices, 32
    iterations."""
    n = args.large_size or 1024
    return bidirectional_scene(args, M, stream, W.config_bdpt_heightfield(n, n), 77, False, unaware=True)


def largest_scene(args, M, stream):
    """The large bidirectional workload: 512 x 512 quads = 524k triangles, 4096
    GGX spheres, 8 area lights, 2048 x 2048, D = 12, 64 iterations, with the
    float32 versus float64 statistics comparison at this size."""
    n = args.large_size or 2048
    return bidirectional_scene(args, M, stream, W.config_bdpt_large(n, n), 91, True, unaware=True)


def serving(args):
    """Serving stream: seeded render requests arriving Poisson at --serve-rate per
    second (square resolutions 64..512, 16..4096 spheres in a room, 4..16
    fixed-point iterations each) submitted to a continuous-batching server with a
    40 GB device-memory budget; per-iteration latency p50 / p99 over all
    iterations of all jobs, job latency (arrival to completion) and aggregate
    vertex throughput over the stream."""
    import paper_2410_20429_gb300 as M
    reqs = W.serving_requests(args.serve_requests, rate=args.serve_rate, seed=11)
    srv = M.Server(40 << 30, args.serve_slots)
    t0 = time.perf_counter()
    ids = []
    for r in reqs:
        wait = r["arrival_s"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids.append(srv.submit(r["scene"], grid_n=r["grid_n"], techniques=r["techniques"],
                              max_depth=r["max_depth"], iterations=r["iterations"], warmup=r["warmup"],
                              seed=r["seed"], key=r["key"], graphs=not args.serve_no_graphs))
    done = {}
    while len(done) < len(ids):
        for j in ids:
            if j not in done:
                st, _ = srv.poll(j)
                if st["state"] in (M.MARS_JOB_DONE, M.MARS_JOB_FAILED):
                    done[j] = st
        time.sleep(0.005)
    lats = [srv.latencies(j) for j in ids]
    lat = np.concatenate(lats)
    slow = sorted(((float(l.max()), int(l.argmax()), r["scene"].width, len(r["scene"].spheres), r["iterations"])
                   for l, r in zip(lats, reqs) if l.size), reverse=True)[:5]
    sts = [done[j] for j in ids]
    job_s = np.array([s["end_s"] - s["submit_s"] for s in sts])
    span = max(s["end_s"] for s in sts) - min(s["submit_s"] for s in sts)
    verts = sum(s["vertices"] for s in sts)
    starts = sorted((s["start_s"], 1) for s in sts) + sorted((s["end_s"], -1) for s in sts)
    cur = peak = 0
    for _, dlt in sorted(starts):
        cur += dlt
        peak = max(peak, cur)
    srv.close()
    return {"requests": len(ids), "rate_per_s": args.serve_rate, "slots": args.serve_slots,
            "graphs": not args.serve_no_graphs,
            "budget_gb": 40, "failed": sum(s["state"] != M.MARS_JOB_DONE for s in sts),
            "iterations": int(lat.size), "iter_ms_p50": round(float(np.percentile(lat, 50)), 3),
            "iter_ms_p99": round(float(np.percentile(lat, 99)), 3),
            "job_s_p50": round(float(np.percentile(job_s, 50)), 3),
            "job_s_p99": round(float(np.percentile(job_s, 99)), 3),
            "throughput_mvertices_s": round(verts / span / 1e6, 2), "span_s": round(span, 2),
            "max_resident": peak,
            "slowest_iterations": [{"ms": round(a, 1), "iteration": b, "resolution": c, "spheres": d2,
                                    "iterations": e} for a, b, c, d2, e in slow],
            "failures": sorted(set(s.get("message", "")[:120] for s in sts if s["state"] != M.MARS_JOB_DONE))[:3]}


def serving_efficiency(args, M, stream):
    """Equal-time efficiency of the served workload (config 4): the first
    request of each resolution of the serving stream, learned over its own
    iterations (its warm-up, then MARS) as the server renders it -- with the
    server's path multiplicity cap -- then the same comparison with fixed-count
    MIS as for the main workload (512-spp reference), MARS rendering with the
    cap too."""
    import torch
    reqs = W.serving_requests(args.serve_requests, rate=args.serve_rate, seed=11)
    picked, seen = [], set()
    for r in reqs:
        if r["scene"].width not in seen:
            seen.add(r["scene"].width)
            picked.append(r)
    out = []
    for r in sorted(picked, key=lambda q: q["scene"].width):
        cfg = W.WorkloadConfig(r["scene"], r["max_depth"], r["grid_n"], r["techniques"], r["iterations"], r["warmup"],
                               r["scene"].name)
        scene = M.Scene(cfg.scene, stream=stream)
        cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream)
        img = torch.zeros(cfg.scene.n_pixels * 3, dtype=torch.float32, device="cuda")
        learn(M, cache, img, r["seed"], cfg.iterations, cfg.warmup, stream, max_mult=SERVE_MULTIPLICITY)
        e = efficiency(args, M, cfg, scene, cache, r["seed"], cfg.iterations, stream, ref_spp=512, unaware=False,
                       max_mult=SERVE_MULTIPLICITY)
        out.append({"scene": cfg.name, "iterations": cfg.iterations, "ratio": round(e["ratio"], 4),
                    "ratio_scaled": round(e["ratio_scaled"], 4),
                    "ratio_vs_own_guide": round(e["ratio_vs_own_guide"], 4),
                    "relmse": [e["mars"]["relmse"], e["fixed_count_mis"]["relmse"]],
                    "seconds": [e["mars"]["seconds"], e["fixed_count_mis"]["seconds"]]})
        del cache, scene
    geo = float(np.exp(np.mean([np.log(max(q["ratio"], 1e-30)) for q in out])))
    return {"requests": out, "ratio_geomean": round(geo, 4),
            "protocol": "the first request of each resolution of the serving stream; efficiency() after its own "
                        "iterations, learned and rendered with the server's path multiplicity cap "
                        f"({SERVE_MULTIPLICITY:g}); fixed-count MIS with the learned guide; 512-spp fixed-count "
                        "reference"}


def precision_study(cfg, cache, seed, it, stream):
    """Float32 versus float64 statistics on the full workload: the next MARS
    iteration rendered from the bench cache's learned state on one cache of
    each precision; relative error of every statistic of the float32 run
    (max and median over the (cell, technique) entries with >= 2 samples)."""
    from paper_2410_20429_gb300 import precision
    g = cache.get_state(stream=stream)
    rep = precision.compare(cfg.scene, cfg.grid_n, cfg.techniques, cfg.max_depth, g["q_rr"], g["q_s"], g["valid"],
                            g["pixel_estimate"], g["run_sum"], g["n_iterations"], iteration=it, seed=seed,
                            stream=stream, guide_cdf=g.get("guide_cdf"))
    out = {k: [float("%.3g" % rep[k]["max"]), float("%.3g" % rep[k]["median"])] for k in precision.STATISTICS}
    out["fields"] = "relative error of float32 vs float64 statistics: [max, median]"
    out["images_equal"] = rep["images_equal"]
    out["entries"] = rep["cells_compared"]
    return out


def learn(M, cache, img, seed, n, warmup, stream, mode=None, weights=None, drop=0, max_mult=0.0):
    """A job of n one-sample renders on `cache` (the first `warmup` of them
    warm-up renders, or all in `mode`), with the count update closing each
    training iteration of the library's schedule (1, 2, 4, ... renders after the
    warm-up ones; Sec. 4.1 "Fixed-point iteration", Sec. 5.1)."""
    weights = M.MARS_WEIGHTS_AWARE if weights is None else weights
    sts = []
    for k in range(n):
        m = mode if mode is not None else (M.MARS_MODE_WARMUP if k < warmup else M.MARS_MODE_MARS)
        sts.append(cache.render_iteration(img, seed=seed, iteration=k, mode=m, weights=weights, update_estimate=True,
                                          vi_drop_brightest=drop, max_multiplicity=max_mult, stream=stream))
        if M.training_step_ends(k, warmup, n):
            cache.update_counts(stream=stream)
    return sts


def efficiency(args, M, cfg, scene, cache, seed, it0, stream, ref_spp=None, cache_kw=None, unaware=True, vi_drop=0,
               max_mult=0.0):
    """Equal-time efficiency 1/(relMSE * s): MARS with the counts learned so far
    (frozen: no statistics, no update) vs fixed-count MIS (beta = 1), both
    timed with CUDA events, against a long fixed-count reference.  Like for
    like: the fixed-count arm samples the guided technique from the MARS
    cache's learned guide (same cells: an octree cache's tree is copied too),
    so the two arms differ in their counts alone; the guided workloads also
    report fixed-count MIS with a guide it learned itself over as many
    iterations, and with the uniform guide of a fresh cache.  Every arm that
    learns follows the library's training schedule, and every arm renders with
    the launch shape the library's autotuner picks for its own iterations."""
    import torch
    npx = cfg.scene.n_pixels
    n_ref = ref_spp or args.ref_spp
    cache_kw = cache_kw or {}
    img = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    ref_cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream, **cache_kw)
    acc = torch.zeros(npx * 3, dtype=torch.float64, device="cuda")
    acc2 = torch.zeros(npx * 3, dtype=torch.float64, device="cuda")
    for k in range(n_ref):
        ref_cache.render_iteration(img, seed=777, iteration=k, mode=M.MARS_MODE_FIXED, collect=False,
                                   update_estimate=False, stream=stream)
        x = img.double()
        acc += x
        acc2 += x * x
    ref_t = acc / n_ref
    # variance of the reference's mean, from the spread of its iterations
    ref_var = ((acc2 / n_ref - ref_t * ref_t).clamp_min(0.0) / max(n_ref - 1, 1)).cpu().numpy().reshape(-1, 3)
    ref = ref_t.cpu().numpy().reshape(-1, 3)
    del ref_cache, acc, acc2
    # relMSE's eps = 1e-2 assumes pixel values of order one (an image exposed
    # for display); the same relMSE at this image's own scale takes eps = 1e-2
    # times its squared mean (what scaling the emitters to a mean of one does)
    ref_mean = float(ref.mean())
    eps_scaled = 1e-2 * max(ref_mean, 1e-30) ** 2

    def timed(c, mode, n, it_base, weights=M.MARS_WEIGHTS_AWARE):
        a = torch.zeros(npx * 3, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rays = 0
        for k in range(n):
            st = c.render_iteration(img, seed=seed + 17, iteration=it_base + k, mode=mode, collect=False,
                                    weights=weights, update_estimate=False, max_multiplicity=max_mult,
                                    stream=stream)
            rays += st["rays"]
            a += img.double()
        e1.record(stream)
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) * 1e-3
        mean = (a / n).cpu().numpy().reshape(-1, 3)
        # a relMSE at or below zero (the reference's own variance exceeds the
        # error) is floored: the comparison then resolves nothing
        r = max(rel_mse(mean, ref, ref_var), 1e-30)
        rs = max(rel_mse(mean, ref, ref_var, eps=eps_scaled), 1e-30)
        return {"relmse": r, "relmse_raw": rel_mse(mean, ref), "seconds": s, "efficiency": 1.0 / (r * s),
                "relmse_scaled": rs, "efficiency_scaled": 1.0 / (rs * s),
                "rays_per_pixel": rays / n / npx, "spp": n}

    def tune(c, mode, weights=M.MARS_WEIGHTS_AWARE):
        # renders without statistics: the learned state is unchanged
        c.autotune(seed=seed + 17, iteration=20000, mode=mode, weights=weights, repeats=1,
                   max_multiplicity=max_mult, stream=stream)

    guided = bool(cfg.techniques & W.TECH_GUIDED)
    tune(cache, M.MARS_MODE_MARS)
    mars = timed(cache, M.MARS_MODE_MARS, args.eff_spp, 20000)
    learned = cache.get_state(stream=stream)
    fixed_cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream, **cache_kw)
    if guided:
        tree = {"oct_nodes": learned["oct_nodes"], "oct_leaf_level": learned["oct_leaf_level"]} \
            if "oct_nodes" in learned else {}
        fixed_cache.set_state(guide_cdf=learned["guide_cdf"], stream=stream, **tree)
    tune(fixed_cache, M.MARS_MODE_FIXED)
    fixed = timed(fixed_cache, M.MARS_MODE_FIXED, args.eff_spp, 20000)
    del fixed_cache
    out = {"mars": mars, "fixed_count_mis": fixed, "ratio": mars["efficiency"] / fixed["efficiency"],
           "ratio_scaled": mars["efficiency_scaled"] / fixed["efficiency_scaled"],
           "reference_mean": ref_mean, "eps_scaled": eps_scaled,
           "reference_spp": n_ref, "learning_iterations": it0,
           "training_schedule": M.training_schedule(it0, cfg.warmup),
           "protocol": f"counts learned over {it0} one-sample renders in training iterations of the library's "
                       "schedule (training_schedule: renders per iteration, one update after each), then frozen; "
                       "every arm autotuned for its own iterations; both arms render "
                       f"{args.eff_spp} fresh iterations with the same learned guide (fixed-count MIS: beta = 1); "
                       f"reference = fixed-count MIS, {n_ref} spp, other random numbers; relMSE with the variance "
                       "of the reference's mean subtracted (relmse_raw without); ratio_scaled: the same with "
                       "relMSE's eps = 1e-2 x the reference's squared mean (the image at its own scale)"}
    if guided:
        # fixed-count MIS that learns its own guide from its own deposits over as
        # many iterations, and with the uniform guide of a fresh cache
        own = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream, **cache_kw)
        learn(M, own, img, seed, it0, cfg.warmup, stream, mode=M.MARS_MODE_FIXED, drop=vi_drop, max_mult=max_mult)
        tune(own, M.MARS_MODE_FIXED)
        f_own = timed(own, M.MARS_MODE_FIXED, args.eff_spp, 20000)
        del own
        uni = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream, **cache_kw)
        tune(uni, M.MARS_MODE_FIXED)
        f_uni = timed(uni, M.MARS_MODE_FIXED, args.eff_spp, 20000)
        del uni
        out["fixed_count_mis_own_guide"] = f_own
        out["ratio_vs_own_guide"] = mars["efficiency"] / f_own["efficiency"]
        out["fixed_count_mis_uniform_guide"] = f_uni
        out["ratio_vs_uniform_guide"] = mars["efficiency"] / f_uni["efficiency"]
    if unaware:
        # the budget-unaware balance heuristic (weights from the sampling densities
        # alone) learns its own counts over as many iterations, then renders alike
        un_cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream, **cache_kw)
        learn(M, un_cache, img, seed, it0, cfg.warmup, stream, weights=M.MARS_WEIGHTS_UNAWARE, drop=vi_drop,
              max_mult=max_mult)
        tune(un_cache, M.MARS_MODE_MARS, M.MARS_WEIGHTS_UNAWARE)
        un = timed(un_cache, M.MARS_MODE_MARS, args.eff_spp, 20000, weights=M.MARS_WEIGHTS_UNAWARE)
        del un_cache
        un["learning_iterations"] = it0
        un["ratio_vs_aware"] = un["efficiency"] / mars["efficiency"]
        out["budget_unaware"] = un
    return out


def box_efficiency(args, M, stream, iterations=None):
    """The box workload (64 x 64, D = 5, BSDF + NEE, 8^3 grid; the paper's own
    failure case, where MARS's overhead can dominate): 1 warm-up render and
    training iterations of 1 and 2 renders learn the counts, then the same equal-time comparison
    with fixed-count MIS as for the main workload, plus the device time of one
    MARS iteration (launch-bound at this size)."""
    import torch
    cfg = W.config_box(64, 64)
    n_iter = iterations or cfg.iterations
    scene = M.Scene(cfg.scene, stream=stream)
    cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream)
    img = torch.zeros(cfg.scene.n_pixels * 3, dtype=torch.float32, device="cuda")
    learn(M, cache, img, 2024, n_iter, cfg.warmup, stream)
    it = n_iter
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    n = 20
    verts = 0
    for k in range(n):
        st = cache.render_iteration(img, seed=2024, iteration=100 + k, mode=M.MARS_MODE_MARS, collect=False,
                                    update_estimate=False, stream=stream)
        verts += st["vertices"]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    eff = efficiency(args, M, cfg, scene, cache, 2024, it, stream)
    eff["workload"] = cfg.name
    eff["learning_iterations"] = n_iter
    eff["iteration_ms"] = round(ms, 4)
    eff["mvertices_s"] = round(verts / n / (ms * 1e-3) / 1e6, 2)
    return eff


_STATE_CACHE = {}


def _mars_inputs(state_path):
    """The teacher-forced MARS inputs (count fields, pixel estimate, guide CDF)
    saved by the GPU run, loaded once per worker process."""
    if state_path not in _STATE_CACHE:
        z = np.load(state_path)
        _STATE_CACHE[state_path] = {k: z[k] for k in z.files}
    d = _STATE_CACHE[state_path]
    return dict(mode=1, q_rr=d["q_rr"], q_s=d["q_s"], valid=d["valid"], est=d["pixel_estimate"],
                guide_cdf=d.get("guide_cdf"))


def _oracle_chunks(job):
    """Worker of the multi-core CPU baseline (a spawned process): render the
    given pixel runs of one iteration with the oracle as it stands -- in MARS
    mode from the GPU run's state when `state_path` is given, else with
    beta = 1; returns (path vertices, seconds)."""
    scene, grid_n, techniques, max_depth, runs, state_path = job
    import oracle
    kw = _mars_inputs(state_path) if state_path else {}
    verts, t = 0, 0.0
    for iteration, b, e in runs:
        t0 = time.perf_counter()
        r = oracle.render(scene, grid_n=grid_n, techniques=techniques, max_depth=max_depth, iteration=iteration,
                          seed=3, px_begin=b, px_end=e, **kw)
        t += time.perf_counter() - t0
        verts += r.vertices
    return verts, t


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_learn_chunk(job):
    """Worker (a spawned process) of the oracle's own fixed-point learning: one
    iteration over a share of the pixels with statistics and guide deposits;
    returns (pixel runs, statistics, guide deposits, counters)."""
    scene, grid_n, techniques, max_depth, runs, iteration, state_path = job
    import oracle
    kw = _mars_inputs(state_path) if state_path else {}
    stats = hist = None
    ctr = np.zeros(8)
    imgs = []
    for b, e in runs:
        r = oracle.render(scene, grid_n=grid_n, techniques=techniques, max_depth=max_depth, iteration=iteration,
                          seed=3, px_begin=b, px_end=e, **kw)
        imgs.append((b, e, r.image[b:e].copy()))
        stats = r.stats if stats is None else stats + r.stats
        hist = r.hist if hist is None else hist + r.hist
        ctr += r.counters
    return imgs, stats, hist, ctr


def oracle_learned_state(cfg, pool, cores, iterations, warmup):
    """The oracle's own MARS state after `iterations` fixed-point iterations of
    the whole image (the first `warmup` with beta = 1), in spawned processes:
    each iteration renders every pixel with statistics, then the image
    statistics, the count update and the guide update run on the sums -- the
    same protocol that produces the GPU's state before its timed steps, with
    every input from the oracle itself.  Returns the path of an .npz with the
    count fields, pixel estimate and guide CDF."""
    import oracle
    sc = cfg.scene
    npx = sc.n_pixels
    cells = cfg.n_cells
    chunk = 4096
    runs = [(b, min(npx, b + chunk)) for b in range(0, npx, chunk)]
    q_rr = np.zeros((cells, 3, 3), np.float32)
    q_s = np.zeros((cells, 3, 3), np.float32)
    valid = np.zeros((cells, 3), np.uint8)
    hist_acc = np.zeros((cells, oracle.GUIDE_BINS))
    cdf = np.tile((np.arange(1, oracle.GUIDE_BINS + 1) / oracle.GUIDE_BINS).astype(np.float32), (cells, 1))
    run_sum = np.zeros((npx, 3))
    est = np.ones((npx, 3), np.float32)
    path = os.path.join(tempfile.gettempdir(), f"mars_oracle_state_{os.getpid()}.npz")
    for it in range(iterations):
        state_path = None
        if it >= warmup:
            np.savez(path, q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, guide_cdf=cdf)
            state_path = path
            _STATE_CACHE.pop(path, None)
        jobs = [(sc, cfg.grid_n, cfg.techniques, cfg.max_depth, runs[k::cores], it, state_path)
                for k in range(cores)]
        res = list(pool.map(_oracle_learn_chunk, jobs))
        img = np.zeros((npx, 3))
        stats = np.zeros((cells, 3, 8))
        ctr = np.zeros(8)
        for imgs, st, h, c in res:
            for b, e, rows in imgs:
                img[b:e] = rows
            if st is not None:
                stats += st
                hist_acc += h
            ctr += c
        vi, run_sum, est64 = oracle.image_stats(sc.width, sc.height, img, run_sum, it)
        est = est64.astype(np.float32)
        q_rr, q_s, valid = oracle.update_counts(stats, vi, ctr[0] / npx, cfg.techniques, q_rr, q_s, valid)
        if cfg.techniques & W.TECH_GUIDED:
            cdf = oracle.guide_update(hist_acc)
    np.savez(path, q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, guide_cdf=cdf)
    return path


def cpu_baseline(cfg, seconds, learn_iterations=3, warmup=3, iteration=3):
    """The CPU oracle as it stands on the host cores, on the work of the GPU's
    timed steps: MARS iterations (index `iteration` on) from the state the
    oracle itself learned over `learn_iterations` iterations of the whole image
    (the first `warmup` with beta = 1; count fields, pixel estimate and guide),
    as the GPU's timed steps start from the state of its own warm-up.  One
    thread on 4096-pixel runs spread evenly over the image (about `seconds` of
    work; runs of that size keep the oracle's per-call set-up, a copy of the
    cache fields and guide tables, from dominating), and the whole image split
    into 4096-pixel runs over one spawned process per host core (started before
    the clock starts)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    sc = cfg.scene
    oracle.build()
    chunk = 4096
    cores = max(1, os.cpu_count() or 1)
    out = {"unit": UNIT, "kind": "oracle", "cpu": _cpu_model(), "nproc": os.cpu_count()}
    # all host cores: spawned workers (a process forked after CUDA was used hangs)
    pool = cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))
    try:
        t0 = time.perf_counter()
        state_path = oracle_learned_state(cfg, pool, cores, learn_iterations, min(warmup, learn_iterations))
        learn_s = time.perf_counter() - t0
    except Exception as exc:  # no spawned processes: learn nothing, time warm-up iterations
        pool.shutdown()
        pool, state_path, learn_s = None, None, 0.0
        out["multi_core_error"] = repr(exc)[:200]
    kw = _mars_inputs(state_path) if state_path else {}
    what = (f"MARS iterations from the oracle's own state after {learn_iterations} whole-image iterations "
            f"({min(warmup, learn_iterations)} with beta = 1; learned in {learn_s:.1f} s)") if state_path \
        else "warm-up iterations (beta = 1)"

    def run(npx_sample, it):
        stride = max(1, sc.n_pixels // npx_sample)
        t = 0.0
        verts = 0.0
        starts = list(range(0, sc.n_pixels, stride * chunk))[: max(1, npx_sample // chunk)]
        for s0 in starts:
            t0 = time.perf_counter()
            r = oracle.render(sc, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                              iteration=it, seed=3, px_begin=s0, px_end=min(sc.n_pixels, s0 + chunk), **kw)
            t += time.perf_counter() - t0
            verts += r.vertices
        return verts, t, len(starts) * chunk

    v, t, n = run(chunk, iteration)
    target = max(chunk, int(chunk * seconds / max(t, 1e-3)))
    v, t, n = run(min(target, sc.n_pixels), iteration + 1)
    single = round(v / t / 1e6, 5)
    out.update({"value": single, "cores": 1,
                "sample": f"{n} pixels of the {sc.width}x{sc.height} workload (4096-pixel runs evenly spread), "
                          f"one iteration: {what}, {int(v)} path vertices in {t:.1f} s"})
    if pool is not None:
        # the whole image, repeated (successive iterations) to about `seconds` of
        # single-core work in all
        images = max(1, int(round(seconds / max(t * sc.n_pixels / max(n, 1), 1e-3))))
        runs = [(iteration + it, b, min(sc.n_pixels, b + chunk)) for it in range(1, images + 1)
                for b in range(0, sc.n_pixels, chunk)]
        jobs = [(sc, cfg.grid_n, cfg.techniques, cfg.max_depth, runs[k::cores], state_path) for k in range(cores)]
        try:
            list(pool.map(_oracle_chunks, [(sc, cfg.grid_n, cfg.techniques, cfg.max_depth, [(0, 0, 64)],
                                            state_path)] * cores))
            t0 = time.perf_counter()
            res = list(pool.map(_oracle_chunks, jobs))
            wall = time.perf_counter() - t0
            verts = sum(r[0] for r in res)
            out.update({"value": round(verts / wall / 1e6, 5), "cores": cores,
                        "sample": f"the whole {sc.width}x{sc.height} image {images} times ({sc.n_pixels} pixels in "
                                  f"4096-pixel runs over {cores} processes), {what}, "
                                  f"{int(verts)} path vertices in {wall:.2f} s",
                        "single_thread": {"value": single, "sample": out["sample"]}})
        except Exception as exc:
            out["multi_core_error"] = repr(exc)[:200]
        pool.shutdown()
    if state_path:
        try:
            os.remove(state_path)
        except OSError:
            pass
    return out


def run_reference(args):
    """Reference arm: the CPU oracle as it stands on the host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    oracle.build()
    cfg = workload(args)
    sc = cfg.scene
    cores = max(1, os.cpu_count() or 1)
    per_step = min(sc.n_pixels, max(64, args.ref_pixels_per_step))
    chunk = max(64, per_step // cores)
    times, verts = [], []
    learn = max(1, args.warmup)
    # one spawned process per host core, started and warmed before the steps;
    # the MARS state comes from the oracle itself: `learn` whole-image
    # iterations with beta = 1 (the GPU arm's warm-up), untimed, as the GPU
    # arm's timed MARS iterations start from the state of its own warm-up
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_oracle_chunks, [(sc, cfg.grid_n, cfg.techniques, cfg.max_depth, [(0, 0, 64)], None)] * cores))
        t0 = time.perf_counter()
        state_path = oracle_learned_state(cfg, pool, cores, learn, learn)
        learn_s = time.perf_counter() - t0
        for k in range(args.warmup + args.steps):
            b = (k * 7919 * 64) % max(1, sc.n_pixels - per_step + 1)
            runs = [(learn + k, b + q, min(b + per_step, b + q + chunk)) for q in range(0, per_step, chunk)]
            jobs = [(sc, cfg.grid_n, cfg.techniques, cfg.max_depth, runs[w::cores], state_path) for w in range(cores)]
            t0 = time.perf_counter()
            res = list(pool.map(_oracle_chunks, jobs))
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                times.append(dt)
                verts.append(sum(r[0] for r in res))
    value = sum(verts) / sum(times) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg.name, "pixels": sc.n_pixels, "max_depth": cfg.max_depth,
                       "grid": cfg.grid_n, "techniques": "bsdf+nee+guided"},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} contiguous pixels per step of the {sc.width}x{sc.height} "
                                       f"workload over {cores} processes, MARS iterations from the oracle's own "
                                       f"state after {learn} whole-image iterations with beta = 1 (learned in "
                                       f"{learn_s:.1f} s, untimed)",
                             "cpu": _cpu_model()},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=13)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mars", choices=["mars", "reference"])
    ap.add_argument("--width", type=int, default=512)
    ap.add_argument("--height", type=int, default=512)
    ap.add_argument("--no-efficiency", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-spp", type=int, default=2048)
    ap.add_argument("--large-ref-spp", type=int, default=256,
                    help="reference iterations of the efficiency comparison on the heightfield workloads")
    ap.add_argument("--eff-spp", type=int, default=32)
    ap.add_argument("--ref-pixels-per-step", type=int, default=65536)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--bvh", default="sah", choices=sorted(BVH_KINDS),
                    help="hierarchy of the closest-hit and shadow queries (results do not depend on it)")
    ap.add_argument("--no-graphs", action="store_true", help="launch every kernel directly (no CUDA graph replay)")
    ap.add_argument("--lanes", type=int, default=2, choices=[1, 2],
                    help="concurrent pixel-tile lanes the cache is created with (the autotuner keeps one or all)")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the bidirectional heightfield sections")
    ap.add_argument("--large-size", type=int, default=0,
                    help="image side of both bidirectional sections (0: 1024 and 2048, their workloads' sizes; "
                         "smaller for profiling captures)")
    ap.add_argument("--serve-requests", type=int, default=256, help="serving-stream requests (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-no-graphs", action="store_true", help="served jobs launch every kernel directly")
    ap.add_argument("--launch", default="", help="fixed wave-kernel launch shape 't,t,t,t:b,b,b,b[:r,r,r,r]' (threads per "
                    "block, blocks per SM and register cap of trace, shade, shadow, reverse); skips the autotuner")
    ap.add_argument("--clocks-csv", default="", help="where the nvidia-smi samples of the timed region go "
                    "('{rank}' is replaced by the rank; default: the temp directory)")
    ap.add_argument("--arena-capacity", type=int, default=0, help="queue arena slots (0 = library default)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mars":
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mars(args)


if __name__ == "__main__":
    main()
