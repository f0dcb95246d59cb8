#!/usr/bin/env python3
"""Benchmark of the irradiance-matrix hot path (arXiv:2103.14137, Sec. IV-C).

One step = one pass of the whole path over one synthetic ward-sized room:
upload/build the scene hierarchy (uvc_build_scene), the occlusion-tested
irradiance matrix with per-source visibility bits (uvc_irradiance_matrix),
the fluence A^T t for 16 dwell vectors (uvc_fluence) and the covered-area
fraction (uvc_coverage).  The metric is occlusion-tested (candidate, patch)
pairs per second, in Gpairs/s, for the whole job.  The same line carries the
second half of the metric, rooms per second: the plain method, the batched
engine and the batched + learned proposal timed on 16 seeded rooms of uneven
size x 12 lamp designs (3 timed steps each), with the proposal's lost
coverage and added dwell time measured on a seeded subset of the timed jobs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ward|tiny|large]

Under torchrun (N > 1) every rank runs its own seeded room of the same size
(independent problems, weak scaling, no data-path collective); rank 0 prints
one JSON line.  `--impl reference` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "irradiance-matrix Gpairs/s (occlusion-tested) and % roofline; rooms/sec batched+learned vs plain"
UNIT = "Gpairs/s"
MU_MIN = 100.0          # 10 mJ/cm^2
NVEC = 16
BL_STEPS = 3            # timed steps of each pipeline in the rooms-per-second block
E2E_TILE = 500          # candidates per tile of A in the end-to-end steps (copied back while the next is computed)
BL_QUALITY_JOBS = 8     # timed jobs (seeded subset) whose proposal quality is measured
L2_BYTES = 129 * 2 ** 20
# ALU work per operation of the traversal (FP32 arithmetic, min/max, compare
# and predicate-combining instructions of the kernels, per lane):
#   segment box test: 6 subtractions, 6 multiplications, 2 three-way near/far
#     combinations, 2 clamps, the far scaling and the comparison = 18
#   triangle test: the watertight segment test = 40
#   segment set-up: TwoSum, error-free dot product, ray set-up, Eq. (7) term = 60
#   wedge box test: 4 subtractions, 4 multiplications, two three-way
#     combinations (2 each), 4 FMAs for the z bounds at both ends, 1 min,
#     1 max, 3 comparisons, 2 ANDs = 23
#   wedge plane test: 3 vertices x (2 subtractions, 1 multiplication, 1 FMA),
#     6 comparisons, 4 ANDs/ORs = 22
OPS_BOX_TEST = 18
OPS_TRI_TEST = 40
OPS_SEGMENT_SETUP = 60
OPS_WEDGE_BOX_TEST = 23
OPS_WEDGE_PLANE_TEST = 22


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["ward", "tiny", "large", "large_tiles", "batched", "learned", "area",
                                          "raster"],
                   default="ward")
    p.add_argument("--resolution", type=int, default=512, help="raster workload: cube face resolution R")
    p.add_argument("--tile", type=int, default=500, help="large_tiles workload: candidates per tile of A")
    p.add_argument("--rooms", type=int, default=16, help="batched workload: number of rooms (x 12 designs)")
    p.add_argument("--keep", type=float, default=0.0,
                   help="learned workload: fraction of the candidates kept (0: the proposal's default)")
    p.add_argument("--pool-gb", type=float, default=96.0, help="batched workload: A buffer pool (GiB)")
    p.add_argument("--candidates", type=int, default=0, help="use only the first N candidates (profiling)")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target CPU time of the oracle sample (per step in --impl reference)")
    p.add_argument("--bl-rooms", type=int, default=16,
                   help="ward workload: rooms (x 12 designs) of the batched/learned/plain rooms-per-second block "
                        "(0 = leave it out)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (weak scaling over independent rooms; no data-path
# collective: only a barrier and a max-reduction of the step time)
# ---------------------------------------------------------------------------

def rank_seeds(name: str, rank: int):
    """Room and dwell-vector seeds of a rank: rank 0 runs the reference room of
    the workload; rank r an independent room of the same size (seed + 1000 r)."""
    base = {"tiny": 0, "ward": 1, "large": 3, "large_tiles": 3}[name]
    return base + 1000 * rank, 2 + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest per-rank value (the job's time is its slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(pairs_per_rank: int, world: int, ms_step: float) -> float:
    """Whole-job throughput in Gpairs/s: every rank's pairs over the slowest step."""
    return world * pairs_per_rank / (ms_step * 1e-3) / 1e9


def make_workload(name: str, rank: int):
    from synth import dwell_vectors, large_floor, tiny_room, ward_room
    room_seed, t_seed = rank_seeds(name, rank)
    if name == "tiny":
        s = tiny_room(seed=room_seed)
    elif name in ("large", "large_tiles"):
        s = large_floor(seed=room_seed)
    else:
        s = ward_room(seed=room_seed)
    nvec = 64 if name in ("large", "large_tiles") else NVEC
    t = dwell_vectors(nvec, s.nc, seed=t_seed)
    return s, t


def workload_config(name, s, nvec, world):
    desc = {
        "ward": "plain method, ward-sized room: 10x8x3 m, 6 beds, 4 cabinets, 2 partitions; K=8 line lamp 1.2 m, P=120 W",
        "tiny": "plain method, tiny room: 4x4x3 m with a table; point lamp P=80 W",
        "large": "large floor: 30x30x3 m, 20 rooms + corridor; K=8 line lamp; streamed A^T t (A not stored)",
        "large_tiles": "large floor: 30x30x3 m, 20 rooms + corridor; K=8 line lamp; FP32 A (10,000 x 994,000, "
                       "40 GB) written tile by tile, then A^T t for 64 dwell vectors",
    }[name]
    return {"workload": desc, "triangles": s.nt, "patches": s.np_, "candidates": s.nc, "sources_K": s.lamp.K,
            "dwell_vectors": nvec, "mu_min_J_m2": MU_MIN, "global_batch_rooms": world,
            "parallelism": f"independent rooms x{world}" if world > 1 else "single GPU",
            "l2": "flushed between steps (256 MiB write)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        load = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def lamp_is_vertical(off) -> bool:
    off = np.asarray(off)
    return off.shape[0] >= 2 and bool(np.all(off[:, :2] == 0))


def l2_read_peak(uvc, nbytes=32 * 2 ** 20, passes=40, reps=10) -> dict:
    """The L2 read bandwidth of this GPU: uvc_probe_l2_read over a 32 MiB
    buffer (well inside the 129 MB L2) read 40 times per launch with L2-only
    16-byte loads; after one warm-up launch, the best of 10 launches timed with
    CUDA events on the launching stream."""
    import torch
    buf = torch.ones(nbytes // 4, dtype=torch.int32, device="cuda")
    sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    uvc.probe_l2_read(buf, passes, sink)
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        uvc.probe_l2_read(buf, passes, sink)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) * 1e-3)
    return {"gbs": nbytes * passes / best / 1e9, "buffer_bytes": nbytes, "passes": passes,
            "method": "uvc_probe_l2_read: 32 MiB resident buffer, 40 passes of ld.global.cg 16-byte loads per "
                      "launch, 4 x 512 threads per SM, best of 10 launches (CUDA events)"}


def memory_roofline(uvc, sc, s, irr_s, pairs, pk, sample_pairs=384_000, seed=11, vis=True) -> dict:
    """Bytes per pair of the wedge traversal from the counting replay
    (replay/, the same hierarchy, task shape and visit order on the CPU, over
    a seeded sample of warp tasks) against the measured L2 and HBM read
    bandwidths."""
    import replay
    ex = uvc.scene_export_traversal(sc)
    cpt = uvc.irradiance_candidates_per_task()
    tasks = replay.sample_tasks(s.nc, s.np_, max(1, sample_pairs // (32 * cpt)), seed, cand_per_task=cpt)
    c = replay.replay(ex, s.cand, s.lamp.offsets, tasks, cand_per_task=cpt)
    bpp = replay.bytes_per_pair(c, s.lamp.K, vis=vis)
    l2 = l2_read_peak(uvc)
    hbm = float(pk.get("hbm_gbs", 6800.0))
    ach_w = bpp["per_warp"] * pairs / irr_s / 1e9
    ach_l = bpp["per_lane"] * pairs / irr_s / 1e9
    return {"bytes_per_pair": {"per_warp": round(bpp["per_warp"], 2), "per_lane": round(bpp["per_lane"], 2),
                               "output": bpp["output"]},
            "achieved_GBs": round(ach_w, 1), "achieved_GBs_per_lane": round(ach_l, 1),
            "peak_l2_GBs": round(l2["gbs"], 1), "peak_hbm_GBs": round(hbm, 1),
            "frac_l2": round(ach_w / l2["gbs"], 4), "frac_hbm": round(ach_w / hbm, 4),
            "frac_l2_per_lane": round(ach_l / l2["gbs"], 4),
            "peak_l2_method": l2["method"],
            "peak_hbm_source": "hbm_gbs of MEASURED_PEAKS.json (copy kernel)" if "hbm_gbs" in pk else "fallback",
            "leaf_step_lane_occupancy": round(bpp["leaf_step_lane_occupancy"], 3),
            "sample": f"{tasks.shape[0]} seeded warp tasks (32 patches x {cpt} candidate(s)) replayed on the CPU, "
                      f"{c['pairs']} pairs"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2103_14137_gb300 as uvc

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    uvc.build()
    s, t_host = make_workload(args.workload, rank)
    if args.candidates:
        s.cand = s.cand[: args.candidates]
        t_host = np.ascontiguousarray(t_host[:, : args.candidates])
    nvec = t_host.shape[0]
    lamp = uvc.Lamp(s.lamp.offsets, s.lamp.weights, s.lamp.power)
    streamed = args.workload == "large"
    tiled = args.workload == "large_tiles"

    host = {"verts": s.verts, "tris": s.tris, "centroid": s.centroid, "normal": s.normal, "area": s.area,
            "excl": s.excl, "cand": s.cand, "t": t_host}
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in host.items()}
    nwords = (s.np_ + 31) // 32
    # rows of A padded to a multiple of 16 bytes, so that the fluence can stream them with tensor-map copies
    lda = (s.np_ + 3) // 4 * 4
    A = None if streamed else torch.empty((s.nc, lda), dtype=torch.float32, device=dev)[:, :s.np_]
    vis = None if (streamed or tiled) else torch.empty((s.lamp.K, s.nc, nwords), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    launches_per_step = [0]

    def step(irr_events=None):
        sc = uvc.build_scene(d["verts"], d["tris"], d["centroid"], d["normal"], d["area"], d["excl"])
        # build: pack_patches, area_total; prepare, morton, 3 x 8 sort passes, gather;
        # karras, refit, pack_nodes, node_depth, collapse4; clearance
        n = 2 + (27 if s.nt > 0 else 0) + (5 if s.nt > 1 else 0) + (1 if s.np_ > 0 else 0)
        if irr_events:
            irr_events[0].record(stream)
        if streamed:
            mu = uvc.fluence_streamed(sc, d["cand"], lamp, d["t"])
            n += 2
        elif tiled:
            for i0 in range(0, s.nc, args.tile):   # A written tile by tile (row slices, lda = np)
                i1 = min(s.nc, i0 + args.tile)
                uvc.irradiance_matrix(sc, d["cand"][i0:i1], lamp, A=A[i0:i1])
                n += 1
        else:
            uvc.irradiance_matrix(sc, d["cand"], lamp, A=A, vis=vis)
            n += 1
        if irr_events:
            irr_events[1].record(stream)
        if not streamed:
            mu = uvc.fluence(sc, A, d["t"])
            n += (nvec + 15) // 16
        ca, cc = uvc.coverage(sc, mu, MU_MIN)
        n += 1
        launches_per_step[0] = n
        return sc, mu, ca

    for _ in range(args.warmup):
        sc, _, _ = step()
        sc.free()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    step_ms, irr_ms = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    scenes = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = ev(), ev()
        ie = (ev(), ev())
        a.record(stream)
        sc, mu, ca = step(ie)
        b.record(stream)
        scenes.append(sc)
        step_ms.append((a, b, ie))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    status = uvc.scene_status(scenes[-1])
    for sc in scenes[:-1]:
        sc.free()
    per_step = [a.elapsed_time(b) for a, b, _ in step_ms]
    irr_ms = [ie[0].elapsed_time(ie[1]) for _, _, ie in step_ms]
    mean_ms = sum(per_step) / len(per_step)
    cov = ca.cpu().numpy().tolist()
    ms_step = max_over_ranks(mean_ms, dist if world > 1 else None, dev)
    pairs = s.nc * s.np_
    value = job_value(pairs, world, ms_step)

    # instrumented run (outside timing) for the dominant kernel's algorithmic work
    sc = scenes[-1]
    if streamed or tiled:
        # the streamed kernel runs the same per-(candidate, patch) search as the
        # matrix kernel, plus nvec FMAs per pair for the dwell-time products:
        # operations from the instrumented matrix run on evenly spaced rows
        # (the tiled matrix: the same without the FMAs)
        rows = np.unique(np.linspace(0, s.nc - 1, min(s.nc, 48)).astype(np.int64))
        ri = torch.from_numpy(rows).to(dev)
        A_s = torch.empty((rows.size, s.np_), dtype=torch.float32, device=dev)
        cnt = uvc.irradiance_counters(sc, d["cand"].index_select(0, ri).contiguous(), lamp, A=A_s)
        del A_s
        pairs_s = rows.size * s.np_
        ops_s = (cnt["lane_box_tests"] * OPS_BOX_TEST + cnt["lane_tri_tests"] * OPS_TRI_TEST
                 + pairs_s * s.lamp.K * OPS_SEGMENT_SETUP + cnt["lane_wedge_box_tests"] * OPS_WEDGE_BOX_TEST
                 + cnt["lane_wedge_plane_tests"] * OPS_WEDGE_PLANE_TEST)
        ops = int(ops_s * pairs / pairs_s) + (pairs * nvec if streamed else 0)
        irr_s = (sum(irr_ms) / len(irr_ms)) * 1e-3
        pk = measured_peaks()
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        peak = 152 * 128 * sm_max * 1e6 / 1e12
        achieved = ops / irr_s / 1e12
        # the tiled matrix has no committed capture of its own (the ward's counters include
        # the visibility words this workload does not write): traffic unknown
        traffic = measured_traffic(pairs, STREAMED_SUMMARY) if streamed else None
        roof = {"bound": "alu", "kernel": "k_streamed" if streamed else "k_irradiance", "achieved": round(achieved, 3),
                "peak": round(peak, 3), "unit": "Tops/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"152 SMs x 128 lanes x {sm_max:.0f} MHz (sm_max_mhz of measured)",
                "ops_per_launch": ops, "launch_ms": round(irr_s * 1e3, 3),
                "ops_sample": f"search operations counted on {rows.size} evenly spaced rows (uvc_irradiance_counters) "
                              f"and scaled to all {s.nc} candidates" + (f", plus {nvec} FMAs per pair" if streamed
                                                                        else ""),
                "counters_sample": cnt}
        if tiled:
            roof["launch_ms_note"] = f"all {(s.nc + args.tile - 1) // args.tile} tile launches of one step"
            if lamp_is_vertical(s.lamp.offsets):
                roof["memory"] = memory_roofline(uvc, sc, s, irr_s, pairs, pk, vis=False)
    else:
        cnt = uvc.irradiance_counters(sc, d["cand"], lamp, A=A)
        segments = pairs * s.lamp.K
        ops = (cnt["lane_box_tests"] * OPS_BOX_TEST + cnt["lane_tri_tests"] * OPS_TRI_TEST
               + segments * OPS_SEGMENT_SETUP + cnt["lane_wedge_box_tests"] * OPS_WEDGE_BOX_TEST
               + cnt["lane_wedge_plane_tests"] * OPS_WEDGE_PLANE_TEST)
        irr_s = (sum(irr_ms) / len(irr_ms)) * 1e-3
        pk = measured_peaks()
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        peak = 152 * 128 * sm_max * 1e6 / 1e12      # lane-instructions per second, in T/s
        achieved = ops / irr_s / 1e12
        traffic = measured_traffic(pairs, TRAFFIC_SUMMARY)
        roof = {"bound": "alu", "kernel": "k_irradiance", "achieved": round(achieved, 3),
                "peak": round(peak, 3), "unit": "Tops/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "peak_source": f"152 SMs x 128 lanes x {sm_max:.0f} MHz (sm_max_mhz of measured)",
                "ops_per_launch": ops, "launch_ms": round(irr_s * 1e3, 3),
                "counters": cnt}
        if lamp_is_vertical(s.lamp.offsets):
            roof["memory"] = memory_roofline(uvc, sc, s, irr_s, pairs, pk)
    sc.free()

    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.workload, s, nvec, world),
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": launches_per_step[0] * args.steps,
        "breakdown_ms": {"irradiance_or_streamed": round(sum(irr_ms) / len(irr_ms), 3),
                         "rest_of_step": round(mean_ms - sum(irr_ms) / len(irr_ms), 3)},
        "status": uvc.status_string(status),
        "coverage_last_step": [round(c, 5) for c in cov[:4]],
        "wall_s": round(wall, 3),
    }
    if not args.no_e2e:
        out["e2e"] = run_e2e(args, s, host, lamp, streamed, nvec, world, dist if world > 1 else None,
                             tile=args.tile if tiled else 0)
    if world == 1 and args.workload == "ward" and args.bl_rooms > 0 and not args.candidates:
        A = vis = None
        torch.cuda.empty_cache()
        out["batched_learned"] = batched_learned(uvc, dev, args.bl_rooms, BL_STEPS, args.pool_gb, BL_QUALITY_JOBS)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(s, args.cpu_seconds)
        out["cpu_baseline_bvh"] = cpu_baseline_bvh(s, args.cpu_seconds)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_e2e(args, s, host, lamp, streamed, nvec, world, dist, tile=0):
    """Same metric through the public API from pinned host buffers: inputs
    copied host->device and results (A, mu, coverage) device->host inside the
    timed region of every step.  With tile > 0 (the tiled large floor) A is
    computed and copied back tile by tile through one pinned tile buffer.
    Otherwise A is computed in row tiles of E2E_TILE candidates and each tile
    is copied back on a second stream while the next one is computed (the
    step ends when every copy has)."""
    import torch

    import paper_2103_14137_gb300 as uvc
    dev = torch.cuda.current_device()
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in host.items()}
    dbuf = {k: torch.empty(v.shape, dtype=v.dtype, device=dev) for k, v in pin.items()}
    lda = (s.np_ + 3) // 4 * 4   # padded rows, as in the device-side steps
    A = None if streamed else torch.empty((s.nc, lda), dtype=torch.float32, device=dev)[:, :s.np_]
    host_rows = min(s.nc, tile) if tile else s.nc
    A_host = None if streamed else torch.empty((host_rows, s.np_), dtype=torch.float32).pin_memory()
    mu_host = torch.empty((nvec, s.np_), dtype=torch.float32).pin_memory()
    cov_host = torch.empty((nvec,), dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in pin.values())
    d2h = mu_host.numel() * 4 + cov_host.numel() * 4 + (0 if streamed else s.nc * s.np_ * 4)
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    pipelined = not streamed and not tile

    def step():
        for k in pin:
            dbuf[k].copy_(pin[k], non_blocking=True)
        sc = uvc.build_scene(dbuf["verts"], dbuf["tris"], dbuf["centroid"], dbuf["normal"], dbuf["area"],
                             dbuf["excl"])
        if streamed:
            mu = uvc.fluence_streamed(sc, dbuf["cand"], lamp, dbuf["t"])
        elif tile:
            for i0 in range(0, s.nc, tile):   # each tile copied back once written (stream order)
                i1 = min(s.nc, i0 + tile)
                uvc.irradiance_matrix(sc, dbuf["cand"][i0:i1], lamp, A=A[i0:i1])
                A_host[:i1 - i0].copy_(A[i0:i1], non_blocking=True)
            mu = uvc.fluence(sc, A, dbuf["t"])
        elif pipelined:
            for i0 in range(0, s.nc, E2E_TILE):
                i1 = min(s.nc, i0 + E2E_TILE)
                uvc.irradiance_matrix(sc, dbuf["cand"][i0:i1], lamp, A=A[i0:i1])
                ready = torch.cuda.Event()
                ready.record(stream)
                copy_stream.wait_event(ready)
                with torch.cuda.stream(copy_stream):
                    A_host[i0:i1].copy_(A[i0:i1], non_blocking=True)
            mu = uvc.fluence(sc, A, dbuf["t"])
        else:
            uvc.irradiance_matrix(sc, dbuf["cand"], lamp, A=A)
            mu = uvc.fluence(sc, A, dbuf["t"])
            A_host.copy_(A, non_blocking=True)
        ca, _ = uvc.coverage(sc, mu, MU_MIN)
        mu_host.copy_(mu, non_blocking=True)
        cov_host.copy_(ca, non_blocking=True)
        if pipelined:
            done = torch.cuda.Event()
            done.record(copy_stream)
            stream.wait_event(done)   # the step's end includes the last tile's copy
        return sc

    for _ in range(max(1, args.warmup)):
        step().free()
    torch.cuda.synchronize()
    n = max(1, args.steps)   # the same number of timed steps as the device-side value
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    scs = [step() for _ in range(n)]
    b.record(stream)
    torch.cuda.synchronize()
    for sc in scs:
        sc.free()
    ms = max_over_ranks(a.elapsed_time(b) / n, dist, dev)
    return {"value": round(job_value(s.nc * s.np_, world, ms), 4), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(ms, 3),
            "steps": n, "a_copy": ("row tiles of %d candidates copied on a second stream while the next tile is "
                                   "computed" % E2E_TILE) if pipelined else ("tile by tile" if tile else
                                                                              ("none (A not stored)" if streamed
                                                                               else "after the matrix"))}


_KERNEL_FILES = ("irradiance.cu", "traverse.cuh", "uvc_internal.cuh")
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_irradiance_ward.txt")
STREAMED_SUMMARY = os.path.join(ROOT, "profiles", "k_streamed_large.txt")


def measured_traffic(pairs, summary):
    """DRAM bytes of one launch from the committed ncu summary of the same
    kernel: its full-size capture when the launch has the same pairs, else its
    bytes per pair scaled to this launch; null once the kernel has changed."""
    try:
        kv = dict(line.split(":", 1) for line in open(summary) if ":" in line)
        if kv.get("kernel_source_hash", "").strip() != kernel_hash():
            return None
        if "dram_bytes_per_launch" in kv and int(kv.get("pairs_per_launch", "-1")) == int(pairs):
            return float(kv["dram_bytes_per_launch"])
        if "dram_bytes_per_pair" in kv:
            return float(kv["dram_bytes_per_pair"]) * pairs
        return None
    except (OSError, ValueError, KeyError):
        return None


def _code_only(text: str) -> str:
    """Source text without comments and whitespace, so that a comment edit does
    not count as a change of the kernel."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return "".join(text.split())


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in _KERNEL_FILES:
        h.update(_code_only(open(os.path.join(ROOT, "paper_2103_14137_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_rate(s, n_pairs, seed, threads):
    import oracle
    rng = np.random.default_rng(seed)
    pairs = np.stack([rng.integers(0, s.nc, n_pairs), rng.integers(0, s.np_, n_pairs)], axis=1)
    t0 = time.perf_counter()
    oracle.irradiance_scene(s, pairs=pairs, flags=False, threads=threads)
    return time.perf_counter() - t0


def cpu_baseline(s, seconds: float):
    """The FP64 brute-force oracle as it stands, on all host cores, on a seeded
    sample of the workload's pairs sized to about `seconds` of CPU time."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.build()
    # calibrate on enough pairs that thread start-up does not dominate the estimate
    probe = 64
    dt = _oracle_rate(s, probe, 101, threads)
    probe = int(min(max(probe, probe * 0.1 * seconds / max(dt, 1e-6)), 200_000))
    dt = _oracle_rate(s, probe, 103, threads)
    n = int(min(max(probe, probe * seconds / max(dt, 1e-6)), 2_000_000))
    dt = _oracle_rate(s, n, 102, threads)
    rate = n / dt
    return {"value": round(rate / 1e9, 9), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} seeded (candidate, patch) pairs of the same workload, K={s.lamp.K} sources, "
                      f"brute force against all {s.nt} triangles, FP64, {dt:.1f} s",
            "threads_available": oracle.max_threads()}


def cpu_baseline_bvh(s, seconds: float):
    """The oracle's CPU-BVH mode (the same entries as its brute force) on all
    host cores, on whole rows of the workload's matrix sized to about
    `seconds` of CPU time."""
    import oracle
    threads = os.cpu_count() or 1

    def rows_rate(rows):
        pairs = np.stack([np.repeat(rows, s.np_), np.tile(np.arange(s.np_), rows.size)], axis=1)
        t0 = time.perf_counter()
        oracle.irradiance_scene(s, pairs=pairs, flags=False, threads=threads, bvh=True)
        return time.perf_counter() - t0

    rng = np.random.default_rng(104)
    probe = min(s.nc, 8)   # enough rows that thread start-up does not dominate the estimate
    dt = rows_rate(rng.choice(s.nc, probe, replace=False))
    nrows = int(min(s.nc, max(1, probe * seconds / max(dt, 1e-6))))
    rows = np.sort(rng.choice(s.nc, nrows, replace=False))
    dt = rows_rate(rows)
    rate = nrows * s.np_ / dt
    return {"value": round(rate / 1e9, 9), "unit": UNIT, "cores": threads, "kind": "oracle (CPU-BVH mode)",
            "sample": f"{nrows} seeded whole rows ({nrows * s.np_} (candidate, patch) pairs) of the same workload, "
                      f"K={s.lamp.K} sources, FP64 bounding-volume hierarchy over {s.nt} triangles, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    s, _ = make_workload(args.workload, 0)
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    # size each step so that warmup + steps end within a few minutes
    per_step_s = max(1.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    dt = _oracle_rate(s, 64, 7, threads)
    n = int(min(max(64, 64 * per_step_s / max(dt, 1e-6)), 2_000_000))
    for k in range(args.warmup):
        _oracle_rate(s, max(64, n // 8), 1000 + k, threads)
    times = [_oracle_rate(s, n, 2000 + k, threads) for k in range(args.steps)]
    mean = sum(times) / len(times)
    value = n / mean / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 9), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(mean * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(args.workload, s, NVEC, 1),
           "cpu_baseline": {"value": round(value, 9), "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": f"{n} seeded pairs per step, K={s.lamp.K}, brute force over {s.nt} triangles"},
           "e2e": {"value": round(value, 9), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# batched rooms x designs (one persistent launch per wave, CUDA graph)
# ---------------------------------------------------------------------------

def setup_rooms(n_rooms: int, dev, base_seed: int = 100, keep: float = 0.0):
    """Rooms of uneven size x the 12 designs, resident on the device: per room
    the scene, the probe scene (1 % of the patches, for the learned proposal)
    and per (room, design) job the candidates, the full and kept dwell vectors
    and the buffers of the kept candidates (the proposal's fraction `keep`,
    its default when 0)."""
    import torch

    import paper_2103_14137_gb300 as uvc
    from paper_2103_14137_gb300 import proposal as prop
    from synth import dwell_vectors
    from synth.batched import batch

    t_gen = time.perf_counter()
    data = batch(n_rooms, base_seed=base_seed)
    t_gen = time.perf_counter() - t_gen
    lamps = [uvc.Lamp(L.offsets, L.weights, L.power) for _, L, _ in data[0][1]]   # the 12 designs' lamps
    Td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    rooms = []
    for room, jobs in data:
        sc = uvc.build_scene(Td(room.verts), Td(room.tris), Td(room.centroid), Td(room.normal), Td(room.area),
                             Td(room.excl))
        probe, half = prop.probe_columns(room.np_, seed=room.info["seed"] * 977)
        psc = uvc.build_scene(Td(room.verts), Td(room.tris), Td(room.centroid[probe]), Td(room.normal[probe]),
                              Td(room.area[probe]), Td(room.excl[probe]))
        js = []
        for cand, _, d in jobs:
            nc = cand.shape[0]
            k = prop.keep_count(nc, keep if keep > 0 else prop.KEEP)
            js.append({"cand": Td(cand), "d": d, "nc": nc, "k": k, "t_full": Td(dwell_vectors(NVEC, nc, seed=d)),
                       "t_kept": Td(dwell_vectors(NVEC, k, seed=d)),
                       "kept": torch.zeros((k, 3), dtype=torch.float32, device=dev),
                       "idx": torch.zeros(k, dtype=torch.int32, device=dev)})
        rooms.append({"seed": room.info["seed"], "sc": sc, "psc": psc, "area": Td(room.area.astype(np.float32)),
                      "area_p": Td(room.area[probe].astype(np.float32)), "half": half, "P": int(probe.size),
                      "np": room.np_, "nt": room.nt, "jobs": js})
    q = 0
    for R in rooms:
        for j in R["jobs"]:
            j["q"] = q
            q += 1
    return lamps, rooms, t_gen


def free_rooms(rooms):
    for R in rooms:
        R["sc"].free()
        R["psc"].free()


def _waves(rooms, need, pool_floats):
    """Whole rooms grouped into waves whose buffers fit the pool."""
    waves, cur, used = [], [], 0
    for r, R in enumerate(rooms):
        n = need(R)
        if cur and used + n > pool_floats:
            waves.append(cur)
            cur, used = [], 0
        cur.append(r)
        used += n
    waves.append(cur)
    return waves


def _post(uvc, sc, A, t, mu):
    """Fluence (16 dwell vectors) and coverage of one job's matrix."""
    mu = uvc.fluence(sc, A, t, mu=mu)
    uvc.coverage(sc, mu, MU_MIN)


def timed_steps(fn, steps: int, warmup: int = 1):
    """Milliseconds of each of `steps` calls of fn (CUDA events on the current
    stream, synchronised on both sides), after `warmup` untimed calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def plain_pipeline(uvc, rooms, lamps, dev):
    """The plain method, job by job: every candidate's full matrix, its fluence
    and coverage (one A buffer, reused)."""
    import torch
    full = torch.empty(max(j["nc"] * R["np"] for R in rooms for j in R["jobs"]), dtype=torch.float32, device=dev)
    mus = torch.empty(NVEC * max(R["np"] for R in rooms), dtype=torch.float32, device=dev)

    def job(R, j):
        A = full[:j["nc"] * R["np"]].view(j["nc"], R["np"])
        uvc.irradiance_matrix(R["sc"], j["cand"], lamps[j["d"]], A=A)
        _post(uvc, R["sc"], A, j["t_full"], mus[:NVEC * R["np"]].view(NVEC, R["np"]))

    def run():
        for R in rooms:
            for j in R["jobs"]:
                job(R, j)
    return run, job


def batched_pipeline(uvc, rooms, lamps, dev, pool_gb: float):
    """All matrices of a wave of rooms in one persistent launch, with every
    job's fluence and coverage, captured as one CUDA graph per wave; A lives in
    a pool reused by the waves.  Returns (run, free, info)."""
    import torch
    pool_floats = int(pool_gb * 2 ** 30 / 4)
    waves = _waves(rooms, lambda R: sum(j["nc"] * R["np"] for j in R["jobs"]), pool_floats)
    pool = torch.empty(max(sum(j["nc"] * rooms[r]["np"] for r in w for j in rooms[r]["jobs"]) for w in waves),
                       dtype=torch.float32, device=dev)
    graphs, batches, keep, tuned = [], [], [], None
    for w in waves:
        views, off = [], 0
        for r in w:
            R = rooms[r]
            for j in R["jobs"]:
                n = j["nc"] * R["np"]
                views.append((R["sc"], j, pool[off:off + n].view(j["nc"], R["np"])))
                off += n
        b = uvc.Batch([(sc, j["cand"], j["d"], A, None) for sc, j, A in views], lamps)
        if tuned is None:
            tuned = b.autotune(0.02)
        else:
            b.set_config(*tuned)
        mus = [torch.empty((NVEC, sc.np), device=dev) for sc, _, _ in views]

        def wave(b=b, views=views, mus=mus):
            b.launch()
            for (sc, j, A), mu in zip(views, mus):
                _post(uvc, sc, A, j["t_full"], mu)
        wave()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            wave()
        graphs.append(g)
        batches.append(b)
        keep.append(mus)

    def run():
        for g in graphs:
            g.replay()

    def free():
        for b in batches:
            b.free()
        graphs.clear()
        keep.clear()

    return run, free, {"waves": len(waves), "tuned": {"cand_per_task": tuned[0], "blocks_per_sm": tuned[1]}}


def learned_pipeline(uvc, rooms, lamps, dev, pool_gb: float, plain_job):
    """Batched + learned proposal.  Per job: the irradiance of all candidates
    on the probe patches (one batched launch), the scorer features, one scorer
    pass over all jobs, the best source of every sketch patch plus the best
    scores kept (20 % in all), the lit probe area the kept set loses, and the
    exact matrix of the kept candidates (a second batched launch) with its
    fluence and coverage: one CUDA graph per wave.  After the graphs the check
    is read back once and the jobs that fail it are recomputed on all
    candidates (plain_job).  Returns (run, free, info); run() returns the
    number of fallback jobs."""
    import torch

    from paper_2103_14137_gb300 import proposal as prop
    total_nc = sum(j["nc"] for R in rooms for j in R["jobs"])
    njobs = sum(len(R["jobs"]) for R in rooms)
    scorer = prop.Scorer.load(max_batch=max(1, total_nc))
    pool_floats = int(pool_gb * 2 ** 30 / 4)
    need = lambda R: sum(j["k"] * R["np"] + j["nc"] * R["P"] for j in R["jobs"])  # noqa: E731
    waves = _waves(rooms, need, pool_floats)
    pool = torch.empty(max(sum(need(rooms[r]) for r in w) for w in waves), dtype=torch.float32, device=dev)
    flags = torch.zeros(njobs, dtype=torch.float32, device=dev)
    work = uvc.probe_features_work(max(R["half"] for R in rooms), dev)
    lost_scratch = torch.empty(max(1, max(R["P"] - R["half"] for R in rooms)), dtype=torch.float32, device=dev)
    feat = torch.empty((max(1, total_nc), prop.IN_DIM), dtype=torch.float32, device=dev)
    score = torch.empty(max(1, total_nc), dtype=torch.float32, device=dev)
    mus_flat = torch.empty(NVEC * max(R["np"] for R in rooms), dtype=torch.float32, device=dev)

    def layout(w):
        off, row, lay = 0, 0, []
        for r in w:
            R = rooms[r]
            for j in R["jobs"]:
                lay.append([R, j, pool[off:off + j["nc"] * R["P"]].view(j["nc"], R["P"]), None, row])
                off += j["nc"] * R["P"]
                row += j["nc"]
        for e in lay:
            R, j = e[0], e[1]
            e[3] = pool[off:off + j["k"] * R["np"]].view(j["k"], R["np"])
            off += j["k"] * R["np"]
        return lay, row

    def wave(lay, nrows, bprobe, bred):
        bprobe.launch()
        for R, j, Ap, Ar, row0 in lay:
            prop.features(R["sc"], j["cand"], Ap[:, :R["half"]], R["area_p"][:R["half"]],
                          feat=feat[row0:row0 + j["nc"]], work=work)
        scorer.scores(feat[:nrows], out=score[:nrows])
        for R, j, Ap, Ar, row0 in lay:
            sj = score[row0:row0 + j["nc"]]
            if prop.GROUP > 1:
                uvc.group_boost(sj, prop.GROUP)
            uvc.mark_best(Ap[:, :R["half"]], sj, rare=prop.rare_count(j["nc"]))
            uvc.select_top(sj, j["k"], cand=j["cand"], out_cand=j["kept"], out_idx=j["idx"])
            uvc.probe_lost(Ap[:, R["half"]:], j["idx"], R["area_p"][R["half"]:], out=flags[j["q"]:j["q"] + 1],
                           lost=lost_scratch[:R["P"] - R["half"]])
        bred.launch()
        for R, j, Ap, Ar, row0 in lay:
            _post(uvc, R["sc"], Ar, j["t_kept"], mus_flat[:NVEC * R["np"]].view(NVEC, R["np"]))

    graphs, batches, tuned = [], [], None
    for w in waves:
        lay, nrows = layout(w)
        bprobe = uvc.Batch([(R["psc"], j["cand"], j["d"], Ap, None) for R, j, Ap, Ar, _ in lay], lamps)
        bred = uvc.Batch([(R["sc"], j["kept"], j["d"], Ar, None) for R, j, Ap, Ar, _ in lay], lamps)
        if tuned is None:
            tuned = bprobe.autotune(0.05)
        bprobe.set_config(*tuned)
        bred.set_config(*tuned)
        wave(lay, nrows, bprobe, bred)          # eager pass: fills the kept buffers
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            wave(lay, nrows, bprobe, bred)
        graphs.append(g)
        batches += [bprobe, bred]
    jobs = [(R, j) for R in rooms for j in R["jobs"]]
    last = {"fallback": []}

    def run():
        for g in graphs:
            g.replay()
        fl = (flags > prop.LOST_MAX).cpu().numpy()      # the check, read back on the host
        fb = [(R, j) for R, j in jobs if fl[j["q"]]]
        for R, j in fb:
            plain_job(R, j)
        last["fallback"] = [j["q"] for _, j in fb]
        return len(fb)

    def free():
        for b in batches:
            b.free()
        graphs.clear()
        scorer.close()

    return run, free, {"waves": len(waves), "tuned": list(tuned), "last": last}


def proposal_quality(uvc, rooms, lamps, dev, qjobs, fallback, workers: int):
    """Lost coverage and added dwell time of the learned proposal on the jobs
    `qjobs` (job numbers), measured on the kept sets the timed run produced:
    the dwell-time LP of Eq. (9) (row generation over every patch) on all
    candidates (the plain method) and on the kept candidates (all of them for a
    job that fell back), coverage at 100 J/m^2 of every patch from the exact
    matrix."""
    import torch

    from paper_2103_14137_gb300 import proposal as prop
    sel = [(R, j) for R in rooms for j in R["jobs"] if j["q"] in set(qjobs)]
    full, red, meta = [], [], []
    for R, j in sel:
        A, _ = uvc.irradiance_matrix(R["sc"], j["cand"], lamps[j["d"]])
        fb = j["q"] in set(fallback)
        rows = np.arange(j["nc"]) if fb else np.sort(j["idx"].cpu().numpy().astype(np.int64))
        seed = R["seed"] * 16 + j["d"]
        full.append({"A": A, "rows": None, "area": R["area"], "seed": seed, "scene": R["sc"]})
        red.append({"A": A, "rows": rows, "area": R["area"], "seed": seed, "scene": R["sc"]})
        meta.append({"room": R["seed"], "design": j["d"], "nc": j["nc"], "np": R["np"], "kept": int(rows.size),
                     "fallback": fb})
    t0 = time.perf_counter()
    sols = prop.dwell_rowgen(full + red, workers)
    lp_s = time.perf_counter() - t0
    n = len(sel)
    for k, m in enumerate(meta):
        t_full, mu_full = sols[k][0], sols[k][1]
        t_red, mu_red = sols[n + k][0], sols[n + k][1]
        cf, cr = prop.coverage_of(sel[k][0]["area"], mu_full), prop.coverage_of(sel[k][0]["area"], mu_red)
        m.update({"cov_full": round(cf, 6), "cov_kept": round(cr, 6), "lost_coverage": max(0.0, cf - cr),
                  "dwell_full_s": round(float(t_full.sum()), 2), "dwell_kept_s": round(float(t_red.sum()), 2),
                  "added_dwell": float(t_red.sum() / max(t_full.sum(), 1e-30) - 1.0)})
    del full, red, sols
    torch.cuda.empty_cache()
    lost = np.array([m["lost_coverage"] for m in meta])
    added = np.array([m["added_dwell"] for m in meta])
    return {"jobs": len(meta), "lost_coverage_mean": float(lost.mean()), "lost_coverage_max": float(lost.max()),
            "added_dwell_mean": float(added.mean()), "added_dwell_max": float(added.max()),
            "lp_wall_s": round(lp_s, 1), "lp_workers": workers, "per_job": meta}


def batched_learned(uvc, dev, n_rooms: int, steps: int, pool_gb: float = 96.0, quality_jobs: int = 8,
                    pipelines=("plain", "batched", "learned"), base_seed: int = 100, keep: float = 0.0):
    """Rooms/s of the plain method (job by job), the batched engine and the
    batched + learned proposal on the same seeded rooms x 12 designs, each
    timed over `steps` steps after one warm-up (a step = every job of every
    room: all matrices, or the learned pipeline's probe, selection and kept
    matrices with its fallbacks, plus every job's fluence and coverage), and
    the learned proposal's quality on a seeded subset of the same timed jobs."""
    import torch
    lamps, rooms, t_gen = setup_rooms(n_rooms, dev, base_seed, keep)
    njobs = sum(len(R["jobs"]) for R in rooms)
    pairs = sum(j["nc"] * R["np"] for R in rooms for j in R["jobs"])
    plain_run, plain_job = plain_pipeline(uvc, rooms, lamps, dev)
    out = {"rooms": n_rooms, "designs": 12, "jobs": njobs, "pairs": pairs, "steps": steps, "warmup": 1,
           "room_seeds": [rooms[0]["seed"], rooms[-1]["seed"]], "generation_s": round(t_gen, 1)}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if "plain" in pipelines:
        ms = timed_steps(plain_run, steps)
        out["plain"] = {"rooms_per_s": round(n_rooms / (np.mean(ms) * 1e-3), 4), "ms_per_step": round(float(np.mean(ms)), 1),
                        "ms_steps": [round(x, 1) for x in ms], "gpairs_per_s": round(pairs / (np.mean(ms) * 1e-3) / 1e9, 4)}
    if "batched" in pipelines:
        run, free, info = batched_pipeline(uvc, rooms, lamps, dev, pool_gb)
        ms = timed_steps(run, steps)
        free()
        torch.cuda.empty_cache()
        out["batched"] = {"rooms_per_s": round(n_rooms / (np.mean(ms) * 1e-3), 4), "ms_per_step": round(float(np.mean(ms)), 1),
                          "ms_steps": [round(x, 1) for x in ms], "gpairs_per_s": round(pairs / (np.mean(ms) * 1e-3) / 1e9, 4),
                          **{k: v for k, v in info.items() if k != "last"}}
    fallback = []
    if "learned" in pipelines:
        run, free, info = learned_pipeline(uvc, rooms, lamps, dev, pool_gb, plain_job)
        nfb = []
        ms = timed_steps(lambda: nfb.append(run()), steps)
        fallback = info["last"]["fallback"]
        free()
        torch.cuda.empty_cache()
        out["learned"] = {"rooms_per_s": round(n_rooms / (np.mean(ms) * 1e-3), 4), "ms_per_step": round(float(np.mean(ms)), 1),
                          "ms_steps": [round(x, 1) for x in ms], "fallback_jobs": nfb[-1], "waves": info["waves"],
                          "tuned": info["tuned"]}
    out["clocks"] = clocks.stop()
    if "plain" in out and "batched" in out:
        out["batched_over_plain"] = round(out["plain"]["ms_per_step"] / out["batched"]["ms_per_step"], 4)
    if "plain" in out and "learned" in out:
        out["learned_over_plain"] = round(out["plain"]["ms_per_step"] / out["learned"]["ms_per_step"], 4)
        if quality_jobs > 0:
            rng = np.random.default_rng(2103)
            qjobs = sorted(rng.choice(njobs, size=min(quality_jobs, njobs), replace=False).tolist())
            workers = max(1, (os.cpu_count() or 2) - 1)
            out["quality"] = proposal_quality(uvc, rooms, lamps, dev, qjobs, fallback, workers)
            out["quality"]["sample"] = (f"{len(qjobs)} of the {njobs} timed jobs (seeded), the kept sets of the "
                                        f"last timed step")
    free_rooms(rooms)
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    """Rooms of uneven size x 12 lamp designs: all matrices A plus the fluence
    (16 dwell vectors) and coverage of every (room, design) job, through the
    batched engine (one captured graph per wave of rooms) against the plain
    job-by-job calls.  Metric: rooms per second."""
    _run_rooms(args, ("plain", "batched"), "batched", 0)


def run_learned(args):
    """Batched + learned proposal against the plain method, in rooms/s, with
    the proposal's lost coverage and added dwell time measured on a seeded
    subset of the timed jobs."""
    _run_rooms(args, ("plain", "learned"), "learned", 8)


def _run_rooms(args, pipelines, key, quality_jobs):
    import torch

    import paper_2103_14137_gb300 as uvc
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    uvc.build()
    steps = max(3, args.steps)
    r = batched_learned(uvc, dev, args.rooms, steps, args.pool_gb, quality_jobs, pipelines, 100 + 1000 * rank,
                        args.keep)
    ms = r[key]["ms_per_step"]
    out = {"metric": METRIC, "value": r[key]["rooms_per_s"], "unit": "rooms/s", "n_gpus": 1, "steps": steps,
           "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if key == "batched" else "f32 (scorer bf16)", "data": "synthetic",
           "config": {"workload": f"{key}: {args.rooms} seeded rooms of uneven size (10k-200k triangles, 5k-300k "
                                  "patches, 500-5,000 candidates, log-uniform) x 12 designs (lamp-bottom heights "
                                  "0.3/0.5/0.8/1.1 m x line lamps 0.6/1.2/1.8 m, K = 4/8/12); fluence (16 vectors) and "
                                  "coverage of every job", "rooms": args.rooms, "pool_gib": args.pool_gb,
                      **({"keep": args.keep} if key == "learned" and args.keep > 0 else {})},
           **{k: v for k, v in r.items() if k not in ("steps",)}}
    print(json.dumps(out), flush=True)


def run_area(args):
    """Area-mean irradiance (uvc_irradiance_area_mean: solid-angle closed form
    with vertex checks, centroid sample as fallback) on the ward room, timed
    beside the centroid-sample matrix (uvc_irradiance_matrix) on the same
    inputs; A > L2, so no flush is needed between steps.  Metric: pairs/s."""
    import torch

    import paper_2103_14137_gb300 as uvc
    from synth import ward_room

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    uvc.build()
    s = ward_room(seed=1 + 1000 * rank)
    if args.candidates:
        s.cand = s.cand[:args.candidates]
    Td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    sc = uvc.build_scene(Td(s.verts), Td(s.tris), Td(s.centroid), Td(s.normal), Td(s.area), Td(s.excl))
    cand, ptri = Td(s.cand), Td(s.ptri)
    lamp = uvc.Lamp(s.lamp.offsets, s.lamp.weights, s.lamp.power)
    A = torch.empty((s.nc, s.np_), dtype=torch.float32, device=dev)
    ncl = torch.empty((s.nc, s.np_), dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(k):
            a, b = ev(), ev()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    clocks = ClockSampler(local)
    clocks.start()
    ms_area = timed(lambda: uvc.irradiance_area_mean(sc, cand, lamp, ptri, A=A), args.steps, args.warmup)
    clk = clocks.stop()
    uvc.irradiance_area_mean(sc, cand, lamp, ptri, A=A, with_closed=True)
    closed_frac = float(uvc.irradiance_area_mean(sc, cand, lamp, ptri, A=A, with_closed=True)[1].float().mean()
                        .item()) / s.lamp.offsets.shape[0]
    ms_point = timed(lambda: uvc.irradiance_matrix(sc, cand, lamp, A=A), args.steps, args.warmup)
    assert uvc.scene_status(sc) == 0
    pairs = s.nc * s.np_
    out = {"metric": METRIC, "value": round(pairs / (ms_area * 1e-3) / 1e9, 4), "unit": "Gpairs/s (area mean)",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_area, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "area-mean irradiance, ward-sized room (51k triangles, 102k bisected triangle "
                                  "patches, K=8 line lamp)", "candidates": s.nc, "patches": s.np_},
           "area_mean": {"ms": round(ms_area, 3), "gpairs_per_s": round(pairs / (ms_area * 1e-3) / 1e9, 4),
                         "closed_form_source_fraction": round(closed_frac, 4)},
           "centroid_sample": {"ms": round(ms_point, 3), "gpairs_per_s": round(pairs / (ms_point * 1e-3) / 1e9, 4)},
           "area_over_point_time": round(ms_area / ms_point, 3), "clocks": clk}
    sc.free()
    print(json.dumps(out), flush=True)


def run_raster(args):
    """The paper's own estimator (visibility cube, uvc_irradiance_raster) at
    its configuration (R = 512 per face) on the ward room: per candidate one
    column of mean irradiances over all triangles, K = 8 cubes per candidate.
    Metric: ms per column (the paper states "milliseconds") and the
    (candidate, triangle) pair rate.  Default: the first 64 candidates."""
    import torch

    import paper_2103_14137_gb300 as uvc
    from synth import ward_room

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    uvc.build()
    s = ward_room(seed=1 + 1000 * rank)
    nc = args.candidates or 64
    cand_h = s.cand[:nc]
    Td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    # per-triangle normals: the ward's patches are pieces of triangles (parent in excl[:, 0])
    tnrm = np.zeros((s.nt, 3), np.float32)
    tnrm[s.excl[:, 0]] = s.normal
    sc = uvc.build_scene(Td(s.verts), Td(s.tris), Td(s.centroid), Td(s.normal), Td(s.area), Td(s.excl))
    lamp = uvc.Lamp(s.lamp.offsets, s.lamp.weights, s.lamp.power)
    cand, nrm = Td(cand_h), Td(tnrm)
    R = args.resolution
    per_batch = 4
    ws = uvc.raster_workspace(sc, lamp, R, per_batch, dev)
    A = torch.empty((nc, s.nt), dtype=torch.float32, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for _ in range(max(1, args.warmup)):
        uvc.irradiance_raster(sc, nrm, cand[:per_batch], lamp, R=R, A=A[:per_batch], workspace=ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    a, b = ev(), ev()
    a.record()
    uvc.irradiance_raster(sc, nrm, cand, lamp, R=R, A=A, workspace=ws)
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b)
    areas = torch.from_numpy(0.5 * np.linalg.norm(np.cross(
        s.verts[s.tris[:, 1]].astype(np.float64) - s.verts[s.tris[:, 0]],
        s.verts[s.tris[:, 2]].astype(np.float64) - s.verts[s.tris[:, 0]]), axis=1)).to(dev)
    flux = (A.double() * areas[None, :]).sum(1)
    out = {"metric": METRIC, "value": round(ms / nc, 4), "unit": "ms per irradiance column (visibility cube)",
           "n_gpus": 1, "steps": 1, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 (flux in 2^-40 W fixed point)", "data": "synthetic",
           "config": {"workload": f"visibility-cube estimator, ward-sized room (51k triangles), R = {R} per face, "
                                  f"K = 8 cubes per candidate, {nc} candidates", "resolution": R, "candidates": nc,
                      "triangles": s.nt, "cubes": nc * 8},
           "pairs_per_s": round(nc * s.nt / (ms * 1e-3), 1),
           "absorbed_flux_fraction_mean": round(float(flux.mean().item()) / s.lamp.power, 6),
           "paper_context": "the paper states milliseconds per column at 512x512 (unnamed GPU, OpenGL)",
           "clocks": clk}
    sc.free()
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "area":
        run_area(args)
    elif args.workload == "raster":
        run_raster(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
