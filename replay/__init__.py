"""Counting replay of the traversal kernels (traversal_replay.c) for the memory
roofline of the irradiance matrix.

A measurement tool used by bench.py and its tests: it replays, on the CPU and
in FP32, the visit order of the wedge traversal (vertical line lamps) over the
hierarchy the library built, for a sample of warp tasks, and converts the
counts into algorithmic bytes per (candidate, patch) pair:

  per warp   128 B per node visit (one warp-uniform node load), 48 B per
             distinct triangle of each leaf step, 48 B per cached-occluder
             test, 40 B of patch record per lane and task, plus the output
             (4 B of A and K/8 B of visibility per pair)
  per lane   128 B per node visit per searching lane, 48 B per leaf per lane,
             plus the same output bytes

It is not the oracle (it checks nothing and shares nothing with it) and not
the product (the library never calls it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "traversal_replay.c")
_LIB = os.path.join(_HERE, "libtraversal_replay.so")
_lib = None

NODE_BYTES = 128
TRI_BYTES = 48
PATCH_BYTES = 40
COUNTERS = ("node_visits", "leaf_loads", "traversals", "tri_tests", "search_segments", "box_tests", "plane_tests",
            "leaf_steps", "leaf_step_lanes", "leaf_step_unique", "cache_loads", "lane_node_visits", "pairs", "tasks")


def build(force: bool = False) -> str:
    """Compile the replay with gcc (OpenMP, no floating-point contraction:
    every fused multiply-add is written out as fmaf, as in the kernels)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.replay_wedge_tasks.argtypes = [P, P, P, P, P, i64, i64, i32, ctypes.c_float, P, i64, P, i32, i32,
                                           ctypes.c_float, ctypes.c_float, i32, P, i64, P, ctypes.c_int]
        lib.replay_wedge_tasks.restype = ctypes.c_int
        lib.replay_num_counters.restype = ctypes.c_int
        assert lib.replay_num_counters() == len(COUNTERS)
        _lib = lib
    return _lib


def uniform_lamp(oz, coord_bound: float):
    """(wuniform, wz0, wrdz) of a vertical lamp with source heights oz, as the
    library decides them: evenly spaced within 1/64 of a step, and the step at
    least 2^-16 (16 B + 3 max|oz|) with B the scene's coordinate bound."""
    oz = np.asarray(oz, np.float32)
    K = oz.size
    z0 = float(oz[0])
    dz = (float(oz[K - 1]) - z0) / (K - 1)
    even = dz > 0.0 and np.isfinite(1.0 / dz)
    if even:
        even = all(abs(float(oz[m]) - (z0 + m * dz)) <= dz / 64.0 for m in range(K))
    offmax = float(np.abs(oz.astype(np.float64)).max())
    if even and not dz >= np.ldexp(16.0 * float(coord_bound) + 3.0 * offmax, -16):
        even = False
    return int(even), np.float32(z0), np.float32(1.0 / dz) if even else np.float32(0.0)


def sample_tasks(nc: int, np_: int, n: int, seed: int, cand_per_task: int = 4):
    """n distinct seeded tasks (candidate chunk, patch block) of an nc x np matrix."""
    nchunk = (nc + cand_per_task - 1) // cand_per_task
    njb = (np_ + 31) // 32
    total = nchunk * njb
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(total, size=min(n, total), replace=False))
    return np.stack([pick % nchunk, pick // nchunk], axis=1).astype(np.int64)


def replay(exported: dict, cand, lamp_offsets, tasks, cand_per_task: int = 4, threads: int = 0) -> dict:
    """Counters of the wedge traversal over `tasks` ((n, 2) int64 of (chunk,
    patch block)); `exported` is paper_2103_14137_gb300.scene_export_traversal's
    dict; lamp_offsets (K, 3) must be vertical."""
    off = np.asarray(lamp_offsets, np.float32).reshape(-1, 3)
    if np.any(off[:, :2] != 0):
        raise ValueError("the replay covers vertical line lamps (the wedge search)")
    oz = np.ascontiguousarray(off[:, 2])
    wu, wz0, wrdz = uniform_lamp(oz, exported["coord_bound"])
    cand = np.ascontiguousarray(cand, np.float32).reshape(-1, 3)
    tasks = np.ascontiguousarray(tasks, np.int64).reshape(-1, 2)
    out = np.zeros(len(COUNTERS), np.uint64)
    e = exported
    nt, np_ = e["tri"].shape[0], e["patch_s"].shape[0]
    ptr = lambda a: ctypes.c_void_p(np.ascontiguousarray(a).ctypes.data)  # noqa: E731
    keep = [np.ascontiguousarray(e[k]) for k in ("nodes4", "tri", "patch_s", "patch_n", "patch_excl")]
    rc = _load().replay_wedge_tasks(*[ptr(a) for a in keep], nt, np_, int(e["root"]), float(e["diameter"]),
                                    ptr(cand), cand.shape[0], ptr(oz), oz.size, wu, float(wz0), float(wrdz),
                                    int(cand_per_task), ptr(tasks), tasks.shape[0], ptr(out), int(threads))
    if rc != 0:
        raise ValueError("replay: invalid arguments")
    return dict(zip(COUNTERS, (int(x) for x in out)))


def bytes_per_pair(c: dict, K: int, vis: bool = True) -> dict:
    """Algorithmic bytes per pair from replay counters (per warp: fetched by
    the warp's loads; per lane: summed over the lanes that need them); the
    output is 4 B of A plus, when the visibility words are written, K bits."""
    pairs = max(1, c["pairs"])
    out_b = 4.0 + (K / 8.0 if vis else 0.0)
    per_warp = (c["node_visits"] * NODE_BYTES + c["leaf_step_unique"] * TRI_BYTES + c["cache_loads"] * TRI_BYTES
                + c["tasks"] * 32 * PATCH_BYTES) / pairs + out_b
    per_lane = (c["lane_node_visits"] * NODE_BYTES + c["leaf_loads"] * TRI_BYTES + c["cache_loads"] * TRI_BYTES
                + c["tasks"] * 32 * PATCH_BYTES) / pairs + out_b
    return {"per_warp": per_warp, "per_lane": per_lane, "output": out_b,
            "leaf_step_lane_occupancy": c["leaf_step_lanes"] / max(1, c["leaf_steps"]) / 32.0}
