"""Seeded rooms of uneven size and the robot-design sweep for batched runs.

Room r (seed = base + r) has log-uniform targets nt in [1e4, 2e5] triangles,
np in [5e3, 3e5] patches and nc in [500, 5000] candidates; a random box room
(3 m high) with furniture boxes standing on the floor.  The design sweep
crosses 4 lamp-bottom heights with 3 vertical line lamps (length, K):
(0.6 m, 4), (1.2 m, 8), (1.8 m, 12), all 120 W.  Geometry and inputs only.
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import MeshBuilder, mesh_box
from .scenes import (Scene, _clear_of, _finish, _grid_xy, line_lamp, patches_bisected,
                     patches_per_triangle, patches_quads)

HEIGHTS = (0.3, 0.5, 0.8, 1.1)
LAMPS = ((0.6, 4), (1.2, 8), (1.8, 12))
POWER = 120.0


def designs():
    """The 12 designs: (lamp-bottom height, lamp length, K)."""
    return [(h, L, K) for h in HEIGHTS for (L, K) in LAMPS]


def _log_uniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def room_targets(seed: int):
    rng = np.random.default_rng(seed)
    return (int(_log_uniform(rng, 1e4, 2e5)), int(_log_uniform(rng, 5e3, 3e5)), int(_log_uniform(rng, 500, 5000)))


def batched_room(seed: int) -> Scene:
    """One room of the batch, without candidates (they depend on the design)."""
    nt_t, np_t, nc_t = room_targets(seed)
    rng = np.random.default_rng(seed + 7919)
    W, D, H = rng.uniform(5.0, 14.0), rng.uniform(4.0, 11.0), 3.0
    boxes = []
    tries = 0
    nbox = int(rng.integers(2, 9))
    while len(boxes) < nbox and tries < 200:
        tries += 1
        w, d, h = rng.uniform(0.5, 2.2), rng.uniform(0.4, 1.2), rng.uniform(0.4, 1.9)
        x0, y0 = rng.uniform(0.05, W - w - 0.05), rng.uniform(0.05, D - d - 0.05)
        lo, hi = np.array([x0, y0, 0.0]), np.array([x0 + w, y0 + d, h])
        if all(hi[0] + 0.05 < b[0][0] or lo[0] > b[1][0] + 0.05 or hi[1] + 0.05 < b[0][1] or lo[1] > b[1][1] + 0.05
               for b in boxes):
            boxes.append((lo, hi))
    area = 2 * W * D + 2 * H * (W + D) + sum(
        (hi[0] - lo[0]) * (hi[1] - lo[1]) + 2 * hi[2] * ((hi[0] - lo[0]) + (hi[1] - lo[1])) for lo, hi in boxes)
    h = math.sqrt(area / (nt_t / 2.0))
    mb = MeshBuilder()
    mb.add(mesh_box([0, 0, 0], [W, D, H], h, free_side="in", jitter=min(0.01, 0.1 * h), rng=rng))
    for lo, hi in boxes:
        mb.add(mesh_box(lo, hi, h, free_side="out", omit=((2, 0),), jitter=min(0.01, 0.1 * h), rng=rng))
    verts, tris, tnrm, tcell = mb.finish()
    nt = tris.shape[0]
    if np_t >= nt:
        cen, nrm, ar, excl, ptri = patches_bisected(verts, tris, tnrm, float(area) / np_t, with_tris=True)
    elif np_t >= nt // 2:
        cen, nrm, ar, excl, ptri = patches_per_triangle(verts, tris, tnrm, with_tris=True)
    else:
        cen, nrm, ar, excl, ptri = patches_quads(verts, tris, tnrm, tcell, with_tris=True)
    if cen.shape[0] > np_t:        # seeded subset, kept in spatial order
        keep = np.sort(rng.choice(cen.shape[0], size=np_t, replace=False))
        cen, nrm, ar, excl, ptri = cen[keep], nrm[keep], ar[keep], excl[keep], ptri[keep]
    s = _finish(f"batch{seed}", verts, tris, cen, nrm, ar, excl, np.zeros((0, 3)), None,
                {"seed": seed, "room": [W, D, H], "boxes": len(boxes), "cell": h, "targets": [nt_t, np_t, nc_t]},
                ptri)
    s.info["box_list"] = boxes
    return s


def design_candidates(room: Scene, height: float, length: float, n: int, seed: int) -> np.ndarray:
    """n candidate lamp positions (lamp bottom) on a free floor grid at `height`,
    0.15 m clear of furniture over the lamp's length; seeded subsample."""
    W, D, _ = room.info["room"]
    free_area = W * D
    step = max(0.05, math.sqrt(free_area / (1.6 * n)))
    rng = np.random.default_rng(seed)
    while True:
        xy = _grid_xy(W, D, step, max(0.2, step))
        ok = _clear_of(xy, height, height + length, room.info["box_list"], 0.15)
        xy = xy[ok]
        if xy.shape[0] >= n or step < 0.06:
            break
        step *= 0.8
    pick = np.sort(rng.choice(xy.shape[0], size=min(n, xy.shape[0]), replace=False))
    xy = xy[pick]
    return np.concatenate([xy, np.full((xy.shape[0], 1), height)], axis=1).astype(np.float32)


def batch(n_rooms: int = 64, base_seed: int = 100):
    """Rooms and, per room and design, (candidates, lamp)."""
    out = []
    for r in range(n_rooms):
        room = batched_room(base_seed + r)
        nc = room.info["targets"][2]
        jobs = []
        for d, (hgt, L, K) in enumerate(designs()):
            cand = design_candidates(room, hgt, L, nc, seed=(base_seed + r) * 16 + d)
            jobs.append((cand, line_lamp(L, K, POWER), d))
        out.append((room, jobs))
    return out
