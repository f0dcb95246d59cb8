"""Seeded synthetic rooms, patches, candidate lamp positions, lamps and dwell vectors.

The paper evaluates on a hospital-ward CAD model decimated to 60k triangles with
8547 vantage candidates (Sec. V-C); that model is not available, so these seeded
procedural rooms of the same scale stand in for it.  Nothing here evaluates the
irradiance law: it only produces inputs, identical for the CUDA path and the oracle.

Scene arrays (all C-contiguous):
  verts    (nv,3) float32     tris  (nt,3) int32
  centroid (np,3) float32     normal (np,3) float32 (unit, into free space)
  area     (np,)  float32     excl  (np,2) int32 (triangles a patch sits on, -1 = none)
  cand     (nc,3) float32     lamp offsets (K,3) float32, weights (K,) float32, power P
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mesh import MeshBuilder, mesh_box


@dataclass
class Lamp:
    """A lamp made of K point sources: source m sits at candidate + offsets[m]
    and emits weights[m] * power watts (Sec. IV-C, non-point light sources)."""
    offsets: np.ndarray   # (K,3) float32
    weights: np.ndarray   # (K,)  float32, sums to 1
    power: float          # total radiant flux P in watts

    @property
    def K(self) -> int:
        return int(self.offsets.shape[0])


def point_lamp(power: float) -> Lamp:
    return Lamp(np.zeros((1, 3), np.float32), np.ones(1, np.float32), float(power))


def line_lamp(length: float, K: int, power: float) -> Lamp:
    """Vertical tube from the candidate point (its bottom) up to +length, as K
    evenly spaced equal-power point sources at the midpoints of K equal pieces."""
    z = length * (np.arange(K, dtype=np.float64) + 0.5) / K
    off = np.zeros((K, 3), np.float64)
    off[:, 2] = z
    return Lamp(off.astype(np.float32), np.full(K, 1.0 / K, np.float32), float(power))


@dataclass
class Scene:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    centroid: np.ndarray
    normal: np.ndarray
    area: np.ndarray
    excl: np.ndarray
    cand: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.float32))
    lamp: Lamp | None = None
    info: dict = field(default_factory=dict)
    ptri: np.ndarray | None = None   # (np, 2, 3, 3) patch geometry: one or two triangles (second all zero if unused)

    @property
    def nt(self):
        return int(self.tris.shape[0])

    @property
    def np_(self):
        return int(self.centroid.shape[0])

    @property
    def nc(self):
        return int(self.cand.shape[0])

    def diameter(self) -> float:
        """Diagonal of the axis-aligned box around the mesh (FP64)."""
        v = self.verts.astype(np.float64)
        return float(np.linalg.norm(v.max(axis=0) - v.min(axis=0)))


# ---------------------------------------------------------------------------
# patches
# ---------------------------------------------------------------------------

def _tri_geom(verts64, tris):
    a, b, c = verts64[tris[:, 0]], verts64[tris[:, 1]], verts64[tris[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    return a, b, c, area


def _ptri(a, b, c, a2=None, b2=None, c2=None):
    out = np.zeros((a.shape[0], 2, 3, 3), np.float32)
    out[:, 0, 0], out[:, 0, 1], out[:, 0, 2] = a, b, c
    if a2 is not None:
        out[:, 1, 0], out[:, 1, 1], out[:, 1, 2] = a2, b2, c2
    return out


def patches_per_triangle(verts, tris, tri_normal, with_tris=False):
    """One patch per triangle: its centroid, area and free-side normal (and,
    with_tris, the patch geometry (np, 2, 3, 3))."""
    v = verts.astype(np.float64)
    a, b, c, area = _tri_geom(v, tris)
    cen = (a + b + c) / 3.0
    excl = np.stack([np.arange(tris.shape[0]), -np.ones(tris.shape[0], np.int64)], axis=1)
    if with_tris:
        return cen, tri_normal, area, excl, _ptri(a, b, c)
    return cen, tri_normal, area, excl


def patches_bisected(verts, tris, tri_normal, amax, with_tris=False):
    """Split every triangle at the midpoint of its longest edge until each piece
    has area <= amax; each piece is a patch whose parent triangle is excluded."""
    v = verts.astype(np.float64)
    a, b, c, area = _tri_geom(v, tris)
    parent = np.arange(tris.shape[0])
    done_c, done_a, done_p, done_t = [], [], [], []
    while a.shape[0]:
        small = area <= amax
        done_c.append((a[small] + b[small] + c[small]) / 3.0)
        done_a.append(area[small])
        done_p.append(parent[small])
        if with_tris:
            done_t.append(_ptri(a[small], b[small], c[small]))
        a, b, c, parent, area = a[~small], b[~small], c[~small], parent[~small], area[~small]
        if not a.shape[0]:
            break
        lab = np.linalg.norm(b - a, axis=1)
        lbc = np.linalg.norm(c - b, axis=1)
        lca = np.linalg.norm(a - c, axis=1)
        # rotate so that the longest edge is (a,b)
        r1 = (lbc >= lab) & (lbc >= lca)
        r2 = (lca > lab) & (lca > lbc)
        a2 = np.where(r1[:, None], b, np.where(r2[:, None], c, a))
        b2 = np.where(r1[:, None], c, np.where(r2[:, None], a, b))
        c2 = np.where(r1[:, None], a, np.where(r2[:, None], b, c))
        m = 0.5 * (a2 + b2)
        a = np.concatenate([a2, m])
        b = np.concatenate([m, b2])
        c = np.concatenate([c2, c2])
        parent = np.concatenate([parent, parent])
        area = np.concatenate([area, area]) * 0.5
    cen = np.concatenate(done_c)
    ar = np.concatenate(done_a)
    par = np.concatenate(done_p)
    order = np.lexsort((np.arange(par.size), par))   # keep triangle order (spatial)
    cen, ar, par = cen[order], ar[order], par[order]
    excl = np.stack([par, -np.ones(par.size, np.int64)], axis=1)
    if with_tris:
        return cen, tri_normal[par], ar, excl, np.concatenate(done_t)[order]
    return cen, tri_normal[par], ar, excl


def patches_quads(verts, tris, tri_normal, tri_cell, with_tris=False):
    """One patch per cell (a quad made of two consecutive triangles): the area
    centroid of the quad; both triangles are excluded."""
    assert tris.shape[0] % 2 == 0 and np.all(tri_cell[0::2] == tri_cell[1::2])
    v = verts.astype(np.float64)
    a, b, c, area = _tri_geom(v, tris)
    g = (a + b + c) / 3.0
    w0, w1 = area[0::2], area[1::2]
    cen = (g[0::2] * w0[:, None] + g[1::2] * w1[:, None]) / (w0 + w1)[:, None]
    idx = np.arange(0, tris.shape[0], 2)
    excl = np.stack([idx, idx + 1], axis=1)
    if with_tris:
        return cen, tri_normal[0::2], w0 + w1, excl, _ptri(a[0::2], b[0::2], c[0::2], a[1::2], b[1::2], c[1::2])
    return cen, tri_normal[0::2], w0 + w1, excl


def _finish(name, verts, tris, cen, nrm, area, excl, cand, lamp, info, ptri=None):
    return Scene(
        ptri=None if ptri is None else np.ascontiguousarray(ptri, np.float32),
        name=name,
        verts=np.ascontiguousarray(verts, np.float32),
        tris=np.ascontiguousarray(tris, np.int32),
        centroid=np.ascontiguousarray(cen, np.float32),
        normal=np.ascontiguousarray(nrm, np.float32),
        area=np.ascontiguousarray(area, np.float32),
        excl=np.ascontiguousarray(excl, np.int32),
        cand=np.ascontiguousarray(cand, np.float32),
        lamp=lamp,
        info=info,
    )


# ---------------------------------------------------------------------------
# candidates
# ---------------------------------------------------------------------------

def _grid_xy(W, D, step, inset):
    xs = np.arange(inset, W - inset + 1e-9, step)
    ys = np.arange(inset, D - inset + 1e-9, step)
    gx, gy = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel()], axis=1)


def _clear_of(xy, z0, z1, boxes, margin):
    """True where the vertical segment x=y=xy, z in [z0,z1] keeps `margin`
    away from every box (lo, hi)."""
    ok = np.ones(xy.shape[0], bool)
    for lo, hi in boxes:
        inside_xy = ((xy[:, 0] > lo[0] - margin) & (xy[:, 0] < hi[0] + margin) &
                     (xy[:, 1] > lo[1] - margin) & (xy[:, 1] < hi[1] + margin))
        overlap_z = (z1 > lo[2] - margin) & (z0 < hi[2] + margin)
        ok &= ~(inside_xy & overlap_z)
    return ok


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def tiny_room(seed: int = 0, n_cand: int = 200) -> Scene:
    """4x4x3 m room with one 1x0.6x0.75 m table; ~1,000 triangles; one patch per
    triangle; 200 candidates on a 0.25 m floor grid at 1.0 m; point lamp, 80 W."""
    rng = np.random.default_rng(seed)
    W, D, H = 4.0, 4.0, 3.0
    mb = MeshBuilder()
    mb.add(mesh_box([0, 0, 0], [W, D, H], 0.42, free_side="in", jitter=0.01, rng=rng))
    tx = 1.3 + rng.uniform(0.0, 0.2)
    ty = 1.6 + rng.uniform(0.0, 0.2)
    table = (np.array([tx, ty, 0.0]), np.array([tx + 1.0, ty + 0.6, 0.75]))
    mb.add(mesh_box(table[0], table[1], 0.42, free_side="out", omit=((2, 0),), jitter=0.01, rng=rng))
    verts, tris, tnrm, tcell = mb.finish()
    cen, nrm, area, excl, ptri = patches_per_triangle(verts, tris, tnrm, with_tris=True)
    xy = _grid_xy(W, D, 0.25, 0.25)
    ok = _clear_of(xy, 1.0, 1.0, [table], 0.1)
    xy = xy[ok][:n_cand]
    cand = np.concatenate([xy, np.full((xy.shape[0], 1), 1.0)], axis=1)
    return _finish("tiny", verts, tris, cen, nrm, area, excl, cand, point_lamp(80.0),
                   {"seed": seed, "room": [W, D, H]}, ptri)


def ward_room(seed: int = 1, n_cand: int = 2000, h: float = 0.1165, amax: float = 0.005,
              lamp_len: float = 1.2, K: int = 8, power: float = 120.0) -> Scene:
    """10x8x3 m ward with 6 beds (2x1x0.6 m), 4 cabinets and 2 partition walls;
    ~50k triangles, each bisected into patches of area <= amax (~100k); 2,000
    candidates on a 0.2 m free grid at lamp-bottom heights 0.5/1.0/1.5 m;
    vertical 1.2 m line lamp with K=8 sources and P=120 W."""
    rng = np.random.default_rng(seed)
    W, D, H = 10.0, 8.0, 3.0
    boxes = []
    # beds along the two long walls, seeded offsets off the cell lattice
    for r in range(3):
        for side in (0, 1):
            x0 = 0.6 + 3.1 * r + rng.uniform(0.0, 0.15)
            # beds run along y (2 m) from the wall into the room
            if side == 0:
                lo, hi = [x0, 0.05 + rng.uniform(0, 0.05), 0.0], [x0 + 1.0, 2.05, 0.6]
            else:
                lo, hi = [x0, D - 2.05, 0.0], [x0 + 1.0, D - 0.05 - rng.uniform(0, 0.05), 0.6]
            boxes.append((np.array(lo), np.array(hi)))
    # cabinets beside the head of the first and last beds
    for x0, y0 in ((1.85, 0.04), (8.05, 0.04), (1.85, D - 0.54), (8.05, D - 0.54)):
        x0 += rng.uniform(0.0, 0.08)
        boxes.append((np.array([x0, y0, 0.0]), np.array([x0 + 0.6, y0 + 0.5, 1.8])))
    # two partition walls (not reaching the ceiling) between bed bays
    for x0 in (3.27, 6.37):
        x0 += rng.uniform(0.0, 0.06)
        boxes.append((np.array([x0, 2.4, 0.0]), np.array([x0 + 0.1, 5.6, 2.0])))
    mb = MeshBuilder()
    mb.add(mesh_box([0, 0, 0], [W, D, H], h, free_side="in", jitter=0.01, rng=rng))
    for lo, hi in boxes:
        mb.add(mesh_box(lo, hi, h, free_side="out", omit=((2, 0),), jitter=0.01, rng=rng))
    verts, tris, tnrm, tcell = mb.finish()
    cen, nrm, area, excl, ptri = patches_bisected(verts, tris, tnrm, amax, with_tris=True)
    cands = []
    xy = _grid_xy(W, D, 0.2, 0.2)
    for zb in (0.5, 1.0, 1.5):
        ok = _clear_of(xy, zb, zb + lamp_len, boxes, 0.15)
        cands.append(np.concatenate([xy[ok], np.full((int(ok.sum()), 1), zb)], axis=1))
    cands = np.concatenate(cands)
    pick = np.sort(rng.choice(cands.shape[0], size=min(n_cand, cands.shape[0]), replace=False))
    lamp = line_lamp(lamp_len, K, power)
    return _finish("ward", verts, tris, cen, nrm, area, excl, cands[pick], lamp,
                   {"seed": seed, "room": [W, D, H], "boxes": len(boxes), "cell": h, "amax": amax}, ptri)


def large_floor(seed: int = 3, n_cand: int = 10000, h: float = 0.0638, K: int = 8,
                lamp_len: float = 1.2, power: float = 120.0) -> Scene:
    """30x30x3 m floor: 20 rooms (two rows of 10) joined by a 3 m corridor, with
    doors, furniture boxes; ~2M triangles; one patch per cell (quad of two
    triangles, ~1M); 10,000 candidates at lamp-bottom heights 0.5/1.2 m."""
    rng = np.random.default_rng(seed)
    W, D, H = 30.0, 30.0, 3.0
    t = 0.1
    walls = []
    c0, c1 = 13.5, 16.5
    for yw in (c0 - t, c1):                      # corridor walls with one door per room
        xs = 0.0
        for r in range(10):
            door = r * 3.0 + 1.0 + rng.uniform(0.0, 0.5)
            if door - xs > 0.05:
                walls.append((np.array([xs + 0.02, yw, 0.0]), np.array([door, yw + t, H])))
            xs = door + 1.0
        walls.append((np.array([xs, yw, 0.0]), np.array([W - 0.02, yw + t, H])))
    for r in range(1, 10):                       # partitions between rooms
        x0 = 3.0 * r - t / 2
        walls.append((np.array([x0, 0.02, 0.0]), np.array([x0 + t, c0 - t - 0.02, H])))
        walls.append((np.array([x0, c1 + t + 0.02, 0.0]), np.array([x0 + t, D - 0.02, H])))
    furn = []
    for r in range(10):
        for (ya, yb) in ((0.3, c0 - 0.6), (c1 + 0.6, D - 0.3)):
            x0 = 3.0 * r + 0.4 + rng.uniform(0.0, 0.3)
            y0 = ya + rng.uniform(0.0, 1.0)
            furn.append((np.array([x0, y0, 0.0]), np.array([x0 + 1.0, y0 + 2.0, 0.6])))
            y1 = yb - 1.2 - rng.uniform(0.0, 1.0)
            furn.append((np.array([x0 + 1.3, y1, 0.0]), np.array([x0 + 1.9, y1 + 0.5, 1.5])))
    mb = MeshBuilder()
    mb.add(mesh_box([0, 0, 0], [W, D, H], h, free_side="in", jitter=0.01, rng=rng))
    for lo, hi in walls:
        mb.add(mesh_box(lo, hi, h, free_side="out", omit=((2, 0), (2, 1)), jitter=0.01, rng=rng))
    for lo, hi in furn:
        mb.add(mesh_box(lo, hi, h, free_side="out", omit=((2, 0),), jitter=0.01, rng=rng))
    verts, tris, tnrm, tcell = mb.finish()
    cen, nrm, area, excl = patches_quads(verts, tris, tnrm, tcell)
    boxes = walls + furn
    cands = []
    xy = _grid_xy(W, D, 0.25, 0.25)
    for zb in (0.5, 1.2):
        ok = _clear_of(xy, zb, zb + lamp_len, boxes, 0.15)
        cands.append(np.concatenate([xy[ok], np.full((int(ok.sum()), 1), zb)], axis=1))
    cands = np.concatenate(cands)
    pick = np.sort(rng.choice(cands.shape[0], size=min(n_cand, cands.shape[0]), replace=False))
    return _finish("large", verts, tris, cen, nrm, area, excl, cands[pick], line_lamp(lamp_len, K, power),
                   {"seed": seed, "room": [W, D, H], "boxes": len(boxes), "cell": h})


def dwell_vectors(nvec: int, nc: int, seed: int = 2, tmax: float = 60.0) -> np.ndarray:
    """nvec dwell-time vectors t (seconds), uniform in [0, tmax], (nvec, nc) float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, tmax, size=(nvec, nc)).astype(np.float32)
