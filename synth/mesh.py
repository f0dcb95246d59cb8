"""Seeded triangle meshes of axis-aligned boxes, welded per box.

This module only builds geometry (vertices, triangles, patch points); it holds
none of the irradiance arithmetic.  Both the CUDA path and the CPU oracle take
what it produces as plain FP32/int32 arrays.

Conventions
-----------
* Every triangle is wound so that its geometric normal (v1-v0)x(v2-v0) points
  into the free space (into the room for the shell, out of a furniture box).
* Faces of one box share their edge vertices (no T-junctions inside a box).
* Interior vertices of a face may be jittered tangentially, so faces stay
  exactly planar (all faces are axis-aligned planes).
* Cells of a face are emitted in Z-order (Morton order of the cell lattice),
  so consecutive triangles and patches are spatially close.
"""
from __future__ import annotations

import numpy as np


def _morton2(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Interleave the low 16 bits of a and b (a in the even bits)."""
    def spread(x):
        x = x.astype(np.uint64) & np.uint64(0xFFFF)
        x = (x | (x << np.uint64(8))) & np.uint64(0x00FF00FF)
        x = (x | (x << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        x = (x | (x << np.uint64(2))) & np.uint64(0x33333333)
        x = (x | (x << np.uint64(1))) & np.uint64(0x55555555)
        return x
    return spread(a) | (spread(b) << np.uint64(1))


class BoxMesh:
    """Triangles of one box; arrays in float64 until the scene is finalised."""

    def __init__(self, verts, tris, tri_normal, tri_cell):
        self.verts = verts            # (nv,3) float64 positions (already jittered)
        self.tris = tris              # (nt,3) int64 local vertex ids
        self.tri_normal = tri_normal  # (nt,3) float64 free-side unit normal (axis vector)
        self.tri_cell = tri_cell      # (nt,) int64 cell id local to the box (2 triangles per cell)


def mesh_box(lo, hi, h, free_side="out", omit=(), jitter=0.0, rng=None) -> BoxMesh:
    """Mesh the surface of the box [lo, hi] with cells of edge about h.

    free_side: "out" for a solid object (normals point away from the box),
               "in" for the room shell (normals point into the box).
    omit: faces left out, as (axis, side) pairs, side 0 = min face, 1 = max face.
    jitter: maximum tangential displacement of face-interior vertices (metres).
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ext = hi - lo
    n = np.maximum(1, np.rint(ext / h).astype(np.int64))
    stride = np.array([(n[1] + 1) * (n[2] + 1), n[2] + 1, 1], dtype=np.int64)

    keys_all, tris_all, normals_all, cells_all = [], [], [], []
    cell_base = 0
    for k in range(3):
        ka, kb = (k + 1) % 3, (k + 2) % 3
        nu, nv = int(n[ka]), int(n[kb])
        for s in (0, 1):
            if (k, s) in omit:
                continue
            outward = 1.0 if s == 1 else -1.0
            sign = outward if free_side == "out" else -outward
            a, b = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
            a = a.ravel()
            b = b.ravel()
            order = np.argsort(_morton2(a, b), kind="stable")
            a = a[order]
            b = b[order]

            def key(da, db):
                lat = np.zeros((a.size, 3), dtype=np.int64)
                lat[:, k] = s * n[k]
                lat[:, ka] = a + da
                lat[:, kb] = b + db
                return lat @ stride

            p00, p10, p11, p01 = key(0, 0), key(1, 0), key(1, 1), key(0, 1)
            if sign > 0:
                t1 = np.stack([p00, p10, p11], axis=1)
                t2 = np.stack([p00, p11, p01], axis=1)
            else:
                t1 = np.stack([p00, p11, p10], axis=1)
                t2 = np.stack([p00, p01, p11], axis=1)
            tri = np.empty((2 * a.size, 3), dtype=np.int64)
            tri[0::2] = t1
            tri[1::2] = t2
            nrm = np.zeros(3)
            nrm[k] = sign
            tris_all.append(tri)
            normals_all.append(np.repeat(nrm[None, :], tri.shape[0], axis=0))
            cells_all.append(cell_base + np.repeat(np.arange(a.size), 2))
            cell_base += a.size

    tris = np.concatenate(tris_all)
    used, inv = np.unique(tris.ravel(), return_inverse=True)
    tris = inv.reshape(-1, 3)
    lat = np.stack([used // stride[0], (used // stride[1]) % (n[1] + 1), used % (n[2] + 1)], axis=1)
    verts = lo[None, :] + ext[None, :] * (lat / n[None, :])
    if jitter > 0.0:
        extreme = (lat == 0) | (lat == n[None, :])
        interior = extreme.sum(axis=1) == 1
        d = rng.uniform(-jitter, jitter, size=verts.shape)
        d[extreme] = 0.0          # only tangential axes move
        d[~interior] = 0.0        # edge and corner vertices stay on the box edges
        verts = verts + d
    return BoxMesh(verts, tris, np.concatenate(normals_all), np.concatenate(cells_all))


class MeshBuilder:
    """Accumulates box meshes into one scene mesh."""

    def __init__(self):
        self.parts = []

    def add(self, m: BoxMesh):
        self.parts.append(m)

    def finish(self):
        verts, tris, nrm, cell = [], [], [], []
        vbase = 0
        cbase = 0
        for m in self.parts:
            verts.append(m.verts)
            tris.append(m.tris + vbase)
            nrm.append(m.tri_normal)
            cell.append(m.tri_cell + cbase)
            vbase += m.verts.shape[0]
            cbase += int(m.tri_cell.max()) + 1
        verts = np.concatenate(verts).astype(np.float32)
        tris = np.concatenate(tris).astype(np.int32)
        return verts, tris, np.concatenate(nrm), np.concatenate(cell)
