"""The seeded input generators (synth/) produce the workloads as specified:
sizes, candidate grids and heights, lamps, dwell vectors, and the mesh
conventions both sides rely on - triangles wound towards the free space,
axis-aligned planar faces after the tangential jitter, closed and consistently
oriented room shells (welded, no T-junctions), patches that partition their
triangles, and seed determinism."""
import math
from collections import Counter

import numpy as np
import pytest

from synth import dwell_vectors, large_floor, tiny_room, ward_room
from synth.batched import HEIGHTS, LAMPS, batched_room, design_candidates, designs, room_targets
from synth.scenes import line_lamp


def tri_normals(verts, tris):
    v = verts.astype(np.float64)
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    cr = np.cross(b - a, c - a)
    return cr / np.linalg.norm(cr, axis=1, keepdims=True), 0.5 * np.linalg.norm(cr, axis=1)


def test_tiny_room_sizes_and_candidates():
    s = tiny_room()
    assert (s.nt, s.np_, s.nc) == (988, 988, 200)
    assert s.lamp.K == 1 and s.lamp.power == 80.0 and np.all(s.lamp.offsets == 0)
    assert np.all(s.cand[:, 2] == 1.0)
    g = s.cand[:, :2] / 0.25
    assert np.allclose(g, np.rint(g), atol=1e-5)                        # 0.25 m grid
    assert s.cand[:, :2].min() >= 0.25 - 1e-6 and s.cand[:, :2].max() <= 3.75 + 1e-6
    # the first 200 points of the 15 x 15 grid in x-major order: the 0.1 m
    # clearance from the table box is tested in 3-D, and at 1.0 m every point
    # is already more than 0.1 m above the 0.75 m table top
    xs = np.arange(0.25, 3.75 + 1e-9, 0.25)
    grid = np.stack(np.meshgrid(xs, xs, indexing="ij"), axis=-1).reshape(-1, 2)[:200]
    assert np.allclose(s.cand[:, :2], grid)
    top = s.verts[s.verts[:, 2] == np.float32(0.75)]
    assert top.shape[0] > 0 and 1.0 - 0.75 > 0.1


def test_ward_room_sizes_lamp_and_candidates():
    s = ward_room()
    assert (s.nt, s.np_, s.nc) == (51_048, 102_030, 2_000)
    assert set(np.unique(s.cand[:, 2]).tolist()) == {0.5, 1.0, 1.5}
    g = s.cand[:, :2] / 0.2
    assert np.allclose(g, np.rint(g), atol=1e-4)                        # 0.2 m grid
    L = s.lamp
    assert L.K == 8 and L.power == 120.0
    assert np.all(L.offsets[:, :2] == 0) and np.allclose(L.offsets[:, 2], 1.2 * (np.arange(8) + 0.5) / 8)
    assert np.allclose(L.weights, 1 / 8) and math.isclose(float(L.weights.sum()), 1.0, rel_tol=1e-6)
    assert len(np.unique(s.cand, axis=0)) == s.nc


def test_line_lamp_midpoint_rule():
    L = line_lamp(1.8, 12, 120.0)
    assert np.allclose(np.diff(L.offsets[:, 2]), 0.15) and math.isclose(float(L.offsets[0, 2]), 0.075,
                                                                         rel_tol=1e-6)


@pytest.mark.parametrize("scene", ["tiny", "ward"])
def test_patches_partition_their_triangles(scene):
    s = tiny_room() if scene == "tiny" else ward_room()
    n, tarea = tri_normals(s.verts, s.tris)
    par = s.excl[:, 0]
    assert np.all((par >= 0) & (par < s.nt)) and np.all(s.excl[:, 1] == -1)
    # areas add up per parent triangle; normals are the parent's unit axis normal
    per = np.bincount(par, weights=s.area.astype(np.float64), minlength=s.nt)
    assert np.allclose(per, tarea, rtol=1e-5)
    assert np.allclose(s.normal, n[par], atol=1e-6)
    assert np.all(np.sort(np.abs(s.normal), axis=1)[:, :2] == 0) and np.all(np.abs(s.normal).max(axis=1) == 1)
    if scene == "ward":
        assert s.area.max() <= 0.005 * (1 + 1e-5)
    # the patch point lies on its parent triangle (inside it, on its plane)
    v = s.verts.astype(np.float64)
    a, b, c = v[s.tris[par, 0]], v[s.tris[par, 1]], v[s.tris[par, 2]]
    p = s.centroid.astype(np.float64)
    assert np.allclose(np.einsum("ij,ij->i", p - a, n[par]), 0, atol=1e-6)
    for e0, e1 in ((a, b), (b, c), (c, a)):
        side = np.einsum("ij,ij->i", np.cross(e1 - e0, p - e0), n[par])
        assert side.min() > -1e-9


def test_ptri_is_the_patch_geometry():
    s = ward_room()
    p = s.ptri.astype(np.float64)
    assert np.all(s.ptri[:, 1] == 0)                                     # one triangle per patch
    cr = np.cross(p[:, 0, 1] - p[:, 0, 0], p[:, 0, 2] - p[:, 0, 0])
    assert np.allclose(0.5 * np.linalg.norm(cr, axis=1), s.area, rtol=1e-4)
    assert np.allclose(p[:, 0].mean(axis=1), s.centroid, atol=1e-5)
    assert np.allclose(cr / np.linalg.norm(cr, axis=1, keepdims=True), s.normal, atol=1e-5)


def test_faces_are_axis_planes_and_wound_to_the_free_space():
    s = tiny_room()
    n, _ = tri_normals(s.verts, s.tris)
    ax = np.argmax(np.abs(n), axis=1)
    v = s.verts[s.tris]                                                  # (nt, 3, 3)
    k = np.take_along_axis(v, ax[:, None, None].repeat(3, axis=1), axis=2)[..., 0]
    assert np.all(k == k[:, :1])                                         # exactly planar after the jitter
    # room shell (first 960 triangles): normals point into the room
    W = np.array([4.0, 4.0, 3.0])
    shell = slice(0, 960)
    cen = v[shell].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", W / 2 - cen, n[shell]) > 0)
    # table (the rest): normals point out of the box
    tab = v[960:].reshape(-1, 3)
    mid = (tab.min(axis=0) + tab.max(axis=0)) / 2
    assert np.all(np.einsum("ij,ij->i", v[960:].mean(axis=1) - mid, n[960:]) > 0)


def test_room_shell_is_closed_and_consistently_oriented():
    """Every directed edge of the welded shell appears once and its reverse
    once: a closed, consistently oriented surface with no T-junction."""
    s = tiny_room()
    t = s.tris[:960]
    directed = Counter()
    for a, b, c in t:
        for e in ((a, b), (b, c), (c, a)):
            directed[(int(e[0]), int(e[1]))] += 1
    assert all(cnt == 1 for cnt in directed.values())
    assert all((b, a) in directed for (a, b) in directed)


def test_generators_are_seeded():
    a, b = ward_room(), ward_room()
    for f in ("verts", "tris", "centroid", "normal", "area", "excl", "cand"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = ward_room(seed=1001)
    assert not np.array_equal(a.verts, c.verts)
    t = dwell_vectors(16, 2000)
    assert t.shape == (16, 2000) and t.dtype == np.float32 and t.min() >= 0 and t.max() <= 60
    assert np.array_equal(t, dwell_vectors(16, 2000)) and not np.array_equal(t, dwell_vectors(16, 2000, seed=3))


def test_large_floor_structure_on_a_coarse_lattice():
    """The large floor's construction at a coarse cell size: quad patches of two
    consecutive triangles, both excluded, whose areas add up to the surface."""
    s = large_floor(h=0.5, n_cand=500)
    assert s.nt % 2 == 0 and s.np_ == s.nt // 2 and s.nc == 500
    assert np.array_equal(s.excl[:, 0], 2 * np.arange(s.np_)) and np.array_equal(s.excl[:, 1], s.excl[:, 0] + 1)
    _, tarea = tri_normals(s.verts, s.tris)
    assert np.allclose(s.area, tarea[0::2] + tarea[1::2], rtol=1e-5)
    assert set(np.unique(s.cand[:, 2]).tolist()) == {0.5, float(np.float32(1.2))} and s.lamp.K == 8


def test_batched_rooms_and_designs():
    assert len(designs()) == 12 == len(HEIGHTS) * len(LAMPS)
    for seed in (100, 101, 102, 103):
        nt_t, np_t, nc_t = room_targets(seed)
        assert 1e4 <= nt_t <= 2e5 and 5e3 <= np_t <= 3e5 and 500 <= nc_t <= 5000
        r = batched_room(seed)
        assert 0.8 * nt_t <= r.nt <= 1.25 * nt_t and r.np_ <= np_t
        for h, length, K in designs()[::4] + designs()[2::5]:
            cand = design_candidates(r, h, length, nc_t, seed=seed)
            assert cand.shape[0] <= nc_t and np.all(cand[:, 2] == np.float32(h))
            for lo, hi in r.info["box_list"]:                          # 0.15 m clear of the furniture
                near = np.all((cand[:, :2] > lo[:2] - 0.15) & (cand[:, :2] < hi[:2] + 0.15), axis=1)
                assert not (near & (h < hi[2] + 0.15)).any()
