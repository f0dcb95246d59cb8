"""The oracle's CPU-BVH mode (uvco_irradiance_bvh) against its brute force:
identical entries, visibility bits and grazing flags, bit for bit, on the
tiny room in full, on sampled pairs of the ward room, and on degenerate
scenes (no triangle, one triangle, many copies of one triangle, a lamp inside
a closed box).  The hierarchy only skips triangles, so any difference would
be a box test that rejected a triangle the brute force counts."""
import numpy as np
import pytest

import oracle
from synth import tiny_room, ward_room
from synth.scenes import line_lamp, point_lamp


def _both(verts, tris, cen, nrm, excl, cand, L, pairs=None):
    a = oracle.irradiance(verts, tris, cen, nrm, excl, cand, L.offsets, L.weights, L.power, pairs=pairs)
    b = oracle.irradiance(verts, tris, cen, nrm, excl, cand, L.offsets, L.weights, L.power, pairs=pairs, bvh=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    return a


def test_tiny_room_full_matrix_identical():
    s = tiny_room()
    E, vis, flag = _both(s.verts, s.tris, s.centroid, s.normal, s.excl, s.cand, s.lamp)
    assert 0.2 < vis.mean() < 0.95


def test_tiny_room_line_lamp_identical():
    s = tiny_room(n_cand=40)
    cand = s.cand.copy()
    cand[:, 2] = 0.7
    _both(s.verts, s.tris, s.centroid, s.normal, s.excl, cand, line_lamp(1.0, 6, 90.0))


def test_ward_sampled_pairs_identical():
    s = ward_room()
    rng = np.random.default_rng(17)
    pairs = np.stack([rng.integers(0, s.nc, 1500), rng.integers(0, s.np_, 1500)], axis=1)
    E, vis, flag = _both(s.verts, s.tris, s.centroid, s.normal, s.excl, s.cand, s.lamp, pairs=pairs)
    assert 0.05 < vis.mean() < 0.95


@pytest.mark.parametrize("k", [0, 1, 300])
def test_degenerate_scenes_identical(k):
    rng = np.random.default_rng(k)
    tri = np.array([[-0.5, -0.5, 1], [0.5, -0.5, 1], [0, 0.5, 1]], np.float32)
    verts = np.tile(tri, (k, 1)).reshape(-1, 3) if k else np.zeros((0, 3), np.float32)
    tris = np.arange(3 * k, dtype=np.int32).reshape(-1, 3)
    cen = np.concatenate([rng.uniform(-1.5, 1.5, (60, 2)), np.zeros((60, 1))], axis=1).astype(np.float32)
    nrm = np.tile(np.array([[0, 0, 1]], np.float32), (60, 1))
    ex = -np.ones((60, 2), np.int32)
    cand = np.concatenate([rng.uniform(-1, 1, (7, 2)), np.full((7, 1), 2.0)], axis=1).astype(np.float32)
    _both(verts, tris, cen, nrm, ex, cand, point_lamp(50.0))


def test_closed_box_lamp_inside_identical():
    """Every segment ends on the box's own walls: the hierarchy must still find
    the neighbouring walls that grazing and exclusion are about."""
    s = tiny_room(n_cand=12)
    E, vis, flag = _both(s.verts, s.tris, s.centroid, s.normal, s.excl, s.cand, line_lamp(0.5, 3, 30.0))
    assert vis.any()


def _area_both(s, cand, L, pairs=None):
    args = (s.verts, s.tris, s.centroid, s.normal, s.area, s.excl, s.ptri, cand, L.offsets, L.weights, L.power)
    a = oracle.area_mean(*args, pairs=pairs)
    b = oracle.area_mean(*args, pairs=pairs, bvh=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    return a


def test_area_mean_tiny_room_identical():
    """uvco_area_mean_bvh against its brute force on the whole tiny-room
    matrix, with a line lamp across the table top's plane: the centroid and
    every pulled-in vertex segment go through the hierarchy."""
    s = tiny_room(n_cand=30)
    cand = s.cand.copy()
    cand[:, 2] = np.where(np.arange(30) % 2 == 0, 0.62, 1.0)
    E, ncl, flag = _area_both(s, cand, line_lamp(0.9, 5, 100.0))
    assert (ncl > 0).mean() > 0.2 and (ncl < 5).any()    # closed form and fallbacks both occur


def test_area_mean_ward_sampled_pairs_identical():
    s = ward_room()
    rng = np.random.default_rng(23)
    pairs = np.stack([rng.integers(0, s.nc, 1200), rng.integers(0, s.np_, 1200)], axis=1)
    E, ncl, flag = _area_both(s, s.cand, s.lamp, pairs=pairs)
    assert (ncl > 0).mean() > 0.05 and (E > 0).mean() > 0.05
