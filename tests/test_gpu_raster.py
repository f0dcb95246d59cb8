"""The visibility-cube rasteriser on the GPU against the FP64 ray-cast oracle:
per-triangle flux within the flux the oracle marks ambiguous (shared edges,
near misses, edge-on hits), the centre of a cube room, and the workspace
contract."""
import numpy as np
import pytest
import torch

import oracle
import paper_2103_14137_gb300 as uvc
from synth import tiny_room
from synth.scenes import line_lamp
from tests.gpu_util import T, build, build_arrays, lamp_of

pytestmark = pytest.mark.gpu


def tri_areas(verts, tris):
    v = np.asarray(verts, np.float32).astype(np.float64)
    t = np.asarray(tris)
    return 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)


def check(verts, tris, nrm, sc, cand, lamp, R):
    A = uvc.irradiance_raster(sc, T(nrm), T(cand), lamp_of(lamp), R=R, cand_per_batch=2)
    torch.cuda.synchronize()
    got = A.cpu().numpy().astype(np.float64) * tri_areas(verts, tris)[None, :]       # flux, W
    F, amb = oracle.raster(verts, tris, nrm, cand, lamp.offsets, lamp.weights, lamp.power, R)
    tol = amb + 1e-6 * F + 1e-9 * lamp.power
    bad = np.abs(got - F) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], F[bad][:5], amb[bad][:5])
    # the flux that reaches front faces never exceeds the lamp's power
    assert np.all(got.sum(1) <= lamp.power * (1 + 1e-6))
    return got, F, amb


@pytest.mark.parametrize("R", [32, 45])
def test_tiny_room_point_lamp(R):
    s = tiny_room()
    sc = build(s)
    cand = s.cand[[0, 37, 101, 199]]
    got, F, amb = check(s.verts, s.tris, s.normal, sc, cand, s.lamp, R)
    assert (amb.sum() / F.sum()) < 0.02                     # most flux is unambiguous
    assert got.sum(1).min() > 0.9 * s.lamp.power             # a closed room absorbs nearly everything
    sc.free()


def test_tiny_room_point_lamp_at_the_benchmark_resolution():
    """R = 512, the resolution the benchmark times, on the tiny room (988
    triangles, table included) from three candidates: every triangle's flux
    within the oracle's ambiguity bound, and under 2 % of the power ambiguous."""
    s = tiny_room()
    sc = build(s)
    cand = s.cand[[0, 112, 187]]
    got, F, amb = check(s.verts, s.tris, s.normal, sc, cand, s.lamp, 512)
    assert (amb.sum() / F.sum()) < 0.02
    assert got.sum(1).min() > 0.99 * s.lamp.power
    sc.free()


def test_tiny_room_line_lamp_batches():
    s = tiny_room()
    sc = build(s)
    lamp = line_lamp(0.6, 4, 120.0)
    cand = s.cand[[3, 50, 150]]                               # 3 candidates in batches of 2 (ragged)
    check(s.verts, s.tris, s.normal, sc, cand, lamp, 24)
    sc.free()


def cube_room(L=2.0):
    c = np.array([[x, y, z] for z in (0, L) for y in (0, L) for x in (0, L)], np.float32)
    i = lambda x, y, z: x + 2 * y + 4 * z  # noqa: E731
    quads = [((i(0, 0, 0), i(1, 0, 0), i(1, 1, 0), i(0, 1, 0)), (0, 0, 1)),
             ((i(0, 0, 1), i(1, 0, 1), i(1, 1, 1), i(0, 1, 1)), (0, 0, -1)),
             ((i(0, 0, 0), i(1, 0, 0), i(1, 0, 1), i(0, 0, 1)), (0, 1, 0)),
             ((i(0, 1, 0), i(1, 1, 0), i(1, 1, 1), i(0, 1, 1)), (0, -1, 0)),
             ((i(0, 0, 0), i(0, 1, 0), i(0, 1, 1), i(0, 0, 1)), (1, 0, 0)),
             ((i(1, 0, 0), i(1, 1, 0), i(1, 1, 1), i(1, 0, 1)), (-1, 0, 0))]
    tris, nrm = [], []
    for (a, b, cc, d), n in quads:
        tris += [(a, b, cc), (a, cc, d)]
        nrm += [n, n]
    return c, np.array(tris, np.int32), np.array(nrm, np.float32)


def test_cube_room_centre_gives_each_wall_a_sixth():
    v, t, n = cube_room()
    cen = v[t].mean(1)
    sc = build_arrays(v, t, cen, n, tri_areas(v, t), np.stack([np.arange(12), -np.ones(12)], 1))
    lamp = uvc.point_lamp(6.0)
    for R in (16, 64, 512):
        A = uvc.irradiance_raster(sc, T(n), T(np.array([[1.0, 1.0, 1.0]], np.float32)), lamp, R=R)
        walls = (A.cpu().numpy()[0].astype(np.float64) * tri_areas(v, t)).reshape(6, 2).sum(1)
        np.testing.assert_allclose(walls, 1.0, rtol=2e-6)
    sc.free()


def test_workspace_too_small_is_rejected():
    s = tiny_room(n_cand=3)
    sc = build(s)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(uvc.UvcError):
        uvc.irradiance_raster(sc, T(s.normal), T(s.cand), lamp_of(s.lamp), R=64, workspace=ws)
    sc.free()
