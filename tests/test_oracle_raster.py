"""Pins of the visibility-cube oracle: a source at the centre of a closed cube
room sends P/6 to each wall (the pixel solid angles of a face sum to 4 pi / 6
and every pixel finds its wall), off-centre wall fluxes converge to the
walls' closed-form solid angles, an occluder casts its shadow, back faces
absorb, and the shared diagonal of each wall is marked ambiguous."""
import math

import numpy as np

import oracle


def cube_room(L=2.0, inward=True):
    """Six walls of [0, L]^3, two triangles each, with normals into the room."""
    c = np.array([[x, y, z] for z in (0, L) for y in (0, L) for x in (0, L)], np.float32)
    idx = lambda x, y, z: x + 2 * y + 4 * z  # noqa: E731
    quads = [  # (corner order around the wall, inward normal)
        ((idx(0, 0, 0), idx(1, 0, 0), idx(1, 1, 0), idx(0, 1, 0)), (0, 0, 1)),     # floor
        ((idx(0, 0, 1), idx(1, 0, 1), idx(1, 1, 1), idx(0, 1, 1)), (0, 0, -1)),    # ceiling
        ((idx(0, 0, 0), idx(1, 0, 0), idx(1, 0, 1), idx(0, 0, 1)), (0, 1, 0)),     # y = 0
        ((idx(0, 1, 0), idx(1, 1, 0), idx(1, 1, 1), idx(0, 1, 1)), (0, -1, 0)),    # y = L
        ((idx(0, 0, 0), idx(0, 1, 0), idx(0, 1, 1), idx(0, 0, 1)), (1, 0, 0)),     # x = 0
        ((idx(1, 0, 0), idx(1, 1, 0), idx(1, 1, 1), idx(1, 0, 1)), (-1, 0, 0)),    # x = L
    ]
    tris, nrm = [], []
    for (a, b, cc, d), n in quads:
        tris += [(a, b, cc), (a, cc, d)]
        nrm += [n, n] if inward else [tuple(-np.array(n))] * 2
    return c, np.array(tris, np.int32), np.array(nrm, np.float32)


def run(verts, tris, nrm, src, R, power=6.0, amb=True):
    return oracle.raster(verts, tris, nrm, np.array([src], np.float32), [[0, 0, 0]], [1.0], power, R,
                         ambiguity=amb)


def test_centre_of_cube_room_each_wall_gets_a_sixth():
    v, t, n = cube_room()
    for R in (8, 33):
        F, amb = run(v, t, n, (1.0, 1.0, 1.0), R)
        walls = F[0].reshape(6, 2).sum(1)
        np.testing.assert_allclose(walls, 1.0, rtol=1e-12)         # P / 6 with P = 6
        assert np.all(amb[0] > 0)                                    # the diagonals are shared edges


def rect_solid_angle(o, corners):
    """Solid angle of a planar quad as two triangles (van Oosterom-Strackee)."""
    def tri(a, b, c):
        R1, R2, R3 = a - o, b - o, c - o
        r1, r2, r3 = map(np.linalg.norm, (R1, R2, R3))
        num = abs(np.dot(R1, np.cross(R2, R3)))
        den = r1 * r2 * r3 + np.dot(R1, R2) * r3 + np.dot(R1, R3) * r2 + np.dot(R2, R3) * r1
        return 2 * math.atan2(num, den)
    a, b, c, d = corners
    return tri(a, b, c) + tri(a, c, d)


def test_off_centre_walls_converge_to_solid_angles():
    v, t, n = cube_room()
    src = np.array([0.6, 1.3, 0.9])
    want = np.array([rect_solid_angle(src, v[[t[2 * w][0], t[2 * w][1], t[2 * w][2], t[2 * w + 1][2]]])
                     for w in range(6)]) * 6.0 / (4 * math.pi)
    assert math.isclose(want.sum(), 6.0, rel_tol=1e-12)
    errs = []
    for R in (16, 32, 64):
        F, _ = run(v, t, n, src, R, amb=False)
        walls = F[0].reshape(6, 2).sum(1)
        assert math.isclose(walls.sum(), 6.0, rel_tol=1e-12)         # every pixel lands on some wall
        errs.append(np.abs(walls - want).max())
    assert errs[2] < errs[0] / 2.5 and errs[2] < 0.02, errs       # first order in the pixel size


def test_occluder_shadow_and_back_faces():
    v, t, n = cube_room()
    # a square facing the source (normal -z) whose projection on the +z face is
    # [-0.5, 0.5]^2, on pixel edges at R = 64: its pixels are exactly the ones it covers
    sq = np.array([[0.75, 0.75, 1.5], [1.25, 0.75, 1.5], [1.25, 1.25, 1.5], [0.75, 1.25, 1.5]], np.float32)
    v2 = np.concatenate([v, sq])
    t2 = np.concatenate([t, np.array([[8, 9, 10], [8, 10, 11]], np.int32)])
    n2 = np.concatenate([n, np.array([[0, 0, -1], [0, 0, -1]], np.float32)])
    src = (1.0, 1.0, 1.0)
    F, _ = run(v2, t2, n2, src, 64, amb=False)
    sq_flux = F[0, 12:].sum()
    want = rect_solid_angle(np.array(src), sq.astype(np.float64)) * 6.0 / (4 * math.pi)
    assert math.isclose(sq_flux, want, rel_tol=1e-12)
    assert math.isclose(F[0, 2:4].sum() + sq_flux, 1.0, rel_tol=1e-12)   # the ceiling loses exactly the shadow
    # the occluder seen from behind absorbs: its flux vanishes, the ceiling still loses the shadow
    F2, _ = run(v2, t2, np.concatenate([n, -n2[12:]]), src, 64, amb=False)
    assert F2[0, 12:].sum() == 0.0 and math.isclose(F2[0, 2:4].sum(), F[0, 2:4].sum(), rel_tol=1e-12)


def test_back_facing_wall_absorbs():
    v, t, n = cube_room()
    n[0:2] *= -1                                                      # floor turned away
    F, _ = run(v, t, n, (1.0, 1.0, 1.0), 16, amb=False)
    walls = F[0].reshape(6, 2).sum(1)
    assert walls[0] == 0.0 and np.allclose(walls[1:], 1.0, rtol=1e-12)


def test_pixel_solid_angles_cover_the_sphere():
    for R in (1, 7, 64):
        assert math.isclose(6 * oracle.pixel_solid_angles(R).sum(), 4 * math.pi, rel_tol=1e-12)


def test_edge_on_triangle_is_an_ambiguous_receiver():
    """A triangle in the plane y = 1 through the source (1, 1, 1) is met
    edge-on by the rays of the middle pixel row of the +z face (odd R, so that
    row's rays have no y component): an FP32 rasteriser may give those pixels
    to it or to the ceiling behind it, so the oracle marks their power
    ambiguous on both, although neither the exact ray cast nor the FP32 one
    hits the edge-on triangle."""
    v, t, n = cube_room()
    R = 9
    edge = np.array([[0.7, 1.0, 1.6], [1.3, 1.0, 1.6], [1.0, 1.0, 1.9]], np.float32)
    v2 = np.concatenate([v, edge])
    t2 = np.concatenate([t, np.array([[8, 9, 10]], np.int32)])
    n2 = np.concatenate([n, np.array([[0, 1, 0]], np.float32)])
    F, amb = run(v2, t2, n2, (1.0, 1.0, 1.0), R)
    assert F[0, 12] == 0.0                              # edge-on: no exact hit
    # pixels of the middle row of the +z face (face 4) whose ray passes through
    # the triangle's interior: u = (2 px + 1)/R - 1 with |u| < 0.5 (at z = 1.6
    # the triangle spans x in [0.7, 1.3]; at its apex it narrows, but the ray at
    # u reaches z = 1.6 inside it)
    om = oracle.pixel_solid_angles(R)                  # [py, px]
    py = (R - 1) // 2
    u = (2 * np.arange(R) + 1) / R - 1
    inside = np.abs(u) < 0.5
    want = 6.0 / (4 * math.pi) * om[py, inside].sum()
    assert want > 0
    assert amb[0, 12] >= want * (1 - 1e-12)
    # the same power is marked on the ceiling triangles that lie behind it
    assert amb[0, 2:4].sum() >= want * (1 - 1e-12)
    # the other pixels of the face stay unambiguous for the edge-on triangle
    assert amb[0, 12] <= 6.0 / (4 * math.pi) * om[py].sum() * (1 + 1e-12)
