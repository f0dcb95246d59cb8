"""Pins of the area-mean oracle: solid angles with known closed forms, dense
quadrature of cos/d^2 over a triangle, the hybrid's fallback to the centroid
sample when a check segment is blocked, the facing rule, and convergence of
the closed form to the centroid sample as the patch shrinks."""
import math

import numpy as np

import oracle


def one_patch(tri_list, normal, area, occluders=(), source=(0.0, 0.0, 0.0), power=1.0):
    """A scene holding the patch's own triangles (excluded) plus occluders."""
    tris = [np.asarray(t, np.float64) for t in tri_list] + [np.asarray(t, np.float64) for t in occluders]
    verts = np.concatenate(tris).astype(np.float32)
    T = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
    ptri = np.zeros((1, 2, 3, 3), np.float32)
    for k, t in enumerate(tri_list):
        ptri[0, k] = t
    w = np.array([0.5 * np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0])) for t in tris[:len(tri_list)]])
    cen = sum(wk * tk.mean(0) for wk, tk in zip(w, tris)) / w.sum()
    excl = np.array([[0, 1 if len(tri_list) == 2 else -1]], np.int32)
    E, ncl, _ = oracle.area_mean(verts, T, cen[None], np.asarray(normal, np.float32)[None], [area], excl, ptri,
                                 np.asarray(source, np.float32)[None], [[0.0, 0.0, 0.0]], [1.0], power, flags=False)
    return float(E[0, 0]), int(ncl[0, 0]), cen


def test_octant_triangle_subtends_an_eighth_of_the_sphere():
    t = np.eye(3)
    area = float(np.float32(math.sqrt(3) / 2))              # the area as the library stores it
    E, ncl, _ = one_patch([t], -np.ones(3) / math.sqrt(3), area)
    # Omega = 4 pi / 8: flux P / 8 over the area
    assert ncl == 1 and math.isclose(E, (1 / 8) / area, rel_tol=1e-12)


def square(a, z=0.0):
    h = a / 2
    p = np.array([[-h, -h, z], [h, -h, z], [h, h, z], [-h, h, z]])
    return [p[[0, 1, 2]], p[[0, 2, 3]]]


def test_square_on_axis():
    for a, h in ((2.0, 1.0), (0.5, 3.0), (3.0, 0.25)):            # all exact in binary32
        E, ncl, _ = one_patch(square(a), [0, 0, 1], a * a, source=(0, 0, h), power=7.0)
        omega = 4 * math.asin(a * a / (a * a + 4 * h * h))
        assert ncl == 1 and math.isclose(E, 7.0 * omega / (4 * math.pi * a * a), rel_tol=1e-9)


def subdivide(t, levels):
    tris = [np.asarray(t, np.float64)]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]), np.array([ab, bc, ca])]
        tris = nxt
    return np.array(tris)


def test_closed_form_equals_dense_quadrature():
    rng = np.random.default_rng(2)
    for _ in range(3):
        t = rng.uniform(-1, 1, (3, 3))
        n = np.cross(t[1] - t[0], t[2] - t[0])
        area = 0.5 * np.linalg.norm(n)
        n /= np.linalg.norm(n)
        src = t.mean(0) + n * rng.uniform(0.8, 2.0) + rng.uniform(-0.3, 0.3, 3)
        t32 = t.astype(np.float32).astype(np.float64)
        src32 = src.astype(np.float32).astype(np.float64)
        E, ncl, _ = one_patch([t32], n, area, source=src32, power=1.0)
        n32 = np.cross(t32[1] - t32[0], t32[2] - t32[0])
        n32 /= np.linalg.norm(n32)

        def quad(levels):                                    # centroid rule on 4^levels pieces
            sub = subdivide(t32, levels)
            g = sub.mean(1)
            w = 0.5 * np.linalg.norm(np.cross(sub[:, 1] - sub[:, 0], sub[:, 2] - sub[:, 0]), axis=1)
            v = src32 - g
            d = np.linalg.norm(v, axis=1)
            return np.sum(w * (v @ n32) / (4 * math.pi * d ** 3)), w.sum()
        (q6, wsum), (q7, _) = quad(6), quad(7)
        flux = q7 + (q7 - q6) / 3                            # Richardson: the rule's error is O(h^2)
        A32 = float(np.float32(area))
        assert ncl == 1 and math.isclose(E * A32, flux, rel_tol=1e-6), (E * A32, flux, q6, q7)


def test_blocked_vertex_falls_back_to_the_centroid_sample():
    occ = np.array([[0.4, 0.4, 1.0], [0.6, 0.4, 1.0], [0.5, 0.6, 1.0]])   # on the way to vertex (1, 1, 0) only
    E, ncl, _ = one_patch(square(2.0), [0, 0, 1], 4.0, occluders=[occ], source=(0, 0, 2), power=3.0)
    assert ncl == 0 and math.isclose(E, 3.0 / (4 * math.pi * 4.0), rel_tol=1e-12)
    # the same occluder moved off the check segments changes nothing
    E2, ncl2, _ = one_patch(square(2.0), [0, 0, 1], 4.0, occluders=[occ + [0, 0, 5.0]], source=(0, 0, 2), power=3.0)
    omega = 4 * math.asin(4.0 / (4.0 + 16.0))
    assert ncl2 == 1 and math.isclose(E2, 3.0 * omega / (4 * math.pi * 4.0), rel_tol=1e-9)


def test_off_axis_fallback_keeps_the_cosine():
    """A source off the patch's axis with only one check segment blocked: the
    centroid sample P cos / (4 pi d^2), cos = h / d."""
    src = np.array([0.625, -0.375, 2.0])                                   # exact in binary32
    occ = np.array([[0.76, 0.26, 1.0], [0.86, 0.26, 1.0], [0.81, 0.36, 1.0]])   # halfway to vertex (1, 1, 0)
    E, ncl, _ = one_patch(square(2.0), [0, 0, 1], 4.0, occluders=[occ], source=src, power=3.0)
    d = float(np.linalg.norm(src))
    assert ncl == 0 and math.isclose(E, 3.0 * (2.0 / d) / (4 * math.pi * d * d), rel_tol=1e-12)


def test_source_behind_the_patch_gives_zero():
    E, ncl, _ = one_patch(square(1.0), [0, 0, 1], 1.0, source=(0.1, 0.2, -1.0))
    assert E == 0.0 and ncl == 0


def test_closed_form_tends_to_the_centroid_sample():
    errs = []
    for a in (0.4, 0.2, 0.1, 0.05):
        E, _, _ = one_patch(square(a), [0, 0, 1], a * a, source=(0.3, 0.1, 1.0))
        v = np.array([0.3, 0.1, 1.0])
        point = v[2] / (4 * math.pi * np.linalg.norm(v) ** 3)
        errs.append(abs(E / point - 1))
    # second-order convergence: halving the patch divides the error by ~4
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.0 < e0 / e1 < 5.0, errs


def closed_box(size, n):
    """The inside of an axis-aligned box [0, size]: every face an n x n grid of
    quad patches (two triangles each, normals into the box)."""
    size = np.asarray(size, np.float64)
    centre = size / 2
    verts, quads = [], []
    for ax in range(3):
        u, v = [k for k in range(3) if k != ax]
        for side in (0.0, size[ax]):
            for i in range(n):
                for j in range(n):
                    q = np.zeros((4, 3))
                    for c, (di, dj) in enumerate(((0, 0), (1, 0), (1, 1), (0, 1))):
                        q[c, ax] = side
                        q[c, u] = size[u] * (i + di) / n
                        q[c, v] = size[v] * (j + dj) / n
                    t0, t1 = q[[0, 1, 2]], q[[0, 2, 3]]
                    nrm = np.cross(t0[1] - t0[0], t0[2] - t0[0])
                    if nrm @ (centre - t0[0]) < 0:          # wind both triangles towards the inside
                        t0, t1 = t0[[0, 2, 1]], t1[[0, 2, 1]]
                    quads.append((t0, t1))
    nq = len(quads)
    tri = np.array([t for q in quads for t in q], np.float32)
    verts = tri.reshape(-1, 3)
    T = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
    ptri = tri.reshape(nq, 2, 3, 3)
    p64 = ptri.astype(np.float64)
    cr = np.cross(p64[:, 0, 1] - p64[:, 0, 0], p64[:, 0, 2] - p64[:, 0, 0])
    normal = (cr / np.linalg.norm(cr, axis=1, keepdims=True)).astype(np.float32)
    area = (0.5 * (np.linalg.norm(cr, axis=1)
                   + np.linalg.norm(np.cross(p64[:, 1, 1] - p64[:, 1, 0], p64[:, 1, 2] - p64[:, 1, 0]), axis=1))
            ).astype(np.float32)
    cen = p64.reshape(nq, 6, 3).mean(axis=1).astype(np.float32)
    excl = np.stack([2 * np.arange(nq), 2 * np.arange(nq) + 1], axis=1).astype(np.int32)
    return verts, T, cen, normal, area, excl, ptri


def test_closed_box_receives_all_the_power():
    """A source inside a closed box sees every patch whole, and the patches'
    solid angles add up to the full sphere: sum_j E_j a_j = P exactly (up to
    FP64 rounding) for a point lamp and for a line lamp, every source using the
    closed form.  A wrong normalisation, solid-angle factor or a dropped
    second patch triangle would miss P."""
    verts, T, cen, nrm, area, excl, ptri = closed_box((4.0, 3.0, 2.5), 5)
    lamps = [([[0.0, 0.0, 0.0]], [1.0]),
             ([[0.0, 0.0, 0.2 + 0.4 * m] for m in range(4)], [0.25] * 4)]
    for off, w in lamps:
        E, ncl, flag = oracle.area_mean(verts, T, cen, nrm, area, excl, ptri, [[1.3, 1.1, 0.55]], off, w, 60.0)
        assert np.all(ncl == len(w))
        flux = float(np.sum(E[0] * area.astype(np.float64)))
        assert math.isclose(flux, 60.0, rel_tol=1e-10), flux
        # the centroid sample alone does not conserve the flux on these coarse patches
        Ec, _, _ = oracle.irradiance(verts, T, cen, nrm, excl, [[1.3, 1.1, 0.55]], off, w, 60.0, flags=False)
        assert abs(float(np.sum(Ec[0] * area)) - 60.0) > 1e-3 * 60.0


def test_partial_shadow_missed_by_the_checks_against_dense_quadrature():
    """How far the hybrid departs from the exact area mean of Eq. (4) when an
    occluder shadows part of a patch but none of its check points: the exact
    mean, by the midpoint rule on a 256 x 256 grid whose every point is tested
    for visibility by the oracle's own brute-force segment test, is smaller
    than the hybrid's closed form by the shadowed share of the flux, and the
    hybrid equals the unoccluded mean.  (Source 2 m above a 2 x 2 m patch, a
    small triangle at 1 m shadowing about 1 % of it near the middle of an
    edge, clear of the centroid and of the vertex checks.)"""
    a, h, P = 2.0, 2.0, 1.0
    occ = np.array([[0.33, -0.08, 1.0], [0.47, -0.08, 1.0], [0.40, 0.08, 1.0]])
    E_h, ncl, _ = one_patch(square(a), [0, 0, 1], a * a, occluders=[occ], source=(0, 0, h), power=P)
    omega = 4 * math.asin(a * a / (a * a + 4 * h * h))
    closed = P * omega / (4 * math.pi * a * a)
    assert ncl == 1 and math.isclose(E_h, closed, rel_tol=1e-9)          # every check passes
    n = 256
    c = (np.arange(n) + 0.5) / n * a - a / 2
    gx, gy = np.meshgrid(c, c, indexing="ij")
    pts = np.stack([gx.ravel(), gy.ravel(), np.zeros(n * n)], 1).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (n * n, 1))
    excl = np.tile(np.array([0, 1], np.int32), (n * n, 1))              # the patch's own triangles

    def grid_mean(with_occluder):
        tris = [np.asarray(t, np.float64) for t in square(a)] + ([occ] if with_occluder else [])
        verts = np.concatenate(tris).astype(np.float32)
        T = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
        E, _, _ = oracle.irradiance(verts, T, pts, nrm, excl, np.array([[0, 0, h]], np.float32),
                                    [[0.0, 0.0, 0.0]], [1.0], P, flags=False)
        return float(E.mean())
    free, shadowed = grid_mean(False), grid_mean(True)
    assert math.isclose(free, closed, rel_tol=2e-5)                        # the grid's own error
    share = 1.0 - shadowed / free
    assert 0.005 < share < 0.02                                            # about 1 % of the flux is shadowed
    departure = E_h / shadowed - 1.0
    assert math.isclose(departure, free / shadowed - 1.0, rel_tol=5e-3)    # the hybrid misses exactly that
    print(f"hybrid area mean {E_h:.6e} vs exact {shadowed:.6e}: {departure * 100:.2f} % high "
          f"({share * 100:.2f} % of the flux shadowed)")
