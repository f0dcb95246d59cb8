"""Pins of the irradiance oracle against facts that do not come from the oracle.

Each pin takes `irr`, a callable with the signature of oracle.irradiance, so the
same checks run on the real oracle (test_oracle_pins.py) and on deliberately
broken copies of it (test_oracle_mutants.py), which must fail at least one pin.

Sources of truth used here:
  * hand-derived closed forms for a three-triangle scene (tests/golden)
  * exact rational arithmetic (fractions.Fraction) for segment/triangle meetings
  * symmetry: a mirror-image scene gives the mirror-image matrix
  * conservation: a lamp inside a closed box sends all of P onto the walls
  * the solid angle of a triangle (van Oosterom & Strackee 1983, cited by the
    paper for the closed-form irradiance of an unoccluded triangle)
  * superposition over lamp sources (Sec. IV-C, non-point light sources)
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np

from synth.mesh import MeshBuilder, mesh_box
from synth.scenes import patches_per_triangle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _expr(s: str) -> float:
    return float(eval(s, {"__builtins__": {}}, {"pi": math.pi}))  # fixture expressions only


def _hand_scene():
    d = json.load(open(os.path.join(GOLDEN, "hand_checked_scene.json")))
    tris_xyz = list(d["triangles"].values())
    verts = np.array([v for t in tris_xyz for v in t], np.float32)
    tris = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
    p = d["patch"]
    return d, verts, tris, p


def pin_hand_checked(irr):
    """Closed forms of the three-triangle scene: facing, off-axis, back-facing,
    occluded, segment-not-ray, exclusion, and a two-source lamp."""
    d, verts, tris, p = _hand_scene()
    cen = np.array([p["centroid"]], np.float32)
    nrm = np.array([p["normal"]], np.float32)
    P = d["power_W"]
    cases = d["point_lamp_cases"]
    cand = np.array([c["lamp"] for c in cases], np.float32)
    E, vis, _ = irr(verts, tris, cen, nrm, np.array([p["excl"]], np.int32), cand,
                    np.zeros((1, 3), np.float32), np.ones(1, np.float32), P)
    for k, c in enumerate(cases):
        want = _expr(c["E"])
        assert vis[k, 0, 0] == c["visible"], (c, vis[k, 0, 0])
        assert abs(E[k, 0] - want) <= 1e-13 * max(1.0, want), (c, E[k, 0], want)
    c = d["excluded_occluder_case"]
    E, vis, _ = irr(verts, tris, cen, nrm, np.array([c["excl"]], np.int32), np.array([c["lamp"]], np.float32),
                    np.zeros((1, 3), np.float32), np.ones(1, np.float32), P)
    assert vis[0, 0, 0] == 1 and abs(E[0, 0] - _expr(c["E"])) <= 1e-13, (E, vis)
    # with no exclusion at all, the patch's own triangle meets the segment only
    # at its end point (tau = 1), which the open segment does not contain
    E, vis, _ = irr(verts, tris, cen, nrm, np.array([[-1, -1]], np.int32), cand,
                    np.zeros((1, 3), np.float32), np.ones(1, np.float32), P)
    for k, c in enumerate(cases):
        assert vis[k, 0, 0] == c["visible"] and abs(E[k, 0] - _expr(c["E"])) <= 1e-13 * max(1.0, _expr(c["E"]))
    c = d["line_lamp_case"]
    E, vis, _ = irr(verts, tris, cen, nrm, np.array([p["excl"]], np.int32), np.array([c["candidate"]], np.float32),
                    np.array(c["offsets"], np.float32), np.array(c["weights"], np.float32), P)
    assert list(vis[0, 0]) == c["visible"]
    assert abs(E[0, 0] - _expr(c["E"])) <= 1e-13, (E[0, 0], _expr(c["E"]))


def _orient(a, b, c, d):
    """Sign of det[b-a, c-a, d-a] in exact rationals."""
    ab = [b[i] - a[i] for i in range(3)]
    ac = [c[i] - a[i] for i in range(3)]
    ad = [d[i] - a[i] for i in range(3)]
    det = (ab[0] * (ac[1] * ad[2] - ac[2] * ad[1]) - ab[1] * (ac[0] * ad[2] - ac[2] * ad[0])
           + ab[2] * (ac[0] * ad[1] - ac[1] * ad[0]))
    return (det > 0) - (det < 0)


def exact_segment_meets_triangle(o, s, a, b, c) -> bool:
    """Exact test: the open segment (o, s) meets the closed triangle abc.
    o and s strictly on opposite sides of the plane, and the line os passes
    through the closed triangle (three edge orientations share a sign)."""
    F = [tuple(Fraction(float(x)) for x in p) for p in (o, s, a, b, c)]
    o, s, a, b, c = F
    so, ss = _orient(a, b, c, o), _orient(a, b, c, s)
    if so == 0 or ss == 0 or so == ss:
        return False
    e = [_orient(o, s, a, b), _orient(o, s, b, c), _orient(o, s, c, a)]
    return all(x >= 0 for x in e) or all(x <= 0 for x in e)


def pin_exact_visibility(irr, seed=11, rounds=6):
    """Random occluders between patches (z<0, facing up) and sources (z>0):
    visibility equals 'no triangle meets the open segment' decided exactly."""
    rng = np.random.default_rng(seed)
    for _ in range(rounds):
        ntri = 6
        verts = np.concatenate([
            rng.uniform(-1.5, 1.5, size=(3 * ntri, 2)),
            rng.uniform(-0.8, 0.8, size=(3 * ntri, 1))], axis=1).astype(np.float32)
        tris = np.arange(3 * ntri, dtype=np.int32).reshape(-1, 3)
        nc, npch = 12, 15
        cand = np.concatenate([rng.uniform(-1, 1, (nc, 2)), rng.uniform(1.0, 2.0, (nc, 1))], axis=1).astype(np.float32)
        cen = np.concatenate([rng.uniform(-1, 1, (npch, 2)), rng.uniform(-2.0, -1.0, (npch, 1))], axis=1).astype(np.float32)
        nrm = np.tile(np.array([[0, 0, 1]], np.float32), (npch, 1))
        excl = -np.ones((npch, 2), np.int32)
        E, vis, flag = irr(verts, tris, cen, nrm, excl, cand, np.zeros((1, 3), np.float32),
                           np.ones(1, np.float32), 10.0, eps=1e-9)
        for i in range(nc):
            for j in range(npch):
                if flag[i, j]:
                    continue
                meets = any(exact_segment_meets_triangle(cand[i], cen[j], *verts[3 * t:3 * t + 3])
                            for t in range(ntri))
                assert vis[i, j, 0] == (0 if meets else 1), (i, j, meets)
                assert (E[i, j] > 0) == (not meets)


def _half_plane_scene():
    # receiver: floor grid on [-2,2]^2 at z=0, normals +z
    mb = MeshBuilder()
    mb.add(mesh_box([-2, -2, -1], [2, 2, 0], 0.25, free_side="out",
                    omit=((0, 0), (0, 1), (1, 0), (1, 1), (2, 0))))
    verts, tris, tnrm, _ = mb.finish()
    cen, nrm, area, excl = patches_per_triangle(verts, tris, tnrm)
    n_recv = tris.shape[0]
    # occluder: rectangle x in [-3,0], y in [-3,3] at z=1 (two triangles)
    occ_v = np.array([[-3, -3, 1], [0, -3, 1], [0, 3, 1], [-3, 3, 1]], np.float32)
    occ_t = np.array([[0, 2, 1], [0, 3, 2]], np.int32) + verts.shape[0]
    verts = np.concatenate([verts, occ_v])
    tris = np.concatenate([tris, occ_t])
    return verts, tris, cen.astype(np.float32), nrm.astype(np.float32), excl.astype(np.int32), n_recv


def pin_half_plane(irr):
    """Lamp at (0,0,2), occluding half-plane at z=1 over x<0: exactly the
    patches with x<0 are dark, the x>0 ones see the lamp unobstructed."""
    verts, tris, cen, nrm, excl, _ = _half_plane_scene()
    cand = np.array([[0, 0, 2]], np.float32)
    E, vis, flag = irr(verts, tris, cen, nrm, excl, cand, np.zeros((1, 3), np.float32), np.ones(1, np.float32), 80.0)
    x = cen[:, 0]
    assert np.all(x != 0)
    assert np.array_equal(vis[0, :, 0], (x > 0).astype(np.uint8))
    assert vis[0, :, 0].sum() * 2 == cen.shape[0]
    # lit side equals the same patches with the occluder removed
    E0, vis0, _ = irr(verts, tris[:-2], cen, nrm, excl, cand, np.zeros((1, 3), np.float32), np.ones(1, np.float32), 80.0)
    assert np.all(vis0 == 1)
    lit = x > 0
    assert np.array_equal(E[0, lit], E0[0, lit])
    assert np.all(E[0, ~lit] == 0.0)
    # the unoccluded field is symmetric under (x,y) -> (-x,-y) about the lamp axis
    key = {(round(float(a), 5), round(float(b), 5)): k for k, (a, b) in enumerate(cen[:, :2])}
    pairs = [(k, key[(round(-float(a), 5), round(-float(b), 5))]) for k, (a, b) in enumerate(cen[:, :2])
             if (round(-float(a), 5), round(-float(b), 5)) in key]
    assert len(pairs) > 100
    for k, m in pairs:
        assert abs(E0[0, k] - E0[0, m]) <= 1e-12 * E0[0, k]


def mirror_room():
    """A room mirror-symmetric about x=0: the half x>=0 (room half + half table)
    and its mirror image (x negated exactly, winding reversed); patches of the
    mirrored half are the exact mirror images of the original ones."""
    rng = np.random.default_rng(5)
    mb = MeshBuilder()
    mb.add(mesh_box([0, 0, 0], [2, 4, 3], 0.4, free_side="in", omit=((0, 0),), jitter=0.01, rng=rng))
    mb.add(mesh_box([0, 1.37, 0], [0.53, 2.01, 0.75], 0.2, free_side="out", omit=((0, 0), (2, 0)),
                    jitter=0.01, rng=rng))
    v, t, tn, _ = mb.finish()
    cen, nrm, area, excl = patches_per_triangle(v, t, tn)
    cen = cen.astype(np.float32)
    nrm = nrm.astype(np.float32)
    nt_half = t.shape[0]
    vm = v.copy()
    vm[:, 0] = -vm[:, 0]
    verts = np.concatenate([v, vm])
    tris = np.concatenate([t, t[:, [0, 2, 1]] + v.shape[0]])
    flip = np.array([-1, 1, 1], np.float32)
    cen = np.concatenate([cen, cen * flip])
    nrm = np.concatenate([nrm, nrm * flip])
    excl = np.concatenate([excl, np.where(excl >= 0, excl + nt_half, -1)]).astype(np.int32)
    mirror_patch = np.concatenate([np.arange(nt_half) + nt_half, np.arange(nt_half)])
    cand_half = np.array([[0.41, 0.77, 1.0], [1.33, 2.9, 1.6], [0.77, 3.31, 0.4], [1.6, 0.5, 2.2],
                          [0.25, 1.7, 1.1]], np.float32)
    cand = np.concatenate([cand_half, cand_half * flip])
    mirror_cand = np.concatenate([np.arange(5) + 5, np.arange(5)])
    return verts, tris, cen, nrm, excl, cand, mirror_cand, mirror_patch


def pin_mirror(irr):
    """Mirror-symmetric room: A[i', j'] = A[i, j] and identical visibility."""
    verts, tris, cen, nrm, excl, cand, mc, mp = mirror_room()
    # mirror centroids must be exact mirror images for the pin to hold
    assert np.array_equal(cen[mp, 0], -cen[:, 0]) and np.array_equal(cen[mp, 1:], cen[:, 1:])
    E, vis, flag = irr(verts, tris, cen, nrm, excl, cand, np.zeros((1, 3), np.float32), np.ones(1, np.float32), 80.0)
    Em = E[mc][:, mp]
    vm = vis[mc][:, mp]
    ok = (flag == 0) & (flag[mc][:, mp] == 0)
    assert ok.mean() > 0.99
    assert np.array_equal(vis[ok], vm[ok])
    assert np.all(np.abs(E[ok] - Em[ok]) <= 1e-12 * np.abs(E[ok]))
    assert 0.2 < (E > 0).mean() < 1.0     # the table occludes a part of the room


def closed_box(h):
    mb = MeshBuilder()
    mb.add(mesh_box([0, 0, 0], [4, 4, 3], h, free_side="in"))
    verts, tris, tnrm, _ = mb.finish()
    cen, nrm, area, excl = patches_per_triangle(verts, tris, tnrm)
    return verts, tris, cen.astype(np.float32), nrm.astype(np.float32), area, excl.astype(np.int32)


def pin_flux_conservation(irr):
    """A point lamp inside a closed box: sum_j E_j a_j -> P as patches shrink
    (every ray leaves through exactly one wall point; total solid angle 4 pi)."""
    P = 80.0
    errs = []
    for h in (0.5, 0.25):
        verts, tris, cen, nrm, area, excl = closed_box(h)
        cand = np.array([[1.7, 2.2, 1.3]], np.float32)
        E, vis, _ = irr(verts, tris, cen, nrm, excl, cand, np.zeros((1, 3), np.float32), np.ones(1, np.float32), P,
                        flags=False)
        assert np.all(vis == 1)
        errs.append(abs(float(E[0] @ area) - P) / P)
    assert errs[1] < 0.01, errs
    assert errs[1] < 0.5 * errs[0], errs       # converges with refinement


def solid_angle(o, a, b, c):
    """Solid angle of triangle abc seen from o (van Oosterom & Strackee 1983)."""
    r1, r2, r3 = (np.asarray(p, np.float64) - np.asarray(o, np.float64) for p in (a, b, c))
    l1, l2, l3 = (np.linalg.norm(r) for r in (r1, r2, r3))
    num = abs(np.dot(r1, np.cross(r2, r3)))
    den = l1 * l2 * l3 + np.dot(r1, r2) * l3 + np.dot(r1, r3) * l2 + np.dot(r2, r3) * l1
    return 2.0 * math.atan2(num, den)


def pin_solid_angle_limit(irr):
    """Unoccluded small triangle: E(centroid) * area -> P * Omega / (4 pi), the
    flux through the triangle, with an error shrinking like the size squared."""
    P = 80.0
    o = np.array([0.3, -0.2, 2.0])
    rels = []
    for size in (0.4, 0.2, 0.1):
        a = np.array([0.5, 0.1, 0.0])
        b = a + np.array([size, 0.0, 0.0])
        c = a + np.array([0.2 * size, 0.9 * size, 0.0])
        verts = np.array([a, b, c], np.float32)
        av, bv, cv = verts.astype(np.float64)
        cen = ((av + bv + cv) / 3.0).astype(np.float32)[None]
        area = 0.5 * np.linalg.norm(np.cross(bv - av, cv - av))
        E, vis, _ = irr(verts, np.array([[0, 1, 2]], np.int32), cen, np.array([[0, 0, 1]], np.float32),
                        np.array([[0, -1]], np.int32), o.astype(np.float32)[None],
                        np.zeros((1, 3), np.float32), np.ones(1, np.float32), P)
        flux = P * solid_angle(o.astype(np.float32), av, bv, cv) / (4.0 * math.pi)
        rels.append(abs(E[0, 0] * area - flux) / flux)
    assert rels[-1] < 1e-3, rels
    assert rels[1] < 0.35 * rels[0] and rels[2] < 0.35 * rels[1], rels


def pin_superposition(irr):
    """Lamp made of K sources = sum of K point lamps of power w_m P placed at
    fl32(c + off_m); K coincident sources = one source of the full power."""
    verts, tris, cen, nrm, excl, cand, _, _ = mirror_room()
    cand = cand[:4]
    P = 120.0
    off = np.array([[0, 0, 0.1], [0, 0, 0.4], [0.05, 0, 0.7]], np.float32)
    w = np.array([0.5, 0.3, 0.2], np.float32)
    E, vis, _ = irr(verts, tris, cen, nrm, excl, cand, off, w, P, flags=False)
    total = np.zeros_like(E)
    for m in range(3):
        src = (cand + off[m]).astype(np.float32)       # the FP32 source point
        Em, vm, _ = irr(verts, tris, cen, nrm, excl, src, np.zeros((1, 3), np.float32),
                        np.ones(1, np.float32), float(np.float64(w[m]) * P), flags=False)
        total += Em
        assert np.array_equal(vis[..., m], vm[..., 0])
    assert np.all(np.abs(E - total) <= 1e-12 * np.abs(total) + 1e-300)
    K = 4
    Ek, vk, _ = irr(verts, tris, cen, nrm, excl, cand, np.zeros((K, 3), np.float32),
                    np.full(K, 1.0 / K, np.float32), P, flags=False)
    E1, v1, _ = irr(verts, tris, cen, nrm, excl, cand, np.zeros((1, 3), np.float32), np.ones(1, np.float32), P,
                    flags=False)
    assert np.all(np.abs(Ek - E1) <= 1e-12 * E1 + 1e-300)
    assert np.all(vk == v1)


def pin_grazing_flags(irr):
    """Flag bits: segment through an occluder edge (bit 0), a triangle touching
    the source point (bit 1), source in the patch plane (bit 2); none otherwise."""
    cen = np.array([[0, 0, 0]], np.float32)
    nrm = np.array([[0, 0, 1]], np.float32)
    ex = np.array([[-1, -1]], np.int32)
    z3 = np.zeros((1, 3), np.float32)
    one = np.ones(1, np.float32)
    lamp = np.array([[0, 0, 2]], np.float32)

    def run(tri_v, cand=lamp):
        return irr(np.array(tri_v, np.float32), np.array([[0, 1, 2]], np.int32), cen, nrm, ex, cand, z3, one, 80.0,
                   eps=1e-6)

    _, _, f = run([[0, -1, 1], [0, 1, 1], [1, 0, 1]])          # edge x=0 crosses the segment
    assert f[0, 0] & 1
    _, _, f = run([[0.1, -1, 1], [0.1, 1, 1], [1, 0, 1]])      # 0.1 m clear
    assert f[0, 0] == 0
    _, _, f = run([[-1, -1, 2], [1, -1, 2], [0, 1, 2]])        # plane through the source point
    assert f[0, 0] & 2
    _, _, f = run([[5, 5, 1], [6, 5, 1], [5, 6, 1]], cand=np.array([[1, 0, 0]], np.float32))
    assert f[0, 0] & 4


ALL_PINS = [pin_hand_checked, pin_exact_visibility, pin_half_plane, pin_mirror, pin_flux_conservation,
            pin_solid_angle_limit, pin_superposition, pin_grazing_flags]
