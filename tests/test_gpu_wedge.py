"""Wedge traversal of vertical line lamps (uvc_set_wedge_traversal) against
the source-by-source traversal and the FP64 oracle.

The wedge path must give each source the visibility its own segment search
gives: A and the visibility words are compared bit for bit with the
per-source path on whole matrices, and any pair where they differ must be one
the oracle flags as grazing (none is expected).  Lamps cover the wedge's
cases: sources in any order, a lamp straddling a patch's plane (some sources
facing, some not), segments shorter than the clearance cut, K = 2 and the
largest K of the wedge path, and lamps the wedge path must leave alone
(tilted, K = 1, K above the limit)."""
import contextlib
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2103_14137_gb300 as uvc
from synth import tiny_room, ward_room
from synth.scenes import Lamp, line_lamp
from tests._compare import GRAZE_CAP, compare_irradiance
from tests.gpu_util import T, build, build_arrays, lamp_of

pytestmark = pytest.mark.gpu


@contextlib.contextmanager
def wedge(enable):
    prev = uvc.set_wedge_traversal(enable)
    try:
        yield
    finally:
        uvc.set_wedge_traversal(prev)


def _matrix(sc, cand, lamp, enable):
    with wedge(enable):
        A, vis = uvc.irradiance_matrix(sc, T(np.asarray(cand, np.float32)), lamp, with_vis=True)
    torch.cuda.synchronize()
    assert uvc.scene_status(sc) == 0
    return A, vis


def _same_as_per_source(s_arrays, sc, cand, L):
    """Whole matrix both ways; differing pairs must be oracle-grazing."""
    verts, tris, cen, nrm, excl = s_arrays
    lamp = lamp_of(L)
    Aw, vw = _matrix(sc, cand, lamp, True)
    Ap, vp = _matrix(sc, cand, lamp, False)
    same_vis = torch.equal(vw, vp)
    same_A = torch.equal(Aw, Ap)
    if same_vis and same_A:
        return Aw, vw, 0
    bw, bp = uvc.vis_to_bool(vw, sc.np), uvc.vis_to_bool(vp, sc.np)
    diff = np.argwhere((bw != bp).any(axis=-1) | (Aw != Ap).cpu().numpy())
    _, _, flag = oracle.irradiance(verts, tris, cen, nrm, excl, np.asarray(cand, np.float32), L.offsets, L.weights,
                                   L.power, pairs=diff)
    assert np.all(flag != 0), f"{int((flag == 0).sum())} non-grazing pairs differ between wedge and per-source"
    cap = math.floor(GRAZE_CAP * Aw.numel() * L.K)
    assert diff.shape[0] <= cap, f"{diff.shape[0]} grazing differences > cap {cap}"
    return Aw, vw, diff.shape[0]


def _tiny_lamps():
    rng = np.random.default_rng(11)
    shuffled = line_lamp(1.1, 7, 90.0)
    perm = rng.permutation(7)
    shuffled = Lamp(shuffled.offsets[perm].copy(), shuffled.weights[perm].copy(), shuffled.power)
    w = rng.uniform(0.5, 1.5, 6).astype(np.float32)
    uneven = Lamp(line_lamp(1.4, 6, 100.0).offsets, (w / w.sum()).astype(np.float32), 100.0)
    below = line_lamp(1.0, 5, 80.0)
    below.offsets[:, 2] -= 0.53          # the tube reaches below the candidate point (no source on a surface)
    return {"K2": line_lamp(0.8, 2, 60.0), "K8": line_lamp(1.2, 8, 120.0), "K16": line_lamp(1.6, 16, 150.0),
            "shuffled": shuffled, "uneven_weights": uneven, "below": below}


@pytest.mark.parametrize("name", list(_tiny_lamps()))
def test_tiny_room_wedge_matches_oracle_and_per_source(name):
    """Tiny room, ragged candidate count, candidates at heights that put the
    tube across the table top's plane (0.75 m): parity with the oracle on the
    full matrix and bitwise equality with the per-source path."""
    L = _tiny_lamps()[name]
    s = tiny_room(n_cand=45)
    cand = s.cand.copy()
    cand[:, 2] = np.where(np.arange(45) % 3 == 0, 0.3, np.where(np.arange(45) % 3 == 1, 0.62, 1.0))
    sc = build(s)
    Aw, vw, ndiff = _same_as_per_source((s.verts, s.tris, s.centroid, s.normal, s.excl), sc, cand, L)
    E, ovis, flag = oracle.irradiance(s.verts, s.tris, s.centroid, s.normal, s.excl, cand, L.offsets, L.weights,
                                      L.power)
    st = compare_irradiance(Aw.cpu().numpy(), uvc.vis_to_bool(vw, s.np_), E, ovis, flag)
    assert st["excused_bits"] == 0 and ndiff == 0
    # some pairs have facing and non-facing sources at once (the lamp crosses a patch plane)
    o = cand[:, None, None, :] + L.offsets[None, None, :, :]
    nv = np.einsum("cpkx,px->cpk", o - s.centroid[None, :, None, :], s.normal)
    assert ((nv > 0).any(axis=-1) & (nv <= 0).any(axis=-1)).any()
    sc.free()


def test_lamps_outside_the_wedge_path_are_unchanged():
    """Tilted lamp, point lamp and K above the wedge limit: the switch changes
    nothing (these always take the per-source path)."""
    s = tiny_room(n_cand=20)
    sc = build(s)
    tilted = line_lamp(1.0, 6, 80.0)
    tilted.offsets[:, 0] = np.linspace(0.0, 0.3, 6, dtype=np.float32)
    for L in (tilted, s.lamp, line_lamp(1.0, 17, 80.0)):
        Aw, vw = _matrix(sc, s.cand, lamp_of(L), True)
        Ap, vp = _matrix(sc, s.cand, lamp_of(L), False)
        assert torch.equal(Aw, Ap) and torch.equal(vw, vp)
    sc.free()


def test_single_triangle_and_empty_scene_with_line_lamp():
    """Degenerate trees (one triangle: no node to traverse; no triangle)."""
    L = line_lamp(1.0, 4, 40.0)
    rng = np.random.default_rng(3)
    cen = np.concatenate([rng.uniform(-2, 2, (70, 2)), np.zeros((70, 1))], axis=1).astype(np.float32)
    nrm = np.tile(np.array([[0, 0, 1]], np.float32), (70, 1))
    ex = -np.ones((70, 2), np.int32)
    cand = np.concatenate([rng.uniform(-1, 1, (5, 2)), np.full((5, 1), 0.6)], axis=1).astype(np.float32)
    for k in (0, 1):
        verts = np.array([[-1, -1, 1], [1, -1, 1], [0, 1, 1]], np.float32)[: 3 * k]
        tris = np.arange(3 * k, dtype=np.int32).reshape(-1, 3)
        sc = build_arrays(verts, tris, cen, nrm, np.ones(70, np.float32), ex)
        Aw, vw, _ = _same_as_per_source((verts, tris, cen, nrm, ex), sc, cand, L)
        E, ovis, flag = oracle.irradiance(verts, tris, cen, nrm, ex, cand, L.offsets, L.weights, L.power)
        compare_irradiance(Aw.cpu().numpy(), uvc.vis_to_bool(vw, 70), E, ovis, flag)
        sc.free()


def test_ward_whole_matrix_equals_per_source():
    """The full ward workload (2,000 x ~102k pairs, K = 8) both ways, in the
    benchmark's launch configuration."""
    s = ward_room()
    sc = build(s)
    Aw, vw, ndiff = _same_as_per_source((s.verts, s.tris, s.centroid, s.normal, s.excl), sc, s.cand, s.lamp)
    assert Aw.shape == (s.nc, s.np_) and bool(torch.isfinite(Aw).all())
    sc.free()


def test_streamed_fluence_wedge_equals_per_source():
    s = ward_room(n_cand=256)
    sc = build(s)
    rng = np.random.default_rng(5)
    t = T(rng.uniform(0, 60, (4, s.nc)).astype(np.float32))
    with wedge(True):
        mu_w = uvc.fluence_streamed(sc, T(s.cand), lamp_of(s.lamp), t)
    with wedge(False):
        mu_p = uvc.fluence_streamed(sc, T(s.cand), lamp_of(s.lamp), t)
    torch.cuda.synchronize()
    assert torch.equal(mu_w, mu_p)
    sc.free()


def _area(sc, cand, lamp, ptri, enable):
    with wedge(enable):
        A, ncl = uvc.irradiance_area_mean(sc, T(np.asarray(cand, np.float32)), lamp, T(ptri), with_closed=True)
    torch.cuda.synchronize()
    assert uvc.scene_status(sc) == 0
    return A, ncl


@pytest.mark.parametrize("which", ["ward", "quad_patches", "tiny_k5"])
def test_area_mean_wedge_equals_per_source(which):
    """Area-mean irradiance: the wedge searches (centroid and every check
    point) give the per-source kernel's entries and closed-form counts; any
    differing pair must be one the oracle flags as grazing."""
    from synth.batched import batched_room, design_candidates
    if which == "ward":
        s = ward_room()
        cand, L = s.cand[:256], s.lamp
    elif which == "quad_patches":
        s = batched_room(136)
        cand, L = design_candidates(s, 0.8, 1.2, 300, seed=4), line_lamp(1.2, 8, 120.0)
    else:
        s = tiny_room(n_cand=45)
        cand = s.cand.copy()
        cand[:, 2] = 0.62
        L = line_lamp(0.9, 5, 100.0)
    sc = build(s)
    lamp = lamp_of(L)
    Aw, cw = _area(sc, cand, lamp, s.ptri, True)
    Ap, cp = _area(sc, cand, lamp, s.ptri, False)
    if not (torch.equal(Aw, Ap) and torch.equal(cw, cp)):
        diff = np.argwhere(((Aw != Ap) | (cw != cp)).cpu().numpy())
        _, _, flag = oracle.area_mean(s.verts, s.tris, s.centroid, s.normal, s.area, s.excl, s.ptri, cand,
                                      L.offsets, L.weights, L.power, pairs=diff)
        assert np.all(flag != 0), f"{int((flag == 0).sum())} non-grazing pairs differ"
        assert diff.shape[0] <= max(1, int(1e-6 * Aw.numel() * L.K))
    assert (cw > 0).float().mean().item() > 0.2          # the closed form is exercised
    sc.free()
