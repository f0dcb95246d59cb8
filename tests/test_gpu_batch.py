"""Batched irradiance matrices (uvc_batch_*): every job's matrix and visibility
words are bit-identical to uvc_irradiance_matrix's for the same inputs, with
the default configuration, after autotuning, and when the launch is replayed
from a captured CUDA graph."""
import numpy as np
import pytest
import torch

import paper_2103_14137_gb300 as uvc
from synth import tiny_room, ward_room
from synth.batched import LAMPS, batched_room, design_candidates
from synth.scenes import line_lamp
from tests.gpu_util import T, build, lamp_of

pytestmark = pytest.mark.gpu


def _jobs():
    rooms = [tiny_room(), batched_room(103), ward_room(n_cand=40)]
    lamps = [line_lamp(L, K, 120.0) for (L, K) in LAMPS] + [rooms[0].lamp]
    scenes = [build(r) for r in rooms]
    jobs = []
    for r, (room, sc) in enumerate(zip(rooms, scenes)):
        for d in range(len(lamps)):
            if room.nc and d == len(lamps) - 1:
                cand = room.cand[:37]
            else:
                cand = design_candidates(room, 0.5 + 0.1 * d, LAMPS[d % 3][0], 53 + 11 * d, seed=r * 7 + d) \
                    if "box_list" in room.info else room.cand[: 29 + d]
            lda = sc.np + (d % 2) * 5
            A = torch.full((cand.shape[0], lda), -1.0, device="cuda")
            vis = torch.zeros((lamps[d].K, cand.shape[0], (sc.np + 31) // 32), dtype=torch.int32, device="cuda")
            jobs.append((sc, T(cand), d, A, vis))
    return rooms, scenes, [uvc.Lamp(L.offsets, L.weights, L.power) for L in lamps], jobs


def _reference(jobs, lamps):
    out = []
    for sc, cand, d, A, vis in jobs:
        A0, v0 = uvc.irradiance_matrix(sc, cand, lamps[d], with_vis=True)
        out.append((A0, v0))
    return out


def _check(jobs, ref):
    torch.cuda.synchronize()
    for (sc, cand, d, A, vis), (A0, v0) in zip(jobs, ref):
        assert torch.equal(A[:, :sc.np], A0)
        assert torch.all(A[:, sc.np:] == -1.0)
        assert torch.equal(vis, v0)


def test_batch_matches_single_calls():
    rooms, scenes, lamps, jobs = _jobs()
    ref = _reference(jobs, lamps)
    b = uvc.Batch(jobs, lamps)
    info = b.info()
    assert info["total_pairs"] == sum(c.shape[0] * s.np for s, c, _, _, _ in jobs)
    b.launch()
    _check(jobs, ref)
    for sc in scenes:
        assert uvc.scene_status(sc) == 0
    b.free()


def test_batch_autotune_and_configs():
    rooms, scenes, lamps, jobs = _jobs()
    ref = _reference(jobs, lamps)
    b = uvc.Batch(jobs, lamps)
    cpt, bps = b.autotune(0.2)
    assert cpt in (4, 8, 16) and bps in (2, 3)
    for A in (j[3] for j in jobs):
        A.fill_(-1.0)
    b.launch()
    _check(jobs, ref)
    for cfg in ((2, 0), (16, 1)):
        b.set_config(*cfg)
        for A in (j[3] for j in jobs):
            A.fill_(-1.0)
        b.launch()
        _check(jobs, ref)
    b.free()


def test_batch_cuda_graph_replay():
    rooms, scenes, lamps, jobs = _jobs()
    ref = _reference(jobs, lamps)
    b = uvc.Batch(jobs, lamps)
    b.launch()                                  # first call outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.launch()
    for A in (j[3] for j in jobs):
        A.fill_(-1.0)
    for j in jobs:
        j[4].zero_()
    g.replay()
    _check(jobs, ref)
    b.free()


@pytest.mark.parametrize("which", ["line_lamps_only", "point_and_tilted_only"])
def test_batch_path_modes_match_single_calls(which):
    """A batch whose lamps all take the wedge path, and one where none does
    (point lamp, tilted line lamp), against the single-matrix calls."""
    room = batched_room(103)
    sc = build(room)
    if which == "line_lamps_only":
        lamps = [line_lamp(L, K, 120.0) for (L, K) in LAMPS]
    else:
        tilted = line_lamp(1.2, 8, 120.0)
        tilted.offsets[:, 1] = np.linspace(-0.1, 0.1, 8, dtype=np.float32)
        lamps = [tiny_room().lamp, tilted]
    L = [uvc.Lamp(x.offsets, x.weights, x.power) for x in lamps]
    jobs = []
    for d in range(len(lamps)):
        cand = design_candidates(room, 0.5 + 0.2 * d, 1.2, 45 + 7 * d, seed=31 + d)
        A = torch.full((cand.shape[0], sc.np), -1.0, device="cuda")
        vis = torch.zeros((lamps[d].K, cand.shape[0], (sc.np + 31) // 32), dtype=torch.int32, device="cuda")
        jobs.append((sc, T(cand), d, A, vis))
    ref = _reference(jobs, L)
    b = uvc.Batch(jobs, L)
    b.launch()
    _check(jobs, ref)
    b.free()
    sc.free()
