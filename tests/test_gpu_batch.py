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
    assert cpt in (1, 4, 16) and bps in (2, 3)
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


def _oracle_jobs():
    """Uneven rooms (12,346 to 190,386 triangles, 5,899 to 12,526 patches)
    crossed with the robot-design sweep: lamp-bottom heights 0.3-1.1 m x line
    lamps of K = 4, 8, 12 sources, an uneven number of candidates per job."""
    from synth.batched import designs
    rooms = [batched_room(103), batched_room(106), batched_room(113)]
    scenes = [build(r) for r in rooms]
    sweep = designs()
    lamps_g = [line_lamp(L, K, 120.0) for (_, L, K) in sweep]
    jobs, host = [], []
    for r, (room, sc) in enumerate(zip(rooms, scenes)):
        ds = range(len(sweep)) if r != 1 else (0, 5, 10)        # the 190k-triangle room: three designs
        for d in ds:
            h, L, K = sweep[d]
            cand = design_candidates(room, h, L, 9 + 5 * d + 3 * r, seed=1000 + 16 * r + d)
            A = torch.full((cand.shape[0], sc.np), -1.0, device="cuda")
            vis = torch.zeros((K, cand.shape[0], (sc.np + 31) // 32), dtype=torch.int32, device="cuda")
            jobs.append((sc, T(cand), d, A, vis))
            host.append((room, cand, d))
    return rooms, scenes, lamps_g, jobs, host


def _check_against_oracle(jobs, host, lamps_g, cache):
    """Every job's whole matrix against the oracle's CPU-BVH mode (the same
    entries as its brute force, computed once per job into `cache`); pairs
    whose visibility differs get the brute force's grazing flags."""
    import oracle
    from tests._compare import compare_irradiance
    torch.cuda.synchronize()
    excused = 0
    for q, ((sc, _, d, A, vis), (room, cand, _)) in enumerate(zip(jobs, host)):
        L = lamps_g[d]
        if q not in cache:
            cache[q] = oracle.irradiance(room.verts, room.tris, room.centroid, room.normal, room.excl, cand,
                                         L.offsets, L.weights, L.power, bvh=True, flags=False)[:2]
        E, ovis = cache[q]
        visg = uvc.vis_to_bool(vis, sc.np)
        flag = np.zeros(E.shape, np.uint8)
        diff = np.argwhere((visg != ovis.astype(bool)).any(axis=-1))
        if diff.size:
            _, _, f = oracle.irradiance(room.verts, room.tris, room.centroid, room.normal, room.excl, cand,
                                        L.offsets, L.weights, L.power, pairs=diff)
            flag[diff[:, 0], diff[:, 1]] = f
        st = compare_irradiance(A.cpu().numpy(), visg, E, ovis, flag)
        excused += st["excused_bits"]
        assert torch.all(torch.isfinite(A))
    return excused


def test_batch_of_uneven_rooms_and_designs_against_oracle():
    """One persistent launch over 27 (room, design) jobs of uneven size, and
    the same launch replayed from a captured CUDA graph, both against the
    FP64 oracle: visibility bit-exact except on grazing pairs (within the
    cap of each job), entries within 1e-5."""
    rooms, scenes, lamps_g, jobs, host = _oracle_jobs()
    lamps = [uvc.Lamp(L.offsets, L.weights, L.power) for L in lamps_g]
    b = uvc.Batch(jobs, lamps)
    b.autotune(0.2)
    b.launch()
    cache = {}
    _check_against_oracle(jobs, host, lamps_g, cache)
    for sc in scenes:
        assert uvc.scene_status(sc) == 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.launch()
    for _, _, _, A, vis in jobs:
        A.fill_(-1.0)
        vis.zero_()
    g.replay()
    _check_against_oracle(jobs, host, lamps_g, cache)
    for sc in scenes:
        assert uvc.scene_status(sc) == 0
    b.free()
    for sc in scenes:
        sc.free()


def test_batch_with_more_lamps_than_the_parameter_pack():
    """18 lamps (more than the 16 a launch carries in its parameters: the
    kernel then reads them from the batch's device table) over two rooms,
    point, tilted and vertical line lamps mixed; every job against the
    single-matrix call."""
    rooms = [tiny_room(), batched_room(113)]
    scenes = [build(r) for r in rooms]
    lamps_g = [line_lamp(0.3 + 0.1 * k, 2 + k % 11, 100.0) for k in range(16)]
    tilted = line_lamp(1.2, 8, 120.0)
    tilted.offsets[:, 1] = np.linspace(-0.1, 0.1, 8, dtype=np.float32)
    lamps_g += [tiny_room().lamp, tilted]
    L = [uvc.Lamp(x.offsets, x.weights, x.power) for x in lamps_g]
    jobs = []
    for r, (room, sc) in enumerate(zip(rooms, scenes)):
        for d in range(len(L)):
            cand = room.cand[: 7 + d] if room.nc else design_candidates(room, 0.6, 1.0, 9 + d, seed=d)
            A = torch.full((cand.shape[0], sc.np), -1.0, device="cuda")
            vis = torch.zeros((L[d].K, cand.shape[0], (sc.np + 31) // 32), dtype=torch.int32, device="cuda")
            jobs.append((sc, T(cand), d, A, vis))
    ref = _reference(jobs, L)
    b = uvc.Batch(jobs, L)
    b.launch()
    _check(jobs, ref)
    b.free()
    for sc in scenes:
        assert uvc.scene_status(sc) == 0
        sc.free()
