"""The counting replay of the wedge traversal (replay/) against the kernel's
own instrumented counters (uvc_irradiance_counters) on the same tasks: whole
rows of the full-size ward for 32 candidates (8 runs of 4), the benchmark's K = 8
lamp.  The replay re-executes the visit order in FP32 on the CPU; its node
visits, leaf loads, box, plane and triangle tests must agree with the
kernel's to within the rounding of the one approximate reciprocal the kernel
uses (0.1 %), so that the bytes per pair derived from it describe the
kernel's traversal."""
import numpy as np
import pytest
import torch

import paper_2103_14137_gb300 as uvc
import replay
from synth import ward_room
from tests.gpu_util import T, build, lamp_of

pytestmark = pytest.mark.gpu


def test_replay_counts_match_kernel_counters():
    s = ward_room()
    sc = build(s)
    chunks = np.array([0, 61, 122, 200, 263, 333, 401, 499])
    rows = (chunks[:, None] * 4 + np.arange(4)[None, :]).reshape(-1)
    cand = np.ascontiguousarray(s.cand[rows])
    ctr = uvc.irradiance_counters(sc, T(cand), lamp_of(s.lamp))
    torch.cuda.synchronize()
    assert uvc.scene_status(sc) == 0
    ex = uvc.scene_export_traversal(sc)
    njb = (s.np_ + 31) // 32
    cpt = uvc.irradiance_candidates_per_task()
    nchunk = (rows.size + cpt - 1) // cpt
    tasks = np.stack([np.repeat(np.arange(nchunk), njb), np.tile(np.arange(njb), nchunk)], axis=1)
    c = replay.replay(ex, cand, s.lamp.offsets, tasks, cand_per_task=cpt)
    assert c["pairs"] == rows.size * s.np_
    pairs = {"node_visits": "node_visits", "leaf_loads": "leaf_tests", "traversals": "traversals",
             "tri_tests": "lane_tri_tests", "search_segments": "facing_segments",
             "box_tests": "lane_wedge_box_tests", "plane_tests": "lane_wedge_plane_tests"}
    for mine, theirs in pairs.items():
        a, b = c[mine], ctr[theirs]
        assert abs(a - b) <= 1e-3 * b + 2, (mine, a, b)
    bpp = replay.bytes_per_pair(c, s.lamp.K)
    assert bpp["per_lane"] > bpp["per_warp"] > bpp["output"]
    sc.free()
