"""The allocation-free streamed fluence (uvc_fluence_streamed_noalloc).

It exists for callers that cannot allocate device memory during a call: a host
program whose own allocator already holds all the device memory it may use, or
a control loop that forbids allocation after start-up.  It must give the same
fluence as uvc_fluence_streamed, within the fluence tolerance of the other
tests, on consecutive calls (the fixed scratch array keeps the previous call's
contents), and must refuse problems larger than its fixed scratch.

This file is collected after the traversal, fluence and proposal suites, so
that a run stopping at the first failure has already run them; it also passes
alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import paper_2103_14137_gb300 as uvc
from synth import dwell_vectors, tiny_room
from tests.gpu_util import T, build, lamp_of

pytestmark = pytest.mark.gpu
MU_TOL = 1e-5


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30)))


def test_noalloc_matches_streamed_on_two_calls_in_a_row():
    s = tiny_room(n_cand=150)
    sc = build(s)
    cand, lamp = T(s.cand), lamp_of(s.lamp)
    for seed, nvec in ((21, 16), (22, 5)):
        t = T(dwell_vectors(nvec, s.nc, seed=seed))
        want = uvc.fluence_streamed(sc, cand, lamp, t).cpu().numpy()
        mu = torch.full((nvec, s.np_), float("nan"), device="cuda")
        got = uvc.fluence_streamed_noalloc(sc, cand, lamp, t, mu)
        torch.cuda.synchronize()
        assert got.data_ptr() == mu.data_ptr()
        assert _rel(got.cpu().numpy(), want) <= MU_TOL, seed
    assert uvc.scene_status(sc) == 0
    sc.free()


@pytest.mark.parametrize("nvec", [100, 60])
def test_noalloc_with_few_chunks_and_a_line_lamp(nvec):
    """The ward's 102,030 patches with 100 dwell vectors (40.8 MB of partial
    sums per chunk: the fixed scratch holds one chunk) and 60 (24.5 MB: two
    chunks), 64 candidates and the K = 8 vertical line lamp (the wedge
    search): fewer, longer chunks than uvc_fluence_streamed picks, so another
    summation order, still within the fluence tolerance, on two calls in a
    row."""
    from synth import ward_room
    s = ward_room()
    sc = build(s)
    rows = np.linspace(0, s.nc - 1, 64).astype(np.int64)
    cand, lamp = T(s.cand[rows]), lamp_of(s.lamp)
    assert 32 * 2 ** 20 < 4 * 100 * s.np_ <= 64 * 2 ** 20 and 4 * 60 * s.np_ <= 32 * 2 ** 20
    for seed in (31, 32):
        t = T(dwell_vectors(nvec, rows.size, seed=seed))
        want = uvc.fluence_streamed(sc, cand, lamp, t).cpu().numpy()
        mu = torch.full((nvec, s.np_), float("nan"), device="cuda")
        got = uvc.fluence_streamed_noalloc(sc, cand, lamp, t, mu).cpu().numpy()
        assert uvc.scene_status(sc) == 0
        assert _rel(got, want) <= MU_TOL, (nvec, seed)
    sc.free()


def test_noalloc_rejects_problems_beyond_its_scratch():
    s = tiny_room(n_cand=4)
    sc = build(s)
    nvec = 256                                   # 4 * 256 * np > 64 MiB needs np > 65,536
    if 4 * nvec * s.np_ <= 64 * 2 ** 20:
        # a patch count above the limit: replicate the tiny room's patches
        reps = (64 * 2 ** 20) // (4 * nvec * s.np_) + 1
        cen = np.tile(s.centroid, (reps, 1))
        sc.free()
        sc = uvc.build_scene(T(s.verts), T(s.tris), T(cen), T(np.tile(s.normal, (reps, 1))),
                             T(np.tile(s.area, reps)), T(np.tile(s.excl, (reps, 1))))
    t = T(dwell_vectors(nvec, s.nc))
    mu = torch.empty((nvec, sc.np), device="cuda")
    with pytest.raises(uvc.UvcError) as e:
        uvc.fluence_streamed_noalloc(sc, T(s.cand), lamp_of(s.lamp), t, mu)
    assert e.value.status == uvc.uvc.UVC_E_SCRATCH
    sc.free()
