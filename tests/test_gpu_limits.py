"""Failure handling of the traversals without a GPU fault: uvc_scene_set_limits
lowers a scene's stack depth or node-visit cap so that searches stop as they
would on a tree too deep for the stack or on a search that does not end.  The
call must return normally, the status word must name the limit
(UVC_E_STACK / UVC_E_TIMEOUT) and be cleared by reading it, the stopped
entries must be NaN, every other entry and visibility bit must be the
unlimited run's, and restoring the limits must restore the result exactly."""
import numpy as np
import pytest
import torch

import paper_2103_14137_gb300 as uvc
from synth import ward_room
from tests.gpu_util import T, build, lamp_of

pytestmark = pytest.mark.gpu
E_STACK, E_TIMEOUT = uvc.uvc.UVC_E_STACK, uvc.uvc.UVC_E_TIMEOUT


@pytest.fixture(scope="module")
def ward():
    s = ward_room()
    sc = build(s)
    yield s, sc
    sc.free()


def _matrix(sc, cand, lamp):
    A, vis = uvc.irradiance_matrix(sc, cand, lamp, with_vis=True)
    torch.cuda.synchronize()
    return A, vis, uvc.scene_status(sc)


def _check_stopped(A0, v0, A1, v1, np_):
    nan = torch.isnan(A1)
    assert not bool(torch.isinf(A1).any())
    frac = nan.float().mean().item()
    assert 0.01 < frac < 0.999, frac
    ok = ~nan
    assert torch.allclose(A1[ok], A0[ok], rtol=1e-6, atol=0.0)
    b0, b1 = uvc.vis_to_bool(v0, np_), uvc.vis_to_bool(v1, np_)
    okn = ok.cpu().numpy()
    assert np.array_equal(b1[okn], b0[okn])


@pytest.mark.parametrize("wedge", [True, False], ids=["wedge", "per_source"])
@pytest.mark.parametrize("limit", ["stack", "visits"])
def test_limited_search_reports_and_keeps_the_rest(ward, wedge, limit):
    s, sc = ward
    cand, lamp = T(s.cand[:64]), lamp_of(s.lamp)
    prev = uvc.set_wedge_traversal(wedge)
    try:
        A0, v0, st0 = _matrix(sc, cand, lamp)
        assert st0 == 0 and not bool(torch.isnan(A0).any())
        if limit == "stack":
            uvc.scene_set_limits(sc, max_stack=4)
        else:
            uvc.scene_set_limits(sc, max_visits=3)
        A1, v1, st1 = _matrix(sc, cand, lamp)
        assert st1 == (E_STACK if limit == "stack" else E_TIMEOUT)
        assert uvc.scene_status(sc) == 0                                # reading cleared it
        _check_stopped(A0, v0, A1, v1, s.np_)
        uvc.scene_set_limits(sc)                                        # built-in limits again
        A2, v2, st2 = _matrix(sc, cand, lamp)
        assert st2 == 0 and torch.equal(A2, A0) and torch.equal(v2, v0)
    finally:
        uvc.scene_set_limits(sc)
        uvc.set_wedge_traversal(prev)


def test_limited_area_mean_reports_and_keeps_the_rest(ward):
    s, sc = ward
    cand, lamp, ptri = T(s.cand[:32]), lamp_of(s.lamp), T(s.ptri)
    try:
        A0, n0 = uvc.irradiance_area_mean(sc, cand, lamp, ptri, with_closed=True)
        torch.cuda.synchronize()
        assert uvc.scene_status(sc) == 0
        uvc.scene_set_limits(sc, max_stack=4)
        A1, n1 = uvc.irradiance_area_mean(sc, cand, lamp, ptri, with_closed=True)
        torch.cuda.synchronize()
        assert uvc.scene_status(sc) == E_STACK
        nan = torch.isnan(A1)
        assert 0.01 < nan.float().mean().item() < 0.999
        assert torch.allclose(A1[~nan], A0[~nan], rtol=1e-6, atol=0.0)
        assert torch.equal(n1[~nan], n0[~nan])
    finally:
        uvc.scene_set_limits(sc)


def test_limits_are_validated(ward):
    _, sc = ward
    for bad in ((-1, 0), (0, -5)):
        with pytest.raises(uvc.UvcError) as e:
            uvc.scene_set_limits(sc, *bad)
        assert e.value.status == uvc.uvc.UVC_E_INVAL
