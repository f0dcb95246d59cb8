"""GPU hierarchy against the oracle's definitions, bit for bit: Morton keys,
stable order, radix tree children, child boxes."""
import numpy as np
import pytest

from oracle import lbvh
from synth import tiny_room, ward_room
from tests.gpu_util import build, build_arrays

pytestmark = pytest.mark.gpu


def _check(verts, tris, sc):
    g = __import__("paper_2103_14137_gb300").scene_export_bvh(sc)
    o = lbvh.build(verts, tris)
    assert np.array_equal(g["keys"], o["sorted_keys"])
    assert np.array_equal(g["order"], o["order"].astype(np.int32))
    n = tris.shape[0]
    if n < 2:
        return
    ref_l = np.where(o["left_leaf"], ~o["left"], o["left"])
    ref_r = np.where(o["right_leaf"], ~o["right"], o["right"])
    assert np.array_equal(g["children"][:, 0], ref_l)
    assert np.array_equal(g["children"][:, 1], ref_r)
    b = g["boxes"]
    assert np.array_equal(b[:, 0:3], o["lo_l"]) and np.array_equal(b[:, 3:6], o["hi_l"])
    assert np.array_equal(b[:, 6:9], o["lo_r"]) and np.array_equal(b[:, 9:12], o["hi_r"])


def test_tiny_bvh_bit_exact():
    s = tiny_room()
    sc = build(s)
    _check(s.verts, s.tris, sc)
    sc.free()


def test_ward_bvh_bit_exact():
    s = ward_room()
    sc = build(s)
    _check(s.verts, s.tris, sc)
    assert 10 < sc.depth < 96
    sc.free()


@pytest.mark.parametrize("n", [1, 2, 3, 33, 2049, 4097])
def test_sizes_across_sort_tiles_and_duplicates(n):
    rng = np.random.default_rng(n)
    base = rng.uniform(0, 5, size=(n, 3)).astype(np.float32)
    base[: n // 3] = base[0]          # a run of identical keys
    verts = np.repeat(base, 3, axis=0) + np.tile(np.array([[0, 0, 0], [0.01, 0, 0], [0, 0.01, 0]], np.float32), (n, 1))
    tris = np.arange(3 * n, dtype=np.int32).reshape(-1, 3)
    cen = np.zeros((1, 3), np.float32)
    sc = build_arrays(verts, tris, cen, [[0, 0, 1]], [1.0], [[-1, -1]])
    _check(verts, tris, sc)
    sc.free()
