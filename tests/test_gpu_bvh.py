"""GPU hierarchy against the oracle's definitions, bit for bit: Morton keys,
stable order, radix tree children, child boxes (plain LBVH build); and the
surface-area restructured hierarchy: a valid tree over the same triangles with
exact boxes and a lower surface-area cost, giving bit-identical matrices."""
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
    sc = build(s, lbvh_only=True)
    _check(s.verts, s.tris, sc)
    sc.free()


def test_ward_bvh_bit_exact():
    s = ward_room()
    sc = build(s, lbvh_only=True)
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
    sc = build_arrays(verts, tris, cen, [[0, 0, 1]], [1.0], [[-1, -1]], lbvh_only=True)
    _check(verts, tris, sc)
    sc.free()


def _tree_sah(children, boxes, verts, tris, order):
    """Surface-area cost with the restructuring's constants (C_i = 1.2, C_t = 1)."""
    def ha(lo, hi):
        d = np.maximum(hi - lo, 0)
        return d[..., 0] * d[..., 1] + d[..., 1] * d[..., 2] + d[..., 2] * d[..., 0]
    lo_l, hi_l, lo_r, hi_r = boxes[:, 0:3], boxes[:, 3:6], boxes[:, 6:9], boxes[:, 9:12]
    node_area = ha(np.minimum(lo_l, lo_r), np.maximum(hi_l, hi_r))
    leaf_cost = (ha(lo_l, hi_l) * (children[:, 0] < 0)).sum() + (ha(lo_r, hi_r) * (children[:, 1] < 0)).sum()
    return 1.2 * node_area.sum() + leaf_cost


def _check_tree(verts, tris, g):
    n = tris.shape[0]
    ch = g["children"]
    assert sorted(g["order"].tolist()) == list(range(n))
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(n - 1, int)
    for a in ch.ravel():
        (seen_leaf if a < 0 else seen_node)[~a if a < 0 else a] += 1
    assert np.all(seen_leaf == 1) and seen_node[0] == 0 and np.all(seen_node[1:] == 1)
    v = verts[tris[g["order"]]]
    tlo, thi = v.min(axis=1), v.max(axis=1)
    b = g["boxes"]
    # exact boxes: each child box is the min/max over its subtree's triangles
    memo = {}

    def box(ref):
        if ref < 0:
            return tlo[~ref], thi[~ref]
        if ref not in memo:
            l0, l1 = box(ch[ref, 0])
            r0, r1 = box(ch[ref, 1])
            memo[ref] = (np.minimum(l0, r0), np.maximum(l1, r1))
        return memo[ref]
    import sys
    sys.setrecursionlimit(100000)
    for k in range(n - 1):
        l0, l1 = box(ch[k, 0])
        r0, r1 = box(ch[k, 1])
        assert np.array_equal(b[k, 0:3], l0) and np.array_equal(b[k, 3:6], l1)
        assert np.array_equal(b[k, 6:9], r0) and np.array_equal(b[k, 9:12], r1)


def test_restructured_tree_valid_and_cheaper():
    import paper_2103_14137_gb300 as uvc
    s = ward_room()
    sc0 = build(s, lbvh_only=True)
    sc1 = build(s)
    g0, g1 = uvc.scene_export_bvh(sc0), uvc.scene_export_bvh(sc1)
    _check_tree(s.verts, s.tris, g1)
    c0 = _tree_sah(g0["children"], g0["boxes"], s.verts, s.tris, g0["order"])
    c1 = _tree_sah(g1["children"], g1["boxes"], s.verts, s.tris, g1["order"])
    assert c1 < 0.95 * c0, (c0, c1)
    sc0.free()
    sc1.free()


def test_restructured_tree_gives_identical_matrix():
    import paper_2103_14137_gb300 as uvc
    from tests.gpu_util import T, lamp_of
    s = ward_room(n_cand=64)
    sc0 = build(s, lbvh_only=True)
    sc1 = build(s)
    A0, v0 = uvc.irradiance_matrix(sc0, T(s.cand), lamp_of(s.lamp), with_vis=True)
    A1, v1 = uvc.irradiance_matrix(sc1, T(s.cand), lamp_of(s.lamp), with_vis=True)
    import torch
    torch.cuda.synchronize()
    assert torch.equal(A0, A1) and torch.equal(v0, v1)
    sc0.free()
    sc1.free()


def test_four_wide_tree_covers_every_triangle_once():
    """The four-wide tree the traversal reads (uvc_scene_export_traversal): from
    the root every triangle is reached exactly once, empty slots carry no
    child, and every child box holds the triangles below it."""
    import paper_2103_14137_gb300 as uvc
    s = ward_room(n_cand=4)
    for lbvh_only in (False, True):
        sc = build(s, lbvh_only=lbvh_only)
        ex = uvc.scene_export_traversal(sc)
        words = ex["nodes4"]
        q = words[:, :24].view(np.float32).reshape(-1, 6, 4)
        ref = words[:, 24:28].view(np.int32)
        mask = words[:, 28:30].view(np.int32)
        tri = ex["tri"]
        seen = np.zeros(s.nt, np.int64)
        EMPTY = 0x7fffffff

        def child_box(i, c):
            h, k = divmod(c, 2)
            lo = np.array([q[i, 3 * h + a, k] for a in range(3)])
            hi = np.array([q[i, 3 * h + a, 2 + k] for a in range(3)])
            return lo, hi

        def visit(i, depth):
            lo_all, hi_all = np.full(3, np.inf), np.full(3, -np.inf)
            for c in range(4):
                r = int(ref[i, c])
                is_leaf, is_inner = (mask[i, 0] >> c) & 1, (mask[i, 1] >> c) & 1
                if r == EMPTY:
                    assert not is_leaf and not is_inner
                    continue
                lo, hi = child_box(i, c)
                if r < 0:
                    assert is_leaf and not is_inner
                    k = ~r
                    seen[k] += 1
                    v = tri[k, :, :3]
                    tlo, thi = v.min(axis=0), v.max(axis=0)
                else:
                    assert is_inner and not is_leaf
                    tlo, thi = visit(r, depth + 1)
                assert np.all(lo <= tlo) and np.all(hi >= thi), (i, c)
                lo_all, hi_all = np.minimum(lo_all, tlo), np.maximum(hi_all, thi)
            return lo_all, hi_all

        import sys
        sys.setrecursionlimit(100000)
        visit(0, 0)
        assert np.all(seen == 1)
        sc.free()
