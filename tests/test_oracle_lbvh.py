"""Pins of the LBVH oracle: hand-derived Morton keys, stable order, the radix
tree of a hand-derived example, tree invariants on random keys (duplicates
included), and boxes recomputed directly over each node's leaf range."""
import json
import os

import numpy as np

from oracle import lbvh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _degenerate_tris(points):
    """Triangles collapsed to points: their reference point is the point itself."""
    v = np.repeat(np.asarray(points, np.float32), 3, axis=0)
    return v, np.arange(v.shape[0], dtype=np.int32).reshape(-1, 3)


def test_morton_hand_values():
    u = 2.0 ** -21
    pts = [[0, 0, 0], [1, 1, 1], [1.5 * u, 0, 0], [0, 1.5 * u, 0], [0, 0, 1.5 * u], [0.5, 0.25, 0.75]]
    v, t = _degenerate_tris(pts)
    k = lbvh.morton_keys(v, t)
    want = [0, 2 ** 63 - 1, 4, 2, 1, 2 ** 62 + 2 ** 60 + 2 ** 58 + 2 ** 57]
    assert [int(x) for x in k] == want


def test_reference_point_is_the_box_centre():
    """The key of a triangle is taken at the centre of its bounding box
    (worked by hand: boxes [0,2]x[0,4]x[0,6] and [-1,3]x[1,5]x[-2,4])."""
    v = np.array([[0, 0, 0], [2, 0, 0], [0, 4, 6], [1, 5, -2], [3, 1, 0], [-1, 2, 4]], np.float32)
    t = np.arange(6, dtype=np.int32).reshape(2, 3)
    assert np.array_equal(lbvh.reference_points(v, t), np.array([[1, 2, 3], [1, 3, 1]], np.float32))


def test_stable_sort_keeps_triangle_order_on_ties():
    keys = np.array([5, 3, 5, 3, 1, 5], np.uint64)
    sk, order = lbvh.sort_keys(keys)
    assert list(order) == [4, 1, 3, 0, 2, 5]
    assert list(sk) == [1, 3, 3, 5, 5, 5]


def test_radix_tree_hand_example():
    d = json.load(open(os.path.join(GOLDEN, "radix_tree_example.json")))
    keys = np.array([int(b, 2) for b in d["keys_binary"]], np.uint64)
    left, right, ll, rl = lbvh.radix_tree(keys)
    for node, spec in d["internal_nodes"].items():
        n = int(node)
        kind, idx = spec["left"]
        assert left[n] == idx and ll[n] == (kind == "leaf")
        kind, idx = spec["right"]
        assert right[n] == idx and rl[n] == (kind == "leaf")


def _check_tree(keys):
    n = len(keys)
    left, right, ll, rl = lbvh.radix_tree(keys)
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(max(n - 1, 1), int)
    for k in range(n - 1):
        (seen_leaf if ll[k] else seen_node)[left[k]] += 1
        (seen_leaf if rl[k] else seen_node)[right[k]] += 1
    assert np.all(seen_leaf == 1)
    if n > 1:
        assert seen_node[0] == 0 and np.all(seen_node[1:] == 1)

    def span(idx, is_leaf):
        if is_leaf:
            return idx, idx
        a1, _ = span(left[idx], ll[idx])
        _, b2 = span(right[idx], rl[idx])
        return a1, b2

    for k in range(n - 1):
        a, b = span(k, False)
        assert k in (a, b)                        # a node's index is an end of its range
        g = left[k] if not ll[k] else a
        assert span(left[k], ll[k]) == (a, g)     # children split the range
        assert span(right[k], rl[k])[0] == g + 1
        # the split separates keys by the first bit (of key, then position) where a and b differ
        whole = lbvh._prefix(keys, a, b)
        for p in range(a, b + 1):
            assert (lbvh._prefix(keys, a, p) > whole) == (p <= g)


def test_radix_tree_invariants_random_with_duplicates():
    rng = np.random.default_rng(3)
    for n in (2, 3, 17, 200):
        keys = np.sort(rng.integers(0, 40, size=n).astype(np.uint64))
        _check_tree(keys)
        keys = np.sort(rng.integers(0, 2 ** 62, size=n, dtype=np.int64).astype(np.uint64))
        _check_tree(keys)


def test_boxes_equal_range_minmax():
    from synth import tiny_room
    s = tiny_room()
    b = lbvh.build(s.verts, s.tris)
    v = s.verts[s.tris[b["order"]]]                # (nt,3,3) sorted triangles
    lo_t, hi_t = v.min(axis=1), v.max(axis=1)

    def span(idx, is_leaf):
        if is_leaf:
            return idx, idx
        return span(b["left"][idx], b["left_leaf"][idx])[0], span(b["right"][idx], b["right_leaf"][idx])[1]

    for k in range(s.nt - 1):
        a, g = span(b["left"][k], b["left_leaf"][k])
        assert np.array_equal(b["lo_l"][k], lo_t[a:g + 1].min(axis=0))
        assert np.array_equal(b["hi_l"][k], hi_t[a:g + 1].max(axis=0))
        a, g = span(b["right"][k], b["right_leaf"][k])
        assert np.array_equal(b["lo_r"][k], lo_t[a:g + 1].min(axis=0))
        assert np.array_equal(b["hi_r"][k], hi_t[a:g + 1].max(axis=0))
    # keys follow the Z-order: sorted keys are non-decreasing, order is a permutation
    assert np.all(np.diff(b["sorted_keys"].astype(np.float64)) >= 0)
    assert np.array_equal(np.sort(b["order"]), np.arange(s.nt))
