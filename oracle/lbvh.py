"""Oracle for the bounding-volume hierarchy over the triangle mesh.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The hierarchy is a linear BVH in the sense of Karras, "Maximizing Parallelism in
the Construction of BVHs, Octrees, and k-d Trees" (HPG 2012): triangles are
ordered along a Z-order (Morton) curve and the tree is the binary radix tree of
the sorted keys.  Each step here is written from its definition, plainly:

  reference point   centre of the triangle's bounding box, fl32(fl32(lo+hi)*0.5)
  quantisation      q = floor(fl32(fl32(p - lo_s) * fl32(2^21 / (hi_s - lo_s)))),
                    clamped to [0, 2^21 - 1] per axis, where [lo_s, hi_s] bounds
                    all reference points; the FP32 steps are the ones the GPU
                    takes, so both sides make the same integer decisions
  key               63-bit interleave, bit 3b+2 = x_b, 3b+1 = y_b, 3b = z_b
  order             stable sort of the keys (equal keys keep triangle order)
  radix tree        node covering sorted range [a, b] splits after the last
                    position g in [a, b-1] whose common prefix with position a
                    is longer than that of a and b; prefixes are taken over
                    (key, position) so that equal keys still split
  numbering         root = internal node 0; the child covering [a, g] is
                    numbered g, the child covering [g+1, b] is numbered g+1,
                    and a child covering a single position is that leaf
  boxes             leaf = min/max of the triangle's vertices; internal node =
                    min/max of its two children (exact in FP32)
"""
from __future__ import annotations

import numpy as np

BITS = 21


def reference_points(verts, tris):
    v = np.asarray(verts, np.float32).reshape(-1, 3)
    t = np.asarray(tris, np.int64).reshape(-1, 3)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    lo = np.minimum(np.minimum(a, b), c)
    hi = np.maximum(np.maximum(a, b), c)
    return (lo + hi) * np.float32(0.5)


def morton_keys(verts, tris):
    """63-bit Morton key of every triangle (uint64)."""
    p = reference_points(verts, tris)
    if p.shape[0] == 0:
        return np.zeros(0, np.uint64)
    lo = p.min(axis=0)
    hi = p.max(axis=0)
    ext = hi - lo
    scale = np.zeros(3, np.float32)
    nz = ext > 0
    scale[nz] = np.float32(2 ** BITS) / ext[nz]
    q = (p - lo) * scale
    qi = np.minimum(np.floor(q).astype(np.int64), 2 ** BITS - 1).astype(np.uint64)
    key = np.zeros(p.shape[0], np.uint64)
    for bit in range(BITS):
        for axis, pos in ((0, 2), (1, 1), (2, 0)):
            b = (qi[:, axis] >> np.uint64(bit)) & np.uint64(1)
            key |= b << np.uint64(3 * bit + pos)
    return key


def sort_keys(keys):
    """Stable sort: (sorted keys, triangle index at each sorted position)."""
    order = np.argsort(keys, kind="stable")
    return keys[order], order.astype(np.int64)


def _prefix(keys, i, j):
    """Common leading bits of the 64-bit words keys[i], keys[j]; for equal keys,
    64 plus the common leading bits of the 32-bit positions i and j."""
    x = int(keys[i]) ^ int(keys[j])
    if x:
        return 64 - x.bit_length()
    return 64 + 32 - (int(i) ^ int(j)).bit_length()


def radix_tree(sorted_keys):
    """Return (left, right, left_is_leaf, right_is_leaf) for the n-1 internal nodes."""
    n = len(sorted_keys)
    m = max(n - 1, 0)
    left = np.full(m, -1, np.int64)
    right = np.full(m, -1, np.int64)
    lleaf = np.zeros(m, bool)
    rleaf = np.zeros(m, bool)
    if n < 2:
        return left, right, lleaf, rleaf
    stack = [(0, 0, n - 1)]
    while stack:
        node, a, b = stack.pop()
        whole = _prefix(sorted_keys, a, b)
        g = a
        while g + 1 <= b - 1 and _prefix(sorted_keys, a, g + 1) > whole:
            g += 1
        left[node] = g
        right[node] = g + 1
        lleaf[node] = (g == a)
        rleaf[node] = (g + 1 == b)
        if g != a:
            stack.append((g, a, g))
        if g + 1 != b:
            stack.append((g + 1, g + 1, b))
    return left, right, lleaf, rleaf


def boxes(verts, tris, order, left, right, lleaf, rleaf):
    """Per internal node, the boxes of its left and right child: (lo_l, hi_l, lo_r, hi_r)."""
    v = np.asarray(verts, np.float32).reshape(-1, 3)
    t = np.asarray(tris, np.int64).reshape(-1, 3)[order]
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    leaf_lo = np.minimum(np.minimum(a, b), c)
    leaf_hi = np.maximum(np.maximum(a, b), c)
    m = left.shape[0]
    node_lo = np.zeros((m, 3), np.float32)
    node_hi = np.zeros((m, 3), np.float32)
    done = np.zeros(m, bool)

    def child(idx, is_leaf):
        return (leaf_lo[idx], leaf_hi[idx]) if is_leaf else (node_lo[idx], node_hi[idx])

    # post-order over the tree without recursion
    stack = [(0, False)] if m else []
    while stack:
        node, expanded = stack.pop()
        if not expanded:
            stack.append((node, True))
            if not rleaf[node]:
                stack.append((int(right[node]), False))
            if not lleaf[node]:
                stack.append((int(left[node]), False))
            continue
        llo, lhi = child(left[node], lleaf[node])
        rlo, rhi = child(right[node], rleaf[node])
        node_lo[node] = np.minimum(llo, rlo)
        node_hi[node] = np.maximum(lhi, rhi)
        done[node] = True
    lo_l = np.zeros((m, 3), np.float32)
    hi_l = np.zeros((m, 3), np.float32)
    lo_r = np.zeros((m, 3), np.float32)
    hi_r = np.zeros((m, 3), np.float32)
    for k in range(m):
        lo_l[k], hi_l[k] = child(left[k], lleaf[k])
        lo_r[k], hi_r[k] = child(right[k], rleaf[k])
    return lo_l, hi_l, lo_r, hi_r


def build(verts, tris):
    """Everything above in one call; returns a dict of arrays."""
    keys = morton_keys(verts, tris)
    skeys, order = sort_keys(keys)
    left, right, lleaf, rleaf = radix_tree(skeys)
    lo_l, hi_l, lo_r, hi_r = boxes(verts, tris, order, left, right, lleaf, rleaf)
    return dict(keys=keys, sorted_keys=skeys, order=order, left=left, right=right,
                left_leaf=lleaf, right_leaf=rleaf, lo_l=lo_l, hi_l=hi_l, lo_r=lo_r, hi_r=hi_r)
