"""The geometry behind the wedge search of vertical line lamps, checked in
FP64 on random configurations (CPU; the CUDA code itself is checked against
the per-source search and the oracle in tests/test_gpu_wedge.py).

1. Box test: a box meets the triangle spanned by the lamp line and the patch
   point iff its x/y slabs leave a parameter interval [a, b] inside [0, 1] on
   which the wedge's height range, linear in the parameter, overlaps the box's
   z range; checking only the ends a and b is exact.  Every box that some
   segment from a lamp point to the patch point crosses is accepted.
2. Lamp-height interval: a segment from lamp height z to the patch point can
   meet a triangle only if z lies in the central projection, from the patch
   point onto the lamp line, of the triangle's projection onto the wedge's
   vertical plane.  No source whose segment meets the triangle lies outside
   that interval.
"""
import math

import numpy as np


def _wedge_box(c, zlo, zhi, s, lo, hi):
    """The kernel's box test in exact-ish FP64 (no widening): c (2,) lamp
    axis, [zlo, zhi] lamp heights, s (3,) patch point, box lo/hi (3,)."""
    g = s[:2] - c
    a, b = 0.0, 1.0
    for k in range(2):
        if g[k] == 0.0:
            if not (lo[k] <= c[k] <= hi[k]):
                return False
            continue
        t0, t1 = (lo[k] - c[k]) / g[k], (hi[k] - c[k]) / g[k]
        a, b = max(a, min(t0, t1)), min(b, max(t0, t1))
    if a > b:
        return False
    zl = lambda t: zlo + t * (s[2] - zlo)  # noqa: E731
    zh = lambda t: zhi + t * (s[2] - zhi)  # noqa: E731
    return hi[2] >= min(zl(a), zl(b)) and lo[2] <= max(zh(a), zh(b))


def _segment_box(o, s, lo, hi):
    """Does the closed segment o -> s meet the box (slab test in FP64)?"""
    d = s - o
    a, b = 0.0, 1.0
    for k in range(3):
        if d[k] == 0.0:
            if not (lo[k] <= o[k] <= hi[k]):
                return False
            continue
        t0, t1 = (lo[k] - o[k]) / d[k], (hi[k] - o[k]) / d[k]
        a, b = max(a, min(t0, t1)), min(b, max(t0, t1))
    return a <= b


def test_wedge_box_test_accepts_every_box_a_segment_crosses():
    rng = np.random.default_rng(1)
    accepted_extra = crossed = 0
    for _ in range(20000):
        c = rng.uniform(-4, 4, 2)
        zlo = rng.uniform(0.2, 1.5)
        zhi = zlo + rng.uniform(0.0, 1.5)
        s = np.array([*rng.uniform(-4, 4, 2), rng.uniform(0, 3)])
        if rng.uniform() < 0.05:
            s[:2] = c                                          # patch straight below or above the lamp
        if rng.uniform() < 0.5:                                # near the wedge
            t = rng.uniform(0, 1)
            ctr = np.array([c[0] + t * (s[0] - c[0]), c[1] + t * (s[1] - c[1]),
                            rng.uniform(zlo, zhi) * (1 - t) + t * s[2]]) + rng.normal(0, 0.3, 3)
        else:
            ctr = np.array([*rng.uniform(-4, 4, 2), rng.uniform(0, 3)])
        half = rng.uniform(0.01, 1.0, 3)
        if rng.uniform() < 0.2:
            half[rng.integers(3)] = 0.0                        # flat boxes (axis-aligned walls)
        lo, hi = ctr - half, ctr + half
        zs = np.linspace(zlo, zhi, 9)
        hits = [_segment_box(np.array([c[0], c[1], z]), s, lo, hi) for z in zs]
        w = _wedge_box(c, zlo, zhi, s, lo, hi)
        if any(hits):
            crossed += 1
            assert w, (c, zlo, zhi, s, lo, hi)
        elif w:
            accepted_extra += 1                                # the wedge is a solid triangle: allowed
    assert crossed > 5000


def _segment_meets_triangle(o, s, a, b, c):
    d = s - o
    e1, e2 = b - a, c - a
    p = np.cross(d, e2)
    det = e1 @ p
    if abs(det) < 1e-14:
        return False
    r = o - a
    u = (r @ p) / det
    if u < 0 or u > 1:
        return False
    q = np.cross(r, e1)
    v = (d @ q) / det
    if v < 0 or u + v > 1:
        return False
    tau = (e2 @ q) / det
    return 0 < tau < 1


def test_lamp_height_interval_contains_every_blocked_source():
    rng = np.random.default_rng(2)
    delta = 1e-5 * 15.0
    hits = kept = tested = 0
    for _ in range(40000):
        c = rng.uniform(-5, 5, 2)
        K = 8
        oz = rng.uniform(0.3, 1.5) + 1.2 * (np.arange(K) + 0.5) / K
        s = np.array([*rng.uniform(-5, 5, 2), rng.uniform(0, 3)])
        g = s[:2] - c
        lam = rng.uniform(-0.2, 1.0)
        centre = np.array([c[0] + lam * g[0], c[1] + lam * g[1], rng.uniform(0, 3)])
        tri = centre + rng.normal(0, 0.3, (3, 3))
        lv = ((tri[:, :2] - c) @ g) / (g @ g)
        dmax = max(np.linalg.norm(s - np.array([c[0], c[1], z])) for z in oz)
        if lv.max() < 0.9990234375:
            zp = s[2] + (tri[:, 2] - s[2]) / (1 - lv)
            m = delta * dmax / np.sqrt(g @ g) / (1 - lv.max())
            inside = (oz >= zp.min() - m) & (oz <= zp.max() + m)
        else:
            inside = np.ones(K, bool)                          # next to the patch point: keep every source
        for q in range(K):
            h = _segment_meets_triangle(np.array([c[0], c[1], oz[q]]), s, *tri)
            hits += h
            assert not h or inside[q]
        kept += inside.sum()
        tested += K
    assert hits > 5000
    assert kept / tested < 0.5                                 # the filter does remove most sources


def _uniform_range(z0, z1, cz, wz0, wrdz, K):
    """The closed-form source index range of an evenly spaced lamp, in the
    kernel's FP32 operations."""
    f = np.float32
    t0 = min(max(f(f(f(f(z0) - f(cz)) - f(wz0)) * f(wrdz)), f(-4)), f(40))
    t1 = min(max(f(f(f(f(z1) - f(cz)) - f(wz0)) * f(wrdz)), f(-4)), f(40))
    return max(0, int(math.ceil(f(t0 - f(0.03125))))), min(K - 1, int(math.floor(f(t1 + f(0.03125)))))


def _violations(rng, spacing_factor, trials=20000):
    """Sources whose FP32 height lies in [z0, z1] but outside the closed-form
    range, for lamps whose step is spacing_factor times the smallest step the
    library lets take the closed form (2^-16 (16 B + 3 max|off|), B the scene's
    coordinate bound, candidates within 16 B)."""
    bad = 0
    for _ in range(trials):
        B = 10.0 ** rng.uniform(0, 3)
        K = int(rng.integers(2, 17))
        z0off = rng.uniform(-1, 1)
        cz = rng.uniform(-16 * B, 16 * B)
        span = rng.uniform(0.01, 2.0)
        dz_min = 2.0 ** -16 * (16 * B + 3 * (abs(z0off) + span))
        dz = dz_min * spacing_factor
        ideal = z0off + dz * np.arange(K)
        off = (ideal + rng.uniform(-dz / 64, dz / 64, K)).astype(np.float32)
        off[0] = np.float32(z0off)
        d_host = (float(off[-1]) - float(off[0])) / (K - 1)
        if not (d_host > 0 and np.all(np.abs(off.astype(np.float64) - (float(off[0]) + np.arange(K) * d_host))
                                      <= d_host / 64)):
            continue                                            # the host would not take the closed form
        oz = (np.float32(cz) + off).astype(np.float32)          # fl32(c.z + off)
        q = int(rng.integers(0, K))
        z_lo = float(oz[q]) - abs(rng.normal(0, dz)) * rng.integers(0, 2)
        z_hi = float(oz[q]) + abs(rng.normal(0, dz)) * rng.integers(0, 2)
        qlo, qhi = _uniform_range(z_lo, z_hi, cz, float(off[0]), 1.0 / d_host, K)
        inside = np.flatnonzero((oz >= np.float32(z_lo)) & (oz <= np.float32(z_hi)))
        bad += int(np.sum((inside < qlo) | (inside > qhi)))
    return bad


def test_closed_form_source_range_keeps_every_source_at_the_allowed_spacing():
    """At the smallest step the library allows for the closed form, no source
    whose FP32 height lies in the lamp-height interval falls outside the
    closed-form index range; at a thousandth of it some would (which is why
    closer sources take the per-source height test)."""
    rng = np.random.default_rng(5)
    assert _violations(rng, 1.0) == 0
    assert _violations(np.random.default_rng(6), 1e-3, trials=2000) > 0
