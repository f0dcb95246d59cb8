"""Oracle for the candidate features of the learned proposal (FP64 numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Features of a candidate lamp position c (the proposal network's input):
  h_b   b = 0..63: the fraction of the surface area whose patch point lies at a
        distance d = |s_j - c| with E_b <= d^2 < E_{b+1}, where the bin edges are
        log-spaced from 0.1 m to 25 m: e_b = 0.1 * 250^(b/64) (b = 1..63),
        E_b = fl32(e_b^2) (E_0 = 0, E_64 = infinity)
  clear the distance from c to the nearest triangle (point-triangle distance)
  z     the height of c
Distances near a bin edge decide an integer (the bin), so `ambiguous` marks
patches whose d^2 lies within a relative 1e-6 of an edge: an FP32 evaluation
may put them in the neighbouring bin.
"""
from __future__ import annotations

import numpy as np

NBINS = 64
D0, D1 = 0.1, 25.0


def bin_edges_sq():
    """E_1..E_63 as float32 (squared metres)."""
    b = np.arange(1, NBINS, dtype=np.float64)
    e = D0 * (D1 / D0) ** (b / NBINS)
    return (e * e).astype(np.float32)


def _point_triangle_distance(p, a, b, c):
    """Distance from p (3,) to triangles (n,3) each: closest point by regions."""
    ab, ac, ap = b - a, c - a, p - a
    d1, d2 = (ab * ap).sum(1), (ac * ap).sum(1)
    bp = p - b
    d3, d4 = (ab * bp).sum(1), (ac * bp).sum(1)
    cp = p - c
    d5, d6 = (ab * cp).sum(1), (ac * cp).sum(1)
    va = d3 * d6 - d5 * d4
    vb = d5 * d2 - d1 * d6
    vc = d1 * d4 - d3 * d2
    res = np.empty(a.shape[0])
    done = np.zeros(a.shape[0], bool)

    def put(mask, q):
        m = mask & ~done
        res[m] = np.linalg.norm(p - q[m], axis=1)
        done[m] = True
    put((d1 <= 0) & (d2 <= 0), a)
    put((d3 >= 0) & (d4 <= d3), b)
    put((d6 >= 0) & (d5 <= d6), c)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = d1 / (d1 - d3)
        put((vc <= 0) & (d1 >= 0) & (d3 <= 0), a + v[:, None] * ab)
        w = d2 / (d2 - d6)
        put((vb <= 0) & (d2 >= 0) & (d6 <= 0), a + w[:, None] * ac)
        w2 = (d4 - d3) / ((d4 - d3) + (d5 - d6))
        put((va <= 0) & ((d4 - d3) >= 0) & ((d5 - d6) >= 0), b + w2[:, None] * (c - b))
        denom = 1.0 / (va + vb + vc)
        vv, ww = vb * denom, vc * denom
        put(np.ones(a.shape[0], bool), a + ab * vv[:, None] + ac * ww[:, None])
    return res


def features(verts, tris, centroid, area, cand):
    """(nc, 66) features and (nc, np) ambiguity mask."""
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64)
    s = np.asarray(centroid, np.float32).astype(np.float64)
    a = np.asarray(area, np.float32).astype(np.float64)
    cand = np.asarray(cand, np.float32).astype(np.float64)
    E = bin_edges_sq().astype(np.float64)
    tot = a.sum()
    out = np.zeros((cand.shape[0], NBINS + 2))
    amb = np.zeros((cand.shape[0], s.shape[0]), bool)
    A, B, C = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    for i, c in enumerate(cand):
        d2 = ((s - c) ** 2).sum(1)
        b = np.searchsorted(E, d2, side="right")          # number of edges <= d2
        out[i, :NBINS] = np.bincount(b, weights=a, minlength=NBINS) / tot
        rel = np.abs(d2[:, None] - E[None, :]) <= 1e-6 * np.maximum(d2[:, None], 1e-30)
        amb[i] = rel.any(1)
        out[i, NBINS] = _point_triangle_distance(c, A, B, C).min() if t.shape[0] else np.inf
        out[i, NBINS + 1] = c[2]
    return out, amb


EFF_EDGES = np.array([0.5, 0.7, 0.8, 0.9, 0.95], np.float32)
HARD_BINS, EFF_BINS = 8, 6


def probe_features(A, area):
    """(nc, 48) visibility sketch and the per-patch hardness ambiguity mask.

    From the irradiance of all candidates on a probe sample of patches:
    E*_j = max_i A[i][j] (the best any candidate gives patch j), the lit set
    L = {j : E*_j > 0}, Ebar = sum_L a_j E*_j / sum_L a_j; patch j's hardness
    h_j = floor(log2(E*_j / Ebar)) + 4 clamped to [0, 7]; candidate i's
    efficiency on it A[i][j] / E*_j, binned at 0.5, 0.7, 0.8, 0.9, 0.95.
    feat[i][6 h + e] = the lit area in that cell / sum_L a_j.  The ratios that
    pick a bin are taken in FP32 (the kernel's precision), so the efficiency
    bin is exact; Ebar is a sum, so a ratio within 1e-5 of a power of two is
    flagged ambiguous (its hardness bin may differ by one)."""
    A32 = np.asarray(A, np.float32)
    a = np.asarray(area, np.float32).astype(np.float64)
    nc, m = A32.shape
    out = np.zeros((nc, HARD_BINS * EFF_BINS))
    amb = np.zeros(m, bool)
    if nc == 0 or m == 0:
        return out, amb
    emax = A32.max(0)
    lit = emax > 0
    if not lit.any():
        return out, amb
    S1 = a[lit].sum()
    ebar = np.float32((a[lit] * emax[lit].astype(np.float64)).sum() / S1)
    r = emax[lit] / ebar                                   # float32 division
    _, ex = np.frexp(r)
    h = np.clip(ex - 1 + 4, 0, HARD_BINS - 1)
    l2 = np.log2(r.astype(np.float64))
    amb[np.flatnonzero(lit)] = np.abs(l2 - np.round(l2)) <= 1e-5 / np.log(2)
    eff = A32[:, lit] / emax[lit][None, :]                 # float32 division
    eb = np.searchsorted(EFF_EDGES, eff, side="right")     # number of edges <= e
    cell = h[None, :] * EFF_BINS + eb
    w = a[lit] / S1
    for i in range(nc):
        out[i] = np.bincount(cell[i], weights=w, minlength=HARD_BINS * EFF_BINS)
    return out, amb
