"""CPU oracle for the irradiance-matrix hot path (paper Sec. III-B and IV-C).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product package never does.
It shares no code with the CUDA library.

Contents
  irradiance(...)       FP64 brute-force E_ij, per-source visibility and grazing
                        flags (C, uvc_oracle.c), Eq. (7) and its visibility rule
  lbvh.*                Morton codes, stable key sort, binary radix tree and
                        bounding boxes by their definitions (Python/numpy)
  fluence(A, t)         mu = A^T t in FP64 (Eq. (5))
  coverage(mu, area..)  area-weighted fraction of patches with mu >= mu_min

Every function here is pinned by tests in tests/test_oracle_*.py against closed
forms, invariants and brute force; see the module docstrings for which.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "uvc_oracle.c")
_LIB = os.path.join(_HERE, "libuvc_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """ctypes handle on a compiled copy of uvc_oracle.c."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.uvco_irradiance.argtypes = [P, i64, P, i64, P, P, P, i64, P, i64, P, P, ctypes.c_int32,
                                    ctypes.c_double, P, i64, ctypes.c_double, P, P, P, ctypes.c_int]
    lib.uvco_irradiance.restype = ctypes.c_int
    lib.uvco_irradiance_bvh.argtypes = lib.uvco_irradiance.argtypes
    lib.uvco_irradiance_bvh.restype = ctypes.c_int
    lib.uvco_area_mean.argtypes = [P, i64, P, i64, P, P, P, P, P, i64, P, i64, P, P, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_float, P, i64, ctypes.c_double, P, P, P, ctypes.c_int]
    lib.uvco_area_mean.restype = ctypes.c_int
    lib.uvco_area_mean_bvh.argtypes = lib.uvco_area_mean.argtypes
    lib.uvco_area_mean_bvh.restype = ctypes.c_int
    lib.uvco_raster.argtypes = [P, i64, P, i64, P, P, i64, P, P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                ctypes.c_double, P, P, ctypes.c_int]
    lib.uvco_raster.restype = ctypes.c_int
    lib.uvco_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def max_threads() -> int:
    return int(_load().uvco_max_threads())


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def grazing_eps(verts, rel: float = 1e-7) -> float:
    """Grazing distance: rel times the diagonal of the mesh's bounding box."""
    v = np.asarray(verts, np.float64).reshape(-1, 3)
    if v.shape[0] == 0:
        return 0.0
    return rel * float(np.linalg.norm(v.max(axis=0) - v.min(axis=0)))


def irradiance(verts, tris, centroid, normal, excl, cand, offsets, weights, power,
               pairs=None, eps=None, flags=True, threads=0, lib=None, bvh=False):
    """FP64 brute-force irradiance (bvh=True: the same entries through the
    oracle's CPU hierarchy, for large samples).

    pairs: None for the full (nc, np) matrix, else an (npairs, 2) array of (i, j).
    Returns (E, vis, flag): E float64 (nc,np) or (npairs,), vis uint8 (..., K),
    flag uint8 grazing bits (or None when flags=False).
    lib: an alternative compiled copy (load_library), default the built oracle.
    """
    lib = lib or _load()
    verts = _c(verts, np.float32).reshape(-1, 3)
    tris = _c(tris, np.int32).reshape(-1, 3)
    centroid = _c(centroid, np.float32).reshape(-1, 3)
    normal = _c(normal, np.float32).reshape(-1, 3)
    excl = _c(excl, np.int32).reshape(-1, 2)
    cand = _c(cand, np.float32).reshape(-1, 3)
    offsets = _c(offsets, np.float32).reshape(-1, 3)
    weights = _c(weights, np.float32).reshape(-1)
    K = offsets.shape[0]
    assert weights.shape[0] == K
    nc, np_ = cand.shape[0], centroid.shape[0]
    if pairs is None:
        shape = (nc, np_)
        npairs = nc * np_
        pp = None
    else:
        pp = _c(pairs, np.int64).reshape(-1, 2)
        npairs = pp.shape[0]
        shape = (npairs,)
    if eps is None:
        eps = grazing_eps(verts)
    E = np.zeros(npairs, np.float64)
    vis = np.zeros(npairs * K, np.uint8)
    flag = np.zeros(npairs, np.uint8) if flags else None
    ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    fn = lib.uvco_irradiance_bvh if bvh else lib.uvco_irradiance
    rc = fn(ptr(verts), verts.shape[0], ptr(tris), tris.shape[0],
                             ptr(centroid), ptr(normal), ptr(excl), np_, ptr(cand), nc,
                             ptr(offsets), ptr(weights), K, float(power),
                             ptr(pp), npairs, float(eps), ptr(E), ptr(vis), ptr(flag), int(threads))
    if rc != 0:
        raise ValueError(f"oracle: invalid input (rc={rc})")
    E = E.reshape(shape)
    vis = vis.reshape(shape + (K,))
    if flag is not None:
        flag = flag.reshape(shape)
    return E, vis, flag


PULL = 1e-3   # check points: patch vertices moved this fraction of the way to the centroid


def area_mean(verts, tris, centroid, normal, area, excl, ptri, cand, offsets, weights, power, delta=PULL,
              pairs=None, eps=None, flags=True, threads=0, bvh=False):
    """FP64 area-mean irradiance (solid-angle closed form where every check
    segment of a source is unoccluded, centroid sample otherwise), see
    uvco_area_mean.  Returns (E, nclosed, flag) shaped like irradiance().
    bvh=True runs every check segment through the CPU hierarchy
    (uvco_area_mean_bvh): the same results, fast enough for whole rows of
    large rooms."""
    lib = _load()
    verts = _c(verts, np.float32).reshape(-1, 3)
    tris = _c(tris, np.int32).reshape(-1, 3)
    centroid = _c(centroid, np.float32).reshape(-1, 3)
    normal = _c(normal, np.float32).reshape(-1, 3)
    area = _c(area, np.float32).reshape(-1)
    excl = _c(excl, np.int32).reshape(-1, 2)
    ptri = _c(ptri, np.float32).reshape(-1, 18)
    cand = _c(cand, np.float32).reshape(-1, 3)
    offsets = _c(offsets, np.float32).reshape(-1, 3)
    weights = _c(weights, np.float32).reshape(-1)
    K = offsets.shape[0]
    nc, np_ = cand.shape[0], centroid.shape[0]
    assert ptri.shape[0] == np_ and area.shape[0] == np_
    if pairs is None:
        shape, npairs, pp = (nc, np_), nc * np_, None
    else:
        pp = _c(pairs, np.int64).reshape(-1, 2)
        shape, npairs = (pp.shape[0],), pp.shape[0]
    if eps is None:
        eps = grazing_eps(verts)
    E = np.zeros(npairs, np.float64)
    ncl = np.zeros(npairs, np.uint8)
    flag = np.zeros(npairs, np.uint8) if flags else None
    ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    fn = lib.uvco_area_mean_bvh if bvh else lib.uvco_area_mean
    rc = fn(ptr(verts), verts.shape[0], ptr(tris), tris.shape[0], ptr(centroid), ptr(normal), ptr(area), ptr(excl),
            ptr(ptri), np_, ptr(cand), nc, ptr(offsets), ptr(weights), K, float(power), float(delta), ptr(pp), npairs,
            float(eps), ptr(E), ptr(ncl), ptr(flag), int(threads))
    if rc != 0:
        raise ValueError(f"oracle: invalid input (rc={rc})")
    return E.reshape(shape), ncl.reshape(shape), None if flag is None else flag.reshape(shape)


def area_mean_scene(scene, pairs=None, **kw):
    """area_mean() on a synth.Scene that carries its patch geometry."""
    L = scene.lamp
    return area_mean(scene.verts, scene.tris, scene.centroid, scene.normal, scene.area, scene.excl, scene.ptri,
                     scene.cand, L.offsets, L.weights, L.power, pairs=pairs, **kw)


def raster(verts, tris, tri_normal, cand, offsets, weights, power, R, rel=1e-5, ambiguity=True, threads=0):
    """FP64 visibility-cube estimator by ray casting through the pixel centres
    (uvco_raster): per candidate and triangle the flux F (W) and the bound amb
    on the flux an FP32 rasteriser may legitimately move (or None)."""
    lib = _load()
    verts = _c(verts, np.float32).reshape(-1, 3)
    tris = _c(tris, np.int32).reshape(-1, 3)
    tri_normal = _c(tri_normal, np.float32).reshape(-1, 3)
    cand = _c(cand, np.float32).reshape(-1, 3)
    offsets = _c(offsets, np.float32).reshape(-1, 3)
    weights = _c(weights, np.float32).reshape(-1)
    nc, nt = cand.shape[0], tris.shape[0]
    F = np.zeros((nc, nt), np.float64)
    amb = np.zeros((nc, nt), np.float64) if ambiguity else None
    ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    rc = lib.uvco_raster(ptr(verts), verts.shape[0], ptr(tris), nt, ptr(tri_normal), ptr(cand), nc, ptr(offsets),
                         ptr(weights), offsets.shape[0], float(power), int(R), float(rel), ptr(F), ptr(amb),
                         int(threads))
    if rc != 0:
        raise ValueError(f"oracle: invalid input (rc={rc})")
    return F, amb


def pixel_solid_angles(R):
    """(R, R) solid angles of one cube face's pixels (FP64, the closed form
    used by uvco_raster), indexed [py, px]."""
    e = 2.0 * np.arange(R + 1) / R - 1.0
    G = lambda u, v: np.arctan(u * v / np.sqrt(1.0 + u * u + v * v))  # noqa: E731
    U, V = np.meshgrid(e, e, indexing="xy")
    g = G(U, V)
    return g[1:, 1:] - g[1:, :-1] - g[:-1, 1:] + g[:-1, :-1]


def irradiance_scene(scene, pairs=None, **kw):
    """irradiance() on a synth.Scene."""
    L = scene.lamp
    return irradiance(scene.verts, scene.tris, scene.centroid, scene.normal, scene.excl,
                      scene.cand, L.offsets, L.weights, L.power, pairs=pairs, **kw)


def fluence(A, t):
    """mu[v, j] = sum_i t[v, i] A[i, j] in FP64 (Eq. (5): fluence is the dwell-
    time weighted sum of the irradiance columns)."""
    A = np.asarray(A, np.float64)
    t = np.atleast_2d(np.asarray(t, np.float64))
    return t @ A


def coverage(mu, area, mu_min):
    """Fraction of the surface area whose fluence reaches mu_min, per dwell vector,
    and the fraction of patches doing so.  The threshold test is taken in FP32
    (mu and mu_min as FP32), the sums in FP64."""
    mu = np.atleast_2d(np.asarray(mu, np.float32))
    area = np.asarray(area, np.float32).astype(np.float64)
    ok = mu >= np.float32(mu_min)
    total = area.sum()
    by_area = (ok * area[None, :]).sum(axis=1) / total if total > 0 else np.zeros(mu.shape[0])
    by_count = ok.sum(axis=1) / max(1, mu.shape[1])
    return by_area, by_count
