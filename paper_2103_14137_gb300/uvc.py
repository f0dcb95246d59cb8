"""Thin ctypes binding of libuvc (include/uvc.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies device memory and
the current CUDA stream.  Functions carry the C-ABI names without the `uvc_`
prefix.  If libuvc.so is missing the import of this module still works, but
every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# UVC_LIB_PATH selects another build of the library (the checked build in its test)
LIB_PATH = os.environ.get("UVC_LIB_PATH") or os.path.join(_HERE, "libuvc.so")
MAX_SOURCES = 32

UVC_OK, UVC_E_INVAL, UVC_E_NOMEM, UVC_E_CUDA, UVC_E_STACK, UVC_E_TIMEOUT, UVC_E_SCRATCH, UVC_E_BOUNDS = range(8)
UVC_LIB_CHECKED = 1
UVC_BUILD_LBVH_ONLY = 1


class UvcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class _Lamp(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("power", ctypes.c_float),
                ("offsets", (ctypes.c_float * 3) * MAX_SOURCES), ("weight", ctypes.c_float * MAX_SOURCES)]


class _Patches(ctypes.Structure):
    _fields_ = [("centroid", ctypes.c_void_p), ("normal", ctypes.c_void_p),
                ("area", ctypes.c_void_p), ("excl", ctypes.c_void_p)]


class _Job(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("cand", ctypes.c_void_p), ("nc", ctypes.c_int64),
                ("lamp", ctypes.c_int32), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("vis", ctypes.c_void_p)]


class _BatchConfig(ctypes.Structure):
    _fields_ = [("cand_per_task", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


_lib = None


def library():
    """The loaded libuvc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libuvc.so is not built ({LIB_PATH}); run paper_2103_14137_gb300.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "uvc_build_scene": [P, i64, P, i64, ctypes.POINTER(_Patches), i64, P, ctypes.POINTER(P)],
        "uvc_build_scene_ex": [P, i64, P, i64, ctypes.POINTER(_Patches), i64, ctypes.c_uint32, P, ctypes.POINTER(P)],
        "uvc_free_scene": [P],
        "uvc_irradiance_matrix": [P, P, i64, ctypes.POINTER(_Lamp), P, i64, P, P],
        "uvc_fluence": [P, P, i64, i64, P, i32, P, P],
        "uvc_irradiance_area_mean": [P, P, i64, ctypes.POINTER(_Lamp), P, P, i64, P, P],
        "uvc_irradiance_raster": [P, P, P, i64, ctypes.POINTER(_Lamp), i32, P, i64, P, ctypes.c_size_t, P],
        "uvc_irradiance_counters": [P, P, i64, ctypes.POINTER(_Lamp), P, i64, P, P],
        "uvc_fluence_streamed": [P, P, i64, ctypes.POINTER(_Lamp), P, i32, P, P],
        "uvc_fluence_streamed_noalloc": [P, P, i64, ctypes.POINTER(_Lamp), P, i32, P, P],
        "uvc_coverage": [P, P, i32, ctypes.c_float, P, P, P],
        "uvc_scene_status": [P, P],
        "uvc_set_wedge_traversal": [i32, ctypes.POINTER(i32)],
        "uvc_scene_info": [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "uvc_scene_set_limits": [P, i32, i32],
        "uvc_scene_export_bvh": [P, P, P, P, P],
        "uvc_probe_l2_read": [P, ctypes.c_size_t, i32, P, P],
        "uvc_scene_export_traversal": [P, P, P, P, P, P, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float)],
        "uvc_irradiance_candidates_per_task": [],
        "uvc_set_fluence_tensor_cores": [i32, ctypes.POINTER(i32)],
    }
    sig.update({
        "uvc_batch_create": [ctypes.POINTER(_Job), i32, ctypes.POINTER(_Lamp), i32, P, ctypes.c_size_t, P,
                             ctypes.POINTER(P)],
        "uvc_batch_launch": [P, P],
        "uvc_batch_set_config": [P, ctypes.POINTER(_BatchConfig), P],
        "uvc_batch_autotune": [P, ctypes.c_double, ctypes.POINTER(_BatchConfig), P],
        "uvc_batch_info": [P, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(_BatchConfig)],
        "uvc_batch_free": [P],
        "uvc_candidate_features": [P, P, i64, P, i64, P],
        "uvc_probe_features": [P, i64, i64, i64, P, P, P, i64, P],
        "uvc_select_top": [P, i64, i64, P, P, P, P],
        "uvc_probe_lost": [P, i64, i64, i64, P, i64, P, P, P, P],
        "uvc_mark_best": [P, i64, i64, i64, P, ctypes.c_float, i32, P],
        "uvc_group_boost": [P, i64, i32, ctypes.c_float, P],
        "uvc_mlp_create": [i32, i32, i32, ctypes.c_uint64, ctypes.POINTER(P)],
        "uvc_mlp_free": [P],
        "uvc_mlp_params": [P, P, i64, i32],
        "uvc_mlp_forward": [P, P, i32, P, P],
        "uvc_mlp_train_step": [P, P, P, P, i32, ctypes.c_float, P, P],
        "uvc_mlp_grads": [P, P, i64],
    })
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.uvc_batch_workspace_bytes.argtypes = [i32, i32]
    lib.uvc_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.uvc_raster_workspace_bytes.argtypes = [P, ctypes.POINTER(_Lamp), i32, i64]
    lib.uvc_raster_workspace_bytes.restype = ctypes.c_size_t
    lib.uvc_probe_features_work_bytes.argtypes = [i64]
    lib.uvc_probe_features_work_bytes.restype = ctypes.c_size_t
    lib.uvc_mlp_param_count.argtypes = [P]
    lib.uvc_mlp_param_count.restype = i64
    lib.uvc_library_flags.argtypes = []
    lib.uvc_library_flags.restype = ctypes.c_uint32
    lib.uvc_status_string.argtypes = [ctypes.c_int]
    lib.uvc_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def library_flags() -> int:
    """Build flags of the loaded library (UVC_LIB_CHECKED for the checked build)."""
    return int(library().uvc_library_flags())


def status_string(status: int) -> str:
    return library().uvc_status_string(int(status)).decode()


def _check(rc: int, what: str):
    if rc != UVC_OK:
        raise UvcError(rc, what)


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _row_layout(shape, strides, name, nrows: int, ncols: int) -> int:
    """Row stride (lda) of an (nrows, >= ncols) matrix with unit column stride
    whose rows may be padded; rejects every layout the library would read or
    write outside of (too few rows or columns, overlapping rows)."""
    if len(shape) != 2:
        raise TypeError(f"{name} must be 2-D")
    rows, cols = shape
    if rows != nrows:
        raise ValueError(f"{name} must have {nrows} rows, got {rows}")
    if cols < ncols:
        raise ValueError(f"{name} must have at least {ncols} columns, got {cols}")
    if rows * cols == 0:
        return cols
    if strides[1] != 1:
        raise ValueError(f"{name} must have unit column stride")
    if rows > 1 and strides[0] < cols:
        raise ValueError(f"{name} has overlapping rows (row stride {strides[0]} < {cols} columns)")
    return strides[0] if rows > 1 else cols


def _matrix_rows(x: torch.Tensor, name, nrows: int, ncols: int):
    """A float32 CUDA matrix of nrows rows and at least ncols columns, unit
    column stride, rows possibly padded (a view of the first columns of a
    wider buffer): (pointer, row stride)."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    _on_current_device(x, name)
    lda = _row_layout(tuple(x.shape), tuple(x.stride()), name, nrows, ncols)
    return ctypes.c_void_p(x.data_ptr() if x.numel() else 0), lda


def _on_current_device(x: torch.Tensor, name):
    """The library runs on the calling thread's current device; a tensor on
    another GPU would hand its kernels pointers into another device's memory."""
    cur = torch.cuda.current_device()
    if x.device.index != cur:
        raise ValueError(f"{name} is on cuda:{x.device.index}, the current device is cuda:{cur}")


def _dev(x: torch.Tensor, dtype, name, shape=None):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    _on_current_device(x, name)
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(x.shape)}")
    return ctypes.c_void_p(x.data_ptr() if x.numel() else 0)


class Lamp:
    """K point sources: offsets (K,3) metres from the candidate point, weights
    (K,) fractions of the total power P (paper Sec. IV-C, non-point lights)."""

    def __init__(self, offsets, weights, power: float):
        self.offsets = np.asarray(offsets, np.float32).reshape(-1, 3)
        self.weights = np.asarray(weights, np.float32).reshape(-1)
        self.power = float(power)
        if not 1 <= self.offsets.shape[0] <= MAX_SOURCES or self.weights.shape[0] != self.offsets.shape[0]:
            raise ValueError("a lamp has 1..32 sources with one weight each")

    @property
    def K(self) -> int:
        return int(self.offsets.shape[0])

    def _c(self) -> _Lamp:
        c = _Lamp()
        c.K = self.K
        c.power = self.power
        for m in range(self.K):
            for k in range(3):
                c.offsets[m][k] = float(self.offsets[m, k])
            c.weight[m] = float(self.weights[m])
        return c


def point_lamp(power: float) -> Lamp:
    return Lamp(np.zeros((1, 3)), np.ones(1), power)


class Scene:
    """A built scene (uvc_build_scene); owns device memory until free().  It
    lives on the device that was current when it was built and is used only
    while that device is current."""

    def __init__(self, handle, keepalive=()):
        self._h = handle
        self.device = torch.cuda.current_device()
        nt, np_, depth = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(library().uvc_scene_info(handle, ctypes.byref(nt), ctypes.byref(np_), ctypes.byref(depth)),
               "uvc_scene_info")
        self.nt, self.np, self.depth = nt.value, np_.value, depth.value

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("scene already freed")
        cur = torch.cuda.current_device()
        if cur != self.device:
            raise ValueError(f"scene was built on cuda:{self.device}, the current device is cuda:{cur}")
        return self._h

    def free(self):
        if self._h is not None:
            library().uvc_free_scene(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_scene(verts, tris, centroid, normal, area, excl, stream=None, lbvh_only=False) -> Scene:
    """uvc_build_scene (lbvh_only=False) or uvc_build_scene_ex(UVC_BUILD_LBVH_ONLY)."""
    nv, nt, np_ = verts.shape[0], tris.shape[0], centroid.shape[0]
    p = _Patches(_dev(centroid, torch.float32, "centroid", (np_, 3)), _dev(normal, torch.float32, "normal", (np_, 3)),
                 _dev(area, torch.float32, "area", (np_,)), _dev(excl, torch.int32, "excl", (np_, 2)))
    out = ctypes.c_void_p()
    args = (_dev(verts, torch.float32, "verts", (nv, 3)), nv, _dev(tris, torch.int32, "tris", (nt, 3)), nt,
            ctypes.byref(p), np_)
    if lbvh_only:
        rc = library().uvc_build_scene_ex(*args, UVC_BUILD_LBVH_ONLY, _stream(stream), ctypes.byref(out))
        _check(rc, "uvc_build_scene_ex")
    else:
        rc = library().uvc_build_scene(*args, _stream(stream), ctypes.byref(out))
        _check(rc, "uvc_build_scene")
    return Scene(out)


def irradiance_matrix(scene: Scene, cand, lamp: Lamp, A=None, vis=None, with_vis=False, stream=None):
    """A (nc, np) float32 and, if requested, vis (K, nc, ceil(np/32)) uint32 bitmask.
    A may be a larger (nc, lda) buffer; only columns [0, np) are written."""
    nc = cand.shape[0]
    if A is None:
        A = torch.empty((nc, scene.np), dtype=torch.float32, device=cand.device)
    if with_vis and vis is None:
        vis = torch.empty((lamp.K, nc, (scene.np + 31) // 32), dtype=torch.int32, device=cand.device)
    if A.dim() != 2 or A.shape[0] != nc:
        raise ValueError("A must be (nc, lda)")
    vptr = None if vis is None else _dev(vis, torch.int32, "vis", (lamp.K, nc, (scene.np + 31) // 32))
    L = lamp._c()
    aptr, lda = _matrix_rows(A, "A", nc, scene.np)
    rc = library().uvc_irradiance_matrix(scene.handle, _dev(cand, torch.float32, "cand", (nc, 3)), nc,
                                         ctypes.byref(L), aptr, lda, vptr, _stream(stream))
    _check(rc, "uvc_irradiance_matrix")
    return A, vis


COUNTER_NAMES = ("node_visits", "leaf_tests", "traversals", "lane_box_tests", "lane_tri_tests", "facing_segments",
                 "lane_wedge_box_tests", "lane_wedge_plane_tests")


def set_wedge_traversal(enable: bool) -> bool:
    """Search a vertical line lamp's sources as one wedge per (candidate,
    patch) (True, the default) or source by source (False); returns the
    previous setting (see uvc_set_wedge_traversal)."""
    prev = ctypes.c_int32(0)
    _check(library().uvc_set_wedge_traversal(1 if enable else 0, ctypes.byref(prev)), "uvc_set_wedge_traversal")
    return bool(prev.value)


def set_fluence_tensor_cores(enable: bool) -> bool:
    """Run A^T t on the tensor cores (True, the default) or the CUDA cores
    (False) where the rows of A allow it; returns the previous setting (see
    uvc_set_fluence_tensor_cores)."""
    prev = ctypes.c_int32(0)
    _check(library().uvc_set_fluence_tensor_cores(1 if enable else 0, ctypes.byref(prev)),
           "uvc_set_fluence_tensor_cores")
    return bool(prev.value)


def irradiance_counters(scene: Scene, cand, lamp: Lamp, A=None, stream=None) -> dict:
    """Instrumented irradiance run: traversal counts (see uvc_irradiance_counters)."""
    nc = cand.shape[0]
    if A is None:
        A = torch.empty((nc, scene.np), dtype=torch.float32, device=cand.device)
    out = np.zeros(len(COUNTER_NAMES), np.uint64)
    L = lamp._c()
    aptr, lda = _matrix_rows(A, "A", nc, scene.np)
    rc = library().uvc_irradiance_counters(scene.handle, _dev(cand, torch.float32, "cand", (nc, 3)), nc,
                                           ctypes.byref(L), aptr, lda, ctypes.c_void_p(out.ctypes.data),
                                           _stream(stream))
    _check(rc, "uvc_irradiance_counters")
    return dict(zip(COUNTER_NAMES, (int(x) for x in out)))


def irradiance_area_mean(scene: Scene, cand, lamp: Lamp, ptri, A=None, with_closed=False, stream=None):
    """Patch-mean irradiance (nc, np): solid-angle closed form for sources that
    see every check point of a patch, centroid sample otherwise.  ptri is the
    (np, 2, 3, 3) float32 patch geometry.  Returns (A, nclosed or None)."""
    nc = cand.shape[0]
    if A is None:
        A = torch.empty((nc, scene.np), dtype=torch.float32, device=cand.device)
    ncl = torch.empty((nc, scene.np), dtype=torch.uint8, device=cand.device) if with_closed else None
    L = lamp._c()
    aptr, lda = _matrix_rows(A, "A", nc, scene.np)
    rc = library().uvc_irradiance_area_mean(scene.handle, _dev(cand, torch.float32, "cand", (nc, 3)), nc,
                                            ctypes.byref(L), _dev(ptri, torch.float32, "ptri", (scene.np, 2, 3, 3)),
                                            aptr, lda, None if ncl is None else _dev(ncl, torch.uint8, "nclosed"),
                                            _stream(stream))
    _check(rc, "uvc_irradiance_area_mean")
    return A, ncl


def raster_workspace(scene: Scene, lamp: Lamp, R: int, cand_per_batch: int, device="cuda"):
    L = lamp._c()
    n = int(library().uvc_raster_workspace_bytes(scene.handle, ctypes.byref(L), int(R), int(cand_per_batch)))
    if n == 0:
        raise UvcError(UVC_E_INVAL, "uvc_raster_workspace_bytes")
    return torch.empty(n, dtype=torch.uint8, device=device)


def irradiance_raster(scene: Scene, tri_normal, cand, lamp: Lamp, R: int = 512, A=None, workspace=None,
                      cand_per_batch: int = 8, stream=None):
    """The visibility-cube estimator: (nc, nt) mean irradiance per triangle."""
    nc = cand.shape[0]
    if A is None:
        A = torch.empty((nc, scene.nt), dtype=torch.float32, device=cand.device)
    if workspace is None:
        workspace = raster_workspace(scene, lamp, R, max(1, min(cand_per_batch, nc)), cand.device)
    L = lamp._c()
    aptr, lda = _matrix_rows(A, "A", nc, scene.nt)
    rc = library().uvc_irradiance_raster(scene.handle, _dev(tri_normal, torch.float32, "tri_normal", (scene.nt, 3)),
                                         _dev(cand, torch.float32, "cand", (nc, 3)), nc, ctypes.byref(L), int(R),
                                         aptr, lda, _scratch(workspace, 0, "workspace"),
                                         workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "uvc_irradiance_raster")
    return A


def fluence(scene: Scene, A, t, mu=None, stream=None):
    """mu (nvec, np) = t (nvec, nc) @ A (nc, np); A may be a view of the
    first np columns of a wider buffer (padded rows)."""
    nvec, nc = t.shape
    if mu is None:
        mu = torch.empty((nvec, scene.np), dtype=torch.float32, device=t.device)
    aptr, lda = _matrix_rows(A, "A", nc, scene.np)
    rc = library().uvc_fluence(scene.handle, aptr, nc, lda, _dev(t, torch.float32, "t", (nvec, nc)), nvec,
                               _dev(mu, torch.float32, "mu", (nvec, scene.np)), _stream(stream))
    _check(rc, "uvc_fluence")
    return mu


def fluence_streamed(scene: Scene, cand, lamp: Lamp, t, mu=None, stream=None):
    nvec, nc = t.shape
    if mu is None:
        mu = torch.empty((nvec, scene.np), dtype=torch.float32, device=t.device)
    L = lamp._c()
    rc = library().uvc_fluence_streamed(scene.handle, _dev(cand, torch.float32, "cand", (nc, 3)), nc,
                                        ctypes.byref(L), _dev(t, torch.float32, "t", (nvec, nc)), nvec,
                                        _dev(mu, torch.float32, "mu", (nvec, scene.np)), _stream(stream))
    _check(rc, "uvc_fluence_streamed")
    return mu


def fluence_streamed_noalloc(scene: Scene, cand, lamp: Lamp, t, mu, stream=None):
    """fluence_streamed for callers that cannot allocate device memory during
    the call (their allocator holds the device, or allocation is forbidden
    after start-up): the library's partial sums go to its fixed 64 MiB device
    array.  `mu` (nvec, np) must be supplied by the caller; nothing is
    allocated here.  Raises UvcError(UVC_E_SCRATCH) when 4*nvec*np > 64 MiB - 256 B."""
    nvec, nc = t.shape
    L = lamp._c()
    rc = library().uvc_fluence_streamed_noalloc(scene.handle, _dev(cand, torch.float32, "cand", (nc, 3)), nc,
                                                ctypes.byref(L), _dev(t, torch.float32, "t", (nvec, nc)), nvec,
                                                _dev(mu, torch.float32, "mu", (nvec, scene.np)), _stream(stream))
    _check(rc, "uvc_fluence_streamed_noalloc")
    return mu


def coverage(scene: Scene, mu, mu_min: float, stream=None):
    """(cov_area, cov_count), each (nvec,) float32 on the device."""
    nvec = mu.shape[0]
    ca = torch.empty(nvec, dtype=torch.float32, device=mu.device)
    cc = torch.empty(nvec, dtype=torch.float32, device=mu.device)
    rc = library().uvc_coverage(scene.handle, _dev(mu, torch.float32, "mu", (nvec, scene.np)), nvec,
                                float(mu_min), _dev(ca, torch.float32, "cov_area"),
                                _dev(cc, torch.float32, "cov_count"), _stream(stream))
    _check(rc, "uvc_coverage")
    return ca, cc


FEATURES = 66
PROBE_FEATURES = 48


def _rows(feat, nc, min_cols, name):
    if not isinstance(feat, torch.Tensor) or not feat.is_cuda or feat.dtype != torch.float32:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    _on_current_device(feat, name)
    if feat.dim() != 2 or feat.shape[0] != nc or feat.shape[1] < min_cols or feat.stride(1) != 1 \
            or (nc > 1 and feat.stride(0) < min_cols):
        raise ValueError(f"{name} must be ({nc}, >= {min_cols}) with unit column stride")
    return ctypes.c_void_p(feat.data_ptr() if feat.numel() else 0), max(feat.stride(0), min_cols)


def candidate_features(scene: Scene, cand, feat=None, stream=None):
    """(nc, 66) float32 scorer inputs: 64-bin area histogram of squared
    distances to the patch centroids, nearest-triangle distance, height.
    `feat` may be a column slice of a wider row-major buffer."""
    nc = cand.shape[0]
    if feat is None:
        feat = torch.empty((nc, FEATURES), dtype=torch.float32, device=cand.device)
    fp, ld = _rows(feat, nc, FEATURES, "feat")
    rc = library().uvc_candidate_features(scene.handle, _dev(cand, torch.float32, "cand", (nc, 3)), nc, fp, ld,
                                          _stream(stream))
    _check(rc, "uvc_candidate_features")
    return feat


def probe_features_work(np_: int, device="cuda"):
    n = int(library().uvc_probe_features_work_bytes(int(np_)))
    return torch.empty((n + 3) // 4, dtype=torch.float32, device=device)


def _scratch(buf, nbytes: int, name):
    """Device pointer of a caller-supplied scratch buffer of at least nbytes."""
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    _on_current_device(buf, name)
    if buf.numel() * buf.element_size() < nbytes:
        raise ValueError(f"{name} holds {buf.numel() * buf.element_size()} bytes, {nbytes} needed")
    return ctypes.c_void_p(buf.data_ptr())


def probe_features(A, area, feat=None, work=None, stream=None):
    """(nc, 48) visibility sketch from the probe irradiance A (nc, np): area of
    the lit probe patches by hardness and efficiency bin (uvc_probe_features).
    A may be a column slice (unit column stride) of a wider matrix."""
    nc, np_ = A.shape
    aptr, lda = _matrix_rows(A, "A", nc, np_)
    if feat is None:
        feat = torch.empty((nc, PROBE_FEATURES), dtype=torch.float32, device=A.device)
    if work is None:
        work = probe_features_work(np_, A.device)
    wptr = _scratch(work, int(library().uvc_probe_features_work_bytes(int(np_))), "work")
    fp, ld = _rows(feat, nc, PROBE_FEATURES, "feat")
    rc = library().uvc_probe_features(aptr, nc, lda, np_, _dev(area, torch.float32, "area", (np_,)), wptr, fp, ld,
                                      _stream(stream))
    _check(rc, "uvc_probe_features")
    return feat


def select_top(score, k: int, cand=None, out_cand=None, out_idx=None, stream=None):
    """The k best-scoring candidates in ascending index order: (idx int32 (k,),
    cand (k, 3) or None).  Ties go to the lower index."""
    n = score.shape[0]
    dev = score.device
    if out_idx is None:
        out_idx = torch.empty(k, dtype=torch.int32, device=dev)
    if cand is not None and out_cand is None:
        out_cand = torch.empty((k, 3), dtype=torch.float32, device=dev)
    rc = library().uvc_select_top(_dev(score, torch.float32, "score", (n,)), n, int(k),
                                  _dev(cand, torch.float32, "cand", (n, 3)) if cand is not None else None,
                                  _dev(out_cand, torch.float32, "out_cand", (k, 3)) if out_cand is not None else None,
                                  _dev(out_idx, torch.int32, "out_idx", (k,)), _stream(stream))
    _check(rc, "uvc_select_top")
    return out_idx, out_cand


def group_boost(score, group: int, bonus: float = 1e30, stream=None):
    """Add `bonus` to the best score of every group of `group` consecutive candidates."""
    n = score.shape[0]
    _check(library().uvc_group_boost(_dev(score, torch.float32, "score", (n,)), n, int(group), float(bonus),
                                     _stream(stream)), "uvc_group_boost")
    return score


def mark_best(A, score, value=float("inf"), rare: int = 0, stream=None):
    """score[argmax_i A[i, j]] = value for every lit column j of A (nc, np);
    with rare > 0 also every candidate lighting a column lit by <= rare rows."""
    nc, np_ = A.shape
    aptr, lda = _matrix_rows(A, "A", nc, np_)
    rc = library().uvc_mark_best(aptr, nc, lda, np_, _dev(score, torch.float32, "score", (nc,)), float(value),
                                 int(rare), _stream(stream))
    _check(rc, "uvc_mark_best")
    return score


def probe_lost(A, idx, area, out=None, lost=None, stream=None):
    """Area fraction of the probe patches lit by some row of A (nc, np) but by
    none of the rows idx; (1,) float32 on the device."""
    nc, np_ = A.shape
    k = idx.shape[0]
    if out is None:
        out = torch.empty(1, dtype=torch.float32, device=A.device)
    if lost is None:
        lost = torch.empty(np_, dtype=torch.float32, device=A.device)
    aptr, lda = _matrix_rows(A, "A", nc, np_)
    rc = library().uvc_probe_lost(aptr, nc, lda, np_,
                                  _dev(idx, torch.int32, "idx", (k,)), k,
                                  _dev(area, torch.float32, "area", (np_,)), _dev(lost, torch.float32, "lost", (np_,)),
                                  _dev(out, torch.float32, "out", (1,)), _stream(stream))
    _check(rc, "uvc_probe_lost")
    return out


class Mlp:
    """The candidate scorer (uvc_mlp_*): BF16 tensor-core perceptron
    in_dim -> hidden -> hidden -> 1 with FP32 master weights and Adam."""

    def __init__(self, in_dim: int, hidden: int = 256, max_batch: int = 65536, seed: int = 0):
        h = ctypes.c_void_p()
        _check(library().uvc_mlp_create(int(in_dim), int(hidden), int(max_batch), int(seed), ctypes.byref(h)),
               "uvc_mlp_create")
        self.handle, self.in_dim, self.hidden, self.max_batch = h, int(in_dim), int(hidden), int(max_batch)
        self.in_pad = (self.in_dim + 15) // 16 * 16
        self.nparam = int(library().uvc_mlp_param_count(h))

    def close(self):
        if self.handle is not None and self.handle.value:
            library().uvc_mlp_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        _check(library().uvc_mlp_params(self.handle, out.ctypes.data_as(ctypes.c_void_p), self.nparam, 0),
               "uvc_mlp_params")
        return out

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, np.float32)
        if a.size != self.nparam:
            raise ValueError(f"expected {self.nparam} parameters, got {a.size}")
        _check(library().uvc_mlp_params(self.handle, a.ctypes.data_as(ctypes.c_void_p), self.nparam, 1),
               "uvc_mlp_params")

    def split(self, flat) -> dict:
        """Views of a flat parameter (or gradient) array by name."""
        P, H = self.in_pad, self.hidden
        sizes = [("W1", (P, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
        out, o = {}, 0
        for name, shp in sizes:
            n = int(np.prod(shp))
            out[name] = flat[o:o + n].reshape(shp)
            o += n
        return out

    def forward(self, x, logit=None, stream=None):
        B = x.shape[0]
        if logit is None:
            logit = torch.empty(B, dtype=torch.float32, device=x.device)
        _check(library().uvc_mlp_forward(self.handle, _dev(x, torch.float32, "x", (B, self.in_dim)), B,
                                         _dev(logit, torch.float32, "logit", (B,)), _stream(stream)),
               "uvc_mlp_forward")
        return logit

    def train_step(self, x, y, w, lr: float, loss=None, stream=None):
        """One Adam step on the weighted BCE loss; returns the device loss (1,)."""
        B = x.shape[0]
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(library().uvc_mlp_train_step(self.handle, _dev(x, torch.float32, "x", (B, self.in_dim)),
                                            _dev(y, torch.float32, "y", (B,)), _dev(w, torch.float32, "w", (B,)),
                                            B, float(lr), _dev(loss, torch.float32, "loss", (1,)),
                                            _stream(stream)),
               "uvc_mlp_train_step")
        return loss

    def grads(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        _check(library().uvc_mlp_grads(self.handle, out.ctypes.data_as(ctypes.c_void_p), self.nparam),
               "uvc_mlp_grads")
        return out


def scene_status(scene: Scene, stream=None) -> int:
    return int(library().uvc_scene_status(scene.handle, _stream(stream)))


def scene_set_limits(scene: Scene, max_stack: int = 0, max_visits: int = 0) -> None:
    """Lower the scene's traversal stack depth and node-visit cap for later
    calls (0 = the built-in bound), to exercise the failure handling (see
    uvc_scene_set_limits)."""
    _check(library().uvc_scene_set_limits(scene.handle, int(max_stack), int(max_visits)), "uvc_scene_set_limits")


def scene_export_bvh(scene: Scene) -> dict:
    """Host copies of the hierarchy: keys, order, children (nt-1,2), boxes (nt-1,12)."""
    n = scene.nt
    ni = max(n - 1, 0)
    keys = np.zeros(n, np.uint64)
    order = np.zeros(n, np.int32)
    children = np.zeros((ni, 2), np.int32)
    boxes = np.zeros((ni, 12), np.float32)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a.size else None  # noqa: E731
    _check(library().uvc_scene_export_bvh(scene.handle, ptr(keys), ptr(order), ptr(children), ptr(boxes)),
           "uvc_scene_export_bvh")
    return dict(keys=keys, order=order, children=children, boxes=boxes)


def probe_l2_read(buf: torch.Tensor, passes: int, sink: torch.Tensor, stream=None):
    """uvc_probe_l2_read over the bytes of `buf` (a contiguous CUDA tensor);
    `sink` a CUDA tensor of at least one 32-bit word."""
    if not buf.is_contiguous():
        raise ValueError("buf must be contiguous")
    nbytes = buf.numel() * buf.element_size() // 16 * 16
    _check(library().uvc_probe_l2_read(_scratch(buf, nbytes, "buf"), nbytes, int(passes),
                                       _scratch(sink, 4, "sink"), _stream(stream)), "uvc_probe_l2_read")


def scene_export_traversal(scene: Scene) -> dict:
    """Host copies of what the traversal kernels read (uvc_scene_export_traversal):
    nodes4 (nt-1, 32) as raw 32-bit words, tri (nt, 3, 4) float32, patch_s and
    patch_n (np, 4) float32, patch_excl (np, 2) int32, root, diameter, coord_bound."""
    n, np_ = scene.nt, scene.np
    nodes4 = np.zeros((max(n - 1, 0), 32), np.uint32)
    tri = np.zeros((n, 3, 4), np.float32)
    ps = np.zeros((np_, 4), np.float32)
    pn = np.zeros((np_, 4), np.float32)
    pe = np.zeros((np_, 2), np.int32)
    root, diam, cb = ctypes.c_int32(), ctypes.c_float(), ctypes.c_float()
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a.size else None  # noqa: E731
    _check(library().uvc_scene_export_traversal(scene.handle, ptr(nodes4), ptr(tri), ptr(ps), ptr(pn), ptr(pe),
                                                ctypes.byref(root), ctypes.byref(diam), ctypes.byref(cb)),
           "uvc_scene_export_traversal")
    return dict(nodes4=nodes4, tri=tri, patch_s=ps, patch_n=pn, patch_excl=pe, root=root.value,
                diameter=diam.value, coord_bound=cb.value)


def irradiance_candidates_per_task() -> int:
    """Candidates per warp task of the matrix kernel (uvc_irradiance_candidates_per_task)."""
    return int(library().uvc_irradiance_candidates_per_task())


class Batch:
    """Many irradiance matrices in one persistent launch (uvc_batch_*).

    jobs: list of (scene, cand (nc,3) CUDA tensor, lamp index, A (nc, lda) CUDA
    tensor, vis CUDA int32 tensor or None); lamps: list of Lamp.  The caller
    keeps scenes and tensors alive while the batch is used (the batch keeps
    references to the tensors it was given).  launch() may be captured in a
    CUDA graph."""

    def __init__(self, jobs, lamps, stream=None):
        lib = library()
        cj = (_Job * len(jobs))()
        self._keep = []
        for q, (scene, cand, lamp, A, vis) in enumerate(jobs):
            nc = cand.shape[0]
            if not 0 <= int(lamp) < len(lamps):
                raise ValueError(f"job {q}: lamp index {lamp} out of range")
            cj[q].scene = scene.handle
            cj[q].cand = _dev(cand, torch.float32, "cand", (nc, 3))
            cj[q].nc = nc
            cj[q].lamp = int(lamp)
            cj[q].A, cj[q].lda = _matrix_rows(A, "A", nc, scene.np)
            cj[q].vis = None if vis is None else _dev(vis, torch.int32, "vis",
                                                      (lamps[int(lamp)].K, nc, (scene.np + 31) // 32))
            self._keep.append((scene, cand, A, vis))
        cl = (_Lamp * len(lamps))(*[L._c() for L in lamps])
        nbytes = lib.uvc_batch_workspace_bytes(len(jobs), len(lamps))
        dev = jobs[0][1].device
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.workspace.data_ptr()) % 256
        out = ctypes.c_void_p()
        _check(lib.uvc_batch_create(cj, len(jobs), cl, len(lamps), ctypes.c_void_p(self.workspace.data_ptr() + off),
                                    nbytes, _stream(stream), ctypes.byref(out)), "uvc_batch_create")
        self._h = out

    def launch(self, stream=None):
        _check(library().uvc_batch_launch(self._h, _stream(stream)), "uvc_batch_launch")

    def set_config(self, cand_per_task: int, blocks_per_sm: int = 0, stream=None):
        c = _BatchConfig(cand_per_task, blocks_per_sm)
        _check(library().uvc_batch_set_config(self._h, ctypes.byref(c), _stream(stream)), "uvc_batch_set_config")

    def autotune(self, sample_fraction: float = 0.05, stream=None):
        c = _BatchConfig()
        _check(library().uvc_batch_autotune(self._h, float(sample_fraction), ctypes.byref(c), _stream(stream)),
               "uvc_batch_autotune")
        return c.cand_per_task, c.blocks_per_sm

    def info(self):
        tp, cap, c = ctypes.c_int64(), ctypes.c_int32(), _BatchConfig()
        _check(library().uvc_batch_info(self._h, ctypes.byref(tp), ctypes.byref(cap), ctypes.byref(c)),
               "uvc_batch_info")
        return dict(total_pairs=tp.value, stack_cap=cap.value, cand_per_task=c.cand_per_task,
                    blocks_per_sm=c.blocks_per_sm)

    def free(self):
        if getattr(self, "_h", None) is not None:
            library().uvc_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vis_to_bool(vis: torch.Tensor, np_: int) -> np.ndarray:
    """Unpack a (K, nc, nwords) bitmask to a bool array (nc, np, K) on the host."""
    w = vis.cpu().numpy().view(np.uint32)
    K, nc, nwords = w.shape
    bits = ((w[..., None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool)
    bits = bits.reshape(K, nc, nwords * 32)[:, :, :np_]
    return np.transpose(bits, (1, 2, 0))
