"""Helpers for the GPU tests: upload synth scenes and call the C ABI."""
import numpy as np
import torch

import paper_2103_14137_gb300 as uvc

DEV = torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def build(scene_or_arrays, lbvh_only=False):
    s = scene_or_arrays
    return uvc.build_scene(T(s.verts), T(s.tris), T(s.centroid), T(s.normal), T(s.area), T(s.excl),
                           lbvh_only=lbvh_only)


def build_arrays(verts, tris, cen, nrm, area, excl, lbvh_only=False):
    return uvc.build_scene(T(np.asarray(verts, np.float32)), T(np.asarray(tris, np.int32)),
                           T(np.asarray(cen, np.float32)), T(np.asarray(nrm, np.float32)),
                           T(np.asarray(area, np.float32)), T(np.asarray(excl, np.int32)), lbvh_only=lbvh_only)


def lamp_of(L):
    return uvc.Lamp(L.offsets, L.weights, L.power)


def gpu_matrix(scene, cand, lamp):
    A, vis = uvc.irradiance_matrix(scene, T(np.asarray(cand, np.float32)), lamp, with_vis=True)
    torch.cuda.synchronize()
    assert uvc.scene_status(scene) == 0
    return A.cpu().numpy(), uvc.vis_to_bool(vis, scene.np)
