"""GB300-native irradiance-matrix library for UV coverage planning.

Hot path of the two-stage planner of arXiv:2103.14137 (Sec. IV-C): the
occlusion-tested irradiance matrix between candidate lamp positions and surface
patches (Eq. (4), (7)), the fluence A^T t (Eq. (5)) and the covered-area
fraction, as hand-written CUDA for sm_103a behind the C ABI of include/uvc.h.
"""
from ._build import build  # noqa: F401
from .uvc import (FEATURES, PROBE_FEATURES, Batch, Lamp, Mlp, Scene, UvcError, build_scene, candidate_features,  # noqa: F401
                  coverage, fluence, fluence_streamed, fluence_streamed_noalloc, irradiance_area_mean, irradiance_counters, irradiance_raster, raster_workspace,
                  group_boost, irradiance_matrix, library, mark_best, point_lamp, probe_l2_read, probe_features, probe_features_work, probe_lost, scene_export_bvh, scene_export_traversal, scene_set_limits, scene_status, select_top,
                  irradiance_candidates_per_task, set_fluence_tensor_cores, set_wedge_traversal, status_string, vis_to_bool)
