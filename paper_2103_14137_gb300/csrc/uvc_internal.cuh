// Internal declarations of libuvc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "uvc.h"

namespace uvc {

// One internal BVH node: the boxes of both children and both child
// references, 64 bytes, loaded with four 16-byte loads.  Bounds are grouped
// by axis with the left and right child side by side, so that both children
// are tested with packed FP32x2 arithmetic:
//   x = (L.lo.x, R.lo.x, L.hi.x, R.hi.x)
//   y = (L.lo.y, R.lo.y, L.hi.y, R.hi.y)
//   z = (L.lo.z, R.lo.z, L.hi.z, R.hi.z)
//   r = (left ref, right ref, parent, 0); ref >= 0 internal node, ref < 0 leaf ~k
struct __align__(16) Node {
    float4 x, y, z;
    int4 r;
};

// Four-wide node used by the traversal: the binary tree collapsed two levels
// at a time (a node at even depth keeps its grandchildren; a leaf child stays a
// leaf).  Children are tested in pairs (0,1) and (2,3) with packed FP32x2:
//   q[0..2] = x, y, z of (c0.lo, c1.lo, c0.hi, c1.hi)
//   q[3..5] = x, y, z of (c2.lo, c3.lo, c2.hi, c3.hi)
//   r = child refs: >= 0 four-wide node (indexed like the binary node it came
//       from), < 0 leaf ~k, kEmptyChild for an unused slot (its box is a point
//       far outside the scene, so no segment enters it)
//   m = (bit c set: child c is a leaf, bit c set: child c is a four-wide node, 0, 0)
constexpr int kEmptyChild = 0x7fffffff;
struct __align__(16) Node4 {
    float4 q[6];
    int4 r;
    int4 m;
};

// Largest lamp for the wedge traversal of vertical line lamps (its shared
// memory per warp grows with K), and largest scene (its queue packs leaf
// indices into 27 bits).
constexpr int kWedgeMaxK = 16;
constexpr int64_t kWedgeMaxTris = int64_t(1) << 27;

// Lamp as seen by the kernels: source offsets and source powers w_m * P.
// wedge = 1: every offset is vertical (x = y = 0), 2 <= K <= kWedgeMaxK, and
// the wedge traversal is switched on (uvc_set_wedge_traversal).
// Wedge lamps whose offsets rise evenly (off_m.z within 1/64 of a step of
// wz0 + m dz, dz > 0) have wuniform = 1 and wz0, wrdz = 1/dz set: the
// sources in a height interval are then a range of indices.
struct LampDev {
    int K;
    int wedge;
    int wuniform;
    float wz0, wrdz;
    float ox[UVC_MAX_SOURCES], oy[UVC_MAX_SOURCES], oz[UVC_MAX_SOURCES];
    float pw[UVC_MAX_SOURCES];
};

// Host: validate a lamp and convert it (api.cu); coord_bound is the largest
// coordinate magnitude and max_tris the largest triangle count of the
// scene(s) it will be used with.
int lamp_to_device(const uvc_lamp* lamp, LampDev* out, float coord_bound, int64_t max_tris);

}  // namespace uvc

struct uvc_scene {
    int device = 0;
    int64_t nt = 0, np = 0;
    int32_t depth = 0;     // edges from the root to the deepest leaf
    int32_t root = 0;      // root reference (0, or ~0 for a single triangle)
    float diameter = 0.f;  // diagonal of the triangles' bounding box
    float coord_bound = 0.f;  // largest |coordinate| of that box
    // device buffers, carved out of one allocation
    void* block = nullptr;
    float4* tri = nullptr;        // [nt][3]: (v0, id bits), (v1, 0), (v2, 0) in sorted order
    uvc::Node* nodes = nullptr;   // [nt-1]
    uvc::Node4* nodes4 = nullptr; // [nt-1], used at even-depth binary indices only
    int32_t depth4 = 0;           // depth of the four-wide tree
    uint64_t* keys = nullptr;     // [nt] sorted Morton keys
    int32_t* order = nullptr;     // [nt] triangle index per sorted position
    float4* patch_s = nullptr;    // [np] (centroid, area)
    float4* patch_n = nullptr;    // [np] (normal, clearance): see k_clearance
    int2* patch_excl = nullptr;   // [np]
    float* area_total = nullptr;  // [1]
    int* status = nullptr;        // [1] device status word (0 = ok)
    cudaStream_t build_stream = nullptr;
    // lowered traversal limits (uvc_scene_set_limits); 0 = the built-in bound
    int32_t limit_stack = 0;
    int32_t limit_visits = 0;
};

namespace uvc {

constexpr int kWarpsPerBlock = 8;
constexpr int kThreads = kWarpsPerBlock * 32;

int sm_count();
int status_from_cuda(cudaError_t e);

// BVH build (build_bvh.cu)
int build_scene(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const uvc_patches* patches,
                int64_t np, uint32_t flags, cudaStream_t stream, uvc_scene** out);

// irradiance (irradiance.cu)
int irradiance_matrix(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, float* A,
                      int64_t lda, uint32_t* vis, cudaStream_t stream);
int irradiance_counters(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, float* A,
                        int64_t lda, unsigned long long* out6, cudaStream_t stream);
int fluence_streamed(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, const float* t,
                     int32_t nvec, float* mu, cudaStream_t stream);
int fluence_streamed_noalloc(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, const float* t,
                             int32_t nvec, float* mu, cudaStream_t stream);

// area-mean irradiance (solid_angle.cu)
int irradiance_area_mean(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, const float* ptri,
                         float* A, int64_t lda, uint8_t* nclosed, cudaStream_t stream);

// visibility-cube estimator (raster.cu)
size_t raster_workspace_bytes(int64_t nt, int K, int R, int64_t cand_per_batch);
int irradiance_raster(const uvc_scene* sc, const float* tri_normal, const float* cand, int64_t nc, const LampDev& L,
                      int R, float* A, int64_t lda, void* work, size_t bytes, cudaStream_t stream);

// fluence and coverage (fluence.cu)
int fluence(const uvc_scene* sc, const float* A, int64_t nc, int64_t lda, const float* t, int32_t nvec,
            float* mu, cudaStream_t stream);
int coverage(const uvc_scene* sc, const float* mu, int32_t nvec, float mu_min, float* cov_area,
             float* cov_count, cudaStream_t stream);
void launch_area_total(const float4* patch_s, int64_t np, float* out, cudaStream_t stream);

// bandwidth probe (probe.cu)
int probe_l2_read(const void* buf, size_t bytes, int32_t passes, uint32_t* sink, cudaStream_t stream);
int irradiance_cand_per_task();   // candidates per warp task of k_irradiance

// learned-proposal features (features.cu)
int candidate_features(const uvc_scene* sc, const float* cand, int64_t nc, float* feat, int64_t ldf,
                       cudaStream_t stream);
int probe_features(const float* A, int64_t nc, int64_t lda, int64_t np, const float* area, float* work,
                   float* feat, int64_t ldf, cudaStream_t stream);
int group_boost(float* score, int64_t n, int group, float bonus, cudaStream_t stream);
int mark_best(const float* A, int64_t nc, int64_t lda, int64_t np, float* score, float value, int rare,
              cudaStream_t stream);
int probe_lost(const float* A, int64_t nc, int64_t lda, int64_t np, const int32_t* idx, int64_t k,
               const float* area, float* lost, float* out, cudaStream_t stream);
int select_top(const float* score, int64_t n, int64_t k, const float* cand, float* out_cand, int32_t* out_idx,
               cudaStream_t stream);

}  // namespace uvc
