// extern "C" entry points of libuvc: argument checks, lamp conversion, and
// dispatch to the kernels.  See include/uvc.h for the contract of each call.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "uvc_internal.cuh"

namespace uvc {

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

int status_from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return UVC_OK;
    return e == cudaErrorMemoryAllocation ? UVC_E_NOMEM : UVC_E_CUDA;
}

namespace {

const int64_t kLimit = int64_t(1) << 31;

bool count_ok(int64_t n) { return n >= 0 && n < kLimit; }

std::atomic<int> g_wedge{1};

}  // namespace
// uvc_fluence's kernel where the rows of A allow a tensor map: 1 = tensor cores,
// 0 = CUDA cores (defined in fluence.cu)
extern std::atomic<int> g_fluence_tc;

int lamp_to_device(const uvc_lamp* lamp, LampDev* out, float coord_bound, int64_t max_tris) {
    if (!lamp || lamp->K < 1 || lamp->K > UVC_MAX_SOURCES) return UVC_E_INVAL;
    if (!std::isfinite(lamp->power) || lamp->power < 0.f) return UVC_E_INVAL;
    std::memset(out, 0, sizeof(*out));
    out->K = lamp->K;
    for (int m = 0; m < lamp->K; ++m) {
        const float w = lamp->weight[m];
        if (!std::isfinite(w) || w < 0.f) return UVC_E_INVAL;
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(lamp->offsets[m][k])) return UVC_E_INVAL;
        out->ox[m] = lamp->offsets[m][0];
        out->oy[m] = lamp->offsets[m][1];
        out->oz[m] = lamp->offsets[m][2];
        out->pw[m] = w * lamp->power;   // source power w_m P (one FP32 rounding)
    }
    bool vertical = lamp->K >= 2 && lamp->K <= kWedgeMaxK;
    for (int m = 0; m < lamp->K && vertical; ++m) vertical = out->ox[m] == 0.f && out->oy[m] == 0.f;
    // the wedge search queues leaf indices in 27 bits (larger scenes search source by source)
    out->wedge = vertical && max_tris <= kWedgeMaxTris && g_wedge.load(std::memory_order_relaxed) ? 1 : 0;
    if (out->wedge) {
        const int K = lamp->K;
        const double z0 = out->oz[0], dz = ((double)out->oz[K - 1] - z0) / (K - 1);
        bool even = dz > 0.0 && std::isfinite(1.0 / dz);
        for (int m = 0; m < K && even; ++m) even = std::fabs((double)out->oz[m] - (z0 + m * dz)) <= dz / 64.0;
        // The closed-form index range of the wedge search leaves 1/64 of a
        // step for FP32 rounding: the source heights fl32(c.z + off) and the
        // interval ends carry errors of about 2^-24 of the coordinates, so the
        // step must be at least 2^-16 of them.  Candidates are taken to lie
        // within 16 times the scene's coordinate bound; closer sources take
        // the source-by-source height test (exact at any spacing).
        double offmax = 0.0;
        for (int m = 0; m < K; ++m) offmax = std::max(offmax, std::fabs((double)out->oz[m]));
        if (even && !(dz >= std::ldexp(16.0 * (double)coord_bound + 3.0 * offmax, -16))) even = false;
        out->wuniform = even ? 1 : 0;
        out->wz0 = (float)z0;
        out->wrdz = even ? (float)(1.0 / dz) : 0.f;
    }
    return UVC_OK;
}

}  // namespace uvc

extern "C" {

int uvc_build_scene(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const uvc_patches* patches,
                    int64_t np, uvc_stream_t stream, uvc_scene** out) {
    return uvc::build_scene(verts, nv, tris, nt, patches, np, 0u, (cudaStream_t)stream, out);
}

int uvc_build_scene_ex(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const uvc_patches* patches,
                       int64_t np, uint32_t flags, uvc_stream_t stream, uvc_scene** out) {
    if (flags & ~(uint32_t)UVC_BUILD_LBVH_ONLY) {
        if (out) *out = nullptr;
        return UVC_E_INVAL;
    }
    return uvc::build_scene(verts, nv, tris, nt, patches, np, flags, (cudaStream_t)stream, out);
}

int uvc_free_scene(uvc_scene* scene) {
    if (!scene) return UVC_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (scene->block) cudaFree(scene->block);
    delete scene;
    return uvc::status_from_cuda(e);
}

int uvc_set_wedge_traversal(int32_t enable, int32_t* previous) {
    if (enable != 0 && enable != 1) return UVC_E_INVAL;
    const int prev = uvc::g_wedge.exchange(enable);
    if (previous) *previous = prev;
    return UVC_OK;
}

int uvc_set_fluence_tensor_cores(int32_t enable, int32_t* previous) {
    if (enable != 0 && enable != 1) return UVC_E_INVAL;
    const int prev = uvc::g_fluence_tc.exchange(enable);
    if (previous) *previous = prev;
    return UVC_OK;
}

int uvc_irradiance_matrix(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp, float* A,
                          int64_t lda, uint32_t* vis, uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc)) return UVC_E_INVAL;
    uvc::LampDev L;
    int rc = uvc::lamp_to_device(lamp, &L, scene->coord_bound, scene->nt);
    if (rc != UVC_OK) return rc;
    if (lda < scene->np) return UVC_E_INVAL;
    if (nc == 0 || scene->np == 0) return UVC_OK;
    if (!cand || !A) return UVC_E_INVAL;
    return uvc::irradiance_matrix(scene, cand, nc, L, A, lda, vis, (cudaStream_t)stream);
}

int uvc_irradiance_counters(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                            float* A, int64_t lda, uint64_t* counters, uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc) || !counters) return UVC_E_INVAL;
    uvc::LampDev L;
    int rc = uvc::lamp_to_device(lamp, &L, scene->coord_bound, scene->nt);
    if (rc != UVC_OK) return rc;
    if (lda < scene->np) return UVC_E_INVAL;
    if (nc > 0 && scene->np > 0 && (!cand || !A)) return UVC_E_INVAL;
    return uvc::irradiance_counters(scene, cand, nc, L, A, lda, reinterpret_cast<unsigned long long*>(counters),
                                    (cudaStream_t)stream);
}

int uvc_irradiance_area_mean(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                             const float* ptri, float* A, int64_t lda, uint8_t* nclosed, uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc) || nc > INT32_MAX) return UVC_E_INVAL;
    uvc::LampDev L;
    int rc = uvc::lamp_to_device(lamp, &L, scene->coord_bound, scene->nt);
    if (rc != UVC_OK) return rc;
    if (lda < scene->np) return UVC_E_INVAL;
    if (nc > 0 && scene->np > 0 && (!cand || !A || !ptri)) return UVC_E_INVAL;
    return uvc::irradiance_area_mean(scene, cand, nc, L, ptri, A, lda, nclosed, (cudaStream_t)stream);
}

size_t uvc_raster_workspace_bytes(const uvc_scene* scene, const uvc_lamp* lamp, int32_t R, int64_t cand_per_batch) {
    if (!scene || !lamp || lamp->K < 1 || lamp->K > UVC_MAX_SOURCES || R < 1 || R > 4096 || cand_per_batch < 1)
        return 0;
    return uvc::raster_workspace_bytes(scene->nt, lamp->K, R, cand_per_batch);
}

int uvc_irradiance_raster(const uvc_scene* scene, const float* tri_normal, const float* cand, int64_t nc,
                          const uvc_lamp* lamp, int32_t R, float* A, int64_t lda, void* workspace, size_t bytes,
                          uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc) || nc > INT32_MAX || R < 1 || R > 4096) return UVC_E_INVAL;
    uvc::LampDev L;
    int rc = uvc::lamp_to_device(lamp, &L, scene->coord_bound, scene->nt);
    if (rc != UVC_OK) return rc;
    if (lda < scene->nt) return UVC_E_INVAL;
    if (nc > 0 && scene->nt > 0 && (!cand || !A || !tri_normal || !workspace)) return UVC_E_INVAL;
    return uvc::irradiance_raster(scene, tri_normal, cand, nc, L, R, A, lda, workspace, bytes, (cudaStream_t)stream);
}

int uvc_fluence(const uvc_scene* scene, const float* A, int64_t nc, int64_t lda, const float* t, int32_t nvec,
                float* mu, uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc) || nvec < 1 || nvec > 256 || lda < scene->np) return UVC_E_INVAL;
    if (scene->np == 0) return UVC_OK;
    if (!mu || (nc > 0 && (!A || !t))) return UVC_E_INVAL;
    return uvc::fluence(scene, A, nc, lda, t, nvec, mu, (cudaStream_t)stream);
}

int uvc_fluence_streamed(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                         const float* t, int32_t nvec, float* mu, uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc) || nvec < 1 || nvec > 256) return UVC_E_INVAL;
    uvc::LampDev L;
    int rc = uvc::lamp_to_device(lamp, &L, scene->coord_bound, scene->nt);
    if (rc != UVC_OK) return rc;
    if (scene->np == 0) return UVC_OK;
    if (!mu || (nc > 0 && (!cand || !t))) return UVC_E_INVAL;
    return uvc::fluence_streamed(scene, cand, nc, L, t, nvec, mu, (cudaStream_t)stream);
}

int uvc_fluence_streamed_noalloc(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                                 const float* t, int32_t nvec, float* mu, uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc) || nvec < 1 || nvec > 256) return UVC_E_INVAL;
    uvc::LampDev L;
    int rc = uvc::lamp_to_device(lamp, &L, scene->coord_bound, scene->nt);
    if (rc != UVC_OK) return rc;
    if (scene->np == 0) return UVC_OK;
    if (!mu || (nc > 0 && (!cand || !t))) return UVC_E_INVAL;
    return uvc::fluence_streamed_noalloc(scene, cand, nc, L, t, nvec, mu, (cudaStream_t)stream);
}

int uvc_coverage(const uvc_scene* scene, const float* mu, int32_t nvec, float mu_min, float* cov_area,
                 float* cov_count, uvc_stream_t stream) {
    if (!scene || nvec < 1 || nvec > 65535 || !cov_area || !std::isfinite(mu_min)) return UVC_E_INVAL;
    if (scene->np > 0 && !mu) return UVC_E_INVAL;
    return uvc::coverage(scene, mu, nvec, mu_min, cov_area, cov_count, (cudaStream_t)stream);
}

int uvc_candidate_features(const uvc_scene* scene, const float* cand, int64_t nc, float* feat, int64_t ldf,
                           uvc_stream_t stream) {
    if (!scene || !uvc::count_ok(nc) || nc > INT32_MAX || ldf < 66) return UVC_E_INVAL;
    if (nc > 0 && (!cand || !feat)) return UVC_E_INVAL;
    return uvc::candidate_features(scene, cand, nc, feat, ldf, (cudaStream_t)stream);
}

size_t uvc_probe_features_work_bytes(int64_t np) {
    return np < 0 ? 0 : (size_t)(np + 4) * sizeof(float) + (size_t)np + 16;
}

int uvc_probe_features(const float* A, int64_t nc, int64_t lda, int64_t np, const float* area, void* work,
                       float* feat, int64_t ldf, uvc_stream_t stream) {
    if (!uvc::count_ok(nc) || !uvc::count_ok(np) || nc > INT32_MAX || np > INT32_MAX || lda < np || ldf < 48)
        return UVC_E_INVAL;
    if (nc > 0 && (!feat || !work || (np > 0 && (!A || !area)))) return UVC_E_INVAL;
    if (reinterpret_cast<uintptr_t>(work) % 4) return UVC_E_INVAL;
    return uvc::probe_features(A, nc, lda, np, area, static_cast<float*>(work), feat, ldf, (cudaStream_t)stream);
}

int uvc_select_top(const float* score, int64_t n, int64_t k, const float* cand, float* out_cand, int32_t* out_idx,
                   uvc_stream_t stream) {
    if (n < 0 || n > 16384 || k < 0 || k > n) return UVC_E_INVAL;
    if (k > 0 && (!score || (!out_cand && !out_idx) || (out_cand && !cand))) return UVC_E_INVAL;
    return uvc::select_top(score, n, k, cand, out_cand, out_idx, (cudaStream_t)stream);
}

int uvc_group_boost(float* score, int64_t n, int32_t group, float bonus, uvc_stream_t stream) {
    if (n < 0 || n > INT32_MAX || group < 1 || (n > 0 && !score)) return UVC_E_INVAL;
    return uvc::group_boost(score, n, group, bonus, (cudaStream_t)stream);
}

int uvc_mark_best(const float* A, int64_t nc, int64_t lda, int64_t np, float* score, float value, int32_t rare,
                  uvc_stream_t stream) {
    if (!uvc::count_ok(nc) || !uvc::count_ok(np) || nc > INT32_MAX || np > INT32_MAX || lda < np || rare < 0)
        return UVC_E_INVAL;
    if (nc > 0 && np > 0 && (!A || !score)) return UVC_E_INVAL;
    return uvc::mark_best(A, nc, lda, np, score, value, rare, (cudaStream_t)stream);
}

int uvc_probe_lost(const float* A, int64_t nc, int64_t lda, int64_t np, const int32_t* idx, int64_t k,
                   const float* area, float* lost, float* out, uvc_stream_t stream) {
    if (!uvc::count_ok(nc) || !uvc::count_ok(np) || np > INT32_MAX || nc > INT32_MAX || k < 0 || k > nc ||
        lda < np || !out)
        return UVC_E_INVAL;
    if (np > 0 && (!area || !lost || (nc > 0 && !A) || (k > 0 && !idx))) return UVC_E_INVAL;
    return uvc::probe_lost(A, nc, lda, np, idx, k, area, lost, out, (cudaStream_t)stream);
}

uint32_t uvc_library_flags(void) {
#ifdef UVC_CHECKED
    return UVC_LIB_CHECKED;
#else
    return 0u;
#endif
}

const char* uvc_status_string(int status) {
    switch (status) {
        case UVC_OK: return "ok";
        case UVC_E_INVAL: return "invalid argument";
        case UVC_E_NOMEM: return "out of device memory";
        case UVC_E_CUDA: return "CUDA runtime error";
        case UVC_E_STACK: return "traversal stack overflow";
        case UVC_E_TIMEOUT: return "traversal exceeded its node-visit cap";
        case UVC_E_BOUNDS: return "traversal index out of range (checked build)";
        case UVC_E_SCRATCH: return "problem too large for the fixed scratch of the allocation-free call";
        default: return "unknown status";
    }
}

int uvc_scene_status(const uvc_scene* scene, uvc_stream_t stream) {
    if (!scene) return UVC_E_INVAL;
    int v = 0;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(&v, scene->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(scene->status, 0, sizeof(int));
    if (e != cudaSuccess) return uvc::status_from_cuda(e);
    return v;
}

int uvc_scene_set_limits(uvc_scene* scene, int32_t max_stack, int32_t max_visits) {
    if (!scene || max_stack < 0 || max_visits < 0) return UVC_E_INVAL;
    scene->limit_stack = max_stack;   // host fields: read when a later call builds its launch
    scene->limit_visits = max_visits;
    return UVC_OK;
}

int uvc_scene_info(const uvc_scene* scene, int64_t* nt, int64_t* np, int32_t* depth) {
    if (!scene) return UVC_E_INVAL;
    if (nt) *nt = scene->nt;
    if (np) *np = scene->np;
    if (depth) *depth = scene->depth;
    return UVC_OK;
}

int uvc_probe_l2_read(const void* buf, size_t bytes, int32_t passes, uint32_t* sink, uvc_stream_t stream) {
    if (!buf || !sink || bytes < 16 || bytes % 16 != 0 || reinterpret_cast<uintptr_t>(buf) % 16 != 0 || passes < 1)
        return UVC_E_INVAL;
    return uvc::probe_l2_read(buf, bytes, passes, sink, (cudaStream_t)stream);
}

int uvc_scene_export_traversal(const uvc_scene* scene, void* nodes4, float* tri, float* patch_s, float* patch_n,
                               int32_t* patch_excl, int32_t* root, float* diameter,
                               float* coord_bound) {
    if (!scene) return UVC_E_INVAL;
    const int64_t n = scene->nt, ni = n > 1 ? n - 1 : 0, np = scene->np;
    cudaError_t e = cudaStreamSynchronize(scene->build_stream);
    if (e == cudaSuccess && nodes4 && ni)
        e = cudaMemcpy(nodes4, scene->nodes4, sizeof(uvc::Node4) * ni, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && tri && n) e = cudaMemcpy(tri, scene->tri, sizeof(float4) * 3 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && patch_s && np)
        e = cudaMemcpy(patch_s, scene->patch_s, sizeof(float4) * np, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && patch_n && np)
        e = cudaMemcpy(patch_n, scene->patch_n, sizeof(float4) * np, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && patch_excl && np)
        e = cudaMemcpy(patch_excl, scene->patch_excl, sizeof(int2) * np, cudaMemcpyDeviceToHost);
    if (root) *root = scene->root;
    if (diameter) *diameter = scene->diameter;
    if (coord_bound) *coord_bound = scene->coord_bound;
    return uvc::status_from_cuda(e);
}

int32_t uvc_irradiance_candidates_per_task(void) { return uvc::irradiance_cand_per_task(); }

int uvc_scene_export_bvh(const uvc_scene* scene, uint64_t* keys, int32_t* order, int32_t* children, float* boxes) {
    if (!scene) return UVC_E_INVAL;
    const int64_t n = scene->nt, ni = n > 1 ? n - 1 : 0;
    cudaError_t e = cudaStreamSynchronize(scene->build_stream);
    if (e == cudaSuccess && keys && n)
        e = cudaMemcpy(keys, scene->keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && order && n)
        e = cudaMemcpy(order, scene->order, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && (children || boxes) && ni) {
        uvc::Node* h = new (std::nothrow) uvc::Node[ni];
        if (!h) return UVC_E_NOMEM;
        e = cudaMemcpy(h, scene->nodes, sizeof(uvc::Node) * ni, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            for (int64_t k = 0; k < ni; ++k) {
                if (children) {
                    children[2 * k] = h[k].r.x;
                    children[2 * k + 1] = h[k].r.y;
                }
                if (boxes) {
                    const uvc::Node& q = h[k];
                    const float v[12] = {q.x.x, q.y.x, q.z.x, q.x.z, q.y.z, q.z.z,    // left lo, hi
                                         q.x.y, q.y.y, q.z.y, q.x.w, q.y.w, q.z.w};   // right lo, hi
                    std::memcpy(boxes + 12 * k, v, sizeof(v));
                }
            }
        }
        delete[] h;
    }
    return uvc::status_from_cuda(e);
}

}  // extern "C"
