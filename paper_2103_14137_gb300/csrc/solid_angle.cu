// Area-mean irradiance of patches with known geometry: the mean of Eq. (4)
// over each patch rather than its centroid sample, which is what the paper's
// raster estimator measures (flux over area, Sec. IV-C).  For an isotropic
// point source of power P that sees all of a triangle, the flux it receives
// is P Omega / (4 pi) with Omega the triangle's solid angle (van Oosterom and
// Strackee, IEEE Trans. Biomed. Eng. 30(2), 1983), so a fully lit patch gets
// P sum_t Omega_t / (4 pi a_j) exactly.  "Fully lit" is checked with
// segments to the centroid and to the patch vertices pulled a fraction kPull
// towards the centroid; a source that fails a check contributes its centroid
// sample instead (the same value as uvc_irradiance_matrix).
//
// Work unit as in irradiance.cu: one warp = 32 patches x one source, walking
// the four-wide tree as a packet; the vertex checks are further packets from
// the same source point.  Vertical line lamps take the wedge searches instead
// (one per check point for all sources).
#include "traverse.cuh"

namespace uvc {
namespace {

constexpr int kAreaCandPerTask = 4;
constexpr float kPull = 1e-3f;

// v = a - o as an exact pair (hi, lo) (TwoSum).
__device__ __forceinline__ void two_diff(float a, float o, float& h, float& l) {
    h = __fsub_rn(a, o);
    const float q = __fsub_rn(h, a);
    l = __fadd_rn(__fsub_rn(a, __fsub_rn(h, q)), __fsub_rn(-o, q));
}

// <n, h + l> with TwoProduct and TwoSum: exact up to the final rounding.
__device__ __forceinline__ float dot_ef(float nx, float ny, float nz, float hx, float hy, float hz, float lx, float ly,
                                        float lz) {
    float acc = __fmul_rn(nx, hx);
    float err = __fmaf_rn(nx, hx, -acc);
    err = __fmaf_rn(nx, lx, err);
    const float n2[2] = {ny, nz}, h2[2] = {hy, hz}, l2[2] = {ly, lz};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float p = __fmul_rn(n2[k], h2[k]);
        const float e = __fmaf_rn(n2[k], h2[k], -p);
        const float s = __fadd_rn(acc, p);
        const float z = __fsub_rn(s, acc);
        const float q = __fadd_rn(__fsub_rn(acc, __fsub_rn(s, z)), __fsub_rn(p, z));
        acc = s;
        err = __fadd_rn(err, __fadd_rn(q, e));
        err = __fmaf_rn(n2[k], l2[k], err);
    }
    return __fadd_rn(acc, err);
}

// Solid angle of triangle (a, b, c) seen from o:
//   tan(Omega / 2) = |R1 . (E1 x E2)| / (r1 r2 r3 + (R1.R2) r3 + (R1.R3) r2 + (R2.R3) r1)
// with R_k = vertex - o, E1 = b - a, E2 = c - a; the numerator (the triple
// product) is evaluated error-free from R1 = a - o, so grazing sources keep
// their relative accuracy.
__device__ float solid_angle(float ox, float oy, float oz, float3 a, float3 b, float3 c) {
    float hx, hy, hz, lx, ly, lz;
    two_diff(a.x, ox, hx, lx);
    two_diff(a.y, oy, hy, ly);
    two_diff(a.z, oz, hz, lz);
    const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    const float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    const float cx = __fsub_rn(__fmul_rn(e1y, e2z), __fmul_rn(e1z, e2y));
    const float cy = __fsub_rn(__fmul_rn(e1z, e2x), __fmul_rn(e1x, e2z));
    const float cz = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
    const float num = fabsf(dot_ef(cx, cy, cz, hx, hy, hz, lx, ly, lz));
    const float r1x = hx, r1y = hy, r1z = hz;
    const float r2x = b.x - ox, r2y = b.y - oy, r2z = b.z - oz;
    const float r3x = c.x - ox, r3y = c.y - oy, r3z = c.z - oz;
    const float r1 = sqrtf(r1x * r1x + r1y * r1y + r1z * r1z);
    const float r2 = sqrtf(r2x * r2x + r2y * r2y + r2z * r2z);
    const float r3 = sqrtf(r3x * r3x + r3y * r3y + r3z * r3z);
    const float d12 = r1x * r2x + r1y * r2y + r1z * r2z;
    const float d13 = r1x * r3x + r1y * r3y + r1z * r3z;
    const float d23 = r2x * r3x + r2y * r3y + r2z * r3z;
    const float den = r1 * r2 * r3 + d12 * r3 + d13 * r2 + d23 * r1;
    return 2.f * atan2f(num, den);
}

// A check point: vertex v moved the fraction kPull towards the centroid s.
__device__ __forceinline__ float3 pulled(float3 v, float4 s) {
    return make_float3(__fadd_rn(v.x, __fmul_rn(kPull, __fsub_rn(s.x, v.x))),
                       __fadd_rn(v.y, __fmul_rn(kPull, __fsub_rn(s.y, v.y))),
                       __fadd_rn(v.z, __fmul_rn(kPull, __fsub_rn(s.z, v.z))));
}

// Vertex k (0..5) of a patch's geometry g = ptri + 18 j.
__device__ __forceinline__ float3 vertex(const float* g, int k) {
    return make_float3(__ldg(g + 3 * k), __ldg(g + 3 * k + 1), __ldg(g + 3 * k + 2));
}

// Bit t set when the patch's triangle t (0, 1) has a non-zero cross product;
// an unused second triangle is stored as zeros.
__device__ __forceinline__ int used_triangles(const float* g, bool valid) {
    if (!valid) return 0;
    int mask = 0;
    for (int t = 0; t < 2; ++t) {
        const float3 a = vertex(g, 3 * t), b = vertex(g, 3 * t + 1), c = vertex(g, 3 * t + 2);
        const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z, fx = c.x - a.x, fy = c.y - a.y, fz = c.z - a.z;
        const float cx = ey * fz - ez * fy, cy = ez * fx - ex * fz, cz = ex * fy - ey * fx;
        if (cx != 0.f || cy != 0.f || cz != 0.f) mask |= 1 << t;
    }
    return mask;
}

// One packet query from o to each lane's point p (lanes in `want`); returns
// the lanes found occluded and ORs failed lanes into `failed_all`.
__device__ __forceinline__ uint32_t packet_to(const SceneView& S, float ox, float oy, float oz, float3 p, int2 ex,
                                              uint32_t want, int* stack, int lane, int& cache, uint32_t& failed_all) {
    Ray r;
    r.ox = ox; r.oy = oy; r.oz = oz;
    r.dx = __fsub_rn(p.x, ox); r.dy = __fsub_rn(p.y, oy); r.dz = __fsub_rn(p.z, oz);
    r.ex0 = ex.x; r.ex1 = ex.y;
    setup_ray(r);
    r.tend = 1.f;
    const bool mine = (want >> lane) & 1u;
    bool cached_hit = false;
    if (mine && cache >= 0) {
        const float4* t = S.tri + 3 * (size_t)cache;
        cached_hit = seg_tri(r, __ldg(t), __ldg(t + 1), __ldg(t + 2));
    }
    const uint32_t cached_mask = __ballot_sync(kFull, cached_hit);
    uint32_t failed;
    int hit_tri = -1;
    const uint32_t occl =
        cached_mask | warp_occluded<false>(S, r, want & ~cached_mask, stack, lane, failed, nullptr, hit_tri);
    if (hit_tri >= 0) cache = hit_tri;
    failed_all |= failed;
    return occl;
}

// Vertical line lamps (WEDGE): the centroid and each check point get one wedge
// search for all of a candidate's sources that still need it (see the wedge
// traversal in traverse.cuh); the per-source results, and so the entries, are
// those of the source-by-source searches.
template <bool WEDGE>
__global__ void __launch_bounds__(kThreads, UVC_IRR_MIN_BLOCKS)
    k_area_mean(SceneView S, const float* __restrict__ cand, int nc, LampDev L, const float* __restrict__ ptri,
                float* __restrict__ A, int64_t lda, uint8_t* __restrict__ nclosed) {
    extern __shared__ __align__(16) int smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = smem + warp * S.stack_cap;
    WedgeSmem ws;
    if (WEDGE) ws = wedge_smem(reinterpret_cast<char*>(smem) + stack_smem_bytes(S.stack_cap), L.K, warp);
    const int njb = (S.np + 31) >> 5;
    const int nchunk = (nc + kAreaCandPerTask - 1) / kAreaCandPerTask;
    const int64_t ntask = (int64_t)nchunk * njb;
    for (int64_t task = (int64_t)blockIdx.x * kWarpsPerBlock + warp; task < ntask;
         task += (int64_t)gridDim.x * kWarpsPerBlock) {
        const int jb = (int)(task / nchunk), ic = (int)(task % nchunk);
        const int j = jb * 32 + lane;
        const PatchLane P = load_patch(S, j);
        const float* g = ptri + 18 * (size_t)(P.valid ? j : 0);
        const int tmask = used_triangles(g, P.valid);
        const float inv_area = P.valid && P.s.w > 0.f ? __frcp_rn(__fmul_rn(kFourPi, P.s.w)) : 0.f;
        int cache = -1;
        const int i1 = min(nc, (ic + 1) * kAreaCandPerTask);
        for (int i = ic * kAreaCandPerTask; i < i1; ++i) {
            const float cx = __ldg(&cand[3 * (size_t)i]), cy = __ldg(&cand[3 * (size_t)i + 1]),
                        cz = __ldg(&cand[3 * (size_t)i + 2]);
            float E = 0.f;
            int closed = 0;
            uint32_t failed_all = 0;
            if (WEDGE) {
                uint32_t want;
                float lend, dmax, gx, gy;
                const uint32_t facing = wedge_setup_patch(S, L, cx, cy, cz, P, lane, ws, want, lend, dmax, gx, gy);
                uint32_t vis_c = 0u, all = 0u;   // all: sources that saw every check point so far
                // q = -1: the centroid; q = 0..5: the check points.  One call site of
                // the (large, inlined) wedge search keeps the kernel's code small.
                for (int q = -1; q < 6; ++q) {
                    uint32_t want_q = want;
                    float szq = P.s.z, gxq = gx, gyq = gy, lq = lend, dq = dmax;
                    if (q >= 0) {
                        want_q = ((tmask >> (q / 3)) & 1) ? all : 0u;
                        if (!__any_sync(kFull, want_q != 0u)) continue;
                        const float3 pq = want_q ? pulled(vertex(g, q), P.s) : make_float3(0.f, 0.f, 0.f);
                        dq = 0.f;
                        gxq = 0.f;
                        gyq = 0.f;
                        if (want_q) wedge_setup_point(L, cx, cy, cz, pq, want_q, lane, ws, dq, gxq, gyq);
                        szq = pq.z;
                        lq = 1.f;
                    }
                    uint32_t fq;
                    const uint32_t oc = wedge_search<false>(S, L, cx, cy, cz, szq, gxq, gyq, want_q, lq, dq, P.ex,
                                                            lane, stack, ws, cache, fq, nullptr);
                    failed_all |= fq;
                    if (q < 0) {
                        vis_c = ((fq >> lane) & 1u) ? 0u : (facing & ~oc);
                        all = tmask != 0 ? vis_c : 0u;
                    } else {
                        all &= ~oc;
                    }
                }
                for (int m = 0; m < L.K; ++m) {
                    if ((all >> m) & 1u) {
                        const float ox = __fadd_rn(cx, L.ox[m]), oy = __fadd_rn(cy, L.oy[m]),
                                    oz = __fadd_rn(cz, L.oz[m]);
                        float om = 0.f;
                        for (int t = 0; t < 2; ++t)
                            if ((tmask >> t) & 1)
                                om = __fadd_rn(om, solid_angle(ox, oy, oz, vertex(g, 3 * t), vertex(g, 3 * t + 1),
                                                               vertex(g, 3 * t + 2)));
                        E = __fadd_rn(E, __fmul_rn(__fmul_rn(L.pw[m], om), inv_area));
                        ++closed;
                    } else if ((vis_c >> m) & 1u) {
                        E = __fadd_rn(E, ws.term[m * 32 + lane]);
                    }
                }
            }
            for (int m = 0; m < (WEDGE ? 0 : L.K); ++m) {
                const float ox = __fadd_rn(cx, L.ox[m]), oy = __fadd_rn(cy, L.oy[m]), oz = __fadd_rn(cz, L.oz[m]);
                float hx, hy, hz, lx, ly, lz;   // v = o - s exactly
                two_diff(ox, P.s.x, hx, lx);
                two_diff(oy, P.s.y, hy, ly);
                two_diff(oz, P.s.z, hz, lz);
                const float nv = dot_ef(P.n.x, P.n.y, P.n.z, hx, hy, hz, lx, ly, lz);
                const float d2 = __fmaf_rn(hx, hx, __fmaf_rn(hy, hy, __fmul_rn(hz, hz)));
                const float d = sqrtf(d2);
                const bool facing = P.valid && nv > 0.f && d2 > 0.f;
                // centroid segment: as uvc_irradiance_matrix, with the clearance cut
                Ray r;
                r.ox = ox; r.oy = oy; r.oz = oz;
                r.dx = -hx; r.dy = -hy; r.dz = -hz;
                r.ex0 = P.ex.x; r.ex1 = P.ex.y;
                setup_ray(r);
                const float cut = __fmaf_rn(0.99f, P.n.w, -S.cut_eps);
                r.tend = cut > 0.f ? 1.f - cut * __frcp_rn(d) : 1.f;
                const bool settled = facing && r.tend <= 0.f;
                bool cached_hit = false;
                if (facing && !settled && cache >= 0) {
                    const float4* t = S.tri + 3 * (size_t)cache;
                    cached_hit = seg_tri(r, __ldg(t), __ldg(t + 1), __ldg(t + 2));
                }
                const uint32_t facing_mask = __ballot_sync(kFull, facing);
                const uint32_t cached_mask = __ballot_sync(kFull, cached_hit);
                const uint32_t settled_mask = __ballot_sync(kFull, settled);
                uint32_t failed;
                int hit_tri = -1;
                const uint32_t occl = cached_mask | warp_occluded<false>(S, r, facing_mask & ~cached_mask & ~settled_mask,
                                                                         stack, lane, failed, nullptr, hit_tri);
                if (hit_tri >= 0) cache = hit_tri;
                failed_all |= failed;
                const uint32_t visible = facing_mask & ~occl & ~failed;
                const bool vis_c = (visible >> lane) & 1u;
                // vertex checks for the lanes whose centroid is lit
                bool all = vis_c && tmask != 0;
                for (int q = 0; q < 6; ++q) {
                    const bool use = all && ((tmask >> (q / 3)) & 1);
                    const uint32_t want = __ballot_sync(kFull, use);
                    if (want == 0) continue;
                    const float3 pq = use ? pulled(vertex(g, q), P.s) : make_float3(0.f, 0.f, 0.f);
                    const uint32_t oc = packet_to(S, ox, oy, oz, pq, P.ex, want, stack, lane, cache, failed_all);
                    if ((oc >> lane) & 1u) all = false;
                }
                if (all) {
                    float om = 0.f;
                    for (int t = 0; t < 2; ++t)
                        if ((tmask >> t) & 1)
                            om = __fadd_rn(om, solid_angle(ox, oy, oz, vertex(g, 3 * t), vertex(g, 3 * t + 1),
                                                           vertex(g, 3 * t + 2)));
                    E = __fadd_rn(E, __fmul_rn(__fmul_rn(L.pw[m], om), inv_area));
                    ++closed;
                } else if (vis_c) {
                    E = __fadd_rn(E, __fmul_rn(L.pw[m], __fdiv_rn(nv, __fmul_rn(__fmul_rn(kFourPi, d2), d))));
                }
            }
            if (P.valid) {
                A[(size_t)i * lda + j] = ((failed_all >> lane) & 1u) ? __int_as_float(0x7fffffff) : E;
                if (nclosed) nclosed[(size_t)i * S.np + j] = (uint8_t)closed;
            }
        }
    }
}

}  // namespace

int irradiance_area_mean(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, const float* ptri,
                         float* A, int64_t lda, uint8_t* nclosed, cudaStream_t stream) {
    if (nc == 0 || sc->np == 0) return UVC_OK;
    SceneView S = view_of(sc);
    const bool wedge = lamp.wedge != 0;
    const size_t smem = stack_smem_bytes(S.stack_cap) + (wedge ? wedge_smem_bytes(lamp.K) : 0);
    const void* kern = wedge ? (const void*)k_area_mean<true> : (const void*)k_area_mean<false>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return status_from_cuda(e);
    }
    const int njb = (S.np + 31) / 32;
    const int64_t ntask = ((nc + kAreaCandPerTask - 1) / kAreaCandPerTask) * njb;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int grid = per_sm * sm_count();
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (wedge)
        k_area_mean<true><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, ptri, A, lda, nclosed);
    else
        k_area_mean<false><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, ptri, A, lda, nclosed);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
