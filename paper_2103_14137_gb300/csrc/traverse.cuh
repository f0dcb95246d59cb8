// Device code of the segment queries shared by the single-matrix, streamed
// and batched kernels: scene view, ray set-up, watertight segment/triangle
// test, four-wide packet traversal, and one irradiance entry (paper Sec.
// IV-C, Eq. (7) with its visibility rule).  See irradiance.cu for the design.
#pragma once

#include <algorithm>
#include <cmath>

#include "uvc_internal.cuh"

namespace uvc {
namespace {

// Resident blocks per SM the traversal kernels are compiled for (register cap
// 65536 / (256 * this)); tuning constants, measured on the ward workload.
#ifndef UVC_IRR_MIN_BLOCKS
#define UVC_IRR_MIN_BLOCKS 3
#endif
#ifndef UVC_STREAMED_MIN_BLOCKS
#define UVC_STREAMED_MIN_BLOCKS 3
#endif

constexpr unsigned kFull = 0xffffffffu;
constexpr float kFourPi = 12.566370614359172f;
// 1 + 2^-20: widening of the far slab distance; covers the relative rounding
// of (b - o) * (1/d) (three roundings) with a wide margin.
constexpr float kFarScale = 1.0f + 9.5367431640625e-07f;

struct SceneView {
    const float4* __restrict__ tri;
    const Node4* __restrict__ nodes4;
    const float4* __restrict__ ps;
    const float4* __restrict__ pn;
    const int2* __restrict__ pe;
    int nt, np, root, stack_cap, visit_cap;
    float cut_eps;   // absolute slack (metres) subtracted from a patch's clearance
    int* status;
};

SceneView view_of(const uvc_scene* sc) {
    SceneView v;
    v.tri = sc->tri;
    v.nodes4 = sc->nodes4;
    v.ps = sc->patch_s;
    v.pn = sc->patch_n;
    v.pe = sc->patch_excl;
    v.nt = (int)sc->nt;
    v.np = (int)sc->np;
    v.root = sc->root;
    v.stack_cap = 3 * (sc->depth4 + 1) + 1;   // at most 3 pushes per four-wide level
    v.visit_cap = (int)sc->nt + 64;
    v.cut_eps = 1e-5f * sc->diameter;
    v.status = sc->status;
    return v;
}

struct Ray {
    float ox, oy, oz;   // segment start (the source point, warp-uniform)
    float dx, dy, dz;   // segment vector: end = start + d
    float ix, iy, iz;   // 1/d with zero components replaced by +-1e-30
    float sx, sy, sz;   // shear constants of the watertight test
    float tend;         // box tests stop at this segment parameter (<= 1), see clearance
    int kx, ky, kz;     // axis permutation of the watertight test
    int ex0, ex1;       // triangles that never occlude this segment
};

__device__ __forceinline__ float pick(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

__device__ __forceinline__ float safe_rcp(float d) {
    float a = fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d;
    return __frcp_rn(a);
}

__device__ __forceinline__ void setup_ray(Ray& r) {
    r.ix = safe_rcp(r.dx);
    r.iy = safe_rcp(r.dy);
    r.iz = safe_rcp(r.dz);
    float ax = fabsf(r.dx), ay = fabsf(r.dy), az = fabsf(r.dz);
    int kz = ax > ay ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dkz = pick(r.dx, r.dy, r.dz, kz);
    if (dkz < 0.f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.sx = __fdiv_rn(pick(r.dx, r.dy, r.dz, kx), dkz);
    r.sy = __fdiv_rn(pick(r.dx, r.dy, r.dz, ky), dkz);
    r.sz = __fdiv_rn(1.0f, dkz);
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Watertight segment/triangle test: hit iff the segment's line passes through
// the closed triangle (all edge functions of one sign, non-degenerate) and
// the parameter tau = T/det lies in the open interval (0, 1).
__device__ __forceinline__ bool seg_tri(const Ray& r, float4 a, float4 b, float4 c) {
    float Ax = __fsub_rn(a.x, r.ox), Ay = __fsub_rn(a.y, r.oy), Az = __fsub_rn(a.z, r.oz);
    float Bx = __fsub_rn(b.x, r.ox), By = __fsub_rn(b.y, r.oy), Bz = __fsub_rn(b.z, r.oz);
    float Cx = __fsub_rn(c.x, r.ox), Cy = __fsub_rn(c.y, r.oy), Cz = __fsub_rn(c.z, r.oz);
    float akz = pick(Ax, Ay, Az, r.kz), bkz = pick(Bx, By, Bz, r.kz), ckz = pick(Cx, Cy, Cz, r.kz);
    float ax = __fmaf_rn(-r.sx, akz, pick(Ax, Ay, Az, r.kx));
    float ay = __fmaf_rn(-r.sy, akz, pick(Ax, Ay, Az, r.ky));
    float bx = __fmaf_rn(-r.sx, bkz, pick(Bx, By, Bz, r.kx));
    float by = __fmaf_rn(-r.sy, bkz, pick(Bx, By, Bz, r.ky));
    float cx = __fmaf_rn(-r.sx, ckz, pick(Cx, Cy, Cz, r.kx));
    float cy = __fmaf_rn(-r.sy, ckz, pick(Cx, Cy, Cz, r.ky));
    float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    float det = U + V + W;
    if (det == 0.f) return false;
    float T = U * __fmul_rn(r.sz, akz) + V * __fmul_rn(r.sz, bkz) + W * __fmul_rn(r.sz, ckz);
    // tau = T / det in (0, 1), compared without dividing
    unsigned sgn = __float_as_uint(det) & 0x80000000u;
    float Ts = __uint_as_float(__float_as_uint(T) ^ sgn);
    float ds = __uint_as_float(__float_as_uint(det) ^ sgn);
    return Ts > 0.f && Ts < ds;
}

__device__ __forceinline__ uint32_t test_leaf(const SceneView& S, int k, const Ray& r, uint32_t mask, int lane) {
    const float4* t = S.tri + 3 * (size_t)k;
    float4 a = __ldg(t), b = __ldg(t + 1), c = __ldg(t + 2);
    int id = __float_as_int(a.w);
    bool hit = ((mask >> lane) & 1u) && id != r.ex0 && id != r.ex1 && seg_tri(r, a, b, c);
    return __ballot_sync(kFull, hit);
}

// Traversal counters of the instrumented variant (one launch, outside timing):
// [0] warp node visits, [1] warp leaf tests, [2] warp traversals,
// [3] lane box tests (alive lanes x 4 per node), [4] lane triangle tests,
// [5] facing segments.
constexpr int kNumCounters = 6;

// Both boxes of a child pair (packed FP32x2).  Each lane loads, per axis, the
// pair of planes its segment meets first (near) and last (far): the near
// planes are the lower bounds when the direction component is positive, the
// upper bounds when it is negative (the sign of 1/d is that of d, zero
// components included), so no per-axis minimum or maximum is needed:
// t = (b - o) * (1/d), t_near = max(0, near values), t_far = min(tend, far
// values), and a child is entered when t_near <= t_far * (1 + 2^-20)
// (conservative).  tend < 1 skips the part of the segment next to the patch
// point that lies within the patch's clearance: no triangle there can
// occlude it (k_clearance).
__device__ __forceinline__ void pair_hits(const Ray& r, float2 nox, float2 noy, float2 noz, float2 ix, float2 iy,
                                          float2 iz, float2 nx, float2 fx, float2 ny, float2 fy, float2 nz,
                                          float2 fz, bool& h0, bool& h1) {
    const float2 tnx = __fmul2_rn(__fadd2_rn(nx, nox), ix), tfx = __fmul2_rn(__fadd2_rn(fx, nox), ix);
    const float2 tny = __fmul2_rn(__fadd2_rn(ny, noy), iy), tfy = __fmul2_rn(__fadd2_rn(fy, noy), iy);
    const float2 tnz = __fmul2_rn(__fadd2_rn(nz, noz), iz), tfz = __fmul2_rn(__fadd2_rn(fz, noz), iz);
    const float tn0 = max3f(tnx.x, tny.x, fmaxf(tnz.x, 0.f));
    const float tf0 = min3f(tfx.x, tfy.x, fminf(tfz.x, r.tend));
    const float tn1 = max3f(tnx.y, tny.y, fmaxf(tnz.y, 0.f));
    const float tf1 = min3f(tfx.y, tfy.y, fminf(tfz.y, r.tend));
    h0 = tn0 <= tf0 * kFarScale;
    h1 = tn1 <= tf1 * kFarScale;
}

__device__ __forceinline__ float2 ldg2(const char* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

__device__ __forceinline__ int pick4(int4 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }

// Packet traversal of the four-wide tree from `node` with the lanes `alive`:
// returns the lanes found occluded; `failed` gets lanes whose search hit the
// visit cap; `hit_tri` receives the occluding leaf of each occluded lane.
// Children are entered in slot order (with the occluder cache in front, the
// order of children hardly changes the work).
template <bool COUNT>
__device__ __forceinline__ uint32_t traverse4(const SceneView& S, const Ray& r, uint32_t alive, int* stack, int lane,
                                           uint32_t& failed, unsigned long long* ctr, int& hit_tri) {
    const float2 nox = make_float2(-r.ox, -r.ox), noy = make_float2(-r.oy, -r.oy), noz = make_float2(-r.oz, -r.oz);
    const float2 ix = make_float2(r.ix, r.ix), iy = make_float2(r.iy, r.iy), iz = make_float2(r.iz, r.iz);
    // byte offset of the near pair inside an axis record (lo pair at 0, hi pair at 8)
    const int onx = (int)(__float_as_uint(r.dx) >> 31) * 8, ony = (int)(__float_as_uint(r.dy) >> 31) * 8,
              onz = (int)(__float_as_uint(r.dz) >> 31) * 8;
    uint32_t occl = 0;
    int top = 0, node = 0, visits = 0;
    unsigned long long c_leaf = 0, c_box = 0, c_tri = 0;
    while (true) {
        if (++visits > S.visit_cap) {
            failed = alive;
            if (lane == 0) atomicCAS(S.status, 0, UVC_E_TIMEOUT);
            break;
        }
        const Node4* nd = S.nodes4 + node;
        const char* b = reinterpret_cast<const char*>(nd);
        const char *bnx = b + onx, *bfx = b + (8 - onx), *bny = b + 16 + ony, *bfy = b + 16 + (8 - ony);
        const char *bnz = b + 32 + onz, *bfz = b + 32 + (8 - onz);
        const int4 rr = __ldg(&nd->r);
        const int4 mm = __ldg(&nd->m);
        bool h0, h1, h2, h3;
        pair_hits(r, nox, noy, noz, ix, iy, iz, ldg2(bnx), ldg2(bfx), ldg2(bny), ldg2(bfy), ldg2(bnz), ldg2(bfz), h0, h1);
        pair_hits(r, nox, noy, noz, ix, iy, iz, ldg2(bnx + 48), ldg2(bfx + 48), ldg2(bny + 48), ldg2(bfy + 48),
                  ldg2(bnz + 48), ldg2(bfz + 48), h2, h3);
        if (COUNT) c_box += 4 * __popc(alive);
        // which children any searching lane enters (one warp OR-reduction)
        const unsigned nib = ((alive >> lane) & 1u) ? (unsigned)h0 | ((unsigned)h1 << 1) | ((unsigned)h2 << 2) |
                                                          ((unsigned)h3 << 3)
                                                    : 0u;
        const unsigned hit = __reduce_or_sync(kFull, nib);
        unsigned leaves = hit & (unsigned)mm.x;
        while (leaves) {                   // leaf children: test their triangle
            const int c = __ffs(leaves) - 1;
            leaves &= leaves - 1;
            const uint32_t m = __ballot_sync(kFull, (nib >> c) & 1u) & alive;
            if (!m) continue;
            const int leaf = ~pick4(rr, c);
            if (COUNT) { ++c_leaf; c_tri += __popc(m); }
            const uint32_t h = test_leaf(S, leaf, r, m, lane);
            if ((h >> lane) & 1u) hit_tri = leaf;
            occl |= h;
            alive &= ~h;
        }
        if (!alive) break;
        unsigned inner = hit & (unsigned)mm.y;
        if ((leaves = hit & (unsigned)mm.x) != 0 && inner) {
            // lanes that just became occluded may have been the only ones wanting a child
            const unsigned nib2 = ((alive >> lane) & 1u) ? nib : 0u;
            inner &= __reduce_or_sync(kFull, nib2);
        }
        if (inner) {
            const int first = __ffs(inner) - 1;
            if (top + 3 > S.stack_cap) {
                failed = alive;
                if (lane == 0) atomicCAS(S.status, 0, UVC_E_STACK);
                break;
            }
            // push the others, highest slot first (branch-free)
            const unsigned rest = inner & (inner - 1);
            stack[top] = rr.w; top += (rest >> 3) & 1u;
            stack[top] = rr.z; top += (rest >> 2) & 1u;
            stack[top] = rr.y; top += (rest >> 1) & 1u;
            node = pick4(rr, first);
        } else {
            if (top == 0) break;
            node = stack[--top];
        }
    }
    if (COUNT && lane == 0) {
        atomicAdd(&ctr[0], (unsigned long long)visits);
        atomicAdd(&ctr[1], c_leaf);
        atomicAdd(&ctr[2], 1ull);
        atomicAdd(&ctr[3], c_box);
        atomicAdd(&ctr[4], c_tri);
    }
    return occl;
}

// Packet occlusion query for the lanes `alive`.
template <bool COUNT>
__device__ uint32_t warp_occluded(const SceneView& S, const Ray& r, uint32_t alive, int* stack, int lane,
                                  uint32_t& failed, unsigned long long* ctr, int& hit_tri) {
    failed = 0;
    if (COUNT && lane == 0) atomicAdd(&ctr[5], (unsigned long long)__popc(alive));
    if (S.nt == 0 || alive == 0) return 0;
    if (S.root < 0) {
        if (COUNT && lane == 0) {
            atomicAdd(&ctr[1], 1ull);
            atomicAdd(&ctr[2], 1ull);
            atomicAdd(&ctr[4], (unsigned long long)__popc(alive));
        }
        const uint32_t h = test_leaf(S, ~S.root, r, alive, lane);
        if ((h >> lane) & 1u) hit_tri = ~S.root;
        return h;
    }
    return traverse4<COUNT>(S, r, alive, stack, lane, failed, ctr, hit_tri);
}

// The patch of one lane: sample point, normal, excluded triangles.
struct PatchLane {
    float4 s, n;   // n.w = clearance (metres)
    int2 ex;
    bool valid;
};

__device__ __forceinline__ PatchLane load_patch(const SceneView& S, int j) {
    PatchLane P;
    P.valid = j < S.np;
    P.s = make_float4(0.f, 0.f, 0.f, 0.f);
    P.n = P.s;
    P.ex = make_int2(-1, -1);
    if (P.valid) {
        P.s = __ldg(&S.ps[j]);
        P.n = __ldg(&S.pn[j]);
        P.ex = __ldg(&S.pe[j]);
    }
    return P;
}

// Irradiance of candidate i at this lane's patch (lanes beyond np give 0).
// Writes the K visibility words when vis != nullptr.  Returns NaN for a lane
// whose search failed (and records UVC_E_TIMEOUT / UVC_E_STACK).
// `cache` is the lane's last occluding triangle (sorted index, -1 = none): it
// is tested first, and a hit settles the segment without a traversal (the
// same predicate the traversal would apply to that triangle).
template <bool COUNT = false>
__device__ __forceinline__ float irradiance_entry(const SceneView& S, const float* __restrict__ cand, int nc,
                                                  const LampDev& L, int i, int jb, int lane, int* stack,
                                                  uint32_t* __restrict__ vis, int nwords, const PatchLane& P,
                                                  int& cache, unsigned long long* ctr = nullptr) {
    const float4 s4 = P.s, n4 = P.n;
    const float cx = __ldg(&cand[3 * (size_t)i]), cy = __ldg(&cand[3 * (size_t)i + 1]),
                cz = __ldg(&cand[3 * (size_t)i + 2]);
    float E = 0.f;
    bool bad = false;
    for (int m = 0; m < L.K; ++m) {
        const float ox = __fadd_rn(cx, L.ox[m]), oy = __fadd_rn(cy, L.oy[m]), oz = __fadd_rn(cz, L.oz[m]);
        // v = o - s exactly as hi + lo (TwoSum)
        float hx = __fsub_rn(ox, s4.x), hy = __fsub_rn(oy, s4.y), hz = __fsub_rn(oz, s4.z);
        float qx = __fsub_rn(hx, ox), qy = __fsub_rn(hy, oy), qz = __fsub_rn(hz, oz);
        float lx = __fadd_rn(__fsub_rn(ox, __fsub_rn(hx, qx)), __fsub_rn(-s4.x, qx));
        float ly = __fadd_rn(__fsub_rn(oy, __fsub_rn(hy, qy)), __fsub_rn(-s4.y, qy));
        float lz = __fadd_rn(__fsub_rn(oz, __fsub_rn(hz, qz)), __fsub_rn(-s4.z, qz));
        // <n, v> with TwoProduct / TwoSum (error-free dot product)
        float p = __fmul_rn(n4.x, hx);
        float err = __fmaf_rn(n4.x, hx, -p);
        err = __fmaf_rn(n4.x, lx, err);
        float acc = p;
        {
            float p2 = __fmul_rn(n4.y, hy);
            float e2 = __fmaf_rn(n4.y, hy, -p2);
            float s = __fadd_rn(acc, p2);
            float z = __fsub_rn(s, acc);
            float q = __fadd_rn(__fsub_rn(acc, __fsub_rn(s, z)), __fsub_rn(p2, z));
            acc = s;
            err = __fadd_rn(err, __fadd_rn(q, e2));
            err = __fmaf_rn(n4.y, ly, err);
        }
        {
            float p3 = __fmul_rn(n4.z, hz);
            float e3 = __fmaf_rn(n4.z, hz, -p3);
            float s = __fadd_rn(acc, p3);
            float z = __fsub_rn(s, acc);
            float q = __fadd_rn(__fsub_rn(acc, __fsub_rn(s, z)), __fsub_rn(p3, z));
            acc = s;
            err = __fadd_rn(err, __fadd_rn(q, e3));
            err = __fmaf_rn(n4.z, lz, err);
        }
        const float nv = __fadd_rn(acc, err);
        const float d2 = __fmaf_rn(hx, hx, __fmaf_rn(hy, hy, __fmul_rn(hz, hz)));
        const float d = sqrtf(d2);
        const bool facing = P.valid && nv > 0.f && d2 > 0.f;
        Ray r;
        r.ox = ox; r.oy = oy; r.oz = oz;
        r.dx = -hx; r.dy = -hy; r.dz = -hz;
        r.ex0 = P.ex.x; r.ex1 = P.ex.y;
        setup_ray(r);
        // the last `cut` metres before the patch point need no box tests; a
        // segment shorter than the cut meets no triangle at all
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
        const uint32_t occl = cached_mask | warp_occluded<COUNT>(S, r, facing_mask & ~cached_mask & ~settled_mask,
                                                                 stack, lane, failed, ctr, hit_tri);
        if (hit_tri >= 0) cache = hit_tri;
        const uint32_t visible = facing_mask & ~occl & ~failed;
        if (vis && lane == 0) vis[((size_t)m * nc + i) * nwords + jb] = visible;
        if ((failed >> lane) & 1u) bad = true;
        if ((visible >> lane) & 1u) {
            E = __fadd_rn(E, __fmul_rn(L.pw[m], __fdiv_rn(nv, __fmul_rn(__fmul_rn(kFourPi, d2), d))));
        }
    }
    return bad ? __int_as_float(0x7fffffff) : E;
}

}  // namespace
}  // namespace uvc
