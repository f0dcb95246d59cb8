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

// Checked build (UVC_CHECKED): every node, leaf and cached-triangle index of the
// traversals is tested against its array before it is used; an index out of
// range sets UVC_E_BOUNDS in the scene's status word and the access is
// skipped (the search ends for the lanes concerned, whose entries become NaN).
// The normal build compiles no checks.
#ifdef UVC_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool out_of_range(int* status, int idx, int n) {
    if (!kChecked || (idx >= 0 && idx < n)) return false;
    atomicCAS(status, 0, UVC_E_BOUNDS);
    return true;
}

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
    if (sc->limit_stack > 0 && sc->limit_stack < v.stack_cap) v.stack_cap = sc->limit_stack;
    if (sc->limit_visits > 0 && sc->limit_visits < v.visit_cap) v.visit_cap = sc->limit_visits;
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
    r.sz = __frcp_rn(dkz);   // the shear constants need no particular rounding, only one value per segment
    r.sx = __fmul_rn(pick(r.dx, r.dy, r.dz, kx), r.sz);
    r.sy = __fmul_rn(pick(r.dx, r.dy, r.dz, ky), r.sz);
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
// the parameter tau = T/det lies in the open interval (0, 1).  The segment is
// given by its start (ox, oy, oz) and the shear constants of setup_ray.
__device__ __forceinline__ bool seg_tri_k(float ox, float oy, float oz, int kx, int ky, int kz, float sx, float sy,
                                          float sz, float4 a, float4 b, float4 c) {
    float Ax = __fsub_rn(a.x, ox), Ay = __fsub_rn(a.y, oy), Az = __fsub_rn(a.z, oz);
    float Bx = __fsub_rn(b.x, ox), By = __fsub_rn(b.y, oy), Bz = __fsub_rn(b.z, oz);
    float Cx = __fsub_rn(c.x, ox), Cy = __fsub_rn(c.y, oy), Cz = __fsub_rn(c.z, oz);
    float akz = pick(Ax, Ay, Az, kz), bkz = pick(Bx, By, Bz, kz), ckz = pick(Cx, Cy, Cz, kz);
    float ax = __fmaf_rn(-sx, akz, pick(Ax, Ay, Az, kx));
    float ay = __fmaf_rn(-sy, akz, pick(Ax, Ay, Az, ky));
    float bx = __fmaf_rn(-sx, bkz, pick(Bx, By, Bz, kx));
    float by = __fmaf_rn(-sy, bkz, pick(Bx, By, Bz, ky));
    float cx = __fmaf_rn(-sx, ckz, pick(Cx, Cy, Cz, kx));
    float cy = __fmaf_rn(-sy, ckz, pick(Cx, Cy, Cz, ky));
    float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    float det = U + V + W;
    if (det == 0.f) return false;
    float T = U * __fmul_rn(sz, akz) + V * __fmul_rn(sz, bkz) + W * __fmul_rn(sz, ckz);
    // tau = T / det in (0, 1), compared without dividing
    unsigned sgn = __float_as_uint(det) & 0x80000000u;
    float Ts = __uint_as_float(__float_as_uint(T) ^ sgn);
    float ds = __uint_as_float(__float_as_uint(det) ^ sgn);
    return Ts > 0.f && Ts < ds;
}

__device__ __forceinline__ bool seg_tri(const Ray& r, float4 a, float4 b, float4 c) {
    return seg_tri_k(r.ox, r.oy, r.oz, r.kx, r.ky, r.kz, r.sx, r.sy, r.sz, a, b, c);
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
// [3] lane segment box tests (alive lanes x 4 per node), [4] lane triangle
// tests (one segment against one triangle), [5] facing segments, [6] lane
// wedge box tests, [7] lane wedge plane tests (see the wedge traversal).
constexpr int kNumCounters = 8;

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
        if (out_of_range(S.status, node, S.nt - 1)) {
            failed = alive;
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
            if (out_of_range(S.status, leaf, S.nt)) {
                failed = alive;
                alive = 0;
                break;
            }
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

// One source's terms for the patch point s (normal n): v = o - s as the
// rounded difference h plus its exact error (TwoSum), <n, v> with an
// error-free dot product (TwoProduct + TwoSum) rounded once, and |h|^2.  Both
// traversal paths call this, so their Eq. (7) terms agree bit for bit.
__device__ __forceinline__ void source_terms(float ox, float oy, float oz, float4 s4, float4 n4, float& hx, float& hy,
                                             float& hz, float& nv, float& d2) {
    hx = __fsub_rn(ox, s4.x);
    hy = __fsub_rn(oy, s4.y);
    hz = __fsub_rn(oz, s4.z);
    const float qx = __fsub_rn(hx, ox), qy = __fsub_rn(hy, oy), qz = __fsub_rn(hz, oz);
    const float lx = __fadd_rn(__fsub_rn(ox, __fsub_rn(hx, qx)), __fsub_rn(-s4.x, qx));
    const float ly = __fadd_rn(__fsub_rn(oy, __fsub_rn(hy, qy)), __fsub_rn(-s4.y, qy));
    const float lz = __fadd_rn(__fsub_rn(oz, __fsub_rn(hz, qz)), __fsub_rn(-s4.z, qz));
    const float p = __fmul_rn(n4.x, hx);
    float err = __fmaf_rn(n4.x, hx, -p);
    err = __fmaf_rn(n4.x, lx, err);
    float acc = p;
    {
        const float p2 = __fmul_rn(n4.y, hy);
        const float e2 = __fmaf_rn(n4.y, hy, -p2);
        const float s = __fadd_rn(acc, p2);
        const float z = __fsub_rn(s, acc);
        const float q = __fadd_rn(__fsub_rn(acc, __fsub_rn(s, z)), __fsub_rn(p2, z));
        acc = s;
        err = __fadd_rn(err, __fadd_rn(q, e2));
        err = __fmaf_rn(n4.y, ly, err);
    }
    {
        const float p3 = __fmul_rn(n4.z, hz);
        const float e3 = __fmaf_rn(n4.z, hz, -p3);
        const float s = __fadd_rn(acc, p3);
        const float z = __fsub_rn(s, acc);
        const float q = __fadd_rn(__fsub_rn(acc, __fsub_rn(s, z)), __fsub_rn(p3, z));
        acc = s;
        err = __fadd_rn(err, __fadd_rn(q, e3));
        err = __fmaf_rn(n4.z, lz, err);
    }
    nv = __fadd_rn(acc, err);
    d2 = __fmaf_rn(hx, hx, __fmaf_rn(hy, hy, __fmul_rn(hz, hz)));
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
        float hx, hy, hz, nv, d2;
        source_terms(ox, oy, oz, s4, n4, hx, hy, hz, nv, d2);
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
        if (facing && !settled && cache >= 0 && !out_of_range(S.status, cache, S.nt)) {
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

// ---------------------------------------------------------------------------
// Wedge traversal for vertical line lamps
// ---------------------------------------------------------------------------
// When every source offset is vertical (x = y = 0), the sources of candidate
// c are o_m = (c.x, c.y, fl32(c.z + off_m.z)), all on the vertical line
// through c, and the segments from them to a patch point s lie in one
// triangle, the wedge conv(o_lo, o_hi, s) (o_lo, o_hi: the lowest and highest
// source still searching).  One packet traversal of the wedges replaces the K
// segment traversals: a child box is entered when it meets the lane's wedge,
// widened by delta, and every triangle reached is tested, with the same
// watertight segment test, against each source still searching that can meet
// it: none if the triangle lies entirely on one side of the wedge's vertical
// plane (farther than delta), else those in its lamp-height interval
// (lamp_interval).  A source stops at its first hit, a lane when all its
// sources have stopped, and the wedge narrows as its outer sources stop.
//
// Every triangle that a source's own segment traversal would reach is reached
// here (each segment lies inside the wedge, and delta = 1e-5 D exceeds the
// segment box test's widening), so each source gets the result of its own
// traversal; the only exception would be a triangle hit inside the patch's
// clearance, which only a triangle in the patch's own plane touching the
// patch point can be (a grazing pair).
//
// Coordinates: the horizontal part g of every segment of the lane is the same
// (the ray direction's x and y, rounded once in the set-up), so the point at
// segment parameter tau lies above c.xy + tau g whatever the source, and
// lambda = tau is a common parameter.  At lambda the wedge spans
//   zlow(lambda)  = z_lo + lambda (s.z - z_lo)  to
//   zhigh(lambda) = z_hi + lambda (s.z - z_hi).
// A box (widened by delta) meets the wedge iff its x and y slabs leave a
// lambda interval [a, b] inside [0, lambda_end] with z1 >= min(zlow(a),
// zlow(b)) and z0 <= max(zhigh(a), zhigh(b)) (both bounds are linear in
// lambda).  lambda_end is the largest clearance cut (tend) of the lane's
// searching sources.

struct WedgeLane {
    float2 oxn, oxf, oyn, oyf;   // -(c.x + delta sgn g.x) / g.x, -(c.x - delta sgn g.x) / g.x, same in y
    float2 igx, igy;             // 1/g.x, 1/g.y (as safe_rcp)
    float2 zl, zh, sl, sh;       // z_lo - delta, z_hi + delta, s.z - z_lo, s.z - z_hi
    float lend;                  // lambda_end
    float ig2;                   // 1 / |g|^2
    float mz;                    // delta * (longest segment) / |g|: margin of lamp_interval before 1/(1 - lambda)
    int onx, ony;                // byte offsets of the near planes in an axis record
};

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// z range of the searching sources `want` (bit m = source m).
__device__ __forceinline__ void wedge_z(WedgeLane& w, uint32_t want, float cz, const LampDev& L, float sz,
                                        float delta) {
    float zlo = 3.0e38f, zhi = -3.0e38f;
    for (uint32_t b = want; b; b &= b - 1) {
        const float oz = __fadd_rn(cz, L.oz[__ffs(b) - 1]);
        zlo = fminf(zlo, oz);
        zhi = fmaxf(zhi, oz);
    }
    w.zl = dup2(zlo - delta);
    w.zh = dup2(zhi + delta);
    w.sl = dup2(sz - zlo);
    w.sh = dup2(sz - zhi);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The sources of `want` whose segment can meet triangle (a, b, c).  Project
// the triangle orthogonally onto the wedge's vertical plane (the projection
// holds every point where the triangle meets the plane, and a segment that
// passes within e of the triangle passes within e of the projection) and then
// centrally from s onto the lamp line: a segment from height z meets the
// projection iff z lies in the image, which is the interval spanned by the
// images z_s + (z_V - z_s) / (1 - lambda_V) of the three vertices while all
// lambda_V < 1.  The interval is widened by mz / (1 - lambda_max): a
// displacement e of a segment at parameter lambda moves its lamp end by at
// most e |d| / (|g| (1 - lambda)), and mz = delta |d|max / |g| with delta
// far above the rounding of the segment test and of this projection.  A
// triangle reaching lambda >= 1 - 2^-10 (next to s or beyond) keeps every
// source, as does a degenerate g (NaN comparisons fail).
__device__ __forceinline__ uint32_t lamp_interval(float ig2, float mz, uint32_t want, float4 a, float4 b, float4 c,
                                                  float cx, float cy, float cz, float sz, float gx, float gy,
                                                  const LampDev& L) {
    const float la = __fmul_rn(__fmaf_rn(__fsub_rn(a.x, cx), gx, __fmul_rn(__fsub_rn(a.y, cy), gy)), ig2);
    const float lb = __fmul_rn(__fmaf_rn(__fsub_rn(b.x, cx), gx, __fmul_rn(__fsub_rn(b.y, cy), gy)), ig2);
    const float lc = __fmul_rn(__fmaf_rn(__fsub_rn(c.x, cx), gx, __fmul_rn(__fsub_rn(c.y, cy), gy)), ig2);
    const float lmax = max3f(la, lb, lc);
    if (!(lmax < 0.9990234375f)) return want;
    const float za = __fmaf_rn(__fsub_rn(a.z, sz), rcp_approx(__fsub_rn(1.f, la)), sz);
    const float zb = __fmaf_rn(__fsub_rn(b.z, sz), rcp_approx(__fsub_rn(1.f, lb)), sz);
    const float zc = __fmaf_rn(__fsub_rn(c.z, sz), rcp_approx(__fsub_rn(1.f, lc)), sz);
    const float m = __fmul_rn(mz, rcp_approx(__fsub_rn(1.f, lmax)));
    const float z0 = __fsub_rn(min3f(za, zb, zc), m), z1 = __fadd_rn(max3f(za, zb, zc), m);
    if (L.wuniform) {
        // source q sits at fl32(cz + off_q), off_q within dz/64 of wz0 + q dz:
        // every q with a height in [z0, z1] lies in [ceil(t0 - 1/32), floor(t1 + 1/32)]
        const float t0 = fminf(fmaxf((z0 - cz - L.wz0) * L.wrdz, -4.f), 40.f);
        const float t1 = fminf(fmaxf((z1 - cz - L.wz0) * L.wrdz, -4.f), 40.f);
        const int qlo = max(0, (int)ceilf(t0 - 0.03125f)), qhi = min(L.K - 1, (int)floorf(t1 + 0.03125f));
        if (qhi < qlo) return 0u;
        return want & ((2u << qhi) - 1u) & ~((1u << qlo) - 1u);
    }
    uint32_t in = 0;
    for (uint32_t bits = want; bits; bits &= bits - 1) {
        const int q = __ffs(bits) - 1;
        const float oz = __fadd_rn(cz, L.oz[q]);
        if (oz >= z0 && oz <= z1) in |= 1u << q;
    }
    return in;
}

// The slab parameters lambda = (x - X) / g come as one FMA, x (1/g) + (-X / g),
// with -X / g rounded once per lane: the rounding moves a plane by about
// 2^-24 of the coordinates, far inside the delta the boxes are widened by.
__device__ __forceinline__ void wedge_pair_hits(const WedgeLane& w, float2 nx, float2 fx, float2 ny, float2 fy,
                                                float2 z0, float2 z1, bool& h0, bool& h1) {
    const float2 lnx = __ffma2_rn(nx, w.igx, w.oxn), lfx = __ffma2_rn(fx, w.igx, w.oxf);
    const float2 lny = __ffma2_rn(ny, w.igy, w.oyn), lfy = __ffma2_rn(fy, w.igy, w.oyf);
    const float2 a = make_float2(max3f(lnx.x, lny.x, 0.f), max3f(lnx.y, lny.y, 0.f));
    const float2 b = make_float2(min3f(lfx.x, lfy.x, w.lend), min3f(lfx.y, lfy.y, w.lend));
    const float2 la = __ffma2_rn(a, w.sl, w.zl), lb = __ffma2_rn(b, w.sl, w.zl);
    const float2 ha = __ffma2_rn(a, w.sh, w.zh), hb = __ffma2_rn(b, w.sh, w.zh);
    h0 = a.x <= b.x && z1.x >= fminf(la.x, lb.x) && z0.x <= fmaxf(ha.x, hb.x);
    h1 = a.y <= b.y && z1.y >= fminf(la.y, lb.y) && z0.y <= fmaxf(ha.y, hb.y);
}

// Per (source, lane) data of the wedge path, in shared memory (one warp's
// slice): shear constants and axis permutation of the source's segment, and
// its Eq. (7) term w_m P <n, v> / (4 pi |v|^3); and the warp's queue of leaf
// tests (see wedge_traverse): a ring of items (lane << 27 | leaf), and per
// lane the sources found occluded by the last batch and the leaf that did it.
// The packed items need leaf indices below 2^27 (kWedgeMaxTris); larger
// scenes take the per-source traversal.
// The queue is worked off, up to 32 items at a time, once kLeafFlush items
// wait (a tuning constant: fewer waiting items stop lanes sooner, more keep
// the batches fuller; on the ward 16: 76.7, 24: 75.9, 32: 77.1, 48: 80.4 ms
// per matrix).
#ifndef UVC_LEAF_FLUSH
#define UVC_LEAF_FLUSH 24
#endif
constexpr int kLeafQueue = 256;       // ring entries per warp (< kLeafFlush waiting + at most 4 x 32 new)
constexpr int kLeafBatch = 32;        // items per batch: one per lane
constexpr int kLeafFlush = UVC_LEAF_FLUSH;
static_assert(kLeafFlush - 1 + 4 * 32 <= kLeafQueue && (kLeafQueue & (kLeafQueue - 1)) == 0,
              "the ring holds the waiting items plus one node's");
constexpr uint32_t kOobBit = 0x80000000u;   // checked build: a leaf index out of range (sources use bits 0..15)
constexpr int kItemLeafBits = 27;
constexpr uint32_t kItemLeafMask = (1u << kItemLeafBits) - 1u;
struct WedgeSmem {
    float4* shear;            // [K][32]: (sx, sy, sz, kx | ky << 2 | kz << 4)
    float* term;              // [K][32]
    uint32_t* qitem;          // [kLeafQueue]: lane << 27 | leaf
    uint32_t* occ;            // [32]
    int* qhit;                // [32]
};

// Shared memory of a block of the traversal kernels: the warps' stacks
// (16-byte aligned size), then kernel-specific staging, then the wedge arrays
// of all warps (shear of every warp, then term of every warp).
__host__ __device__ inline size_t stack_smem_bytes(int stack_cap) {
    return ((size_t)kWarpsPerBlock * stack_cap * sizeof(int) + 15) & ~size_t(15);
}
constexpr size_t kWedgeQueueBytes = kLeafQueue * sizeof(uint32_t) + 32 * (sizeof(uint32_t) + sizeof(int));
inline size_t wedge_smem_bytes(int K) {
    return (size_t)kWarpsPerBlock * (K * 32 * (sizeof(float4) + sizeof(float)) + kWedgeQueueBytes);
}

__device__ __forceinline__ WedgeSmem wedge_smem(char* base, int K, int warp) {
    WedgeSmem w;
    const size_t per_src = (size_t)kWarpsPerBlock * K * 32;
    w.shear = reinterpret_cast<float4*>(base) + (size_t)warp * K * 32;
    w.term = reinterpret_cast<float*>(base + per_src * sizeof(float4)) + (size_t)warp * K * 32;
    char* q = base + per_src * (sizeof(float4) + sizeof(float));   // 4-byte aligned
    w.qitem = reinterpret_cast<uint32_t*>(q) + (size_t)warp * kLeafQueue;
    q += (size_t)kWarpsPerBlock * kLeafQueue * sizeof(uint32_t);
    w.occ = reinterpret_cast<uint32_t*>(q) + (size_t)warp * 32;
    q += (size_t)kWarpsPerBlock * 32 * sizeof(uint32_t);
    w.qhit = reinterpret_cast<int*>(q) + (size_t)warp * 32;
    return w;
}

// One batch of queued leaf tests: lane k of the warp takes item head + k
// (k < n), a leaf wanted by some lane `own` of the warp, and tests it with
// own's wedge (the plane and lamp-height filters) and own's searching
// sources (the watertight segment test with own's shear constants), as own
// would have done itself; the sources found occluded are OR-ed into own's
// word, which own folds into `want` after the batch (narrowing its wedge).
// Items whose lane has stopped are skipped.  Every lane of the warp calls it.
template <bool COUNT>
__device__ __forceinline__ void wedge_leaf_batch(const SceneView& S, const LampDev& L, WedgeLane& w, uint32_t& want,
                                                 int lane, const WedgeSmem& ws, int head, int n, float cx, float cy,
                                                 float cz, float sz, float gx, float gy, float mh, int ex0, int ex1,
                                                 unsigned& c_leaf, unsigned& c_tri, int& hit_tri, bool& oob) {
    const bool has = lane < n;
    const uint32_t item = has ? ws.qitem[(head + lane) & (kLeafQueue - 1)] : (uint32_t)lane << kItemLeafBits;
    const int own = (int)(item >> kItemLeafBits);
    const int leaf = (int)(item & kItemLeafMask);
    const uint32_t owant = __shfl_sync(kFull, want, own);
    const float osz = __shfl_sync(kFull, sz, own);
    const float ogx = __shfl_sync(kFull, gx, own);
    const float ogy = __shfl_sync(kFull, gy, own);
    const float omh = __shfl_sync(kFull, mh, own);
    const float oig2 = __shfl_sync(kFull, w.ig2, own);
    const float omz = __shfl_sync(kFull, w.mz, own);
    const int oex0 = __shfl_sync(kFull, ex0, own);
    const int oex1 = __shfl_sync(kFull, ex1, own);
    if (has && owant) {
        uint32_t occl = 0;
        if (out_of_range(S.status, leaf, S.nt)) {
            occl = kOobBit;
        } else {
            const float4* t = S.tri + 3 * (size_t)leaf;
            const float4 ta = __ldg(t), tb = __ldg(t + 1), tc = __ldg(t + 2);
            const int id = __float_as_int(ta.w);
            if (COUNT) ++c_leaf;
            if (id != oex0 && id != oex1) {
                // triangle entirely on one side of the wedge's vertical plane,
                // farther than delta: no segment of the lane can meet it
                const float qa = __fmaf_rn(__fsub_rn(ta.x, cx), -ogy, __fmul_rn(__fsub_rn(ta.y, cy), ogx));
                const float qb = __fmaf_rn(__fsub_rn(tb.x, cx), -ogy, __fmul_rn(__fsub_rn(tb.y, cy), ogx));
                const float qc = __fmaf_rn(__fsub_rn(tc.x, cx), -ogy, __fmul_rn(__fsub_rn(tc.y, cy), ogx));
                const bool beside = (qa > omh && qb > omh && qc > omh) || (qa < -omh && qb < -omh && qc < -omh);
                if (!beside) {
                    const uint32_t test = owant & lamp_interval(oig2, omz, owant, ta, tb, tc, cx, cy, cz, osz, ogx,
                                                                ogy, L);
                    for (uint32_t bits = test; bits; bits &= bits - 1) {
                        const int q = __ffs(bits) - 1;
                        const float4 sh = ws.shear[q * 32 + own];
                        const int kb = __float_as_int(sh.w);
                        if (COUNT) ++c_tri;
                        if (seg_tri_k(cx, cy, __fadd_rn(cz, L.oz[q]), kb & 3, (kb >> 2) & 3, (kb >> 4) & 3, sh.x,
                                      sh.y, sh.z, ta, tb, tc))
                            occl |= 1u << q;
                    }
                }
            }
        }
        if (occl) {
            atomicOr(&ws.occ[own], occl);
            atomicMax(&ws.qhit[own], leaf);   // the lane caches the highest such leaf (deterministic)
        }
    }
    __syncwarp();
    const uint32_t o = ws.occ[lane];
    if (o) {
        ws.occ[lane] = 0u;
        if (kChecked && (o & kOobBit)) {
            oob = true;
            want = 0u;
        }
        const uint32_t nw = want & ~o;
        if (nw != want) {
            want = nw;
            hit_tri = ws.qhit[lane];
            if (want) wedge_z(w, want, cz, L, sz, S.cut_eps);
        }
        ws.qhit[lane] = -1;
    }
    __syncwarp();
}

// Lane-level wedge search.  `want` holds the lane's searching sources and
// loses the bit of each source found occluded; `hit_tri` gets the last
// occluding leaf.
//
// The leaf children a lane's wedge enters are not tested at once: they go to
// the warp's queue (shared memory), and whenever 32 items wait the whole warp
// works off 32 of them, one per lane, whichever lane wanted them.  Lanes want
// leaves unevenly (a few lanes near dense geometry, the rest none), so testing
// them where they arise would leave most lanes idle; the queue keeps the leaf
// tests nearly fully occupied at the price of narrowing a lane's wedge (and
// stopping it) up to a batch later.  The sources a lane finds occluded are
// those of its own search: every leaf its wedge enters while a source is
// still searching is tested against that source.
template <bool COUNT>
__device__ __forceinline__ void wedge_traverse(const SceneView& S, const LampDev& L, WedgeLane& w, uint32_t& want,
                                               uint32_t alive, int* stack, int lane, const WedgeSmem& ws, float cx,
                                               float cy, float cz, float sz, float gx, float gy, float mh, int ex0,
                                               int ex1, uint32_t& failed, unsigned long long* ctr, int& hit_tri) {
    int top = 0, node = 0, visits = 0, head = 0, tail = 0;
    unsigned long long c_box = 0;
    unsigned c_leaf = 0, c_tri = 0;
    bool oob = false;   // checked build: this lane met an index out of range
    ws.occ[lane] = 0u;
    ws.qhit[lane] = -1;
    __syncwarp();
    while (true) {
        if (++visits > S.visit_cap) {
            failed = alive;
            if (lane == 0) atomicCAS(S.status, 0, UVC_E_TIMEOUT);
            break;
        }
        if (out_of_range(S.status, node, S.nt - 1)) {
            failed = alive;
            break;
        }
        const Node4* nd = S.nodes4 + node;
        const int4 rr = __ldg(&nd->r);
        const int4 mm = __ldg(&nd->m);
        bool h0, h1, h2, h3;
        {
            const char* b = reinterpret_cast<const char*>(nd);
            const char *bnx = b + w.onx, *bfx = b + (8 - w.onx), *bny = b + 16 + w.ony, *bfy = b + 16 + (8 - w.ony);
            const char* bz = b + 32;
            wedge_pair_hits(w, ldg2(bnx), ldg2(bfx), ldg2(bny), ldg2(bfy), ldg2(bz), ldg2(bz + 8), h0, h1);
            wedge_pair_hits(w, ldg2(bnx + 48), ldg2(bfx + 48), ldg2(bny + 48), ldg2(bfy + 48), ldg2(bz + 48),
                            ldg2(bz + 56), h2, h3);
        }
        if (COUNT) c_box += 4 * __popc(alive);
        const unsigned nib = ((alive >> lane) & 1u) ? (unsigned)h0 | ((unsigned)h1 << 1) | ((unsigned)h2 << 2) |
                                                          ((unsigned)h3 << 3)
                                                    : 0u;
        const unsigned hit = __reduce_or_sync(kFull, nib);
        if (hit & (unsigned)mm.x) {
            // queue the lane's leaf children (prefix sum of the counts, at most 4 each)
            const unsigned mine = nib & (unsigned)mm.x;
            const unsigned cnt = __popc(mine), lt = (1u << lane) - 1u;
            const unsigned b0 = __ballot_sync(kFull, cnt & 1u), b1 = __ballot_sync(kFull, cnt & 2u),
                           b2 = __ballot_sync(kFull, cnt & 4u);
            int pos = tail + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
            tail += __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
            for (unsigned m = mine; m; m &= m - 1) {
                ws.qitem[pos & (kLeafQueue - 1)] = ((uint32_t)lane << kItemLeafBits) | (uint32_t)~pick4(rr, __ffs(m) - 1);
                ++pos;
            }
            __syncwarp();
            if (tail - head >= kLeafFlush) {
                do {
                    const int n = min(kLeafBatch, tail - head);
                    wedge_leaf_batch<COUNT>(S, L, w, want, lane, ws, head, n, cx, cy, cz, sz, gx, gy, mh, ex0, ex1,
                                            c_leaf, c_tri, hit_tri, oob);
                    head += n;
                } while (tail - head >= kLeafFlush);
                if (kChecked) failed |= __ballot_sync(kFull, oob);
                alive &= __ballot_sync(kFull, want != 0u);
                if (!alive) break;
            }
        }
        unsigned inner = hit & (unsigned)mm.y;
        if (inner) {
            const int first = __ffs(inner) - 1;
            if (top + 3 > S.stack_cap) {
                failed = alive;
                if (lane == 0) atomicCAS(S.status, 0, UVC_E_STACK);
                break;
            }
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
    if (tail > head) {   // the leaves still queued when the traversal ends
        wedge_leaf_batch<COUNT>(S, L, w, want, lane, ws, head, tail - head, cx, cy, cz, sz, gx, gy, mh, ex0, ex1,
                                c_leaf, c_tri, hit_tri, oob);
        if (kChecked) failed |= __ballot_sync(kFull, oob);
    }
    if (COUNT && lane == 0) {
        atomicAdd(&ctr[0], (unsigned long long)visits);
        atomicAdd(&ctr[2], 1ull);
        atomicAdd(&ctr[6], c_box);
    }
    if (COUNT) {   // leaf loads (each with its plane test) and triangle tests, by the lanes that made them
        const unsigned nleaf = __reduce_add_sync(kFull, c_leaf);
        const unsigned ntri = __reduce_add_sync(kFull, c_tri);
        if (lane == 0) {
            atomicAdd(&ctr[1], (unsigned long long)nleaf);
            atomicAdd(&ctr[7], (unsigned long long)nleaf);
            atomicAdd(&ctr[4], (unsigned long long)ntri);
        }
    }
}

// Per-source set-up of the segments from candidate c's sources to the lane's
// patch point (the arithmetic of irradiance_entry, source by source): shear
// constants and Eq. (7) terms go to shared memory; returns the facing sources
// and, in `want`, those that need a search (facing, longer than the clearance
// cut), with the largest cut parameter `lend`, the longest such segment
// `dmax` and the common horizontal direction (gx, gy).
__device__ __forceinline__ uint32_t wedge_setup_patch(const SceneView& S, const LampDev& L, float cx, float cy,
                                                      float cz, const PatchLane& P, int lane, const WedgeSmem& ws,
                                                      uint32_t& want, float& lend, float& dmax, float& gx,
                                                      float& gy) {
    const float4 s4 = P.s, n4 = P.n;
    uint32_t facing = 0;
    want = 0;
    lend = 0.f;
    dmax = 0.f;
    gx = 0.f;
    gy = 0.f;
    for (int m = 0; m < L.K; ++m) {
        const float ox = __fadd_rn(cx, L.ox[m]), oy = __fadd_rn(cy, L.oy[m]), oz = __fadd_rn(cz, L.oz[m]);
        float hx, hy, hz, nv, d2;
        source_terms(ox, oy, oz, s4, n4, hx, hy, hz, nv, d2);
        const float d = sqrtf(d2);
        const bool fac = P.valid && nv > 0.f && d2 > 0.f;
        Ray r;
        r.ox = ox; r.oy = oy; r.oz = oz;
        r.dx = -hx; r.dy = -hy; r.dz = -hz;
        setup_ray(r);
        const float cut = __fmaf_rn(0.99f, P.n.w, -S.cut_eps);
        const float tend = cut > 0.f ? 1.f - cut * __frcp_rn(d) : 1.f;
        ws.shear[m * 32 + lane] = make_float4(r.sx, r.sy, r.sz, __int_as_float(r.kx | (r.ky << 2) | (r.kz << 4)));
        ws.term[m * 32 + lane] = fac ? __fmul_rn(L.pw[m], __fdiv_rn(nv, __fmul_rn(__fmul_rn(kFourPi, d2), d))) : 0.f;
        if (fac) {
            facing |= 1u << m;
            if (tend > 0.f) {   // a segment shorter than the cut meets no triangle at all
                want |= 1u << m;
                lend = fmaxf(lend, tend);
                dmax = fmaxf(dmax, d);
            }
        }
        gx = r.dx;
        gy = r.dy;
    }
    return facing;
}

// Per-source set-up of the segments from the sources in `want` to point p
// (direction p - o rounded once, as a plain segment query; no clearance cut):
// shear constants to shared memory, the longest segment `dmax` and the common
// horizontal direction (gx, gy).
__device__ __forceinline__ void wedge_setup_point(const LampDev& L, float cx, float cy, float cz, float3 p,
                                                  uint32_t want, int lane, const WedgeSmem& ws, float& dmax,
                                                  float& gx, float& gy) {
    dmax = 0.f;
    gx = __fsub_rn(p.x, cx);
    gy = __fsub_rn(p.y, cy);
    for (uint32_t bits = want; bits; bits &= bits - 1) {
        const int m = __ffs(bits) - 1;
        Ray r;
        r.ox = __fadd_rn(cx, L.ox[m]); r.oy = __fadd_rn(cy, L.oy[m]); r.oz = __fadd_rn(cz, L.oz[m]);
        r.dx = __fsub_rn(p.x, r.ox); r.dy = __fsub_rn(p.y, r.oy); r.dz = __fsub_rn(p.z, r.oz);
        setup_ray(r);
        ws.shear[m * 32 + lane] = make_float4(r.sx, r.sy, r.sz, __int_as_float(r.kx | (r.ky << 2) | (r.kz << 4)));
        dmax = fmaxf(dmax, sqrtf(__fmaf_rn(r.dx, r.dx, __fmaf_rn(r.dy, r.dy, __fmul_rn(r.dz, r.dz)))));
    }
}

// The wedge search from the lamp line of candidate c to the lane's point
// (height sz, horizontal direction (gx, gy) from c) for the sources in `want`
// (shear constants already in shared memory): the lane's cached occluder
// first, then the packet traversal.  Returns the sources found occluded;
// `failed` gets the lanes whose search hit the visit cap or the stack limit.
template <bool COUNT>
__device__ __forceinline__ uint32_t wedge_search(const SceneView& S, const LampDev& L, float cx, float cy, float cz,
                                                 float sz, float gx, float gy, uint32_t want, float lend, float dmax,
                                                 int2 ex, int lane, int* stack, const WedgeSmem& ws, int& cache,
                                                 uint32_t& failed, unsigned long long* ctr) {
    const float delta = S.cut_eps;
    WedgeLane w;
    const float g2 = __fmaf_rn(gx, gx, __fmul_rn(gy, gy));
    const float gn = sqrtf(g2);
    const float mh = delta * gn;   // plane margin (the plane's normal (-g.y, g.x) is not normalised)
    w.ig2 = 1.f / g2;
    w.mz = delta * dmax / gn;
    // the lane's last occluder first, against the searching sources it can reach
    uint32_t occl = 0;
    if (want && cache >= 0 && !out_of_range(S.status, cache, S.nt)) {
        const float4* t = S.tri + 3 * (size_t)cache;
        const float4 ta = __ldg(t), tb = __ldg(t + 1), tc = __ldg(t + 2);
        const float qa = __fmaf_rn(__fsub_rn(ta.x, cx), -gy, __fmul_rn(__fsub_rn(ta.y, cy), gx));
        const float qb = __fmaf_rn(__fsub_rn(tb.x, cx), -gy, __fmul_rn(__fsub_rn(tb.y, cy), gx));
        const float qc = __fmaf_rn(__fsub_rn(tc.x, cx), -gy, __fmul_rn(__fsub_rn(tc.y, cy), gx));
        const bool beside = (qa > mh && qb > mh && qc > mh) || (qa < -mh && qb < -mh && qc < -mh);
        const uint32_t test = beside ? 0u : lamp_interval(w.ig2, w.mz, want, ta, tb, tc, cx, cy, cz, sz, gx, gy, L);
        for (uint32_t bits = test; bits; bits &= bits - 1) {
            const int q = __ffs(bits) - 1;
            const float4 sh = ws.shear[q * 32 + lane];
            const int kb = __float_as_int(sh.w);
            if (seg_tri_k(cx, cy, __fadd_rn(cz, L.oz[q]), kb & 3, (kb >> 2) & 3, (kb >> 4) & 3, sh.x, sh.y, sh.z, ta,
                          tb, tc))
                occl |= 1u << q;
        }
        want &= ~occl;
    }
    if (COUNT) {   // segments that need a search
        const unsigned nseg = __reduce_add_sync(kFull, (unsigned)__popc(want));
        if (lane == 0) atomicAdd(&ctr[5], (unsigned long long)nseg);
    }
    failed = 0;
    int hit_tri = -1;
    const uint32_t alive = __ballot_sync(kFull, want != 0u);
    if (alive && S.nt > 0) {
        const uint32_t before = want;
        if (S.root < 0) {   // a single triangle: test it directly
            const float4* t = S.tri + 3 * (size_t)(~S.root);
            const float4 ta = __ldg(t), tb = __ldg(t + 1), tc = __ldg(t + 2);
            const int id = __float_as_int(ta.w);
            if (id != ex.x && id != ex.y) {
                for (uint32_t bits = want; bits; bits &= bits - 1) {
                    const int q = __ffs(bits) - 1;
                    const float4 sh = ws.shear[q * 32 + lane];
                    const int kb = __float_as_int(sh.w);
                    if (seg_tri_k(cx, cy, __fadd_rn(cz, L.oz[q]), kb & 3, (kb >> 2) & 3, (kb >> 4) & 3, sh.x, sh.y,
                                  sh.z, ta, tb, tc))
                        want &= ~(1u << q);
                }
                if (want != before) hit_tri = ~S.root;
            }
        } else {
            const float sgx = (__float_as_uint(gx) >> 31) ? -delta : delta;
            const float sgy = (__float_as_uint(gy) >> 31) ? -delta : delta;
            const float igxs = safe_rcp(gx), igys = safe_rcp(gy);
            w.oxn = dup2(__fmul_rn(-(cx + sgx), igxs));
            w.oxf = dup2(__fmul_rn(-(cx - sgx), igxs));
            w.oyn = dup2(__fmul_rn(-(cy + sgy), igys));
            w.oyf = dup2(__fmul_rn(-(cy - sgy), igys));
            w.igx = dup2(igxs);
            w.igy = dup2(igys);
            w.lend = lend;
            w.onx = (int)(__float_as_uint(gx) >> 31) * 8;
            w.ony = (int)(__float_as_uint(gy) >> 31) * 8;
            if (want) wedge_z(w, want, cz, L, sz, delta);
            wedge_traverse<COUNT>(S, L, w, want, alive, stack, lane, ws, cx, cy, cz, sz, gx, gy, mh, ex.x, ex.y,
                                  failed, ctr, hit_tri);
        }
        occl |= before & ~want;
    }
    if (hit_tri >= 0) cache = hit_tri;
    return occl;
}

// Irradiance of candidate i at this lane's patch for a vertical line lamp
// (L.wedge): the same entry as irradiance_entry, with one wedge search per
// candidate instead of one segment search per source.
template <bool COUNT = false>
__device__ __forceinline__ float irradiance_wedge(const SceneView& S, const float* __restrict__ cand, int nc,
                                                  const LampDev& L, int i, int jb, int lane, int* stack,
                                                  const WedgeSmem& ws, uint32_t* __restrict__ vis, int nwords,
                                                  const PatchLane& P, int& cache, unsigned long long* ctr = nullptr) {
    const float cx = __ldg(&cand[3 * (size_t)i]), cy = __ldg(&cand[3 * (size_t)i + 1]),
                cz = __ldg(&cand[3 * (size_t)i + 2]);
    uint32_t want;
    float lend, dmax, gx, gy;
    const uint32_t facing = wedge_setup_patch(S, L, cx, cy, cz, P, lane, ws, want, lend, dmax, gx, gy);
    uint32_t failed;
    const uint32_t occl =
        wedge_search<COUNT>(S, L, cx, cy, cz, P.s.z, gx, gy, want, lend, dmax, P.ex, lane, stack, ws, cache, failed, ctr);
    const bool bad = (failed >> lane) & 1u;
    const uint32_t visible = bad ? 0u : (facing & ~occl);
    float E = 0.f;
    for (int m = 0; m < L.K; ++m) {
        const bool v = (visible >> m) & 1u;
        const uint32_t word = __ballot_sync(kFull, v);
        if (vis && lane == 0) vis[((size_t)m * nc + i) * nwords + jb] = word;
        if (v) E = __fadd_rn(E, ws.term[m * 32 + lane]);
    }
    return bad ? __int_as_float(0x7fffffff) : E;
}

}  // namespace
}  // namespace uvc
