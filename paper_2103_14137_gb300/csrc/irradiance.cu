// Irradiance matrix (paper Sec. IV-C, Eq. (4) and Eq. (7)) by BVH segment
// queries, and the streamed fluence (Eq. (5)) that never stores the matrix.
//
// Work unit: one warp = one candidate i, one lamp source m at a time, and 32
// consecutive patches (one per lane).  All 32 segments of a warp start at the
// same source point, so the warp walks the hierarchy as a packet: one shared
// node stack, every node box tested by every still-searching lane, a child
// entered when any lane's segment overlaps it (ballot), and each lane leaving
// the search at its first occluder (any-hit).  Node and triangle loads are
// warp-uniform, i.e. one 16-byte transaction serves 32 lanes.  A row tile of
// A is written as one coalesced 128-byte store per warp; the visibility word
// of the 32 lanes is the warp ballot itself.
//
// Arithmetic (FP32 only):
//   source      o = fl32(c_i + off_m)
//   v = o - s   as an exact float pair (TwoSum), <n, v> with an error-free
//               dot product (TwoProduct + TwoSum), so the facing test and the
//               cosine keep full relative accuracy even for grazing angles
//   E          += w_m P <n, v> / (4 pi |v|^3)   for facing, unoccluded sources
//   occlusion   open segment o + tau (s - o), 0 < tau < 1, against every
//               triangle except the patch's own (excl), watertight
//               ray/triangle test of Woop, Benthin and Wald (JCGT 2013) with
//               the edge functions evaluated without contraction, and a
//               conservatively widened slab test for the boxes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

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

// Candidates per warp task: the warp keeps its 32 patches (and its occluder
// cache) over this many consecutive candidates.
constexpr int kCandPerTask = 8;

template <bool COUNT>
__global__ void __launch_bounds__(kThreads, UVC_IRR_MIN_BLOCKS) k_irradiance(SceneView S, const float* __restrict__ cand, int nc,
                                                         LampDev L, float* __restrict__ A, int64_t lda,
                                                         uint32_t* __restrict__ vis, unsigned long long* ctr) {
    extern __shared__ int smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = smem + warp * S.stack_cap;
    const int njb = (S.np + 31) >> 5;
    const int nchunk = (nc + kCandPerTask - 1) / kCandPerTask;
    const int64_t ntask = (int64_t)nchunk * njb;
    for (int64_t task = (int64_t)blockIdx.x * kWarpsPerBlock + warp; task < ntask;
         task += (int64_t)gridDim.x * kWarpsPerBlock) {
        const int jb = (int)(task / nchunk), ic = (int)(task % nchunk);
        const int j = jb * 32 + lane;
        const PatchLane P = load_patch(S, j);
        int cache = -1;
        const int i1 = min(nc, (ic + 1) * kCandPerTask);
        for (int i = ic * kCandPerTask; i < i1; ++i) {
            const float E = irradiance_entry<COUNT>(S, cand, nc, L, i, jb, lane, stack, vis, njb, P, cache, ctr);
            if (P.valid) A[(size_t)i * lda + j] = E;
        }
    }
}

// Streamed fluence, pass 1: warp task = (candidate chunk s, patch block jb).
// E values of up to 32 candidates are staged in shared memory, multiplied by
// the dwell times and added to the chunk's partial sums partial[s][v][j].
__global__ void __launch_bounds__(kThreads, UVC_STREAMED_MIN_BLOCKS) k_streamed(SceneView S, const float* __restrict__ cand, int nc,
                                                       LampDev L, const float* __restrict__ t, int nvec,
                                                       float* __restrict__ partial, int nsplit, int chunk) {
    extern __shared__ int smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = smem + warp * S.stack_cap;
    float* Et = reinterpret_cast<float*>(smem + kWarpsPerBlock * S.stack_cap) + warp * 32 * 32;
    const int njb = (S.np + 31) >> 5;
    const int64_t ntask = (int64_t)nsplit * njb;
    for (int64_t task = (int64_t)blockIdx.x * kWarpsPerBlock + warp; task < ntask;
         task += (int64_t)gridDim.x * kWarpsPerBlock) {
        const int s = (int)(task / njb), jb = (int)(task % njb);
        const int j = jb * 32 + lane;
        const PatchLane P = load_patch(S, j);
        int cache = -1;
        const int i0 = s * chunk, i1 = min(nc, i0 + chunk);
        for (int ib = i0; ib < i1; ib += 32) {
            const int nb = min(32, i1 - ib);
            for (int q = 0; q < nb; ++q)
                Et[q * 32 + lane] = irradiance_entry(S, cand, nc, L, ib + q, jb, lane, stack, nullptr, 0, P, cache);
            __syncwarp();
            if (j < S.np) {
                for (int v = 0; v < nvec; ++v) {
                    const float* tv = t + (size_t)v * nc + ib;
                    float sum = 0.f;
                    for (int q = 0; q < nb; ++q) sum = __fmaf_rn(__ldg(tv + q), Et[q * 32 + lane], sum);
                    float* pp = partial + ((size_t)s * nvec + v) * S.np + j;
                    *pp = (ib == i0) ? sum : __fadd_rn(*pp, sum);
                }
            }
            __syncwarp();
        }
    }
}

// Streamed fluence, pass 2: mu[v][j] = sum over chunks (fixed order, Kahan).
__global__ void k_reduce_partials(const float* __restrict__ partial, int nsplit, int nvec, int np,
                                  float* __restrict__ mu) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nvec * np) return;
    const size_t stride = (size_t)nvec * np;
    float sum = 0.f, c = 0.f;
    for (int s = 0; s < nsplit; ++s) {
        float y = __fsub_rn(partial[(size_t)s * stride + idx], c);
        float t = __fadd_rn(sum, y);
        c = __fsub_rn(__fsub_rn(t, sum), y);
        sum = t;
    }
    mu[idx] = sum;
}

int grid_for(const void* kernel, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * sm_count();
}

}  // namespace

int irradiance_matrix(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, float* A,
                      int64_t lda, uint32_t* vis, cudaStream_t stream) {
    if (nc == 0 || sc->np == 0) return UVC_OK;
    SceneView S = view_of(sc);
    const size_t smem = sizeof(int) * kWarpsPerBlock * S.stack_cap;
    const int njb = (S.np + 31) / 32;
    const int64_t ntask = ((nc + kCandPerTask - 1) / kCandPerTask) * njb;
    int grid = grid_for((const void*)k_irradiance<false>, smem);
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    k_irradiance<false><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, A, lda, vis, nullptr);
    return status_from_cuda(cudaGetLastError());
}

int irradiance_counters(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, float* A,
                        int64_t lda, unsigned long long* out6, cudaStream_t stream) {
    for (int k = 0; k < kNumCounters; ++k) out6[k] = 0;
    if (nc == 0 || sc->np == 0) return UVC_OK;
    SceneView S = view_of(sc);
    const size_t smem = sizeof(int) * kWarpsPerBlock * S.stack_cap;
    unsigned long long* dctr = nullptr;
    if (cudaMallocAsync(&dctr, sizeof(unsigned long long) * kNumCounters, stream) != cudaSuccess) {
        cudaGetLastError();
        return UVC_E_NOMEM;
    }
    cudaError_t e = cudaMemsetAsync(dctr, 0, sizeof(unsigned long long) * kNumCounters, stream);
    const int njb = (S.np + 31) / 32;
    const int64_t ntask = ((nc + kCandPerTask - 1) / kCandPerTask) * njb;
    int grid = grid_for((const void*)k_irradiance<true>, smem);
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (e == cudaSuccess) {
        k_irradiance<true><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, A, lda, nullptr, dctr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out6, dctr, sizeof(unsigned long long) * kNumCounters, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(dctr, stream);
    return status_from_cuda(e);
}

int fluence_streamed(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, const float* t,
                     int32_t nvec, float* mu, cudaStream_t stream) {
    if (sc->np == 0) return UVC_OK;
    SceneView S = view_of(sc);
    if (nc == 0) return status_from_cuda(cudaMemsetAsync(mu, 0, sizeof(float) * (size_t)nvec * S.np, stream));
    const size_t smem = sizeof(int) * kWarpsPerBlock * S.stack_cap + sizeof(float) * kWarpsPerBlock * 32 * 32;
    const int njb = (S.np + 31) / 32;
    int grid = grid_for((const void*)k_streamed, smem);
    // enough (chunk, block) tasks to fill the persistent grid several times over
    const int64_t want = 8 * (int64_t)grid * kWarpsPerBlock;
    int64_t nsplit = (want + njb - 1) / njb;
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, (nc + 31) / 32));
    const int64_t cap = (int64_t(1) << 31) / (4 * (int64_t)nvec * S.np);   // partials <= 2 GiB
    nsplit = std::max<int64_t>(1, std::min(nsplit, cap));
    const int chunk = (int)((nc + nsplit - 1) / nsplit);
    nsplit = (nc + chunk - 1) / chunk;
    float* partial = nullptr;
    if (cudaMallocAsync(&partial, sizeof(float) * (size_t)nsplit * nvec * S.np, stream) != cudaSuccess) {
        cudaGetLastError();
        return UVC_E_NOMEM;
    }
    const int64_t ntask = nsplit * njb;
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    k_streamed<<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, t, nvec, partial, (int)nsplit, chunk);
    const int64_t total = (int64_t)nvec * S.np;
    k_reduce_partials<<<(int)((total + 255) / 256), 256, 0, stream>>>(partial, (int)nsplit, nvec, S.np, mu);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(partial, stream);
    return status_from_cuda(e);
}

}  // namespace uvc

// ---------------------------------------------------------------------------
// Allocation-free streamed fluence
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory while they run: a host
// application whose own allocator has already claimed the device memory it is
// allowed to use, or a control loop that forbids allocation after start-up
// because cudaMalloc/cudaMallocAsync may block, synchronise or fail at a bad
// moment.  For them the chunk partial sums of the streamed fluence live in
// this fixed array instead.  Every GPU that loads the library holds it until
// the process exits.
namespace uvc {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float)];

// Device address of g_noalloc_scratch per device ordinal, resolved once per
// device (the host-side name of the array is only a stand-in, not a device
// address).
constexpr int kMaxDevices = 64;
std::atomic<float*> g_noalloc_ptr[kMaxDevices];
std::mutex g_noalloc_mutex;

int noalloc_scratch(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return UVC_E_CUDA;
    }
    float* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
        if (!p) {
            void* addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess || !addr) {
                cudaGetLastError();
                return UVC_E_CUDA;
            }
            p = static_cast<float*>(addr);
            g_noalloc_ptr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return UVC_OK;
}

}  // namespace

int fluence_streamed_noalloc(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, const float* t,
                             int32_t nvec, float* mu, cudaStream_t stream) {
    if (sc->np == 0) return UVC_OK;
    const size_t per_split = sizeof(float) * (size_t)nvec * (size_t)sc->np;
    if (per_split > kNoAllocScratchBytes) return UVC_E_SCRATCH;
    float* partial = nullptr;
    int rc = noalloc_scratch(&partial);
    if (rc != UVC_OK) return rc;
    SceneView S = view_of(sc);
    if (nc == 0) return status_from_cuda(cudaMemsetAsync(mu, 0, per_split, stream));
    const size_t smem = sizeof(int) * kWarpsPerBlock * S.stack_cap + sizeof(float) * kWarpsPerBlock * 32 * 32;
    const int njb = (S.np + 31) / 32;
    int grid = grid_for((const void*)k_streamed, smem);
    const int64_t want = 8 * (int64_t)grid * kWarpsPerBlock;
    int64_t nsplit = (want + njb - 1) / njb;
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, (nc + 31) / 32));
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, (int64_t)(kNoAllocScratchBytes / per_split)));
    const int chunk = (int)((nc + nsplit - 1) / nsplit);
    nsplit = (nc + chunk - 1) / chunk;
    const int64_t ntask = nsplit * njb;
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    // every partial is written before it is read, so the array needs no clearing
    k_streamed<<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, t, nvec, partial, (int)nsplit, chunk);
    const int64_t total = (int64_t)nvec * S.np;
    k_reduce_partials<<<(int)((total + 255) / 256), 256, 0, stream>>>(partial, (int)nsplit, nvec, S.np, mu);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
