// Scene upload and linear-BVH construction on the GPU.
//
// The environment boundary is a triangle mesh (paper Sec. III-B).  Occlusion
// queries (the visibility rule stated with Eq. (7), Sec. IV-C) are answered by
// a bounding-volume hierarchy built here in five data-parallel steps:
//   1. per triangle: bounding box, reference point (box centre), scene bounds
//   2. 63-bit Morton key of the reference point (21 bits per axis)
//   3. stable LSD radix sort of (key, triangle) in eight 8-bit passes
//   4. binary radix tree over the sorted keys (Karras, HPG 2012): every
//      internal node finds its own key range and split independently
//   5. bottom-up box refit: the second child to finish merges both boxes
// Nodes hold the boxes of both children so that one 64-byte load serves a
// traversal step.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "uvc_internal.cuh"

namespace uvc {
namespace {

constexpr int kSortItems = 8;                      // keys per thread per tile
constexpr int kSortTile = kThreads * kSortItems;   // 2048 keys per tile
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kSortPasses = 8;                     // 64 bits of key

enum : int { kErrTriIndex = 1, kErrVertex = 2, kErrExcl = 4, kErrPatch = 8 };

// Order-preserving map of floats to unsigned integers (for atomic min/max).
__device__ __forceinline__ unsigned int float_to_ordered(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
    return isfinite(x) && isfinite(y) && isfinite(z);
}

// Step 1: triangle boxes and reference points; scene bounds of the references.
__global__ void k_prepare_tris(const float* __restrict__ verts, int64_t nv, const int32_t* __restrict__ tris,
                               int nt, float4* __restrict__ tri_lo, float4* __restrict__ tri_hi,
                               float4* __restrict__ ref, unsigned int* bounds, int* err) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu};
    unsigned int mx[3] = {0u, 0u, 0u};
    unsigned int bmn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu};
    unsigned int bmx[3] = {0u, 0u, 0u};
    if (t < nt) {
        int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
        float3 lo = make_float3(0.f, 0.f, 0.f), hi = lo, p = lo;
        if (ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv) {
            atomicOr(err, kErrTriIndex);
        } else {
            float ax = verts[3 * ia], ay = verts[3 * ia + 1], az = verts[3 * ia + 2];
            float bx = verts[3 * ib], by = verts[3 * ib + 1], bz = verts[3 * ib + 2];
            float cx = verts[3 * ic], cy = verts[3 * ic + 1], cz = verts[3 * ic + 2];
            if (!finite3(ax, ay, az) || !finite3(bx, by, bz) || !finite3(cx, cy, cz)) atomicOr(err, kErrVertex);
            lo = make_float3(fminf(fminf(ax, bx), cx), fminf(fminf(ay, by), cy), fminf(fminf(az, bz), cz));
            hi = make_float3(fmaxf(fmaxf(ax, bx), cx), fmaxf(fmaxf(ay, by), cy), fmaxf(fmaxf(az, bz), cz));
            p = make_float3(__fmul_rn(__fadd_rn(lo.x, hi.x), 0.5f), __fmul_rn(__fadd_rn(lo.y, hi.y), 0.5f),
                            __fmul_rn(__fadd_rn(lo.z, hi.z), 0.5f));
            mn[0] = mx[0] = float_to_ordered(p.x);
            mn[1] = mx[1] = float_to_ordered(p.y);
            mn[2] = mx[2] = float_to_ordered(p.z);
            bmn[0] = float_to_ordered(lo.x); bmn[1] = float_to_ordered(lo.y); bmn[2] = float_to_ordered(lo.z);
            bmx[0] = float_to_ordered(hi.x); bmx[1] = float_to_ordered(hi.y); bmx[2] = float_to_ordered(hi.z);
        }
        tri_lo[t] = make_float4(lo.x, lo.y, lo.z, 0.f);
        tri_hi[t] = make_float4(hi.x, hi.y, hi.z, 0.f);
        ref[t] = make_float4(p.x, p.y, p.z, 0.f);
    }
    for (int k = 0; k < 3; ++k) {
        unsigned int a = __reduce_min_sync(0xffffffffu, mn[k]);
        unsigned int b = __reduce_max_sync(0xffffffffu, mx[k]);
        unsigned int c = __reduce_min_sync(0xffffffffu, bmn[k]);
        unsigned int d = __reduce_max_sync(0xffffffffu, bmx[k]);
        if ((threadIdx.x & 31) == 0) {
            if (a != 0xffffffffu) atomicMin(&bounds[k], a);
            if (b != 0u) atomicMax(&bounds[3 + k], b);
            if (c != 0xffffffffu) atomicMin(&bounds[6 + k], c);
            if (d != 0u) atomicMax(&bounds[9 + k], d);
        }
    }
}

// Patches: validate and pack into the scene's layout.
__global__ void k_pack_patches(uvc_patches p, int np, int nt, float4* __restrict__ ps, float4* __restrict__ pn,
                               int2* __restrict__ pe, int* err) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    float sx = p.centroid[3 * j], sy = p.centroid[3 * j + 1], sz = p.centroid[3 * j + 2];
    float nx = p.normal[3 * j], ny = p.normal[3 * j + 1], nz = p.normal[3 * j + 2];
    float a = p.area[j];
    int e0 = p.excl[2 * j], e1 = p.excl[2 * j + 1];
    if (!finite3(sx, sy, sz) || !finite3(nx, ny, nz) || !isfinite(a)) atomicOr(err, kErrPatch);
    if (e0 < -1 || e0 >= nt || e1 < -1 || e1 >= nt) atomicOr(err, kErrExcl);
    ps[j] = make_float4(sx, sy, sz, a);
    pn[j] = make_float4(nx, ny, nz, 0.f);
    pe[j] = make_int2(e0, e1);
}

__device__ __forceinline__ uint64_t spread21(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Step 2: Morton keys.  q = floor((p - lo) * (2^21 / (hi - lo))) in FP32 steps.
__global__ void k_morton(const float4* __restrict__ ref, int nt, const unsigned int* __restrict__ bounds,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float lo[3], scale[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = ordered_to_float(bounds[k]);
        float ext = __fsub_rn(ordered_to_float(bounds[3 + k]), lo[k]);
        scale[k] = ext > 0.f ? __fdiv_rn(2097152.0f, ext) : 0.f;
    }
    float4 p = ref[t];
    float pc[3] = {p.x, p.y, p.z};
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        float f = floorf(__fmul_rn(__fsub_rn(pc[k], lo[k]), scale[k]));
        q[k] = f >= 2097151.0f ? 2097151u : (uint32_t)f;
    }
    keys[t] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    vals[t] = (uint32_t)t;
}

// Step 3a: per-tile digit histograms, laid out [digit][tile].
__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint64_t* __restrict__ keys, int n, int shift,
                                                         int ntiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kRadixBins];
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) h[d] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int idx = base + k * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & (kRadixBins - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) hist[(size_t)d * ntiles + blockIdx.x] = h[d];
}

// Step 3b: exclusive scan of each digit's row of tile counts; row totals.
__global__ void __launch_bounds__(1024) k_radix_rowscan(uint32_t* __restrict__ hist, int ntiles,
                                                        uint32_t* __restrict__ totals) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    uint32_t* row = hist + (size_t)blockIdx.x * ntiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < ntiles; base += 1024) {
        int idx = base + threadIdx.x;
        uint32_t v = idx < ntiles ? row[idx] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        uint32_t excl = carry + (warp ? warp_sums[warp - 1] : 0u) + x - v;
        if (idx < ntiles) row[idx] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Step 3c: stable scatter.  Within a tile, keys are ranked in index order
// (warp chunk, then iteration, then lane) using warp match masks.
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint64_t* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            uint64_t* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out, int n, int shift,
                                                            int ntiles, const uint32_t* __restrict__ hist,
                                                            const uint32_t* __restrict__ totals) {
    __shared__ uint32_t tile_off[kRadixBins];
    __shared__ uint32_t cnt[kWarpsPerBlock][kRadixBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // digit base = exclusive scan of totals (256 values, by warp 0)
    if (warp == 0) {
        uint32_t v[8], run = 0;
        for (int k = 0; k < 8; ++k) { v[k] = totals[lane * 8 + k]; run += v[k]; }
        uint32_t x = run;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        uint32_t b = x - run;
        for (int k = 0; k < 8; ++k) {
            int d = lane * 8 + k;
            tile_off[d] = b + hist[(size_t)d * ntiles + blockIdx.x];
            b += v[k];
        }
    }
    for (int d = lane; d < kRadixBins; d += 32) cnt[warp][d] = 0;
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const int base = blockIdx.x * kSortTile + warp * (32 * kSortItems);
    uint64_t key[kSortItems];
    uint32_t val[kSortItems], rank[kSortItems], dig[kSortItems];
    for (int k = 0; k < kSortItems; ++k) {
        int idx = base + k * 32 + lane;
        bool ok = idx < n;
        key[k] = ok ? keys_in[idx] : 0ull;
        val[k] = ok ? vals_in[idx] : 0u;
        uint32_t d = ok ? (uint32_t)((key[k] >> shift) & (kRadixBins - 1)) : (uint32_t)(kRadixBins + lane);
        dig[k] = d;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = ok ? cnt[warp][d] : 0u;
        __syncwarp();
        rank[k] = before + __popc(peers & lt);
        if (ok && (31 - __clz(peers)) == lane) cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
        uint32_t run = 0;
        for (int w = 0; w < kWarpsPerBlock; ++w) {
            uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int k = 0; k < kSortItems; ++k) {
        int idx = base + k * 32 + lane;
        if (idx >= n) continue;
        uint32_t d = dig[k];
        uint32_t pos = tile_off[d] + cnt[warp][d] + rank[k];
        keys_out[pos] = key[k];
        vals_out[pos] = val[k];
    }
}

// Sorted triangle records and leaf boxes.
__global__ void k_gather_tris(const uint32_t* __restrict__ order, const float* __restrict__ verts, int64_t nv,
                              const int32_t* __restrict__ tris, int nt, const float4* __restrict__ tri_lo,
                              const float4* __restrict__ tri_hi, float4* __restrict__ tri_out,
                              int32_t* __restrict__ order_out, float4* __restrict__ leaf_lo,
                              float4* __restrict__ leaf_hi) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    int t = (int)order[k];
    int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
    // invalid indices were flagged by k_prepare_tris (the build then fails);
    // clamp so that no read leaves the vertex array meanwhile
    if (ia < 0 || ia >= nv) ia = 0;
    if (ib < 0 || ib >= nv) ib = 0;
    if (ic < 0 || ic >= nv) ic = 0;
    tri_out[3 * k] = make_float4(verts[3 * ia], verts[3 * ia + 1], verts[3 * ia + 2], __int_as_float(t));
    tri_out[3 * k + 1] = make_float4(verts[3 * ib], verts[3 * ib + 1], verts[3 * ib + 2], 0.f);
    tri_out[3 * k + 2] = make_float4(verts[3 * ic], verts[3 * ic + 1], verts[3 * ic + 2], 0.f);
    order_out[k] = t;
    leaf_lo[k] = tri_lo[t];
    leaf_hi[k] = tri_hi[t];
}

// Common prefix of the extended keys (key, position) at sorted positions i, j;
// -1 when j lies outside [0, n).
__device__ __forceinline__ int prefix_len(const uint64_t* __restrict__ keys, int n, int i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    uint64_t a = keys[i], b = keys[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz(i ^ (int)j);
}

// Step 4: binary radix tree, one thread per internal node (Karras 2012).
__global__ void k_karras(const uint64_t* __restrict__ keys, int n, int2* __restrict__ children,
                         int* __restrict__ parent_int, int* __restrict__ parent_leaf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (prefix_len(keys, n, i, i + 1) - prefix_len(keys, n, i, i - 1)) > 0 ? 1 : -1;
    int dmin = prefix_len(keys, n, i, i - d);
    int64_t lmax = 2;
    while (prefix_len(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (prefix_len(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = (int)(i + l * d);
    int dnode = prefix_len(keys, n, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (prefix_len(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = (int)(i + s * d + min(d, 0));
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? ~gamma : gamma;
    int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    children[i] = make_int2(left, right);
    if (left < 0) parent_leaf[~left] = i; else parent_int[left] = i;
    if (right < 0) parent_leaf[~right] = i; else parent_int[right] = i;
    if (i == 0) parent_int[0] = -1;
}

// Step 5: bottom-up refit; one thread per leaf climbs while it is the second
// child to arrive at a node.  Also computes subtree heights (tree depth).
__global__ void k_refit(int n, const int2* __restrict__ children, const int* __restrict__ parent_int,
                        const int* __restrict__ parent_leaf, const float4* __restrict__ leaf_lo,
                        const float4* __restrict__ leaf_hi, float4* node_lo, float4* node_hi, int* height,
                        int* flags, int* depth_out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int p = parent_leaf[k];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;   // first arrival: the sibling finishes p
        __threadfence();
        int2 c = children[p];
        float4 llo, lhi, rlo, rhi;
        int hl = 0, hr = 0;
        if (c.x < 0) { llo = leaf_lo[~c.x]; lhi = leaf_hi[~c.x]; }
        else { llo = __ldcg(&node_lo[c.x]); lhi = __ldcg(&node_hi[c.x]); hl = __ldcg(&height[c.x]); }
        if (c.y < 0) { rlo = leaf_lo[~c.y]; rhi = leaf_hi[~c.y]; }
        else { rlo = __ldcg(&node_lo[c.y]); rhi = __ldcg(&node_hi[c.y]); hr = __ldcg(&height[c.y]); }
        __stcg(&node_lo[p], make_float4(fminf(llo.x, rlo.x), fminf(llo.y, rlo.y), fminf(llo.z, rlo.z), 0.f));
        __stcg(&node_hi[p], make_float4(fmaxf(lhi.x, rhi.x), fmaxf(lhi.y, rhi.y), fmaxf(lhi.z, rhi.z), 0.f));
        int h = 1 + max(hl, hr);
        __stcg(&height[p], h);
        if (p == 0) { *depth_out = h; return; }
        p = parent_int[p];
    }
}

__global__ void k_pack_nodes(int n, const int2* __restrict__ children, const int* __restrict__ parent_int,
                             const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
                             const float4* __restrict__ node_lo, const float4* __restrict__ node_hi,
                             Node* __restrict__ nodes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int2 c = children[i];
    float4 L0 = c.x < 0 ? leaf_lo[~c.x] : node_lo[c.x];
    float4 L1 = c.x < 0 ? leaf_hi[~c.x] : node_hi[c.x];
    float4 R0 = c.y < 0 ? leaf_lo[~c.y] : node_lo[c.y];
    float4 R1 = c.y < 0 ? leaf_hi[~c.y] : node_hi[c.y];
    Node nd;
    nd.x = make_float4(L0.x, R0.x, L1.x, R1.x);
    nd.y = make_float4(L0.y, R0.y, L1.y, R1.y);
    nd.z = make_float4(L0.z, R0.z, L1.z, R1.z);
    nd.r = make_int4(c.x, c.y, parent_int[i], 0);
    nodes[i] = nd;
}

// Depth of every internal node (edges from the root), by walking up; the
// tree depth (deepest leaf) goes to *tree_depth.
__global__ void k_node_depth(int n, const int* __restrict__ parent_int, const int2* __restrict__ children,
                             int* __restrict__ depth, int* tree_depth) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = 0;
    int p = parent_int[i];
    while (p >= 0 && d < n) {
        ++d;
        p = parent_int[p];
    }
    depth[i] = d;
    const int2 c = children[i];
    if (c.x < 0 || c.y < 0) atomicMax(tree_depth, d + 1);
}

// ---------------------------------------------------------------------------
// Treelet restructuring (optional quality pass over the LBVH)
// ---------------------------------------------------------------------------
// The matrix asks 1e9+ segment queries of one hierarchy, so the hierarchy's
// quality matters far more than its build time.  After the refit, every
// internal node is visited bottom-up (second child to finish, as in the refit)
// and the treelet below it - the node's children, repeatedly replacing the
// internal treelet leaf of largest surface area by its two children, up to 7
// treelet leaves - is given the topology of least surface-area cost, found by
// dynamic programming over all subsets of the treelet leaves (Karras & Aila,
// "Fast Parallel Construction of High-Quality Bounding Volume Hierarchies",
// HPG 2013).  Cost of a subtree: C_i * area + children's costs; of a leaf:
// C_t * area.  The set of triangles under every treelet root is unchanged, so
// its box is too; only nodes inside the treelet are rewired.  Treelets of 5
// leaves: the dynamic programme over subsets costs about a ninth of 7
// leaves' (a pass takes ~0.3 ms instead of 2.3 ms on the ward) and one pass
// gives as fast a traversal (ward matrix 75.4 ms with 5, 75.3 with 6, 75.6
// with 7 leaves, 76.1 with 4); a second pass of 5-leaf treelets cuts node
// visits by 3 % (74.0 ms).
constexpr int kTreelet = 5;
constexpr int kRestructurePasses = 2;
constexpr float kCostNode = 1.2f, kCostTri = 1.0f;

__device__ __forceinline__ float half_area(float4 lo, float4 hi) {
    const float dx = fmaxf(hi.x - lo.x, 0.f), dy = fmaxf(hi.y - lo.y, 0.f), dz = fmaxf(hi.z - lo.z, 0.f);
    return dx * dy + dy * dz + dz * dx;
}

struct TreeView {
    int2* children;
    int* parent_int;
    int* parent_leaf;
    const float4* leaf_lo;
    const float4* leaf_hi;
    float4* node_lo;
    float4* node_hi;
    float* cost;
};

__device__ __forceinline__ void ref_box(const TreeView& T, int ref, float4& lo, float4& hi) {
    if (ref < 0) { lo = T.leaf_lo[~ref]; hi = T.leaf_hi[~ref]; }
    else { lo = __ldcg(&T.node_lo[ref]); hi = __ldcg(&T.node_hi[ref]); }
}

__device__ __forceinline__ float ref_cost(const TreeView& T, int ref) {
    if (ref < 0) return kCostTri * half_area(T.leaf_lo[~ref], T.leaf_hi[~ref]);
    return __ldcg(&T.cost[ref]);
}

__device__ void restructure_treelet(const TreeView& T, int root) {
    int tl[kTreelet];          // treelet leaves (refs)
    int ti[kTreelet - 1];      // treelet internal nodes (reused)
    const int2 rc = __ldcg(&T.children[root]);
    tl[0] = rc.x;
    tl[1] = rc.y;
    int nl = 2, nin = 1;
    ti[0] = root;
    while (nl < kTreelet) {
        int best = -1;
        float best_a = -1.f;
        for (int q = 0; q < nl; ++q) {
            if (tl[q] < 0) continue;
            float4 lo, hi;
            ref_box(T, tl[q], lo, hi);
            const float a = half_area(lo, hi);
            if (a > best_a) { best_a = a; best = q; }
        }
        if (best < 0) break;
        const int q = tl[best];
        const int2 c = __ldcg(&T.children[q]);
        ti[nin++] = q;
        tl[best] = c.x;
        tl[nl++] = c.y;
    }
    const float4 rlo = __ldcg(&T.node_lo[root]), rhi = __ldcg(&T.node_hi[root]);
    // current cost of the root's subtree (children are final)
    const float cur = kCostNode * half_area(rlo, rhi) + ref_cost(T, rc.x) + ref_cost(T, rc.y);
    if (nl <= 2) {
        __stcg(&T.cost[root], cur);
        return;
    }
    const int nsub = 1 << nl;
    float4 llo[kTreelet], lhi[kTreelet];
    float copt[1 << kTreelet];
    unsigned char part[1 << kTreelet];
    for (int q = 0; q < nl; ++q) {
        ref_box(T, tl[q], llo[q], lhi[q]);
        copt[1 << q] = ref_cost(T, tl[q]);
    }
    auto set_box = [&](int S, float4& lo, float4& hi) {
        lo = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
        hi = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
        for (int q = 0; q < nl; ++q)
            if (S & (1 << q)) {
                lo = make_float4(fminf(lo.x, llo[q].x), fminf(lo.y, llo[q].y), fminf(lo.z, llo[q].z), 0.f);
                hi = make_float4(fmaxf(hi.x, lhi[q].x), fmaxf(hi.y, lhi[q].y), fmaxf(hi.z, lhi[q].z), 0.f);
            }
    };
    for (int S = 1; S < nsub; ++S) {
        const int low = S & -S;
        if (S == low) continue;
        float best = 3.0e38f;
        int bp = low;
        // partitions (P, S\P) with P holding S's lowest leaf
        for (int P = (S - 1) & S; P != 0; P = (P - 1) & S) {
            if (!(P & low)) continue;
            const float c = copt[P] + copt[S ^ P];
            if (c < best) { best = c; bp = P; }
        }
        float4 lo, hi;
        set_box(S, lo, hi);
        copt[S] = kCostNode * half_area(lo, hi) + best;
        part[S] = (unsigned char)bp;
    }
    const int full = nsub - 1;
    if (!(copt[full] < cur * 0.999f)) {
        __stcg(&T.cost[root], cur);
        return;
    }
    // rewire: the root keeps its index and parent; other internal nodes are reused
    int st_set[kTreelet], st_node[kTreelet];
    int top = 0, next = 1;
    st_set[top] = full;
    st_node[top] = root;
    ++top;
    while (top > 0) {
        --top;
        const int S = st_set[top], node = st_node[top];
        const int P = part[S], Q = S ^ P;
        int ref[2];
        const int sets[2] = {P, Q};
        for (int h = 0; h < 2; ++h) {
            const int X = sets[h];
            if ((X & (X - 1)) == 0) {
                ref[h] = tl[__ffs(X) - 1];
            } else {
                const int m = ti[next++];
                ref[h] = m;
                st_set[top] = X;
                st_node[top] = m;
                ++top;
            }
            if (ref[h] < 0) T.parent_leaf[~ref[h]] = node;
            else T.parent_int[ref[h]] = node;
        }
        float4 lo, hi;
        set_box(S, lo, hi);
        __stcg(&T.children[node], make_int2(ref[0], ref[1]));
        __stcg(&T.node_lo[node], lo);
        __stcg(&T.node_hi[node], hi);
        __stcg(&T.cost[node], copt[S]);
    }
}

__global__ void k_restructure(int n, TreeView T, const int* __restrict__ leaf_parent0, int* flags) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int p = leaf_parent0[k];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;   // the sibling subtree finishes p
        __threadfence();
        restructure_treelet(T, p);
        __threadfence();
        if (p == 0) return;
        p = T.parent_int[p];
    }
}

// Collapse to the four-wide tree, top down, one level of four-wide nodes per
// launch: a four-wide node (kept at the index of the binary node it starts
// from) takes that node's two children and, while it has fewer than four,
// replaces the internal child of largest surface area by its two children
// (in place, so the slots keep the binary tree's left-to-right order); its
// internal children are the next level's four-wide nodes.  Fuller nodes than
// taking the grandchildren of every node at even depth (a leaf child there
// leaves a slot empty): on the ward, 4 % fewer node visits per query.
__device__ __forceinline__ float box_half_area(const float* lo, const float* hi) {
    const float dx = fmaxf(hi[0] - lo[0], 0.f), dy = fmaxf(hi[1] - lo[1], 0.f), dz = fmaxf(hi[2] - lo[2], 0.f);
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_collapse_level(const Node* __restrict__ nodes, const int* __restrict__ fin,
                                 const int* __restrict__ nin, int* __restrict__ fout, int* __restrict__ nout,
                                 Node4* __restrict__ nodes4) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *nin) return;
    const int i = fin[k];
    int ref[4];
    float lo[4][3], hi[4][3];
    int cnt = 0;
    auto kids = [&](int b, int at) {   // the two children of binary node b into slots at, at + 1
        const Node nd = nodes[b];
        ref[at] = nd.r.x;
        ref[at + 1] = nd.r.y;
        lo[at][0] = nd.x.x; lo[at][1] = nd.y.x; lo[at][2] = nd.z.x;
        hi[at][0] = nd.x.z; hi[at][1] = nd.y.z; hi[at][2] = nd.z.z;
        lo[at + 1][0] = nd.x.y; lo[at + 1][1] = nd.y.y; lo[at + 1][2] = nd.z.y;
        hi[at + 1][0] = nd.x.w; hi[at + 1][1] = nd.y.w; hi[at + 1][2] = nd.z.w;
    };
    kids(i, 0);
    cnt = 2;
    while (cnt < 4) {
        int best = -1;
        float ba = -1.f;
        for (int q = 0; q < cnt; ++q)
            if (ref[q] >= 0) {
                const float a = box_half_area(lo[q], hi[q]);
                if (a > ba) { ba = a; best = q; }
            }
        if (best < 0) break;
        const int b = ref[best];
        for (int q = cnt - 1; q > best; --q) {   // make room: slots after best move up by one
            ref[q + 1] = ref[q];
            for (int a = 0; a < 3; ++a) { lo[q + 1][a] = lo[q][a]; hi[q + 1][a] = hi[q][a]; }
        }
        kids(b, best);
        ++cnt;
    }
    const float far = 1e30f;
    for (int q = cnt; q < 4; ++q) {
        ref[q] = kEmptyChild;
        for (int a = 0; a < 3; ++a) { lo[q][a] = far; hi[q][a] = far; }
    }
    Node4 o;
    for (int h = 0; h < 2; ++h)
        for (int a = 0; a < 3; ++a)
            o.q[3 * h + a] = make_float4(lo[2 * h][a], lo[2 * h + 1][a], hi[2 * h][a], hi[2 * h + 1][a]);
    o.r = make_int4(ref[0], ref[1], ref[2], ref[3]);
    int leafmask = 0, innermask = 0, ninner = 0;
    for (int c = 0; c < 4; ++c) {
        if (ref[c] < 0) leafmask |= 1 << c;
        else if (ref[c] != kEmptyChild) { innermask |= 1 << c; ++ninner; }
    }
    o.m = make_int4(leafmask, innermask, 0, 0);
    nodes4[i] = o;
    if (ninner) {
        int at = atomicAdd(nout, ninner);
        for (int c = 0; c < 4; ++c)
            if ((innermask >> c) & 1) fout[at++] = ref[c];
    }
}

__global__ void k_collapse_start(int* frontier, int* counters, int nlevels) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nlevels) counters[k] = k == 0 ? 1 : 0;
    if (k == 0) frontier[0] = 0;
}

// Collapse to the four-wide tree: every internal node at even depth gets a
// four-wide node holding its children (leaf children) or grandchildren.
// (Kept for UVC_BUILD_LBVH_ONLY, whose four-wide tree the LBVH tests know.)
__global__ void k_collapse4(int n, const Node* __restrict__ nodes, const int* __restrict__ depth,
                            Node4* __restrict__ nodes4) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1 || (depth[i] & 1)) return;
    const Node nd = nodes[i];
    float lo[4][3], hi[4][3];
    int ref[4];
    const float far = 1e30f;
    for (int c = 0; c < 2; ++c) {
        const int r = c ? nd.r.y : nd.r.x;
        const float clo[3] = {c ? nd.x.y : nd.x.x, c ? nd.y.y : nd.y.x, c ? nd.z.y : nd.z.x};
        const float chi[3] = {c ? nd.x.w : nd.x.z, c ? nd.y.w : nd.y.z, c ? nd.z.w : nd.z.z};
        if (r < 0) {
            ref[2 * c] = r;
            ref[2 * c + 1] = kEmptyChild;
            for (int k = 0; k < 3; ++k) {
                lo[2 * c][k] = clo[k];
                hi[2 * c][k] = chi[k];
                lo[2 * c + 1][k] = far;
                hi[2 * c + 1][k] = far;
            }
        } else {
            const Node g = nodes[r];
            ref[2 * c] = g.r.x;
            ref[2 * c + 1] = g.r.y;
            lo[2 * c][0] = g.x.x; lo[2 * c][1] = g.y.x; lo[2 * c][2] = g.z.x;
            hi[2 * c][0] = g.x.z; hi[2 * c][1] = g.y.z; hi[2 * c][2] = g.z.z;
            lo[2 * c + 1][0] = g.x.y; lo[2 * c + 1][1] = g.y.y; lo[2 * c + 1][2] = g.z.y;
            hi[2 * c + 1][0] = g.x.w; hi[2 * c + 1][1] = g.y.w; hi[2 * c + 1][2] = g.z.w;
        }
    }
    Node4 o;
    for (int h = 0; h < 2; ++h)
        for (int k = 0; k < 3; ++k)
            o.q[3 * h + k] = make_float4(lo[2 * h][k], lo[2 * h + 1][k], hi[2 * h][k], hi[2 * h + 1][k]);
    o.r = make_int4(ref[0], ref[1], ref[2], ref[3]);
    int leafmask = 0, innermask = 0;
    for (int c = 0; c < 4; ++c) {
        if (ref[c] < 0) leafmask |= 1 << c;
        else if (ref[c] != kEmptyChild) innermask |= 1 << c;
    }
    o.m = make_int4(leafmask, innermask, 0, 0);
    nodes4[i] = o;
}

// Clearance of each patch: a lower bound on the distance from its sample
// point s_j to the nearest triangle that could occlude a segment ending at
// s_j.  Excluded triangles never occlude.  A triangle lying exactly in the
// patch's plane cannot meet a segment that arrives from the free side except
// at s_j itself (tau = 1, outside the open segment), so it is ignored unless
// it comes within `margin` of s_j in the plane (then the clearance is 0).  The
// plane test is exact: it applies when the patch normal is an exact axis
// vector and all three vertices share s_j's coordinate on that axis.  Other
// triangles count with the distance to their bounding box (a lower bound).
// The traversal uses the clearance to stop box tests that far short of s_j.
__device__ __forceinline__ float box_dist2(float px, float py, float pz, float lx, float ly, float lz, float hx,
                                           float hy, float hz) {
    const float dx = fmaxf(fmaxf(lx - px, px - hx), 0.f);
    const float dy = fmaxf(fmaxf(ly - py, py - hy), 0.f);
    const float dz = fmaxf(fmaxf(lz - pz, pz - hz), 0.f);
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ float seg2_dist2(float px, float py, float ax, float ay, float bx, float by) {
    const float ux = bx - ax, uy = by - ay;
    const float L = ux * ux + uy * uy;
    float t = L > 0.f ? ((px - ax) * ux + (py - ay) * uy) / L : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float dx = ax + t * ux - px, dy = ay + t * uy - py;
    return dx * dx + dy * dy;
}

// 2-D distance^2 from p to triangle (a, b, c) (0 inside).
__device__ float tri2_dist2(float px, float py, float ax, float ay, float bx, float by, float cx, float cy) {
    const float e0 = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
    const float e1 = (cx - bx) * (py - by) - (cy - by) * (px - bx);
    const float e2 = (ax - cx) * (py - cy) - (ay - cy) * (px - cx);
    if ((e0 >= 0.f && e1 >= 0.f && e2 >= 0.f) || (e0 <= 0.f && e1 <= 0.f && e2 <= 0.f)) return 0.f;
    return fminf(seg2_dist2(px, py, ax, ay, bx, by), fminf(seg2_dist2(px, py, bx, by, cx, cy),
                                                           seg2_dist2(px, py, cx, cy, ax, ay)));
}

__device__ __forceinline__ float tri_box_dist2(float px, float py, float pz, float4 a, float4 b, float4 c) {
    return box_dist2(px, py, pz, fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                     fminf(fminf(a.z, b.z), c.z), fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                     fmaxf(fmaxf(a.z, b.z), c.z));
}

// One thread per patch: depth-first nearest search, nearer child first,
// pruning boxes that are no closer than the best distance so far.
constexpr int kClearStack = 128;

__global__ void k_clearance(const Node* __restrict__ nodes, const float4* __restrict__ tri, int nt,
                            const float4* __restrict__ ps, float4* __restrict__ pn, const int2* __restrict__ pe,
                            int np, float margin) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const float4 s4 = ps[j];
    float4 n4 = pn[j];
    const int2 ex = pe[j];
    int ax = -1;
    if (fabsf(n4.x) == 1.f && n4.y == 0.f && n4.z == 0.f) ax = 0;
    if (fabsf(n4.y) == 1.f && n4.x == 0.f && n4.z == 0.f) ax = 1;
    if (fabsf(n4.z) == 1.f && n4.x == 0.f && n4.y == 0.f) ax = 2;
    const float sk = ax == 0 ? s4.x : (ax == 1 ? s4.y : s4.z);
    const float su = ax == 0 ? s4.y : s4.x, sv = ax == 2 ? s4.y : s4.z;   // in-plane coordinates
    const float margin2 = margin * margin;
    float best = 3.0e38f;
    int stack[kClearStack];
    int top = 0;
    if (nt > 1) stack[top++] = 0;
    else if (nt == 1) stack[top++] = ~0;
    int guard = 0;
    while (top > 0 && best > 0.f) {
        if (++guard > 4 * nt + 64) { best = 0.f; break; }   // cannot happen on a valid tree; 0 = no trimming
        const int ref = stack[--top];
        if (ref < 0) {
            const int k = ~ref;
            const float4 a = tri[3 * k], b = tri[3 * k + 1], c = tri[3 * k + 2];
            const int id = __float_as_int(a.w);
            if (id == ex.x || id == ex.y) continue;
            const float d2 = tri_box_dist2(s4.x, s4.y, s4.z, a, b, c);
            if (d2 >= best) continue;
            bool coplanar = false;
            if (ax >= 0) {
                const float ak = ax == 0 ? a.x : (ax == 1 ? a.y : a.z);
                const float bk = ax == 0 ? b.x : (ax == 1 ? b.y : b.z);
                const float ck = ax == 0 ? c.x : (ax == 1 ? c.y : c.z);
                coplanar = ak == sk && bk == sk && ck == sk;
            }
            if (coplanar) {
                const float au = ax == 0 ? a.y : a.x, av = ax == 2 ? a.y : a.z;
                const float bu = ax == 0 ? b.y : b.x, bv = ax == 2 ? b.y : b.z;
                const float cu = ax == 0 ? c.y : c.x, cv = ax == 2 ? c.y : c.z;
                if (tri2_dist2(su, sv, au, av, bu, bv, cu, cv) <= margin2) best = 0.f;
            } else {
                best = d2;
            }
            continue;
        }
        const Node nd = nodes[ref];
        const float dL = box_dist2(s4.x, s4.y, s4.z, nd.x.x, nd.y.x, nd.z.x, nd.x.z, nd.y.z, nd.z.z);
        const float dR = box_dist2(s4.x, s4.y, s4.z, nd.x.y, nd.y.y, nd.z.y, nd.x.w, nd.y.w, nd.z.w);
        const bool lfirst = dL <= dR;
        const int far_ref = lfirst ? nd.r.y : nd.r.x, near_ref = lfirst ? nd.r.x : nd.r.y;
        const float far_d = lfirst ? dR : dL, near_d = lfirst ? dL : dR;
        if (top + 2 > kClearStack) { best = 0.f; break; }
        if (far_d < best) stack[top++] = far_ref;
        if (near_d < best) stack[top++] = near_ref;
    }
    n4.w = sqrtf(best);
    pn[j] = n4;
}

// Clearance, warp-packet version over the four-wide tree: a warp takes 32
// consecutive (spatially close) patches and walks the tree once for all of
// them; each lane keeps its own best distance, a child is entered while any
// lane could still find something closer in it, nearest children first (as
// seen from the first lane).  Same definition as k_clearance.
__global__ void __launch_bounds__(kThreads) k_clearance4(const Node4* __restrict__ nodes4,
                                                         const float4* __restrict__ tri, int nt,
                                                         const float4* __restrict__ ps, float4* __restrict__ pn,
                                                         const int2* __restrict__ pe, int np, float margin,
                                                         int stack_cap) {
    extern __shared__ int cl_stack[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = cl_stack + warp * stack_cap;
    const int j = (blockIdx.x * kWarpsPerBlock + warp) * 32 + lane;
    const bool valid = j < np;
    const float4 s4 = valid ? ps[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 n4 = valid ? pn[j] : make_float4(0.f, 0.f, 1.f, 0.f);
    const int2 ex = valid ? pe[j] : make_int2(-1, -1);
    int ax = -1;
    if (fabsf(n4.x) == 1.f && n4.y == 0.f && n4.z == 0.f) ax = 0;
    if (fabsf(n4.y) == 1.f && n4.x == 0.f && n4.z == 0.f) ax = 1;
    if (fabsf(n4.z) == 1.f && n4.x == 0.f && n4.y == 0.f) ax = 2;
    const float sk = ax == 0 ? s4.x : (ax == 1 ? s4.y : s4.z);
    const float su = ax == 0 ? s4.y : s4.x, sv = ax == 2 ? s4.y : s4.z;
    const float margin2 = margin * margin;
    float best = valid ? 3.0e38f : 0.f;
    const uint32_t live = __ballot_sync(0xffffffffu, valid);
    if (!live) return;
    const int src = __ffs(live) - 1;
    int top = 0, node = 0, visits = 0;
    while (true) {
        if (++visits > 4 * nt + 64) { best = 0.f; break; }   // cannot happen on a valid tree
        const Node4* nd = nodes4 + node;
        const float4 q0 = nd->q[0], q1 = nd->q[1], q2 = nd->q[2], q3 = nd->q[3], q4 = nd->q[4], q5 = nd->q[5];
        const int4 rr = nd->r, mm = nd->m;
        float d[4];
        d[0] = box_dist2(s4.x, s4.y, s4.z, q0.x, q1.x, q2.x, q0.z, q1.z, q2.z);
        d[1] = box_dist2(s4.x, s4.y, s4.z, q0.y, q1.y, q2.y, q0.w, q1.w, q2.w);
        d[2] = box_dist2(s4.x, s4.y, s4.z, q3.x, q4.x, q5.x, q3.z, q4.z, q5.z);
        d[3] = box_dist2(s4.x, s4.y, s4.z, q3.y, q4.y, q5.y, q3.w, q4.w, q5.w);
        if (ax >= 0) {
            // a box flat in the patch's own plane holds only coplanar triangles:
            // it matters only if it comes within the margin (in-plane distance)
            const float lo4[4] = {ax == 0 ? q0.x : (ax == 1 ? q1.x : q2.x), ax == 0 ? q0.y : (ax == 1 ? q1.y : q2.y),
                                  ax == 0 ? q3.x : (ax == 1 ? q4.x : q5.x), ax == 0 ? q3.y : (ax == 1 ? q4.y : q5.y)};
            const float hi4[4] = {ax == 0 ? q0.z : (ax == 1 ? q1.z : q2.z), ax == 0 ? q0.w : (ax == 1 ? q1.w : q2.w),
                                  ax == 0 ? q3.z : (ax == 1 ? q4.z : q5.z), ax == 0 ? q3.w : (ax == 1 ? q4.w : q5.w)};
            for (int c = 0; c < 4; ++c)
                if (lo4[c] == sk && hi4[c] == sk && d[c] > margin2) d[c] = 3.0e38f;
        }
        const unsigned nib = (unsigned)(d[0] < best) | ((unsigned)(d[1] < best) << 1) |
                             ((unsigned)(d[2] < best) << 2) | ((unsigned)(d[3] < best) << 3);
        const unsigned hit = __reduce_or_sync(0xffffffffu, nib);
        unsigned leaves = hit & (unsigned)mm.x;
        while (leaves) {
            const int c = __ffs(leaves) - 1;
            leaves &= leaves - 1;
            if (!((nib >> c) & 1u)) continue;
            const int ref = c == 0 ? rr.x : (c == 1 ? rr.y : (c == 2 ? rr.z : rr.w));
            const int k = ~ref;
            const float4 a = tri[3 * k], b = tri[3 * k + 1], cc = tri[3 * k + 2];
            const int id = __float_as_int(a.w);
            if (id == ex.x || id == ex.y || d[c] >= best) continue;
            bool coplanar = false;
            if (ax >= 0) {
                const float ak = ax == 0 ? a.x : (ax == 1 ? a.y : a.z);
                const float bk = ax == 0 ? b.x : (ax == 1 ? b.y : b.z);
                const float ck = ax == 0 ? cc.x : (ax == 1 ? cc.y : cc.z);
                coplanar = ak == sk && bk == sk && ck == sk;
            }
            if (coplanar) {
                const float au = ax == 0 ? a.y : a.x, av = ax == 2 ? a.y : a.z;
                const float bu = ax == 0 ? b.y : b.x, bv = ax == 2 ? b.y : b.z;
                const float cu = ax == 0 ? cc.y : cc.x, cv = ax == 2 ? cc.y : cc.z;
                if (tri2_dist2(su, sv, au, av, bu, bv, cu, cv) <= margin2) best = 0.f;
            } else {
                best = d[c];
            }
        }
        // internal children still wanted (after the leaf updates), nearest first
        const unsigned nib2 = (unsigned)(d[0] < best) | ((unsigned)(d[1] < best) << 1) |
                              ((unsigned)(d[2] < best) << 2) | ((unsigned)(d[3] < best) << 3);
        unsigned inner = __reduce_or_sync(0xffffffffu, nib2) & (unsigned)mm.y;
        if (inner) {
            float key[4];
            for (int c = 0; c < 4; ++c) key[c] = __shfl_sync(0xffffffffu, d[c], src);
            if (top + 4 > stack_cap) { best = 0.f; break; }
            // push farthest first so that the nearest is popped next
            while (inner) {
                int far_c = -1;
                float far_k = -1.f;
                for (int c = 0; c < 4; ++c)
                    if (((inner >> c) & 1u) && key[c] > far_k) { far_k = key[c]; far_c = c; }
                inner &= ~(1u << far_c);
                stack[top++] = far_c == 0 ? rr.x : (far_c == 1 ? rr.y : (far_c == 2 ? rr.z : rr.w));
            }
        }
        if (top == 0) break;
        node = stack[--top];
    }
    if (valid) {
        n4.w = sqrtf(best);
        pn[j] = n4;
    }
}

struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int build_scene(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const uvc_patches* patches,
                int64_t np, uint32_t flags_in, cudaStream_t stream, uvc_scene** out) {
    if (!out) return UVC_E_INVAL;
    *out = nullptr;
    const int64_t lim = int64_t(1) << 31;
    if (nv < 0 || nt < 0 || np < 0 || nv >= lim || nt >= lim || np >= lim || !patches) return UVC_E_INVAL;
    if ((nt > 0 && (!verts || !tris || nv == 0)) || (nv > 0 && !verts)) return UVC_E_INVAL;
    if (np > 0 && (!patches->centroid || !patches->normal || !patches->area || !patches->excl)) return UVC_E_INVAL;

    uvc_scene* sc = new (std::nothrow) uvc_scene();
    if (!sc) return UVC_E_NOMEM;
    cudaGetDevice(&sc->device);
    sc->nt = nt;
    sc->np = np;
    sc->build_stream = stream;
    const int n = (int)nt;
    const int ni = n > 1 ? n - 1 : 0;

    // persistent buffers
    size_t bytes = align256(sizeof(float4) * 3 * (size_t)n) + align256(sizeof(Node) * (size_t)ni) +
                   align256(sizeof(Node4) * (size_t)ni) +
                   align256(sizeof(uint64_t) * (size_t)n) + align256(sizeof(int32_t) * (size_t)n) +
                   2 * align256(sizeof(float4) * (size_t)np) + align256(sizeof(int2) * (size_t)np) +
                   align256(sizeof(float)) + align256(sizeof(int)) + 256;
    if (cudaMallocAsync(&sc->block, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        delete sc;
        return UVC_E_NOMEM;
    }
    Carver pc(sc->block);
    sc->tri = pc.take<float4>(3 * (size_t)n);
    sc->nodes = pc.take<Node>(ni);
    sc->nodes4 = pc.take<Node4>(ni);
    sc->keys = pc.take<uint64_t>(n);
    sc->order = pc.take<int32_t>(n);
    sc->patch_s = pc.take<float4>(np);
    sc->patch_n = pc.take<float4>(np);
    sc->patch_excl = pc.take<int2>(np);
    sc->area_total = pc.take<float>(1);
    sc->status = pc.take<int>(1);

    // temporaries
    const int ntiles = (n + kSortTile - 1) / kSortTile;
    size_t tbytes = 3 * align256(sizeof(float4) * (size_t)n) +            // tri_lo, tri_hi, ref
                    align256(sizeof(uint64_t) * (size_t)n) +                // keys alt
                    2 * align256(sizeof(uint32_t) * (size_t)n) +            // vals, vals alt
                    align256(sizeof(uint32_t) * kRadixBins * (size_t)ntiles) + align256(sizeof(uint32_t) * kRadixBins) +
                    align256(sizeof(int2) * (size_t)ni) + align256(sizeof(int) * (size_t)ni) +   // children, parent_int
                    align256(sizeof(int) * (size_t)n) +                      // parent_leaf
                    2 * align256(sizeof(float4) * (size_t)n) +               // leaf lo/hi
                    2 * align256(sizeof(float4) * (size_t)ni) +              // node lo/hi
                    3 * align256(sizeof(int) * (size_t)ni) +                 // height, flags, depth
                    align256(sizeof(float) * (size_t)ni) +                   // subtree cost
                    align256(sizeof(int) * (size_t)n) +                      // leaf parents at pass start
                    align256(sizeof(unsigned int) * 12) + align256(sizeof(int) * 2) +
                    align256(sizeof(int) * ((size_t)n + 2)) + 256;                    // collapse level counters
    void* tblock = nullptr;
    if (cudaMallocAsync(&tblock, tbytes, stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(sc->block, stream);
        delete sc;
        return UVC_E_NOMEM;
    }
    Carver tc(tblock);
    float4* tri_lo = tc.take<float4>(n);
    float4* tri_hi = tc.take<float4>(n);
    float4* ref = tc.take<float4>(n);
    uint64_t* keys_alt = tc.take<uint64_t>(n);
    uint32_t* vals = tc.take<uint32_t>(n);
    uint32_t* vals_alt = tc.take<uint32_t>(n);
    uint32_t* hist = tc.take<uint32_t>(kRadixBins * (size_t)ntiles);
    uint32_t* totals = tc.take<uint32_t>(kRadixBins);
    int2* children = tc.take<int2>(ni);
    int* parent_int = tc.take<int>(ni);
    int* parent_leaf = tc.take<int>(n);
    float4* leaf_lo = tc.take<float4>(n);
    float4* leaf_hi = tc.take<float4>(n);
    float4* node_lo = tc.take<float4>(ni);
    float4* node_hi = tc.take<float4>(ni);
    int* height = tc.take<int>(ni);
    int* flags = tc.take<int>(ni);
    int* ndepth = tc.take<int>(ni);
    float* cost = tc.take<float>(ni);
    int* leaf_parent0 = tc.take<int>(n);
    unsigned int* bounds = tc.take<unsigned int>(12);   // reference points lo/hi, triangle boxes lo/hi
    int* errdepth = tc.take<int>(2);   // [0] = error bits, [1] = depth
    int* level_counts = tc.take<int>((size_t)n + 2);   // four-wide nodes per level of the collapse

    cudaError_t e = cudaSuccess;
    unsigned int init_bounds[12] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u,
                                    0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    e = cudaMemcpyAsync(bounds, init_bounds, sizeof(init_bounds), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(errdepth, 0, 2 * sizeof(int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->status, 0, sizeof(int), stream);
    if (e == cudaSuccess && ni) e = cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)ni, stream);
    const int B = 256;
    if (e == cudaSuccess && np > 0)
        k_pack_patches<<<(int)((np + B - 1) / B), B, 0, stream>>>(*patches, (int)np, n, sc->patch_s, sc->patch_n,
                                                                   sc->patch_excl, errdepth);
    launch_area_total(sc->patch_s, np, sc->area_total, stream);
    if (e == cudaSuccess && n > 0) {
        k_prepare_tris<<<(n + B - 1) / B, B, 0, stream>>>(verts, nv, tris, n, tri_lo, tri_hi, ref, bounds, errdepth);
        k_morton<<<(n + B - 1) / B, B, 0, stream>>>(ref, n, bounds, sc->keys, vals);
        uint64_t* kin = sc->keys;
        uint64_t* kout = keys_alt;
        uint32_t* vin = vals;
        uint32_t* vout = vals_alt;
        for (int pass = 0; pass < kSortPasses; ++pass) {
            int shift = pass * kRadixBits;
            k_radix_hist<<<ntiles, kThreads, 0, stream>>>(kin, n, shift, ntiles, hist);
            k_radix_rowscan<<<kRadixBins, 1024, 0, stream>>>(hist, ntiles, totals);
            k_radix_scatter<<<ntiles, kThreads, 0, stream>>>(kin, vin, kout, vout, n, shift, ntiles, hist, totals);
            uint64_t* tk = kin; kin = kout; kout = tk;
            uint32_t* tv = vin; vin = vout; vout = tv;
        }
        // eight passes: the sorted keys are back in sc->keys, values in `vals`
        k_gather_tris<<<(n + B - 1) / B, B, 0, stream>>>(vin, verts, nv, tris, n, tri_lo, tri_hi, sc->tri, sc->order,
                                                         leaf_lo, leaf_hi);
        if (n > 1) {
            k_karras<<<(ni + B - 1) / B, B, 0, stream>>>(sc->keys, n, children, parent_int, parent_leaf);
            k_refit<<<(n + B - 1) / B, B, 0, stream>>>(n, children, parent_int, parent_leaf, leaf_lo, leaf_hi,
                                                       node_lo, node_hi, height, flags, errdepth + 1);
            if (!(flags_in & UVC_BUILD_LBVH_ONLY) && n > 2) {
                TreeView T{children, parent_int, parent_leaf, leaf_lo, leaf_hi, node_lo, node_hi, cost};
                for (int pass = 0; pass < kRestructurePasses; ++pass) {
                    cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)ni, stream);
                    cudaMemcpyAsync(leaf_parent0, parent_leaf, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice,
                                    stream);
                    k_restructure<<<(n + 127) / 128, 128, 0, stream>>>(n, T, leaf_parent0, flags);
                }
            }
            cudaMemsetAsync(errdepth + 1, 0, sizeof(int), stream);
            k_pack_nodes<<<(ni + B - 1) / B, B, 0, stream>>>(n, children, parent_int, leaf_lo, leaf_hi, node_lo,
                                                             node_hi, sc->nodes);
            k_node_depth<<<(ni + B - 1) / B, B, 0, stream>>>(n, parent_int, children, ndepth, errdepth + 1);
            if (flags_in & UVC_BUILD_LBVH_ONLY)
                k_collapse4<<<(ni + B - 1) / B, B, 0, stream>>>(n, sc->nodes, ndepth, sc->nodes4);
        }
        e = cudaGetLastError();
    }
    // one synchronisation: validation result, tree depth and the scene diameter
    // (clearance margin, traversal cut tolerance) come back to the host
    unsigned int host_bounds[12];
    int host_ed[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_bounds, bounds, sizeof(host_bounds), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_ed, errdepth, sizeof(host_ed), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    auto fail = [&](int code) {
        cudaGetLastError();
        cudaStreamSynchronize(stream);
        cudaFreeAsync(tblock, stream);
        cudaFree(sc->block);
        delete sc;
        return code;
    };
    if (e != cudaSuccess) return fail(UVC_E_CUDA);
    if (host_ed[0] != 0) return fail(UVC_E_INVAL);
    sc->depth = host_ed[1];
    sc->depth4 = (sc->depth + 1) / 2;
    if (n > 1 && !(flags_in & UVC_BUILD_LBVH_ONLY)) {
        // the greedy collapse, one launch per level of four-wide nodes; a path
        // of the four-wide tree advances at least one binary level per node,
        // so it has at most `depth` levels (the bound the stacks are sized by)
        sc->depth4 = sc->depth;
        int* fa = height;
        int* fb = flags;
        int* counters = level_counts;   // depth + 2 <= n + 1 counters
        const int nlev = sc->depth + 1;
        k_collapse_start<<<(nlev + 1 + B - 1) / B, B, 0, stream>>>(fa, counters, nlev + 1);
        for (int L = 0; L < nlev; ++L) {
            const int64_t bound = L < 15 ? std::min<int64_t>(ni, int64_t(1) << (2 * L)) : ni;
            k_collapse_level<<<(int)((bound + B - 1) / B), B, 0, stream>>>(sc->nodes, L & 1 ? fb : fa, counters + L,
                                                                         L & 1 ? fa : fb, counters + L + 1,
                                                                         sc->nodes4);
        }
        if (cudaGetLastError() != cudaSuccess) return fail(UVC_E_CUDA);
    }
    float diam = 0.f;
    if (n > 0) {
        double d2 = 0.0, cmax = 0.0;
        for (int k = 0; k < 3; ++k) {
            const unsigned int lo_u = host_bounds[6 + k], hi_u = host_bounds[9 + k];
            float lo_f, hi_f;
            unsigned int a = (lo_u & 0x80000000u) ? (lo_u & 0x7fffffffu) : ~lo_u;
            unsigned int b = (hi_u & 0x80000000u) ? (hi_u & 0x7fffffffu) : ~hi_u;
            std::memcpy(&lo_f, &a, 4);
            std::memcpy(&hi_f, &b, 4);
            const double ext = (double)hi_f - (double)lo_f;
            if (std::isfinite(ext)) d2 += ext * ext;
            if (std::isfinite(ext)) cmax = std::max(cmax, std::max(std::fabs((double)lo_f), std::fabs((double)hi_f)));
        }
        diam = (float)std::sqrt(d2);
        sc->coord_bound = (float)cmax;
    }
    sc->diameter = diam;
    if (np > 0) {
        // a patch closer than 2^-14 of the scene diameter to a coplanar triangle gets no clearance
        if (n > 1) {
            const int cap = 3 * (sc->depth4 + 1) + 8;
            const int blocks = (int)((np + kThreads - 1) / kThreads);
            k_clearance4<<<blocks, kThreads, sizeof(int) * kWarpsPerBlock * cap, stream>>>(
                sc->nodes4, sc->tri, n, sc->patch_s, sc->patch_n, sc->patch_excl, (int)np, diam * 6.103515625e-05f,
                cap);
        } else {
            k_clearance<<<(int)((np + B - 1) / B), B, 0, stream>>>(sc->nodes, sc->tri, n, sc->patch_s,
                                                                   sc->patch_n, sc->patch_excl, (int)np,
                                                                   diam * 6.103515625e-05f);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(UVC_E_CUDA);
    }
    cudaFreeAsync(tblock, stream);
    sc->root = n == 1 ? ~0 : 0;
    *out = sc;
    return UVC_OK;
}

}  // namespace uvc
