// Visibility-cube estimator of the paper (Sec. IV-C, Fig. 2) as a CUDA
// software rasteriser: around every source point a cube of six R x R faces
// holds, per pixel, the nearest triangle along the ray through the pixel
// centre (a depth test); each pixel's power w_m P Omega_pixel / (4 pi) is
// added to its triangle when the ray meets the triangle's front side, and the
// flux over the triangle's area is its mean irradiance.
//
// The graphics pipeline of the paper (geometry shader, framebuffer, pixel
// blending) becomes four kernels over a batch of cubes:
//   setup    per (cube, face, triangle): the triangle clipped to the face's
//            near plane and projected; the pixel box that can hold it
//   scan     exclusive prefix sum of the box sizes: one flat index space of
//            candidate fragments, so large and small triangles balance
//   raster   per candidate fragment: watertight ray/triangle test through the
//            pixel centre, 64-bit atomicMin of (depth bits, triangle id)
//   resolve  per pixel: the power (a precomputed table, like the paper's
//            emission texture E) added to the triangle's flux in 2^-40 W
//            fixed point (integer atomics: the sum does not depend on order)
// and a finish pass divides by the triangle areas.
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "uvc_internal.cuh"

namespace uvc {
namespace {

constexpr float kFixOne = 1099511627776.0f;          // 2^40
constexpr float kFixInv = 1.0f / 1099511627776.0f;   // 2^-40
constexpr int kScanBlock = 1024, kScanPer = 4;       // 4096 elements per scan block
constexpr int kSampleShift = 8;                      // one search hint per 256 fragments

struct RasterBatch {
    const float4* tri;        // sorted triangles (v0.w = original id)
    const int32_t* order;     // sorted position -> original id
    int nt, R, C, K;
    const float* cand;        // candidates of this batch
    LampDev L;
    unsigned long long* keys;     // [C][6][R][R]
    unsigned long long* count;    // [E + 1] counts, then exclusive offsets (offsets[E] = total)
    unsigned long long* box;      // [E] x0 | y0 << 16 | w << 32
    unsigned long long* F;        // [C / K][nt] flux, 2^-40 W units, by original id
    const float* e_unit;          // [R][R] Omega_pixel / (4 pi)
    const float* tri_normal;      // [nt][3] by original id
    int* hint;                    // [total / 256 + 2] entry holding fragment 256 s (search hint)
    int64_t hint_cap;             // capacity of hint
};

__device__ __forceinline__ float comp(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

// Pixel-centre coordinate of pixel p on a face: fl32(fl32(2p + 1) / R) - 1.
__device__ __forceinline__ float pix_center(int p, int R) {
    return __fsub_rn(__fdiv_rn((float)(2 * p + 1), (float)R), 1.f);
}

__global__ void k_rs_setup(RasterBatch B, float near_eps) {
    const int64_t E = (int64_t)B.C * 6 * B.nt;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int k = (int)(e % B.nt);
    const int cf = (int)(e / B.nt);
    const int c = cf / 6, f = cf % 6;
    const int a = f >> 1, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    const float s = (f & 1) ? -1.f : 1.f;
    const int ci = c / B.K, m = c % B.K;
    const float ox = B.cand[3 * ci] + B.L.ox[m], oy = B.cand[3 * ci + 1] + B.L.oy[m],
                oz = B.cand[3 * ci + 2] + B.L.oz[m];
    float w[3], u[3], v[3];
    for (int q = 0; q < 3; ++q) {
        const float4 p = B.tri[3 * (size_t)k + q];
        const float rx = p.x - ox, ry = p.y - oy, rz = p.z - oz;
        w[q] = s * comp(rx, ry, rz, a);
        u[q] = comp(rx, ry, rz, b1);
        v[q] = comp(rx, ry, rz, b2);
    }
    // clip the triangle to w >= near_eps (Sutherland-Hodgman, one plane)
    float cw[4], cu[4], cv[4];
    int n = 0;
    for (int q = 0; q < 3; ++q) {
        const int r = (q + 1) % 3;
        const bool in_q = w[q] >= near_eps, in_r = w[r] >= near_eps;
        if (in_q) {
            cw[n] = w[q]; cu[n] = u[q]; cv[n] = v[q]; ++n;
        }
        if (in_q != in_r) {
            const float t = (near_eps - w[q]) / (w[r] - w[q]);
            cw[n] = near_eps; cu[n] = u[q] + t * (u[r] - u[q]); cv[n] = v[q] + t * (v[r] - v[q]); ++n;
        }
    }
    unsigned long long cnt = 0, bx = 0;
    if (n > 0) {
        float umin = 3e38f, umax = -3e38f, vmin = 3e38f, vmax = -3e38f;
        for (int q = 0; q < n; ++q) {
            const float pu = cu[q] / cw[q], pv = cv[q] / cw[q];
            umin = fminf(umin, pu); umax = fmaxf(umax, pu);
            vmin = fminf(vmin, pv); vmax = fmaxf(vmax, pv);
        }
        if (umax >= -1.f && umin <= 1.f && vmax >= -1.f && vmin <= 1.f) {
            umin = fmaxf(umin, -1.f); umax = fminf(umax, 1.f);
            vmin = fmaxf(vmin, -1.f); vmax = fminf(vmax, 1.f);
            const float h = 0.5f * B.R;
            // pixel centres (2p + 1) / R - 1 inside [min, max], widened by one pixel
            const int x0 = max(0, (int)floorf((umin + 1.f) * h - 0.5f) - 1);
            const int x1 = min(B.R - 1, (int)ceilf((umax + 1.f) * h - 0.5f) + 1);
            const int y0 = max(0, (int)floorf((vmin + 1.f) * h - 0.5f) - 1);
            const int y1 = min(B.R - 1, (int)ceilf((vmax + 1.f) * h - 0.5f) + 1);
            if (x1 >= x0 && y1 >= y0) {
                const unsigned long long wdt = (unsigned long long)(x1 - x0 + 1);
                cnt = wdt * (unsigned long long)(y1 - y0 + 1);
                bx = (unsigned long long)x0 | ((unsigned long long)y0 << 16) | (wdt << 32);
            }
        }
    }
    B.count[e] = cnt;
    B.box[e] = bx;
}

// Exclusive scan of n uint64 values in place (three passes).
__global__ void k_scan_blocks(unsigned long long* x, int64_t n, unsigned long long* sums) {
    __shared__ unsigned long long warp_tot[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanPer + (int64_t)threadIdx.x * kScanPer;
    unsigned long long v[kScanPer], run = 0;
    for (int q = 0; q < kScanPer; ++q) {
        v[q] = base + q < n ? x[base + q] : 0ull;
        run += v[q];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < kScanBlock / 32 ? warp_tot[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanBlock / 32) warp_tot[lane] = t;   // inclusive
    }
    __syncthreads();
    unsigned long long pre = (w > 0 ? warp_tot[w - 1] : 0ull) + inc - run;
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < n) x[base + q] = pre;
        pre += v[q];
    }
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = warp_tot[kScanBlock / 32 - 1];
}

__global__ void k_scan_sums(unsigned long long* sums, int nb, unsigned long long* total) {
    // one warp, chunks of 32 with a running carry
    const int lane = threadIdx.x;
    unsigned long long carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        const unsigned long long v = b0 + lane < nb ? sums[b0 + lane] : 0ull;
        unsigned long long inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (b0 + lane < nb) sums[b0 + lane] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) *total = carry;
}

__global__ void k_scan_add(unsigned long long* x, int64_t n, const unsigned long long* sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += sums[i / (kScanBlock * kScanPer)];
}

__global__ void k_fill64(unsigned long long* x, int64_t n, unsigned long long v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// hint[s] = the entry that holds fragment s << kSampleShift (thread per entry;
// entries own disjoint fragment ranges, so every hint slot is written once).
__global__ void k_rs_hints(RasterBatch B) {
    const int64_t E = (int64_t)B.C * 6 * B.nt;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const unsigned long long lo = B.count[e], hi = B.count[e + 1];
    if (hi == lo) return;
    const unsigned long long step = 1ull << kSampleShift;
    for (unsigned long long g = (lo + step - 1) & ~(step - 1); g < hi; g += step) {
        const unsigned long long s = g >> kSampleShift;
        if ((int64_t)s < B.hint_cap) B.hint[s] = (int)e;
    }
}

// Watertight ray/triangle test (Woop, Benthin and Wald, JCGT 2013) for the ray
// o + t d, t > 0; returns t (or a negative value for a miss).
__device__ __forceinline__ float ray_tri(float ox, float oy, float oz, float dx, float dy, float dz, float4 A4,
                                         float4 B4, float4 C4) {
    const float ax_ = fabsf(dx), ay_ = fabsf(dy), az_ = fabsf(dz);
    int kz = ax_ > ay_ ? (ax_ > az_ ? 0 : 2) : (ay_ > az_ ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dkz = comp(dx, dy, dz, kz);
    if (dkz < 0.f) {
        const int t = kx; kx = ky; ky = t;
    }
    const float sx = __fdiv_rn(comp(dx, dy, dz, kx), dkz), sy = __fdiv_rn(comp(dx, dy, dz, ky), dkz),
                sz = __fdiv_rn(1.f, dkz);
    const float Ax = __fsub_rn(A4.x, ox), Ay = __fsub_rn(A4.y, oy), Az = __fsub_rn(A4.z, oz);
    const float Bx = __fsub_rn(B4.x, ox), By = __fsub_rn(B4.y, oy), Bz = __fsub_rn(B4.z, oz);
    const float Cx = __fsub_rn(C4.x, ox), Cy = __fsub_rn(C4.y, oy), Cz = __fsub_rn(C4.z, oz);
    const float akz = comp(Ax, Ay, Az, kz), bkz = comp(Bx, By, Bz, kz), ckz = comp(Cx, Cy, Cz, kz);
    const float ax = __fmaf_rn(-sx, akz, comp(Ax, Ay, Az, kx)), ay = __fmaf_rn(-sy, akz, comp(Ax, Ay, Az, ky));
    const float bx = __fmaf_rn(-sx, bkz, comp(Bx, By, Bz, kx)), by = __fmaf_rn(-sy, bkz, comp(Bx, By, Bz, ky));
    const float cx = __fmaf_rn(-sx, ckz, comp(Cx, Cy, Cz, kx)), cy = __fmaf_rn(-sy, ckz, comp(Cx, Cy, Cz, ky));
    const float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    const float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    const float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return -1.f;
    const float det = U + V + W;
    if (det == 0.f) return -1.f;
    const float T = U * __fmul_rn(sz, akz) + V * __fmul_rn(sz, bkz) + W * __fmul_rn(sz, ckz);
    const float t = __fdiv_rn(T, det);
    return t > 0.f ? t : -1.f;
}

// ray_tri for a pixel ray of face (a, s): the axis a holds the largest
// component (+-1; |u|, |v| < 1 at pixel centres), so the shear of ray_tri
// divides by s = +-1, which is exact: the same values without divisions.
__device__ __forceinline__ float ray_tri_face(float ox, float oy, float oz, float dx, float dy, float dz, int a, float s,
                                              float4 A4, float4 B4, float4 C4) {
    const int kz = a;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (s < 0.f) {
        const int t = kx; kx = ky; ky = t;
    }
    const float sx = s * comp(dx, dy, dz, kx), sy = s * comp(dx, dy, dz, ky), sz = s;
    const float Ax = __fsub_rn(A4.x, ox), Ay = __fsub_rn(A4.y, oy), Az = __fsub_rn(A4.z, oz);
    const float Bx = __fsub_rn(B4.x, ox), By = __fsub_rn(B4.y, oy), Bz = __fsub_rn(B4.z, oz);
    const float Cx = __fsub_rn(C4.x, ox), Cy = __fsub_rn(C4.y, oy), Cz = __fsub_rn(C4.z, oz);
    const float akz = comp(Ax, Ay, Az, kz), bkz = comp(Bx, By, Bz, kz), ckz = comp(Cx, Cy, Cz, kz);
    const float ax = __fmaf_rn(-sx, akz, comp(Ax, Ay, Az, kx)), ay = __fmaf_rn(-sy, akz, comp(Ax, Ay, Az, ky));
    const float bx = __fmaf_rn(-sx, bkz, comp(Bx, By, Bz, kx)), by = __fmaf_rn(-sy, bkz, comp(Bx, By, Bz, ky));
    const float cx = __fmaf_rn(-sx, ckz, comp(Cx, Cy, Cz, kx)), cy = __fmaf_rn(-sy, ckz, comp(Cx, Cy, Cz, ky));
    const float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    const float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    const float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return -1.f;
    const float det = U + V + W;
    if (det == 0.f) return -1.f;
    const float T = U * __fmul_rn(sz, akz) + V * __fmul_rn(sz, bkz) + W * __fmul_rn(sz, ckz);
    const float t = __fdiv_rn(T, det);
    return t > 0.f ? t : -1.f;
}

__global__ void k_rs_raster(RasterBatch B) {
    const int64_t E = (int64_t)B.C * 6 * B.nt;
    const int64_t RR = (int64_t)B.R * B.R;
    // no entry holds more than a face's R x R pixels: a larger total is not a
    // prefix sum of the setup's counts, and the loop below must stay bounded
    const unsigned long long total = B.count[E];
    if (total > (unsigned long long)E * (unsigned long long)RR) return;
    for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (unsigned long long)gridDim.x * blockDim.x) {
        // entry e: the last offset <= g, searched between the hints of the
        // 256-fragment slots around g
        const unsigned long long sl = g >> kSampleShift;
        int64_t lo = 0, hi = E;   // count[lo] <= g < count[hi]
        if ((int64_t)sl + 1 < B.hint_cap) {
            lo = B.hint[sl];
            const unsigned long long nx = (sl + 1) << kSampleShift;
            hi = nx < total ? (int64_t)B.hint[sl + 1] + 1 : E;
            if (lo < 0 || lo >= E || B.count[lo] > g) lo = 0;   // not a valid hint: full range
            if (hi <= lo || hi > E || B.count[hi] <= g) hi = E;
        }
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (B.count[mid] <= g) lo = mid; else hi = mid;
        }
        const int64_t e = lo;
        const unsigned long long local = g - B.count[e], bx = B.box[e];
        const int x0 = (int)(bx & 0xffffull), y0 = (int)((bx >> 16) & 0xffffull), w = (int)(bx >> 32);
        const int px = x0 + (int)(local % (unsigned long long)w), py = y0 + (int)(local / (unsigned long long)w);
        const int k = (int)(e % B.nt);
        const int cf = (int)(e / B.nt);
        const int c = cf / 6, f = cf % 6;
        const int a = f >> 1;
        const float s = (f & 1) ? -1.f : 1.f;
        const float u = pix_center(px, B.R), v = pix_center(py, B.R);
        float d[3];
        d[a] = s; d[(a + 1) % 3] = u; d[(a + 2) % 3] = v;
        const int ci = c / B.K, m = c % B.K;
        const float ox = B.cand[3 * ci] + B.L.ox[m], oy = B.cand[3 * ci + 1] + B.L.oy[m],
                    oz = B.cand[3 * ci + 2] + B.L.oz[m];
        const float4 A4 = __ldg(&B.tri[3 * (size_t)k]), B4 = __ldg(&B.tri[3 * (size_t)k + 1]),
                     C4 = __ldg(&B.tri[3 * (size_t)k + 2]);
        const float t = ray_tri_face(ox, oy, oz, d[0], d[1], d[2], a, s, A4, B4, C4);
        if (t > 0.f) {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(t) << 32) | (unsigned)__float_as_int(A4.w);
            atomicMin(&B.keys[(int64_t)cf * RR + (int64_t)py * B.R + px], key);
        }
    }
}

// Neighbouring pixels mostly see the same triangle: the lanes of a warp that
// add to the same (candidate, triangle) sum their fixed-point powers first
// (lanes grouped with __match_any_sync, the lowest lane adds for the group).
__global__ void k_rs_resolve(RasterBatch B) {
    __shared__ unsigned long long part[8][32];
    const int64_t RR = (int64_t)B.R * B.R;
    const int64_t n = (int64_t)B.C * 6 * RR;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < n; base += nwarps * 32) {
        const int64_t q = base + lane;
        unsigned long long key = q < n ? B.keys[q] : ~0ull;
        long long slot = -1;                  // (candidate, triangle) the lane adds to
        unsigned long long val = 0;
        if (key != ~0ull) {
            const int id = (int)(key & 0xffffffffull);
            const int64_t cf = q / RR;
            const int pix = (int)(q % RR);
            const int px = pix % B.R, py = pix / B.R;
            const int c = (int)(cf / 6), f = (int)(cf % 6);
            const int a = f >> 1;
            const float s = (f & 1) ? -1.f : 1.f;
            float d[3];
            d[a] = s; d[(a + 1) % 3] = pix_center(px, B.R); d[(a + 2) % 3] = pix_center(py, B.R);
            const float* nrm = B.tri_normal + 3 * (size_t)id;
            const float dn = d[0] * nrm[0] + d[1] * nrm[1] + d[2] * nrm[2];
            if (dn < 0.f) {                   // front side; the back side absorbs
                const int ci = c / B.K, m = c % B.K;
                const float pw = __fmul_rn(B.L.pw[m], B.e_unit[pix]);
                val = __float2ull_rn(__fmul_rn(pw, kFixOne));
                slot = (long long)ci * B.nt + id;
            }
        }
        const unsigned group = __match_any_sync(0xffffffffu, slot);
        part[wib][lane] = val;
        __syncwarp();
        if (slot >= 0 && lane == __ffs(group) - 1) {
            unsigned long long sum = 0;
            for (unsigned g = group; g; g &= g - 1) sum += part[wib][__ffs(g) - 1];
            atomicAdd(&B.F[slot], sum);
        }
        __syncwarp();
    }
}

__global__ void k_rs_finish(RasterBatch B, int nb, float* __restrict__ A, int64_t lda) {
    const int64_t n = (int64_t)nb * B.nt;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / B.nt), k = (int)(q % B.nt);
        const float4 a = B.tri[3 * (size_t)k], b = B.tri[3 * (size_t)k + 1], c = B.tri[3 * (size_t)k + 2];
        const int id = __float_as_int(a.w);
        const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z, fx = c.x - a.x, fy = c.y - a.y, fz = c.z - a.z;
        const float cx = ey * fz - ez * fy, cy = ez * fx - ex * fz, cz = ex * fy - ey * fx;
        const float area = 0.5f * sqrtf(cx * cx + cy * cy + cz * cz);
        const float flux = __fmul_rn(__ull2float_rn(B.F[(size_t)i * B.nt + id]), kFixInv);
        A[(size_t)i * lda + id] = area > 0.f ? flux / area : 0.f;
    }
}

// Omega_pixel / (4 pi) for one face (all faces are alike), from the closed
// form of the solid angle of a rectangle on the unit-distance plane:
// Omega = G(u1,v1) - G(u0,v1) - G(u1,v0) + G(u0,v0), G = atan(u v / sqrt(1 + u^2 + v^2)).
const std::vector<float>& pixel_table(int R) {
    static std::mutex mu;
    static std::map<int, std::vector<float>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(R);
    if (it != cache.end()) return it->second;
    std::vector<float> t((size_t)R * R);
    auto G = [](double u, double v) { return std::atan(u * v / std::sqrt(1.0 + u * u + v * v)); };
    for (int py = 0; py < R; ++py) {
        const double v0 = 2.0 * py / R - 1.0, v1 = 2.0 * (py + 1) / R - 1.0;
        for (int px = 0; px < R; ++px) {
            const double u0 = 2.0 * px / R - 1.0, u1 = 2.0 * (px + 1) / R - 1.0;
            t[(size_t)py * R + px] = (float)((G(u1, v1) - G(u0, v1) - G(u1, v0) + G(u0, v0)) / (4.0 * M_PI));
        }
    }
    return cache.emplace(R, std::move(t)).first->second;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Hint slots for a batch of C cubes: fragments are bounded by 8 per pixel on
// average (bounding boxes over-cover; scenes with more depth complexity fall
// back to the full search beyond the slots).
int64_t hint_slots(int64_t C, int R) { return ((C * 6 * (int64_t)R * R * 8) >> kSampleShift) + 2; }

// Workspace layout for nb candidates per batch.
size_t raster_bytes(int64_t nt, int K, int R, int64_t nb) {
    const int64_t C = nb * K, E = C * 6 * nt;
    const int64_t nblk = (E + 1 + kScanBlock * kScanPer - 1) / (kScanBlock * kScanPer);
    return align256(sizeof(int) * (size_t)hint_slots(C, R)) +
           align256(sizeof(unsigned long long) * (size_t)C * 6 * R * R) +
           align256(sizeof(unsigned long long) * (size_t)(E + 1)) + align256(sizeof(unsigned long long) * (size_t)E) +
           align256(sizeof(unsigned long long) * (size_t)(nb * nt)) + align256(sizeof(float) * (size_t)R * R) +
           align256(sizeof(unsigned long long) * (size_t)(nblk + 1)) + 256;
}

}  // namespace

size_t raster_workspace_bytes(int64_t nt, int K, int R, int64_t cand_per_batch) {
    return raster_bytes(nt, K, R, cand_per_batch);
}

int irradiance_raster(const uvc_scene* sc, const float* tri_normal, const float* cand, int64_t nc, const LampDev& L,
                      int R, float* A, int64_t lda, void* work, size_t bytes, cudaStream_t stream) {
    if (nc == 0 || sc->nt == 0) return UVC_OK;
    const int64_t nt = sc->nt;
    int64_t nb = 1;
    if (raster_bytes(nt, L.K, R, 1) > bytes) return UVC_E_INVAL;
    while (nb < nc && raster_bytes(nt, L.K, R, nb * 2) <= bytes) nb *= 2;
    if (nb > nc) nb = nc;
    const std::vector<float>& table = pixel_table(R);
    char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    const int64_t Cmax = nb * L.K, Emax = Cmax * 6 * nt;
    RasterBatch B;
    B.hint = reinterpret_cast<int*>(p);
    B.hint_cap = hint_slots(Cmax, R);
    p += align256(sizeof(int) * (size_t)B.hint_cap);
    B.tri = sc->tri;
    B.order = sc->order;
    B.nt = (int)nt;
    B.R = R;
    B.K = L.K;
    B.L = L;
    B.keys = reinterpret_cast<unsigned long long*>(p);
    p += align256(sizeof(unsigned long long) * (size_t)Cmax * 6 * R * R);
    B.count = reinterpret_cast<unsigned long long*>(p);
    p += align256(sizeof(unsigned long long) * (size_t)(Emax + 1));
    B.box = reinterpret_cast<unsigned long long*>(p);
    p += align256(sizeof(unsigned long long) * (size_t)Emax);
    B.F = reinterpret_cast<unsigned long long*>(p);
    p += align256(sizeof(unsigned long long) * (size_t)(nb * nt));
    float* e_unit = reinterpret_cast<float*>(p);
    p += align256(sizeof(float) * (size_t)R * R);
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(p);
    B.e_unit = e_unit;
    B.tri_normal = tri_normal;
    cudaError_t err = cudaMemcpyAsync(e_unit, table.data(), sizeof(float) * table.size(), cudaMemcpyHostToDevice,
                                      stream);
    if (err != cudaSuccess) return status_from_cuda(err);
    const float near_eps = 1e-6f * fmaxf(sc->diameter, 1e-30f);
    const int grid = sm_count() * 8;
    for (int64_t i0 = 0; i0 < nc; i0 += nb) {
        const int64_t n = std::min<int64_t>(nb, nc - i0);
        B.C = (int)(n * L.K);
        B.cand = cand + 3 * i0;
        const int64_t E = (int64_t)B.C * 6 * nt;
        k_rs_setup<<<(int)((E + 255) / 256), 256, 0, stream>>>(B, near_eps);
        const int64_t nblk = (E + kScanBlock * kScanPer - 1) / (kScanBlock * kScanPer);
        k_scan_blocks<<<(int)nblk, kScanBlock, 0, stream>>>(B.count, E, sums);
        k_scan_sums<<<1, 32, 0, stream>>>(sums, (int)nblk, B.count + E);
        k_scan_add<<<(int)((E + 255) / 256), 256, 0, stream>>>(B.count, E, sums);
        k_rs_hints<<<(int)((E + 255) / 256), 256, 0, stream>>>(B);
        k_fill64<<<grid, 256, 0, stream>>>(B.keys, (int64_t)B.C * 6 * R * R, ~0ull);
        k_fill64<<<grid, 256, 0, stream>>>(B.F, n * nt, 0ull);
        k_rs_raster<<<grid, 256, 0, stream>>>(B);
        k_rs_resolve<<<grid, 256, 0, stream>>>(B);
        k_rs_finish<<<grid, 256, 0, stream>>>(B, (int)n, A + (size_t)i0 * lda, lda);
    }
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
