// Candidate features for the learned candidate proposal: per candidate lamp
// position c, the area-weighted histogram of distances from c to the patch
// points (64 log-spaced bins, 0.1 m to 25 m), the distance from c to the
// nearest triangle, and c's height.  No visibility is involved: the features
// cost one pass over the patches per candidate, a small fraction of the
// occlusion-tested matrix they help to avoid.
#include <cmath>

#include "uvc_internal.cuh"

namespace uvc {
namespace {

constexpr int kBins = 64;
// Probe-column kernels: a block covers 32 columns x 8 row slices; thread
// (slice, column) scans rows slice, slice + 8, ... (coalesced across the 32
// columns), and the 8 slices are combined in shared memory.
constexpr int kColW = 32, kColSlices = 8;
constexpr int kHistThreads = 256;

struct Edges {
    float e[kBins - 1];   // squared bin edges
};

// One block per candidate; each thread keeps its own 64 slots in shared
// memory (no atomics), the slots are then added in a fixed order.
__global__ void __launch_bounds__(kHistThreads) k_feat_hist(const float4* __restrict__ ps, int np,
                                                             const float* __restrict__ area_total,
                                                             const float* __restrict__ cand, Edges E,
                                                             float* __restrict__ feat, int64_t ldf) {
    extern __shared__ float slot[];   // [kBins][kHistThreads]
    __shared__ float edge[kBins - 1];
    const int i = blockIdx.x;
    const int t = threadIdx.x;
    for (int b = t; b < kBins - 1; b += blockDim.x) edge[b] = E.e[b];
    for (int b = 0; b < kBins; ++b) slot[b * kHistThreads + t] = 0.f;
    __syncthreads();
    const float cx = cand[3 * (size_t)i], cy = cand[3 * (size_t)i + 1], cz = cand[3 * (size_t)i + 2];
    for (int j = t; j < np; j += kHistThreads) {
        const float4 s = __ldg(&ps[j]);
        const float dx = s.x - cx, dy = s.y - cy, dz = s.z - cz;
        const float d2 = dx * dx + dy * dy + dz * dz;
        int lo = 0, hi = kBins - 1;   // number of edges <= d2, by bisection
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (edge[mid] <= d2) lo = mid + 1; else hi = mid;
        }
        slot[lo * kHistThreads + t] += s.w;
    }
    __syncthreads();
    const float tot = *area_total;
    for (int b = t; b < kBins; b += blockDim.x) {
        float sum = 0.f;
        for (int q = 0; q < kHistThreads; ++q) sum += slot[b * kHistThreads + q];
        feat[i * ldf + b] = tot > 0.f ? sum / tot : 0.f;
    }
}

// Squared distance from p to triangle abc: the closest point is a vertex, a
// point of an edge or an interior point, decided by the signs of the
// barycentric-style dot products (Voronoi regions of the triangle).
__device__ float point_tri_dist2(float3 p, float3 a, float3 b, float3 c) {
    const float3 ab = make_float3(b.x - a.x, b.y - a.y, b.z - a.z), ac = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
    const float3 ap = make_float3(p.x - a.x, p.y - a.y, p.z - a.z);
    auto dot = [](float3 u, float3 v) { return u.x * v.x + u.y * v.y + u.z * v.z; };
    auto d2of = [&](float3 q) {
        const float x = p.x - q.x, y = p.y - q.y, z = p.z - q.z;
        return x * x + y * y + z * z;
    };
    const float d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) return d2of(a);
    const float3 bp = make_float3(p.x - b.x, p.y - b.y, p.z - b.z);
    const float d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.f && d4 <= d3) return d2of(b);
    const float3 cp = make_float3(p.x - c.x, p.y - c.y, p.z - c.z);
    const float d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.f && d5 <= d6) return d2of(c);
    const float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        const float v = d1 / (d1 - d3);
        return d2of(make_float3(a.x + v * ab.x, a.y + v * ab.y, a.z + v * ab.z));
    }
    const float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        const float w = d2 / (d2 - d6);
        return d2of(make_float3(a.x + w * ac.x, a.y + w * ac.y, a.z + w * ac.z));
    }
    const float va = d3 * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        const float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        return d2of(make_float3(b.x + w * (c.x - b.x), b.y + w * (c.y - b.y), b.z + w * (c.z - b.z)));
    }
    const float den = 1.f / (va + vb + vc);
    const float v = vb * den, w = vc * den;
    return d2of(make_float3(a.x + ab.x * v + ac.x * w, a.y + ab.y * v + ac.y * w, a.z + ab.z * v + ac.z * w));
}

__device__ __forceinline__ float box_d2(float3 p, float lx, float ly, float lz, float hx, float hy, float hz) {
    const float dx = fmaxf(fmaxf(lx - p.x, p.x - hx), 0.f);
    const float dy = fmaxf(fmaxf(ly - p.y, p.y - hy), 0.f);
    const float dz = fmaxf(fmaxf(lz - p.z, p.z - hz), 0.f);
    return dx * dx + dy * dy + dz * dz;
}

// One thread per candidate: nearest-triangle search over the binary tree.
__global__ void k_feat_clear(const Node* __restrict__ nodes, const float4* __restrict__ tri, int nt,
                             const float* __restrict__ cand, int nc, float* __restrict__ feat, int64_t ldf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const float3 p = make_float3(cand[3 * (size_t)i], cand[3 * (size_t)i + 1], cand[3 * (size_t)i + 2]);
    float best = 3.0e38f;
    int stack[128];
    int top = 0;
    if (nt > 1) stack[top++] = 0;
    else if (nt == 1) stack[top++] = ~0;
    int guard = 0;
    while (top > 0 && ++guard < 4 * nt + 64) {
        const int ref = stack[--top];
        if (ref < 0) {
            const int k = ~ref;
            const float4 a = tri[3 * k], b = tri[3 * k + 1], c = tri[3 * k + 2];
            best = fminf(best, point_tri_dist2(p, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                                               make_float3(c.x, c.y, c.z)));
            continue;
        }
        const Node nd = nodes[ref];
        const float dL = box_d2(p, nd.x.x, nd.y.x, nd.z.x, nd.x.z, nd.y.z, nd.z.z);
        const float dR = box_d2(p, nd.x.y, nd.y.y, nd.z.y, nd.x.w, nd.y.w, nd.z.w);
        // never taken: the stack holds at most one pending sibling per level plus
        // the two children just pushed, and candidate_features refuses trees
        // deeper than 126
        if (top + 2 > 128) break;
        const bool lfirst = dL <= dR;
        if ((lfirst ? dR : dL) < best) stack[top++] = lfirst ? nd.r.y : nd.r.x;
        if ((lfirst ? dL : dR) < best) stack[top++] = lfirst ? nd.r.x : nd.r.y;
    }
    feat[i * ldf + kBins] = nt > 0 ? sqrtf(best) : 3.0e38f;
    feat[i * ldf + kBins + 1] = p.z;
}

constexpr int kSelectMax = 16384;
constexpr int kSelectThreads = 1024;

// Order-preserving map of a float score to an unsigned key (NaN lowest).
__device__ __forceinline__ uint32_t score_key(float v) {
    if (v != v) return 0u;
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// The k best of n scores (higher first, ties to the lower index), written in
// ascending index order: a bitonic sort of (inverted key, index) in shared
// memory, a flag per selected index, then a block-wide scan compacts the flags.
__global__ void __launch_bounds__(kSelectThreads) k_select_top(const float* __restrict__ score, int n, int k,
                                                                const float* __restrict__ cand,
                                                                float* __restrict__ out_cand,
                                                                int32_t* __restrict__ out_idx) {
    extern __shared__ unsigned long long key[];   // [m] then flags [n] as bytes
    __shared__ int warp_tot[kSelectThreads / 32];
    int m = 1;
    while (m < n) m <<= 1;
    unsigned char* flag = reinterpret_cast<unsigned char*>(key + m);
    const int t = threadIdx.x;
    for (int i = t; i < m; i += blockDim.x)
        key[i] = i < n ? ((unsigned long long)(~score_key(score[i])) << 32) | (unsigned)i : ~0ull;
    for (int i = t; i < n; i += blockDim.x) flag[i] = 0;
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = t; i < m; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = key[i], b = key[j];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int r = t; r < k; r += blockDim.x) flag[(int)(key[r] & 0xffffffffu)] = 1;
    __syncthreads();
    // each thread owns a run of consecutive indices
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, t * per), hi = min(n, lo + per);
    int cnt = 0;
    for (int i = lo; i < hi; ++i) cnt += flag[i];
    const int lane = t & 31, w = t >> 5;
    int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    int base = 0;
    for (int q = 0; q < w; ++q) base += warp_tot[q];
    int pos = base + inc - cnt;
    for (int i = lo; i < hi; ++i)
        if (flag[i]) {
            if (out_idx) out_idx[pos] = i;
            if (out_cand) {
                out_cand[3 * (size_t)pos] = cand[3 * (size_t)i];
                out_cand[3 * (size_t)pos + 1] = cand[3 * (size_t)i + 1];
                out_cand[3 * (size_t)pos + 2] = cand[3 * (size_t)i + 2];
            }
            ++pos;
        }
}

// Per probe patch j: its area if some candidate lights it (A[i][j] > 0) but
// none of the selected ones does, else 0.
__global__ void k_probe_lost(const float* __restrict__ A, int nc, int64_t lda, int np,
                             const int32_t* __restrict__ idx, int k, const float* __restrict__ area,
                             float* __restrict__ lost) {
    __shared__ unsigned char pf[kColSlices][kColW], pr[kColSlices][kColW];
    const int cx = threadIdx.x % kColW, sl = threadIdx.x / kColW;
    const int j = blockIdx.x * kColW + cx;
    bool full = false, red = false;
    if (j < np) {
        for (int i = sl; i < nc && !full; i += kColSlices) full = A[(int64_t)i * lda + j] > 0.f;
        for (int r = sl; r < k && !red; r += kColSlices) {
            const int i = idx[r];
            if (i >= 0 && i < nc) red = A[(int64_t)i * lda + j] > 0.f;   // rows out of range are ignored
        }
    }
    pf[sl][cx] = full;
    pr[sl][cx] = red;
    __syncthreads();
    if (sl == 0 && j < np) {
        for (int q = 1; q < kColSlices; ++q) {
            full |= pf[q][cx];
            red |= pr[q][cx];
        }
        lost[j] = (full && !red) ? area[j] : 0.f;
    }
}

// out = sum(lost) / sum(area), compensated sums in a fixed order (one block).
__global__ void k_probe_total(const float* __restrict__ lost, const float* __restrict__ area, int np,
                              float* __restrict__ out) {
    __shared__ float sl[256], sa[256];
    float l = 0.f, cl = 0.f, a = 0.f, ca = 0.f;
    for (int j = threadIdx.x; j < np; j += 256) {
        const float yl = lost[j] - cl, tl = l + yl;
        cl = (tl - l) - yl;
        l = tl;
        const float ya = area[j] - ca, ta = a + ya;
        ca = (ta - a) - ya;
        a = ta;
    }
    sl[threadIdx.x] = l;
    sa[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        float L = 0.f, cL = 0.f, S = 0.f, cS = 0.f;
        for (int q = 0; q < 256; ++q) {
            const float yl = sl[q] - cL, tl = L + yl;
            cL = (tl - L) - yl;
            L = tl;
            const float ya = sa[q] - cS, ta = S + ya;
            cS = (ta - S) - ya;
            S = ta;
        }
        *out = S > 0.f ? L / S : 0.f;
    }
}

constexpr int kHardBins = 8, kEffBins = 6, kProbeFeat = kHardBins * kEffBins;
constexpr int kProbeWarps = 4;

// E*_j = max_i A[i][j].
__global__ void k_col_max(const float* __restrict__ A, int nc, int64_t lda, int np, float* __restrict__ emax) {
    __shared__ float part[kColSlices][kColW];
    const int cx = threadIdx.x % kColW, sl = threadIdx.x / kColW;
    const int j = blockIdx.x * kColW + cx;
    float m = 0.f;
    if (j < np)
        for (int i = sl; i < nc; i += kColSlices) m = fmaxf(m, A[(int64_t)i * lda + j]);
    part[sl][cx] = m;
    __syncthreads();
    if (sl == 0 && j < np) {
        for (int q = 1; q < kColSlices; ++q) m = fmaxf(m, part[q][cx]);
        emax[j] = m;
    }
}

// Lit-area-weighted mean of E* (compensated sums, fixed order, one block),
// then each lit patch's hardness bin floor(log2(E*_j / mean)) + 4 clamped to
// [0, 7] (-1 for an unlit patch); stats = (sum a E*, sum a) over lit patches.
__global__ void k_probe_bins(const float* __restrict__ emax, const float* __restrict__ area, int np,
                             float* __restrict__ stats, signed char* __restrict__ hb) {
    __shared__ float s0[256], s1[256];
    __shared__ float mean_sh;
    float a0 = 0.f, c0 = 0.f, a1 = 0.f, c1 = 0.f;
    for (int j = threadIdx.x; j < np; j += 256) {
        const float e = emax[j];
        if (!(e > 0.f)) continue;
        const float y0 = area[j] * e - c0, t0 = a0 + y0;
        c0 = (t0 - a0) - y0;
        a0 = t0;
        const float y1 = area[j] - c1, t1 = a1 + y1;
        c1 = (t1 - a1) - y1;
        a1 = t1;
    }
    s0[threadIdx.x] = a0;
    s1[threadIdx.x] = a1;
    __syncthreads();
    if (threadIdx.x == 0) {
        float A0 = 0.f, C0 = 0.f, A1 = 0.f, C1 = 0.f;
        for (int q = 0; q < 256; ++q) {
            const float y0 = s0[q] - C0, t0 = A0 + y0;
            C0 = (t0 - A0) - y0;
            A0 = t0;
            const float y1 = s1[q] - C1, t1 = A1 + y1;
            C1 = (t1 - A1) - y1;
            A1 = t1;
        }
        stats[0] = A0;
        stats[1] = A1;
        mean_sh = A1 > 0.f ? A0 / A1 : 0.f;
    }
    __syncthreads();
    const float mean = mean_sh;
    for (int j = threadIdx.x; j < np; j += 256) {
        const float e = emax[j];
        if (!(e > 0.f) || !(mean > 0.f)) {
            hb[j] = -1;
            continue;
        }
        int ex;
        frexpf(e / mean, &ex);   // e / mean = f 2^ex, f in [0.5, 1): floor(log2) = ex - 1
        hb[j] = (signed char)min(kHardBins - 1, max(0, ex - 1 + 4));
    }
}

// One warp per candidate: area of the lit probe patches by (hardness bin,
// efficiency bin of A[i][j] / E*_j), over the lit area.  Per-lane slots in
// shared memory, lanes added in a fixed order.
__global__ void __launch_bounds__(kProbeWarps * 32) k_probe_feat(const float* __restrict__ A, int nc, int64_t lda,
                                                                  int np, const float* __restrict__ emax,
                                                                  const signed char* __restrict__ hb,
                                                                  const float* __restrict__ area,
                                                                  const float* __restrict__ stats,
                                                                  float* __restrict__ feat, int64_t ldf) {
    __shared__ float slot[kProbeWarps][kProbeFeat][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kProbeWarps + w;
    if (i >= nc) return;
    for (int b = 0; b < kProbeFeat; ++b) slot[w][b][lane] = 0.f;
    const float* row = A + (int64_t)i * lda;
    for (int j = lane; j < np; j += 32) {
        const int h = hb[j];
        if (h < 0) continue;
        const float e = row[j] / emax[j];
        const int eb = e < 0.5f ? 0 : e < 0.7f ? 1 : e < 0.8f ? 2 : e < 0.9f ? 3 : e < 0.95f ? 4 : 5;
        slot[w][h * kEffBins + eb][lane] += area[j];
    }
    __syncwarp();
    const float lit = stats[1];
    for (int b = lane; b < kProbeFeat; b += 32) {
        float sum = 0.f;
        for (int q = 0; q < 32; ++q) sum += slot[w][b][q];
        feat[(int64_t)i * ldf + b] = lit > 0.f ? sum / lit : 0.f;
    }
}

// For each lit probe patch j, score[argmax_i A[i][j]] = value (the lowest
// index among equal maxima); with rare > 0, also every candidate that lights
// a patch lit by at most `rare` candidates.  Several patches may write the
// same candidate with the same value.
__global__ void k_mark_best(const float* __restrict__ A, int nc, int64_t lda, int np, float* __restrict__ score,
                            float value, int rare) {
    __shared__ float pv[kColSlices][kColW];
    __shared__ int pi[kColSlices][kColW], pn[kColSlices][kColW];
    const int cx = threadIdx.x % kColW, sl = threadIdx.x / kColW;
    const int j = blockIdx.x * kColW + cx;
    float m = 0.f;
    int best = -1, lit = 0;
    if (j < np)
        for (int i = sl; i < nc; i += kColSlices) {
            const float v = A[(int64_t)i * lda + j];
            lit += v > 0.f;
            if (v > m) {        // rows ascend within a slice: the first maximum is kept
                m = v;
                best = i;
            }
        }
    pv[sl][cx] = m;
    pi[sl][cx] = best;
    pn[sl][cx] = lit;
    __syncthreads();
    int total = 0;
    for (int q = 0; q < kColSlices; ++q) total += pn[q][cx];
    if (sl == 0 && j < np) {
        for (int q = 1; q < kColSlices; ++q) {
            const float v = pv[q][cx];
            const int b = pi[q][cx];
            if (b >= 0 && (v > m || (v == m && (best < 0 || b < best)))) {
                m = v;
                best = b;
            }
        }
        if (best >= 0) score[best] = value;
    }
    if (j < np && total > 0 && total <= rare)
        for (int i = sl; i < nc; i += kColSlices)
            if (A[(int64_t)i * lda + j] > 0.f) score[i] = value;
}

// score[winner of each group of `group` consecutive candidates] += bonus;
// the winner is the highest score of the group (lowest index among equals,
// NaN lowest).  One thread per group.
__global__ void k_group_boost(float* __restrict__ score, int n, int group, float bonus) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i0 = g * group;
    if (i0 >= n) return;
    const int i1 = min(n, i0 + group);
    int best = i0;
    uint32_t bk = score_key(score[i0]);
    for (int i = i0 + 1; i < i1; ++i) {
        const uint32_t k = score_key(score[i]);
        if (k > bk) {
            bk = k;
            best = i;
        }
    }
    score[best] = score[best] + bonus;
}

}  // namespace

int group_boost(float* score, int64_t n, int group, float bonus, cudaStream_t stream) {
    const int64_t ng = (n + group - 1) / group;
    if (ng > 0) k_group_boost<<<(int)((ng + 255) / 256), 256, 0, stream>>>(score, (int)n, group, bonus);
    return status_from_cuda(cudaGetLastError());
}

int mark_best(const float* A, int64_t nc, int64_t lda, int64_t np, float* score, float value, int rare,
              cudaStream_t stream) {
    if (np > 0 && nc > 0)
        k_mark_best<<<(int)((np + kColW - 1) / kColW), kColW * kColSlices, 0, stream>>>(A, (int)nc, lda, (int)np,
                                                                                      score, value, rare);
    return status_from_cuda(cudaGetLastError());
}

int probe_features(const float* A, int64_t nc, int64_t lda, int64_t np, const float* area, float* work,
                   float* feat, int64_t ldf, cudaStream_t stream) {
    if (nc == 0) return UVC_OK;
    float* emax = work;
    float* stats = work + np;
    signed char* hb = reinterpret_cast<signed char*>(work + np + 4);
    if (np > 0)
        k_col_max<<<(int)((np + kColW - 1) / kColW), kColW * kColSlices, 0, stream>>>(A, (int)nc, lda, (int)np, emax);
    k_probe_bins<<<1, 256, 0, stream>>>(emax, area, (int)np, stats, hb);
    k_probe_feat<<<(int)((nc + kProbeWarps - 1) / kProbeWarps), kProbeWarps * 32, 0, stream>>>(
        A, (int)nc, lda, (int)np, emax, hb, area, stats, feat, ldf);
    return status_from_cuda(cudaGetLastError());
}

int probe_lost(const float* A, int64_t nc, int64_t lda, int64_t np, const int32_t* idx, int64_t k,
               const float* area, float* lost, float* out, cudaStream_t stream) {
    if (np > 0) {
        k_probe_lost<<<(int)((np + kColW - 1) / kColW), kColW * kColSlices, 0, stream>>>(A, (int)nc, lda, (int)np, idx,
                                                                                       (int)k, area, lost);
    }
    k_probe_total<<<1, 256, 0, stream>>>(lost, area, (int)np, out);
    return status_from_cuda(cudaGetLastError());
}

int select_top(const float* score, int64_t n, int64_t k, const float* cand, float* out_cand, int32_t* out_idx,
               cudaStream_t stream) {
    if (n < 0 || n > kSelectMax || k < 0 || k > n) return UVC_E_INVAL;
    if (k == 0) return UVC_OK;
    int m = 1;
    while (m < n) m <<= 1;
    const size_t smem = sizeof(unsigned long long) * m + (size_t)n;
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_select_top, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kSelectMax + kSelectMax));
    if (attr != cudaSuccess) return status_from_cuda(attr);
    k_select_top<<<1, kSelectThreads, smem, stream>>>(score, (int)n, (int)k, cand, out_cand, out_idx);
    return status_from_cuda(cudaGetLastError());
}

int candidate_features(const uvc_scene* sc, const float* cand, int64_t nc, float* feat, int64_t ldf,
                       cudaStream_t stream) {
    if (nc == 0) return UVC_OK;
    if (sc->depth > 126) return UVC_E_STACK;   // k_feat_clear's fixed stack of 128 entries
    Edges E;
    for (int b = 1; b < kBins; ++b) {
        const double e = 0.1 * std::pow(250.0, (double)b / kBins);
        E.e[b - 1] = (float)(e * e);
    }
    static const cudaError_t attr = cudaFuncSetAttribute(k_feat_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)(sizeof(float) * kBins * kHistThreads));
    if (attr != cudaSuccess) return status_from_cuda(attr);
    k_feat_hist<<<(int)nc, kHistThreads, sizeof(float) * kBins * kHistThreads, stream>>>(
        sc->patch_s, (int)sc->np, sc->area_total, cand, E, feat, ldf);
    k_feat_clear<<<(int)((nc + 127) / 128), 128, 0, stream>>>(sc->nodes, sc->tri, (int)sc->nt, cand, (int)nc, feat,
                                                              ldf);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
