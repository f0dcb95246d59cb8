// Fluence mu = A^T t (paper Eq. (5)) and the covered-area fraction (the dose
// constraint mu >= mu_min of Eq. (8)).
//
// Fluence: one thread per patch column j; the thread walks its column of A
// (coalesced across the warp) and keeps NV dwell-vector accumulators.  Terms
// are summed in blocks of 32 candidates, and the block sums are added with
// Kahan compensation, so the relative error stays near 34 ulp whatever nc is.
// The dwell times of a candidate chunk sit in shared memory (broadcast reads).
// At nvec = 16 the kernel is bound by the HBM read of A (16 FMA per 4 bytes).
#include <algorithm>

#include "uvc_internal.cuh"

namespace uvc {
namespace {

constexpr int kNV = 16;       // dwell vectors per pass
constexpr int kChunk = 128;   // candidates staged per shared-memory fill

__device__ __forceinline__ void kahan_add(float& sum, float& c, float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

__global__ void __launch_bounds__(256) k_fluence(const float* __restrict__ A, int nc, int64_t lda,
                                                 const float* __restrict__ t, int nvec, int v0,
                                                 float* __restrict__ mu, int np) {
    __shared__ float ts[kNV][kChunk];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = j < np;
    float acc[kNV], comp[kNV];
#pragma unroll
    for (int v = 0; v < kNV; ++v) { acc[v] = 0.f; comp[v] = 0.f; }
    for (int i0 = 0; i0 < nc; i0 += kChunk) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < kNV * kChunk; idx += blockDim.x) {
            int v = idx / kChunk, q = idx % kChunk;
            ts[v][q] = (v0 + v < nvec && i0 + q < nc) ? t[(size_t)(v0 + v) * nc + i0 + q] : 0.f;
        }
        __syncthreads();
        const int nb = min(kChunk, nc - i0);
        const float* col = A + (size_t)i0 * lda + j;
        for (int q0 = 0; q0 < nb; q0 += 32) {
            float part[kNV];
#pragma unroll
            for (int v = 0; v < kNV; ++v) part[v] = 0.f;
            const int qe = min(nb, q0 + 32);
            if (qe - q0 == 32) {
#pragma unroll 8
                for (int q = q0; q < q0 + 32; ++q) {
                    const float a = valid ? __ldg(col + (size_t)q * lda) : 0.f;
#pragma unroll
                    for (int v = 0; v < kNV; ++v) part[v] = __fmaf_rn(ts[v][q], a, part[v]);
                }
            } else {
                for (int q = q0; q < qe; ++q) {
                    const float a = valid ? __ldg(col + (size_t)q * lda) : 0.f;
#pragma unroll
                    for (int v = 0; v < kNV; ++v) part[v] = __fmaf_rn(ts[v][q], a, part[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < kNV; ++v) kahan_add(acc[v], comp[v], part[v]);
        }
    }
    if (!valid) return;
#pragma unroll
    for (int v = 0; v < kNV; ++v)
        if (v0 + v < nvec) mu[(size_t)(v0 + v) * np + j] = acc[v];
}

// Deterministic block sum of (float with Kahan terms, count).
__device__ void block_reduce(float& s, unsigned long long& cnt) {
    __shared__ float ss[32];
    __shared__ unsigned long long sc[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        s = __fadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) { ss[warp] = s; sc[warp] = cnt; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        s = lane < nw ? ss[lane] : 0.f;
        cnt = lane < nw ? sc[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            s = __fadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
            cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        }
    }
}

__global__ void __launch_bounds__(1024) k_area_total(const float4* __restrict__ ps, int np, float* out) {
    float s = 0.f, c = 0.f;
    for (int j = threadIdx.x; j < np; j += blockDim.x) kahan_add(s, c, ps[j].w);
    s = __fsub_rn(s, c);
    unsigned long long n = 0;
    block_reduce(s, n);
    if (threadIdx.x == 0) *out = s;
}

// One block per dwell vector.
__global__ void __launch_bounds__(1024) k_coverage(const float* __restrict__ mu, int np, float mu_min,
                                                   const float4* __restrict__ ps, const float* __restrict__ area_total,
                                                   float* __restrict__ cov_area, float* __restrict__ cov_count) {
    const int v = blockIdx.x;
    const float* m = mu + (size_t)v * np;
    float s = 0.f, c = 0.f;
    unsigned long long n = 0;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        if (m[j] >= mu_min) {
            kahan_add(s, c, ps[j].w);
            ++n;
        }
    }
    s = __fsub_rn(s, c);
    block_reduce(s, n);
    if (threadIdx.x == 0) {
        const float tot = *area_total;
        cov_area[v] = tot > 0.f ? __fdiv_rn(s, tot) : 0.f;
        if (cov_count) cov_count[v] = np > 0 ? __fdiv_rn((float)n, (float)np) : 0.f;
    }
}

}  // namespace

void launch_area_total(const float4* patch_s, int64_t np, float* out, cudaStream_t stream) {
    k_area_total<<<1, 1024, 0, stream>>>(patch_s, (int)np, out);
}

int fluence(const uvc_scene* sc, const float* A, int64_t nc, int64_t lda, const float* t, int32_t nvec,
            float* mu, cudaStream_t stream) {
    const int np = (int)sc->np;
    if (np == 0) return UVC_OK;
    if (nc == 0) return status_from_cuda(cudaMemsetAsync(mu, 0, sizeof(float) * (size_t)nvec * np, stream));
    const int grid = (np + 255) / 256;
    for (int v0 = 0; v0 < nvec; v0 += kNV)
        k_fluence<<<grid, 256, 0, stream>>>(A, (int)nc, lda, t, nvec, v0, mu, np);
    return status_from_cuda(cudaGetLastError());
}

int coverage(const uvc_scene* sc, const float* mu, int32_t nvec, float mu_min, float* cov_area, float* cov_count,
             cudaStream_t stream) {
    k_coverage<<<nvec, 1024, 0, stream>>>(mu, (int)sc->np, mu_min, sc->patch_s, sc->area_total, cov_area,
                                          cov_count);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
