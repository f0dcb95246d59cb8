// Fluence mu = A^T t (paper Eq. (5)) and the covered-area fraction (the dose
// constraint mu >= mu_min of Eq. (8)).
//
// Fluence: each lane owns one patch column j and keeps NV dwell-vector
// accumulators; terms are summed in blocks of 32 candidates and the block sums
// are added with Kahan compensation (relative error near 34 ulp whatever nc
// is).  At nvec = 16 the kernel is bound by the HBM read of A (16 FMA per
// 4 bytes).
#include <algorithm>

#include "uvc_internal.cuh"

namespace uvc {
namespace {

constexpr int kNV = 16;       // dwell vectors per pass

__device__ __forceinline__ void kahan_add(float& sum, float& c, float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

constexpr int kRows = 16;     // candidate rows per pipeline stage
constexpr int kStages = 3;    // stages in flight per warp
constexpr size_t kFluenceSmem = sizeof(float) * kWarpsPerBlock * kStages * kRows * (32 + kNV);

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src, bool pred) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int n = pred ? 4 : 0;   // 0: zero-fill, nothing read
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(gmem_src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One block = 32 patch columns; its 8 warps split the candidates into 8
// contiguous ranges.  Each warp streams its rows of A (one coalesced 128-byte
// segment per row) and the matching dwell times through a kStages-deep ring
// of cp.async copies into shared memory, so that many rows are in flight per
// SM without holding them in registers; each lane then reads its column from
// shared memory.  The 8 warp results are added in a fixed order at the end.
__global__ void __launch_bounds__(256, 2) k_fluence(const float* __restrict__ A, int nc, int64_t lda,
                                                    const float* __restrict__ t, int nvec, int v0,
                                                    float* __restrict__ mu, int np) {
    extern __shared__ float4 fluence_smem[];
    auto abuf = reinterpret_cast<float (*)[kStages][kRows][32]>(fluence_smem);
    auto tbuf = reinterpret_cast<float (*)[kStages][kRows][kNV]>(reinterpret_cast<float*>(fluence_smem) +
                                                                 kWarpsPerBlock * kStages * kRows * 32);
    // after the main loop the row buffers are reused for the cross-warp sums
    auto red = reinterpret_cast<float (*)[kNV][33]>(fluence_smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    const bool valid = j < np;
    const int per = (nc + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int i_begin = min(nc, warp * per), i_end = min(nc, i_begin + per);
    const int nstage = (i_end - i_begin + kRows - 1) / kRows;
    const float* colp = A + (valid ? j : 0);

    // stage k covers rows i_begin + k*kRows ...; lane copies its column of each
    // row, and lanes 0..15 copy the dwell times of the stage's rows
    auto issue = [&](int k) {
        if (k < nstage) {
            const int ib = i_begin + k * kRows;
            const int buf = k % kStages;
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int i = ib + q;
                const bool ok = valid && i < i_end;
                cp_async4(&abuf[warp][buf][q][lane], ok ? colp + (size_t)i * lda : A, ok);
            }
            if (lane < kRows) {
                const int i = ib + lane;
#pragma unroll
                for (int v = 0; v < kNV; ++v) {
                    const bool ok = i < i_end && v0 + v < nvec;
                    cp_async4(&tbuf[warp][buf][lane][v], ok ? t + (size_t)(v0 + v) * nc + i : t, ok);
                }
            }
        }
        cp_async_commit();
    };

    float acc[kNV], comp[kNV], part[kNV];
#pragma unroll
    for (int v = 0; v < kNV; ++v) { acc[v] = 0.f; comp[v] = 0.f; part[v] = 0.f; }
#pragma unroll
    for (int k = 0; k < kStages - 1; ++k) issue(k);
    for (int k = 0; k < nstage; ++k) {
        issue(k + kStages - 1);
        cp_async_wait<kStages - 1>();
        __syncwarp();
        const int buf = k % kStages;
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
            const float a = abuf[warp][buf][q][lane];
            const float4* tq = reinterpret_cast<const float4*>(&tbuf[warp][buf][q][0]);
#pragma unroll
            for (int v4 = 0; v4 < kNV / 4; ++v4) {
                const float4 w = tq[v4];
                part[4 * v4 + 0] = __fmaf_rn(w.x, a, part[4 * v4 + 0]);
                part[4 * v4 + 1] = __fmaf_rn(w.y, a, part[4 * v4 + 1]);
                part[4 * v4 + 2] = __fmaf_rn(w.z, a, part[4 * v4 + 2]);
                part[4 * v4 + 3] = __fmaf_rn(w.w, a, part[4 * v4 + 3]);
            }
        }
        __syncwarp();
        if ((k & 1) || k == nstage - 1) {   // blocks of 32 rows (2 stages) into the compensated sums
#pragma unroll
            for (int v = 0; v < kNV; ++v) {
                kahan_add(acc[v], comp[v], part[v]);
                part[v] = 0.f;
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();   // every warp is done with its row buffers
#pragma unroll
    for (int v = 0; v < kNV; ++v) red[warp][v][lane] = __fsub_rn(acc[v], comp[v]);
    __syncthreads();
    // fixed-order (warp 0..7) compensated sum; thread (v, lane) per output
    for (int idx = threadIdx.x; idx < kNV * 32; idx += blockDim.x) {
        const int v = idx >> 5, l = idx & 31;
        const int jj = blockIdx.x * 32 + l;
        if (jj >= np || v0 + v >= nvec) continue;
        float s = 0.f, c = 0.f;
        for (int w = 0; w < kWarpsPerBlock; ++w) kahan_add(s, c, red[w][v][l]);
        mu[(size_t)(v0 + v) * np + jj] = s;
    }
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
    static_assert(kWarpsPerBlock * kNV * 33 <= kWarpsPerBlock * kStages * kRows * (32 + kNV), "red fits");
    // once per process (and so not during a stream capture that follows a first call)
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_fluence, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFluenceSmem);
    if (attr != cudaSuccess) return status_from_cuda(attr);
    const int grid = (np + 31) / 32;
    for (int v0 = 0; v0 < nvec; v0 += kNV)
        k_fluence<<<grid, kThreads, kFluenceSmem, stream>>>(A, (int)nc, lda, t, nvec, v0, mu, np);
    return status_from_cuda(cudaGetLastError());
}

int coverage(const uvc_scene* sc, const float* mu, int32_t nvec, float mu_min, float* cov_area, float* cov_count,
             cudaStream_t stream) {
    k_coverage<<<nvec, 1024, 0, stream>>>(mu, (int)sc->np, mu_min, sc->patch_s, sc->area_total, cov_area,
                                          cov_count);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
