// Fluence mu = A^T t (paper Eq. (5)) and the covered-area fraction (the dose
// constraint mu >= mu_min of Eq. (8)).
//
// Fluence: each thread owns two patch columns of a quarter of the candidate
// rows and keeps NV dwell-vector accumulators per column; terms are summed in
// blocks of 32 candidates and the block sums are added with Kahan
// compensation, the quarters in a fixed order (relative error near 36 ulp
// whatever nc is).  At nvec = 16 the kernel should be bound by the HBM read of
// A (16 FMA per 4 bytes).
#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched through the runtime)

#include <algorithm>
#include <atomic>
#include <mutex>

#include "tcgen05.cuh"
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

// One block = 128 patch columns x all candidates.  Its 256 threads form 4
// row groups of 64 threads; a group takes a contiguous quarter of the
// candidate rows and each of its threads two adjacent columns, read straight
// from global memory as one 8-byte load per row when the row stride allows
// (lda even, A 8-byte aligned), else as two 4-byte loads; a warp reads 256
// contiguous bytes per row.  The dwell times of the group's rows are staged in
// shared memory transposed (row-major, 16 per row), so one 16-byte broadcast
// serves four vectors of both columns, and the 16 products per row and column
// pair run as packed FP32x2 FMAs.  Sums: blocks of 32 rows plain, block sums
// Kahan-compensated, the 4 group results added in a fixed order.
constexpr int kFlGroups = 4;                      // row groups per block
constexpr int kFlGroupThreads = 64;              // threads per row group
constexpr int kFlCols = 2 * kFlGroupThreads;     // columns per block
constexpr int kFlChunk = 128;                     // rows of dwell times staged per group at a time
constexpr int kFlUnroll = 4;                      // rows of A loaded ahead
constexpr size_t kFluenceSmem = sizeof(float) * kFlGroups * kFlChunk * kNV;

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__global__ void __launch_bounds__(256, 2) k_fluence(const float* __restrict__ A, int nc, int64_t lda,
                                                    const float* __restrict__ t, int nvec, int v0,
                                                    float* __restrict__ mu, int np, int vec2) {
    extern __shared__ float4 fluence_smem[];
    const int g = threadIdx.x / kFlGroupThreads, gt = threadIdx.x % kFlGroupThreads;
    float4* ts = fluence_smem + (size_t)g * kFlChunk * (kNV / 4);   // [kFlChunk][kNV / 4]
    const int j0 = blockIdx.x * kFlCols + 2 * gt;
    const bool ok0 = j0 < np, ok1 = j0 + 1 < np;
    const int per = (((nc + kFlGroups - 1) / kFlGroups) + 31) / 32 * 32;   // rows per group, multiple of 32
    const int r0 = min(nc, g * per), r1 = min(nc, r0 + per);
    float2 part[kNV], acc[kNV], comp[kNV];
#pragma unroll
    for (int v = 0; v < kNV; ++v) {
        part[v] = make_float2(0.f, 0.f);
        acc[v] = part[v];
        comp[v] = part[v];
    }
    const int nchunk = (per + kFlChunk - 1) / kFlChunk;   // the same for every group
    for (int ck = 0; ck < nchunk; ++ck) {
        const int c0 = r0 + ck * kFlChunk, c1 = min(r1, c0 + kFlChunk);
        __syncthreads();
        // stage t[v0 + v][c0 .. c1) transposed: ts[row][v]
        float* tsf = reinterpret_cast<float*>(ts);
        for (int e = gt; e < kFlChunk * kNV; e += kFlGroupThreads) {
            const int v = e / kFlChunk, q = e % kFlChunk;
            const int i = c0 + q;
            tsf[q * kNV + v] = (i < c1 && v0 + v < nvec) ? __ldg(&t[(size_t)(v0 + v) * nc + i]) : 0.f;
        }
        __syncthreads();
        for (int q0 = 0; q0 < c1 - c0; q0 += kFlUnroll) {
            float2 a[kFlUnroll];
#pragma unroll
            for (int u = 0; u < kFlUnroll; ++u) {
                const int i = c0 + q0 + u;
                a[u] = make_float2(0.f, 0.f);
                if (i < c1) {
                    const float* row = A + (size_t)i * lda + j0;
                    if (vec2 && ok1) {
                        a[u] = __ldcs(reinterpret_cast<const float2*>(row));
                    } else {
                        if (ok0) a[u].x = __ldcs(row);
                        if (ok1) a[u].y = __ldcs(row + 1);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kFlUnroll; ++u) {
#pragma unroll
                for (int v4 = 0; v4 < kNV / 4; ++v4) {
                    const float4 w = ts[(q0 + u) * (kNV / 4) + v4];   // rows past c1 hold zeros
                    part[4 * v4 + 0] = ffma2(make_float2(w.x, w.x), a[u], part[4 * v4 + 0]);
                    part[4 * v4 + 1] = ffma2(make_float2(w.y, w.y), a[u], part[4 * v4 + 1]);
                    part[4 * v4 + 2] = ffma2(make_float2(w.z, w.z), a[u], part[4 * v4 + 2]);
                    part[4 * v4 + 3] = ffma2(make_float2(w.w, w.w), a[u], part[4 * v4 + 3]);
                }
            }
            if (((q0 + kFlUnroll) & 31) == 0 || q0 + kFlUnroll >= c1 - c0) {   // a block of 32 rows ends
#pragma unroll
                for (int v = 0; v < kNV; ++v) {
                    kahan_add(acc[v].x, comp[v].x, part[v].x);
                    kahan_add(acc[v].y, comp[v].y, part[v].y);
                    part[v] = make_float2(0.f, 0.f);
                }
            }
        }
    }
    // fixed-order (group 0..3) compensated sum of the group results
    __syncthreads();
    float2* red = reinterpret_cast<float2*>(fluence_smem);   // [kFlGroups][kNV][kFlGroupThreads]
#pragma unroll
    for (int v = 0; v < kNV; ++v)
        red[((size_t)g * kNV + v) * kFlGroupThreads + gt] =
            make_float2(__fsub_rn(acc[v].x, comp[v].x), __fsub_rn(acc[v].y, comp[v].y));
    __syncthreads();
    for (int idx = threadIdx.x; idx < kNV * kFlGroupThreads; idx += blockDim.x) {
        const int v = idx / kFlGroupThreads, l = idx % kFlGroupThreads;
        const int jj = blockIdx.x * kFlCols + 2 * l;
        if (v0 + v >= nvec) continue;
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
        for (int w = 0; w < kFlGroups; ++w) {
            const float2 x = red[((size_t)w * kNV + v) * kFlGroupThreads + l];
            kahan_add(s0, c0, x.x);
            kahan_add(s1, c1, x.y);
        }
        if (jj < np) mu[(size_t)(v0 + v) * np + jj] = s0;
        if (jj + 1 < np) mu[(size_t)(v0 + v) * np + jj + 1] = s1;
    }
}

// ---------------------------------------------------------------------------
// Fluence with the rows of A fed by the tensor-memory accelerator
// ---------------------------------------------------------------------------
// The same block shape and summation order as k_fluence (so the same bits),
// but A does not pass through registers: each row group streams its rows
// through a ring of kTmaStages shared-memory tiles of kTmaRows x 128 floats,
// loaded by cp.async.bulk.tensor (one 2-D tensor-map copy per tile, issued by
// the group's first thread) and completed on an mbarrier per tile.  Up to
// 4 groups x kTmaStages tiles = 128 KB per SM are in flight without
// occupying a register, where k_fluence has 16 KB.  The grid is persistent
// (one block per SM, looping over the 128-column strips).  Needs rows that
// start on 16-byte boundaries (lda a multiple of 4, A 16-byte aligned); other
// layouts take k_fluence.  Every wait is bounded: a wait that runs out
// records UVC_E_TIMEOUT in the scene's status word and the block finishes
// without further waiting (its results are then invalid).
constexpr int kTmaRows = 16;                      // rows per tile
constexpr int kTmaStages = 4;                     // tiles in flight per row group
constexpr size_t kTmaTileBytes = sizeof(float) * kTmaRows * kFlCols;
constexpr size_t kTmaSmem = kFlGroups * kTmaStages * kTmaTileBytes   // tiles
                            + kFluenceSmem                          // dwell times (and the group results)
                            + kFlGroups * kTmaStages * sizeof(uint64_t);   // mbarriers
using tc::mbar_arrive;
using tc::mbar_init;
using tc::mbar_wait;
using tc::smem_u32;

__device__ __forceinline__ void tma_load_tile(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"((uint32_t)kTmaTileBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__global__ void __launch_bounds__(256, 1) k_fluence_tma(const __grid_constant__ CUtensorMap amap, int nc,
                                                        const float* __restrict__ t, int nvec, int v0,
                                                        float* __restrict__ mu, int np, int* status) {
    extern __shared__ __align__(128) unsigned char tma_smem[];
    float* tiles = reinterpret_cast<float*>(tma_smem);
    float4* tsbase = reinterpret_cast<float4*>(tma_smem + kFlGroups * kTmaStages * kTmaTileBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tma_smem + kFlGroups * kTmaStages * kTmaTileBytes + kFluenceSmem);
    const int g = threadIdx.x / kFlGroupThreads, gt = threadIdx.x % kFlGroupThreads;
    float4* ts = tsbase + (size_t)g * kFlChunk * (kNV / 4);   // [kFlChunk][kNV / 4]
    float* gtiles = tiles + (size_t)g * kTmaStages * kTmaRows * kFlCols;
    uint64_t* gbar = bars + g * kTmaStages;
    const bool producer = gt == 0;
    if (producer)
        for (int q = 0; q < kTmaStages; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&gbar[q])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const int per = (((nc + kFlGroups - 1) / kFlGroups) + 31) / 32 * 32;
    const int r0 = min(nc, g * per), r1 = min(nc, r0 + per);
    const int nst = (r1 - r0 + kTmaRows - 1) / kTmaRows;   // tiles of this group per strip
    const int nchunk = (per + kFlChunk - 1) / kFlChunk;
    const int nstrip = (np + kFlCols - 1) / kFlCols;
    uint32_t issued = 0, consumed = 0;   // tiles issued / consumed by this group over all strips
    bool ok = true;
    for (int strip = blockIdx.x; strip < nstrip; strip += gridDim.x) {
        const int x0 = strip * kFlCols;
        if (producer) {
            // the slots were last read through the generic proxy (the previous strip)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int k = 0; k < min(kTmaStages, nst); ++k, ++issued)
                tma_load_tile(&amap, &gbar[issued % kTmaStages], gtiles + (size_t)(issued % kTmaStages) * kTmaRows * kFlCols,
                              x0, r0 + k * kTmaRows);
        }
        // accumulators of column c (0, 1) hold the vector pairs (2p, 2p + 1): the
        // dwell times of two vectors are adjacent in a 16-byte broadcast, so
        // each packed FMA takes them as they are and only the A value is paired
        // with itself (same terms, same order as k_fluence for every vector and column)
        float2 part[2][kNV / 2], acc[2][kNV / 2], comp[2][kNV / 2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int p = 0; p < kNV / 2; ++p) {
                part[c][p] = make_float2(0.f, 0.f);
                acc[c][p] = part[c][p];
                comp[c][p] = part[c][p];
            }
        int k = 0;   // tile of this strip
        for (int ck = 0; ck < nchunk; ++ck) {
            const int c0 = r0 + ck * kFlChunk, c1 = min(r1, c0 + kFlChunk);
            asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kFlGroupThreads) : "memory");
            float* tsf = reinterpret_cast<float*>(ts);
            for (int e = gt; e < kFlChunk * kNV; e += kFlGroupThreads) {
                const int v = e / kFlChunk, q = e % kFlChunk;
                const int i = c0 + q;
                tsf[q * kNV + v] = (i < c1 && v0 + v < nvec) ? __ldg(&t[(size_t)(v0 + v) * nc + i]) : 0.f;
            }
            asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kFlGroupThreads) : "memory");
            // the chunk's tiles (a chunk is a whole number of tiles)
            for (int q0 = 0; q0 < c1 - c0; q0 += kTmaRows, ++k) {
                const uint32_t slot = consumed % kTmaStages;
                if (ok && !mbar_wait(&gbar[slot], (consumed / kTmaStages) & 1u)) {
                    ok = false;
                    atomicCAS(status, 0, UVC_E_TIMEOUT);
                }
                const float* tile = gtiles + (size_t)slot * kTmaRows * kFlCols + 2 * gt;
                const int rows = min(kTmaRows, c1 - c0 - q0);
#pragma unroll 4
                for (int u = 0; u < rows; ++u) {
                    const float2 a = *reinterpret_cast<const float2*>(tile + (size_t)u * kFlCols);
                    const float2 a0 = make_float2(a.x, a.x), a1 = make_float2(a.y, a.y);
#pragma unroll
                    for (int v4 = 0; v4 < kNV / 4; ++v4) {
                        const float4 w = ts[(q0 + u) * (kNV / 4) + v4];
                        const float2 w01 = make_float2(w.x, w.y), w23 = make_float2(w.z, w.w);
                        part[0][2 * v4] = __ffma2_rn(w01, a0, part[0][2 * v4]);
                        part[0][2 * v4 + 1] = __ffma2_rn(w23, a0, part[0][2 * v4 + 1]);
                        part[1][2 * v4] = __ffma2_rn(w01, a1, part[1][2 * v4]);
                        part[1][2 * v4 + 1] = __ffma2_rn(w23, a1, part[1][2 * v4 + 1]);
                    }
                    const int q = q0 + u;
                    if (((q + 1) & 31) == 0 || q + 1 == c1 - c0) {   // a block of 32 rows ends
#pragma unroll
                        for (int c = 0; c < 2; ++c)
#pragma unroll
                            for (int p = 0; p < kNV / 2; ++p) {
                                kahan_add(acc[c][p].x, comp[c][p].x, part[c][p].x);
                                kahan_add(acc[c][p].y, comp[c][p].y, part[c][p].y);
                                part[c][p] = make_float2(0.f, 0.f);
                            }
                    }
                }
                ++consumed;
                // every thread of the group is done with the slot: refill it
                asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kFlGroupThreads) : "memory");
                if (producer && k + kTmaStages < nst) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tma_load_tile(&amap, &gbar[issued % kTmaStages],
                                  gtiles + (size_t)(issued % kTmaStages) * kTmaRows * kFlCols, x0,
                                  r0 + (k + kTmaStages) * kTmaRows);
                    ++issued;
                }
            }
        }
        // fixed-order (group 0..3) compensated sum of the group results
        __syncthreads();
        float2* red = reinterpret_cast<float2*>(tsbase);   // [kFlGroups][kNV][kFlGroupThreads]: (col 0, col 1)
#pragma unroll
        for (int p = 0; p < kNV / 2; ++p) {
            red[((size_t)g * kNV + 2 * p) * kFlGroupThreads + gt] =
                make_float2(__fsub_rn(acc[0][p].x, comp[0][p].x), __fsub_rn(acc[1][p].x, comp[1][p].x));
            red[((size_t)g * kNV + 2 * p + 1) * kFlGroupThreads + gt] =
                make_float2(__fsub_rn(acc[0][p].y, comp[0][p].y), __fsub_rn(acc[1][p].y, comp[1][p].y));
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < kNV * kFlGroupThreads; idx += blockDim.x) {
            const int v = idx / kFlGroupThreads, l = idx % kFlGroupThreads;
            const int jj = x0 + 2 * l;
            if (v0 + v >= nvec) continue;
            float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
            for (int w = 0; w < kFlGroups; ++w) {
                const float2 x = red[((size_t)w * kNV + v) * kFlGroupThreads + l];
                kahan_add(s0, c0, x.x);
                kahan_add(s1, c1, x.y);
            }
            if (jj < np) mu[(size_t)(v0 + v) * np + jj] = s0;
            if (jj + 1 < np) mu[(size_t)(v0 + v) * np + jj + 1] = s1;
        }
        __syncthreads();
    }
    // copies still in flight (only after a wait gave up): wait for them, bounded
    if (producer)
        while (consumed < issued) {
            mbar_wait(&gbar[consumed % kTmaStages], (consumed / kTmaStages) & 1u);
            ++consumed;
        }
}

// ---------------------------------------------------------------------------
// Fluence on the tensor cores (tcgen05, TF32 operands split in two)
// ---------------------------------------------------------------------------
// The same product as a matrix multiply on the fifth-generation tensor cores:
// per strip of 128 patches, D (128 patches x 16 vectors, FP32, in tensor
// memory) takes A_strip^T (128 x nc) times t^T (nc x 16).  TF32 keeps 10 of
// FP32's 23 fraction bits, so every operand value x is split as x = hi + lo,
// hi = tf32(x) and lo = tf32(x - hi) (cvt.rna: nearest, ties away), which leaves
// |x - hi - lo| <= 2^-22 |x|; D takes hi*hi + hi*lo + lo*hi + lo*lo, products
// of TF32 values being exact in FP32 (one MMA takes a part of A times both
// parts of t).  Each stage of 32 candidate rows is accumulated from zero into
// one of kTcAccs tensor-memory buffers (128 products per value); the
// converting threads read the stage sum back and add it to per-thread sums
// with Kahan compensation.  The tensor core thus sums within a stage in its
// own order and the stage sums are added in candidate order: the result is
// not bitwise that of k_fluence, and its accuracy is tested against the FP64
// product.
//
// Roles (kTcThreads = 32 (8 kTcGroups + 2)): the first 8 kTcGroups warps form
// kTcGroups converting groups of 8 warps, each an independent pipeline over
// every kTcGroups-th strip of the block (its own tiles of A, operand buffer,
// accumulators and barriers), so that the latency of one group's stage (wait
// for the tile, convert, wait for the MMAs, read the accumulator back)
// overlaps the others' (ward A^T t: one group 0.389 ms, two 0.297, three
// 0.265; four do not fit the shared memory).  A group's threads read the
// stage's tile of A (landed by a tensor-map copy), write the hi / lo operand
// tiles in the tensor core's K-major layout, the same for the stage's dwell
// times, and drain the accumulator of their previous stage.  The next warp's
// lane 0 issues the copies of A for every group; the last warp allocates the
// tensor memory and its lane 0 issues the MMAs of every group in stage order.
// One block per SM (shared memory), persistent over the strips.  Every wait
// is bounded (tc::kSpinCycles); a wait that runs out records UVC_E_TIMEOUT in
// the status word, its thread stops waiting, and the block drains what it
// started before it frees the tensor memory.
constexpr int kTcRows = 32;                       // candidate rows per stage (4 MMA K-steps of 8)
#ifndef UVC_TC_GROUPS
#define UVC_TC_GROUPS 3
#endif
constexpr int kTcGroups = UVC_TC_GROUPS;          // independent converting pipelines per block
constexpr int kTcGroupWarps = 8;
constexpr int kTcGroupThreads = 32 * kTcGroupWarps;
constexpr int kTcSlotsPer = 6 / kTcGroups;       // tiles of A in flight per group
constexpr int kTcConvWarps = kTcGroups * kTcGroupWarps;
constexpr int kTcThreads = 32 * (kTcConvWarps + 2);
constexpr int kTcRowsPer = kTcRows * kFlCols / kTcGroupThreads;   // rows of a stage each converting thread takes
constexpr int kTcDrainCols = kNV * 4 / kTcGroupWarps;             // vectors each converting thread drains
static_assert(kTcRowsPer % 4 == 0 && kTcDrainCols == 8, "converter shape");
constexpr uint32_t kTcTileBytes = sizeof(float) * kTcRows * kFlCols;   // 16 KB
// K-major operand layout without swizzle: 8-row x 16-byte core matrices; for
// one K-step (8 TF32 values) the two core matrices of an 8-row group lie
// kTcLbo apart and consecutive 8-row groups kTcSbo apart.
constexpr uint32_t kTcLbo = 128, kTcSbo = 256;
// The B operand holds t's hi and lo parts as 2 x kNV rows (N = 32), so one MMA
// takes a part of A times both parts of t.
constexpr int kTcN = 2 * kNV;
constexpr uint32_t kTcAStep = (kFlCols / 8) * kTcSbo;   // 4 KB: one K-step of A (128 rows)
constexpr uint32_t kTcBStep = (kTcN / 8) * kTcSbo;      // 1 KB: one K-step of t (32 rows)
constexpr uint32_t kTcAOp = (kTcRows / 8) * kTcAStep;   // 16 KB per stage and part of A
constexpr uint32_t kTcBOp = (kTcRows / 8) * kTcBStep;   // 4 KB per stage
constexpr uint32_t kTcOpBuf = 2 * kTcAOp + kTcBOp;      // hi and lo of A, t
// Per group: kTcSlotsPer tiles of A, one operand buffer, kTcAccs
// tensor-memory accumulators, and its barriers (full / empty per tile;
// opready, mmadone; accfree per accumulator).
constexpr int kTcAccs = 2;
constexpr int kTcBarsPer = 2 * kTcSlotsPer + 2 + kTcAccs;
constexpr int kTcTAhead = 8 / kTcGroups;         // stages of dwell times copied ahead (per group)
constexpr size_t kTcOpsOff = (size_t)kTcGroups * kTcSlotsPer * kTcTileBytes;
constexpr size_t kTcTRingOff = kTcOpsOff + kTcGroups * (size_t)kTcOpBuf;
constexpr size_t kTcTRingBytes = (size_t)kTcGroups * kTcTAhead * 4 * kFlCols * sizeof(float);
constexpr size_t kTcBarOff = kTcTRingOff + kTcTRingBytes;
constexpr size_t kTcSmem = kTcBarOff + (size_t)kTcGroups * kTcBarsPer * sizeof(uint64_t) + 16;
constexpr uint32_t tc_pow2(uint32_t x) { return x <= 32 ? 32 : 2 * tc_pow2((x + 1) / 2); }
constexpr uint32_t kTcTmemCols = tc_pow2(kTcGroups * kTcAccs * kTcN);   // the groups' accumulators (a power of 2 >= 32)

// M = 128 patches, N = both parts of t, TF32 operands, FP32 accumulator
constexpr uint32_t kTcIdesc = tc::idesc_f32acc(tc::kFmtTF32, kFlCols, kTcN);

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tma_load_bytes(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y,
                                               uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Stage (group r, index j) of a block: the group's local strip kTcGroups (j / nst) + r
// (the block's strips alternate between the groups), row tile j % nst.
__device__ __forceinline__ int tc_strip(int r, int j, int nst) {
    return (int)blockIdx.x + (kTcGroups * (j / nst) + r) * (int)gridDim.x;
}

__device__ __forceinline__ void tc_fail(bool& ok, int* fail, int* status) {
    ok = false;
    *fail = 1;
    atomicCAS(status, 0, UVC_E_TIMEOUT);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_fluence_tc(const __grid_constant__ CUtensorMap amap, int nc,
                                                              const float* __restrict__ t, int nvec, int v0,
                                                              float* __restrict__ mu, int np, int* status) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ int fail;
    // per group r: tiles of A [kTcSlotsPer], operand buffer, barriers
    auto slot_of = [&](int r, int s) { return tc_smem + (size_t)(r * kTcSlotsPer + s) * kTcTileBytes; };
    auto ops_of = [&](int r) { return tc_smem + kTcOpsOff + (size_t)r * kTcOpBuf; };
    auto bars_of = [&](int r) { return reinterpret_cast<uint64_t*>(tc_smem + kTcBarOff) + r * kTcBarsPer; };
    // in a group's barriers: full [kTcSlotsPer], empty [kTcSlotsPer], opready, mmadone, accfree [kTcAccs]
    constexpr int kFull = 0, kEmpty = kTcSlotsPer, kOpready = 2 * kTcSlotsPer, kMmadone = kOpready + 1,
                  kAccfree = kMmadone + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_smem + kTcBarOff + (size_t)kTcGroups * kTcBarsPer * 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kProducer = kTcConvWarps, kMma = kTcConvWarps + 1;
    if (threadIdx.x == 0) {
        fail = 0;
        for (int r = 0; r < kTcGroups; ++r) {
            uint64_t* B = bars_of(r);
            for (int q = 0; q < kTcSlotsPer; ++q) {
                mbar_init(&B[kFull + q], 1);
                mbar_init(&B[kEmpty + q], kTcGroupThreads);
            }
            mbar_init(&B[kOpready], kTcGroupThreads);
            mbar_init(&B[kMmadone], 1);
            for (int q = 0; q < kTcAccs; ++q) mbar_init(&B[kAccfree + q], kTcGroupThreads);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMma) {
        tc::alloc(tmem_slot, kTcTmemCols);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nst = (nc + kTcRows - 1) / kTcRows;                // stages per strip
    const int nstrip = (np + kFlCols - 1) / kFlCols;
    const int S = (nstrip - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;   // strips of this block
    int Gr[kTcGroups];                                            // stages of each group
    for (int r = 0; r < kTcGroups; ++r) Gr[r] = (S - r + kTcGroups - 1) / kTcGroups * nst;
    const int Gmax = Gr[0];
    bool ok = true;

    if (warp == kProducer) {
        if (lane == 0)
            for (int j = 0; j < Gmax; ++j)
                for (int r = 0; r < kTcGroups; ++r) {
                    if (j >= Gr[r]) continue;
                    uint64_t* B = bars_of(r);
                    const int s = j % kTcSlotsPer;
                    if (j >= kTcSlotsPer && ok && !mbar_wait(&B[kEmpty + s], ((j / kTcSlotsPer) - 1) & 1u))
                        tc_fail(ok, &fail, status);
                    // the slot was last read through the generic proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tma_load_bytes(&amap, &B[kFull + s], slot_of(r, s), tc_strip(r, j, nst) * kFlCols,
                                   (j % nst) * kTcRows, kTcTileBytes);
                }
    } else if (warp == kMma) {
        if (lane == 0)
            for (int j = 0; j < Gmax; ++j)
                for (int r = 0; r < kTcGroups; ++r) {
                    if (j >= Gr[r]) continue;
                    uint64_t* B = bars_of(r);
                    const int a = j % kTcAccs;
                    if (ok && !mbar_wait(&B[kOpready], j & 1u)) tc_fail(ok, &fail, status);
                    if (j >= kTcAccs && ok && !mbar_wait(&B[kAccfree + a], ((j / kTcAccs) - 1) & 1u))
                        tc_fail(ok, &fail, status);
                    tc::fence_after();
                    const uint32_t ahi = smem_u32(ops_of(r)), alo = ahi + kTcAOp, bt = ahi + 2 * kTcAOp;
                    const uint32_t d = tmem + (uint32_t)((r * kTcAccs + a) * kTcN);
#pragma unroll
                    for (int ks = 0; ks < kTcRows / 8; ++ks) {
                        const uint64_t ah = tc::smem_desc(ahi + ks * kTcAStep, kTcLbo, kTcSbo);
                        const uint64_t al = tc::smem_desc(alo + ks * kTcAStep, kTcLbo, kTcSbo);
                        const uint64_t bd = tc::smem_desc(bt + ks * kTcBStep, kTcLbo, kTcSbo);
                        tc::mma<true>(d, al, bd, kTcIdesc, ks > 0 ? 1u : 0u);   // a stage starts from zero
                        tc::mma<true>(d, ah, bd, kTcIdesc, 1u);
                    }
                    tc::commit(&B[kMmadone]);
                }
    } else {
        const int r = warp / kTcGroupWarps, wl = warp % kTcGroupWarps;   // group, warp in the group
        const int gt = threadIdx.x % kTcGroupThreads;
        const int h = gt / kFlCols, m = gt % kFlCols;             // row part of the stage, patch of the strip
        // dwell values (gt < 128): vector tn, rows tk..tk+3; the 8 lanes of a
        // quarter warp take 8 vectors of one 8-row group (one 128-byte row of stores)
        const int tn = (gt & 7) | (((gt >> 6) & 1) << 3), tk = 4 * ((gt >> 3) & 7);
        const int q = warp & 3, ch = wl >> 2;                     // drain: lane quarter, column group
        uint64_t* B = bars_of(r);
        unsigned char* op = ops_of(r);
        const int G = Gr[r];
        // the thread's 4 dwell values of the next kTcTAhead stages, copied
        // asynchronously into its own slice of a shared ring (cp.async, one
        // group per stage; zero-filled outside t), so that their L2 latency
        // is hidden behind the stages before
        float* tring = reinterpret_cast<float*>(tc_smem + kTcTRingOff) + (size_t)r * kTcTAhead * 4 * kFlCols + 4 * gt;
        auto load_t = [&](int j1) {
            if (gt < kFlCols && j1 < G) {
                const int i0 = (j1 % nst) * kTcRows + tk;
                float* dst = tring + (j1 % kTcTAhead) * (4 * kFlCols);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool in = v0 + tn < nvec && i0 + e < nc;
                    const float* src = in ? &t[(size_t)(v0 + tn) * nc + i0 + e] : t;
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst + e)), "l"(src),
                                 "r"(in ? 4 : 0)
                                 : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        float acc[kTcDrainCols], comp[kTcDrainCols];
#pragma unroll
        for (int c = 0; c < kTcDrainCols; ++c) acc[c] = comp[c] = 0.f;
        for (int j1 = 0; j1 < kTcTAhead; ++j1) load_t(j1);
        for (int j = 0; j <= G; ++j) {
            if (j >= 1) {   // stage j - 1: its MMAs complete frees the operand buffer; drain its accumulator
                const int s = j - 1, a = s % kTcAccs;
                if (ok && !mbar_wait(&B[kMmadone], s & 1u)) tc_fail(ok, &fail, status);
                __syncwarp();
                tc::fence_after();
                float vh[kTcDrainCols], vl[kTcDrainCols];   // the stage's sums against t's hi and lo parts
                tc::load8x2(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((r * kTcAccs + a) * kTcN + kTcDrainCols * ch),
                            kNV, vh, vl);
                tc::fence_before();
                mbar_arrive(&B[kAccfree + a]);
#pragma unroll
                for (int c = 0; c < kTcDrainCols; ++c) kahan_add(acc[c], comp[c], __fadd_rn(vl[c], vh[c]));
                if (s % nst == nst - 1) {   // the strip's last stage: store and restart
                    const int jj = tc_strip(r, s, nst) * kFlCols + 32 * q + lane;
#pragma unroll
                    for (int c = 0; c < kTcDrainCols; ++c) {
                        const int v = v0 + kTcDrainCols * ch + c;
                        if (jj < np && v < nvec) mu[(size_t)v * np + jj] = __fsub_rn(acc[c], comp[c]);
                        acc[c] = comp[c] = 0.f;
                    }
                }
            }
            if (j == G) break;
            const int slot = j % kTcSlotsPer;
            if (ok && !mbar_wait(&B[kFull + slot], (j / kTcSlotsPer) & 1u)) tc_fail(ok, &fail, status);
            const float* tile = reinterpret_cast<const float*>(slot_of(r, slot));
#pragma unroll
            for (int kk = 0; kk < kTcRowsPer / 4; ++kk) {
                const int k0 = kTcRowsPer * h + 4 * kk;
                float a4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) a4[e] = tile[(k0 + e) * kFlCols + m];
                float4 hi, lo;
                hi.x = tf32_rn(a4[0]); lo.x = tf32_rn(__fsub_rn(a4[0], hi.x));
                hi.y = tf32_rn(a4[1]); lo.y = tf32_rn(__fsub_rn(a4[1], hi.y));
                hi.z = tf32_rn(a4[2]); lo.z = tf32_rn(__fsub_rn(a4[2], hi.z));
                hi.w = tf32_rn(a4[3]); lo.w = tf32_rn(__fsub_rn(a4[3], hi.w));
                const uint32_t off = (uint32_t)(k0 >> 3) * kTcAStep + (uint32_t)(m >> 3) * kTcSbo +
                                     (uint32_t)((k0 >> 2) & 1) * kTcLbo + (uint32_t)(m & 7) * 16u;
                *reinterpret_cast<float4*>(op + off) = hi;
                *reinterpret_cast<float4*>(op + kTcAOp + off) = lo;
            }
            if (gt < kFlCols) {
                asm volatile("cp.async.wait_group %0;" ::"n"(kTcTAhead - 1) : "memory");
                float tv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) tv[e] = tring[(j % kTcTAhead) * (4 * kFlCols) + e];
                float4 hi, lo;
                hi.x = tf32_rn(tv[0]); lo.x = tf32_rn(__fsub_rn(tv[0], hi.x));
                hi.y = tf32_rn(tv[1]); lo.y = tf32_rn(__fsub_rn(tv[1], hi.y));
                hi.z = tf32_rn(tv[2]); lo.z = tf32_rn(__fsub_rn(tv[2], hi.z));
                hi.w = tf32_rn(tv[3]); lo.w = tf32_rn(__fsub_rn(tv[3], hi.w));
                // rows tn (hi) and kNV + tn (lo) of the B operand
                const uint32_t off = (uint32_t)(tk >> 3) * kTcBStep + (uint32_t)(tn >> 3) * kTcSbo +
                                     (uint32_t)((tk >> 2) & 1) * kTcLbo + (uint32_t)(tn & 7) * 16u;
                *reinterpret_cast<float4*>(op + 2 * kTcAOp + off) = hi;
                *reinterpret_cast<float4*>(op + 2 * kTcAOp + (kNV / 8) * kTcSbo + off) = lo;
            }
            mbar_arrive(&B[kEmpty + slot]);
            // the operands were written through the generic proxy; the tensor core reads them through the async one
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&B[kOpready]);
            load_t(j + kTcTAhead);   // into the slot just read
        }
    }
    __syncthreads();
    if (fail) {   // only after a wait ran out: let what was started finish (bounded) before the memory goes
        if (warp == kProducer && lane == 0)
            for (int r = 0; r < kTcGroups; ++r)
                for (int j = Gr[r] > kTcSlotsPer ? Gr[r] - kTcSlotsPer : 0; j < Gr[r]; ++j)
                    mbar_wait(&bars_of(r)[kFull + j % kTcSlotsPer], (j / kTcSlotsPer) & 1u);
        if (warp == kMma && lane == 0)
            for (int r = 0; r < kTcGroups; ++r)
                if (Gr[r] > 0) mbar_wait(&bars_of(r)[kMmadone], (Gr[r] - 1) & 1u);
        __syncthreads();
    }
    if (warp == kMma) {
        tc::fence_after();
        tc::dealloc(tmem, kTcTmemCols);
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

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry points (the
// library does not link the driver library itself); nullptr if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        cudaGetLastError();
    });
    return fn;
}

// The tensor map of A (nc rows of lda floats, np used) for `rows` x 128
// tiles; false when the layout does not allow one (rows not 16-byte aligned).
bool fluence_tensor_map(const float* A, int64_t nc, int64_t lda, int np, int rows, CUtensorMap* map) {
    if (lda % 4 != 0 || reinterpret_cast<uintptr_t>(A) % 16 != 0 || np < 1 || nc < 1) return false;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)nc};
    const cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kFlCols, (cuuint32_t)rows};
    const cuuint32_t estride[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

std::atomic<int> g_fluence_tc{1};

int fluence(const uvc_scene* sc, const float* A, int64_t nc, int64_t lda, const float* t, int32_t nvec,
            float* mu, cudaStream_t stream) {
    const int np = (int)sc->np;
    if (np == 0) return UVC_OK;
    if (nc == 0) return status_from_cuda(cudaMemsetAsync(mu, 0, sizeof(float) * (size_t)nvec * np, stream));
    static_assert(sizeof(float2) * kFlGroups * kNV * kFlGroupThreads <= kFluenceSmem, "group results fit");
    static_assert(kFlGroups * kFlGroupThreads == kThreads, "block shape");
    static_assert(kFlChunk % kTmaRows == 0 && kTmaRows * kFlCols * sizeof(float) % 128 == 0, "tile shape");
    CUtensorMap map;
    if (g_fluence_tc.load() && fluence_tensor_map(A, nc, lda, np, kTcRows, &map)) {
        static const cudaError_t cattr =
            cudaFuncSetAttribute(k_fluence_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (cattr != cudaSuccess) return status_from_cuda(cattr);
        const int nstrip = (np + kFlCols - 1) / kFlCols;
        const int grid = std::min(nstrip, sm_count());
        for (int v0 = 0; v0 < nvec; v0 += kNV)
            k_fluence_tc<<<grid, kTcThreads, kTcSmem, stream>>>(map, (int)nc, t, nvec, v0, mu, np, sc->status);
        return status_from_cuda(cudaGetLastError());
    }
    if (fluence_tensor_map(A, nc, lda, np, kTmaRows, &map)) {
        static const cudaError_t tattr =
            cudaFuncSetAttribute(k_fluence_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem);
        if (tattr != cudaSuccess) return status_from_cuda(tattr);
        const int nstrip = (np + kFlCols - 1) / kFlCols;
        const int grid = std::min(nstrip, sm_count());
        for (int v0 = 0; v0 < nvec; v0 += kNV)
            k_fluence_tma<<<grid, kThreads, kTmaSmem, stream>>>(map, (int)nc, t, nvec, v0, mu, np, sc->status);
        return status_from_cuda(cudaGetLastError());
    }
    // once per process (and so not during a stream capture that follows a first call)
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_fluence, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFluenceSmem);
    if (attr != cudaSuccess) return status_from_cuda(attr);
    const int grid = (np + kFlCols - 1) / kFlCols;
    const int vec2 = (lda % 2 == 0) && (reinterpret_cast<uintptr_t>(A) % 8 == 0);
    for (int v0 = 0; v0 < nvec; v0 += kNV)
        k_fluence<<<grid, kThreads, kFluenceSmem, stream>>>(A, (int)nc, lda, t, nvec, v0, mu, np, vec2);
    return status_from_cuda(cudaGetLastError());
}

int coverage(const uvc_scene* sc, const float* mu, int32_t nvec, float mu_min, float* cov_area, float* cov_count,
             cudaStream_t stream) {
    k_coverage<<<nvec, 1024, 0, stream>>>(mu, (int)sc->np, mu_min, sc->patch_s, sc->area_total, cov_area,
                                          cov_count);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
