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
#include <cmath>
#include <mutex>

#include "traverse.cuh"

namespace uvc {
namespace {

// Candidates per warp task: the warp keeps its 32 patches (and its occluder
// cache) over this many consecutive candidates (a tuning constant).  One
// candidate per task measured fastest on the ward (69.6 ms per matrix, against
// 70.2 / 71.5 / 72.2 ms for 3 / 2 / 4): the occluder cache saves less than the
// finer tasks gain, as the warps of a block then take neighbouring candidates
// of the same patches and share their node and triangle loads in L1.
#ifndef UVC_CAND_PER_TASK
#define UVC_CAND_PER_TASK 1
#endif
constexpr int kCandPerTask = UVC_CAND_PER_TASK;

template <bool COUNT, bool WEDGE>
__global__ void __launch_bounds__(kThreads, UVC_IRR_MIN_BLOCKS) k_irradiance(SceneView S, const float* __restrict__ cand, int nc,
                                                         LampDev L, float* __restrict__ A, int64_t lda,
                                                         uint32_t* __restrict__ vis, unsigned long long* ctr) {
    extern __shared__ __align__(16) int smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = smem + warp * S.stack_cap;
    WedgeSmem ws;
    if (WEDGE) ws = wedge_smem(reinterpret_cast<char*>(smem) + stack_smem_bytes(S.stack_cap), L.K, warp);
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
            const float E =
                WEDGE ? irradiance_wedge<COUNT>(S, cand, nc, L, i, jb, lane, stack, ws, vis, njb, P, cache, ctr)
                      : irradiance_entry<COUNT>(S, cand, nc, L, i, jb, lane, stack, vis, njb, P, cache, ctr);
            if (P.valid) A[(size_t)i * lda + j] = E;
        }
    }
}

// Streamed fluence, pass 1: warp task = (candidate chunk s, patch block jb).
// E values of up to kStreamedBlock candidates are staged in shared memory,
// multiplied by the dwell times and added to the chunk's partial sums
// partial[s][v][j].  20 candidates per stage keeps a K = 8 lamp's block within
// a third of an SM's shared memory (three resident blocks).  A task is a whole
// chunk of candidates for 32 patches, and its cost varies with the geometry
// around the patches, so the warps take tasks from a counter (next_task,
// zeroed before the launch) as they finish instead of a fixed share each;
// every task's sums are the same whichever warp takes it.
constexpr int kStreamedBlock = 20;
template <bool WEDGE>
__global__ void __launch_bounds__(kThreads, UVC_STREAMED_MIN_BLOCKS) k_streamed(SceneView S, const float* __restrict__ cand, int nc,
                                                       LampDev L, const float* __restrict__ t, int nvec,
                                                       float* __restrict__ partial, int nsplit, int chunk,
                                                       unsigned long long* next_task) {
    extern __shared__ __align__(16) int smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = smem + warp * S.stack_cap;
    char* after_stacks = reinterpret_cast<char*>(smem) + stack_smem_bytes(S.stack_cap);
    float* Et = reinterpret_cast<float*>(after_stacks) + warp * kStreamedBlock * 32;
    WedgeSmem ws;
    if (WEDGE) ws = wedge_smem(after_stacks + sizeof(float) * kWarpsPerBlock * kStreamedBlock * 32, L.K, warp);
    const int njb = (S.np + 31) >> 5;
    const unsigned long long ntask = (unsigned long long)nsplit * (unsigned long long)njb;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(next_task, 1ull);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk >= ntask) break;
        const int64_t task = (int64_t)tk;
        const int s = (int)(task / njb), jb = (int)(task % njb);
        const int j = jb * 32 + lane;
        const PatchLane P = load_patch(S, j);
        int cache = -1;
        const int i0 = s * chunk, i1 = min(nc, i0 + chunk);
        for (int ib = i0; ib < i1; ib += kStreamedBlock) {
            const int nb = min(kStreamedBlock, i1 - ib);
            for (int q = 0; q < nb; ++q)
                Et[q * 32 + lane] =
                    WEDGE ? irradiance_wedge(S, cand, nc, L, ib + q, jb, lane, stack, ws, nullptr, 0, P, cache)
                          : irradiance_entry(S, cand, nc, L, ib + q, jb, lane, stack, nullptr, 0, P, cache);
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


// Dynamic shared memory above 48 KiB must be opted into per kernel.
int allow_smem(const void* kernel, size_t smem) {
    if (smem <= 48 * 1024) return UVC_OK;
    return status_from_cuda(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
}

// k_streamed for this lamp: shared memory, grid, launch.
size_t streamed_smem(const SceneView& S, const LampDev& lamp) {
    return stack_smem_bytes(S.stack_cap) + sizeof(float) * kWarpsPerBlock * kStreamedBlock * 32 +
           (lamp.wedge ? wedge_smem_bytes(lamp.K) : 0);
}

const void* streamed_kernel(const LampDev& lamp) {
    return lamp.wedge ? (const void*)k_streamed<true> : (const void*)k_streamed<false>;
}

int streamed_grid(const SceneView& S, const LampDev& lamp, int* grid) {
    const int rc = allow_smem(streamed_kernel(lamp), streamed_smem(S, lamp));
    *grid = grid_for(streamed_kernel(lamp), streamed_smem(S, lamp));
    return rc;
}

// next_task: a device counter the launch zeroes first (the warps' task counter).
int launch_streamed(int grid, const SceneView& S, const float* cand, int64_t nc, const LampDev& lamp,
                    const float* t, int32_t nvec, float* partial, int64_t nsplit, int chunk,
                    unsigned long long* next_task, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(next_task, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    const size_t smem = streamed_smem(S, lamp);
    if (lamp.wedge)
        k_streamed<true><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, t, nvec, partial, (int)nsplit,
                                                           chunk, next_task);
    else
        k_streamed<false><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, t, nvec, partial, (int)nsplit,
                                                            chunk, next_task);
    return UVC_OK;
}

template <bool COUNT>
int launch_irradiance(const SceneView& S, const float* cand, int64_t nc, const LampDev& lamp, float* A, int64_t lda,
                      uint32_t* vis, unsigned long long* ctr, cudaStream_t stream) {
    const bool wedge = lamp.wedge != 0;
    const size_t smem = stack_smem_bytes(S.stack_cap) + (wedge ? wedge_smem_bytes(lamp.K) : 0);
    const void* kern = wedge ? (const void*)k_irradiance<COUNT, true> : (const void*)k_irradiance<COUNT, false>;
    int rc = allow_smem(kern, smem);
    if (rc != UVC_OK) return rc;
    const int njb = (S.np + 31) / 32;
    const int64_t ntask = ((nc + kCandPerTask - 1) / kCandPerTask) * njb;
    int grid = grid_for(kern, smem);
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (wedge)
        k_irradiance<COUNT, true><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, A, lda, vis, ctr);
    else
        k_irradiance<COUNT, false><<<grid, kThreads, smem, stream>>>(S, cand, (int)nc, lamp, A, lda, vis, ctr);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace

int irradiance_cand_per_task() { return kCandPerTask; }

int irradiance_matrix(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, float* A,
                      int64_t lda, uint32_t* vis, cudaStream_t stream) {
    if (nc == 0 || sc->np == 0) return UVC_OK;
    return launch_irradiance<false>(view_of(sc), cand, nc, lamp, A, lda, vis, nullptr, stream);
}

int irradiance_counters(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, float* A,
                        int64_t lda, unsigned long long* out6, cudaStream_t stream) {
    for (int k = 0; k < kNumCounters; ++k) out6[k] = 0;
    if (nc == 0 || sc->np == 0) return UVC_OK;
    SceneView S = view_of(sc);
    unsigned long long* dctr = nullptr;
    if (cudaMallocAsync(&dctr, sizeof(unsigned long long) * kNumCounters, stream) != cudaSuccess) {
        cudaGetLastError();
        return UVC_E_NOMEM;
    }
    cudaError_t e = cudaMemsetAsync(dctr, 0, sizeof(unsigned long long) * kNumCounters, stream);
    if (e == cudaSuccess) {
        const int rc = launch_irradiance<true>(S, cand, nc, lamp, A, lda, nullptr, dctr, stream);
        if (rc != UVC_OK) {
            cudaFreeAsync(dctr, stream);
            return rc;
        }
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
    const int njb = (S.np + 31) / 32;
    int grid = 0;
    int rc = streamed_grid(S, lamp, &grid);
    if (rc != UVC_OK) return rc;
    // enough (chunk, block) tasks that every warp of the persistent grid gets
    // some 32 of them: with few, large tasks the last ones leave SMs idle
    const int64_t want = 32 * (int64_t)grid * kWarpsPerBlock;
    int64_t nsplit = (want + njb - 1) / njb;
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, (nc + 31) / 32));
    const int64_t cap = (int64_t(1) << 31) / (4 * (int64_t)nvec * S.np);   // partials <= 2 GiB
    nsplit = std::max<int64_t>(1, std::min(nsplit, cap));
    const int chunk = (int)((nc + nsplit - 1) / nsplit);
    nsplit = (nc + chunk - 1) / chunk;
    // the task counter in the first 256 bytes, the partial sums after it
    char* block = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&block), 256 + sizeof(float) * (size_t)nsplit * nvec * S.np,
                        stream) != cudaSuccess) {
        cudaGetLastError();
        return UVC_E_NOMEM;
    }
    float* partial = reinterpret_cast<float*>(block + 256);
    const int64_t ntask = nsplit * njb;
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    rc = launch_streamed(grid, S, cand, nc, lamp, t, nvec, partial, nsplit, chunk,
                         reinterpret_cast<unsigned long long*>(block), stream);
    cudaError_t e = cudaSuccess;
    if (rc == UVC_OK) {
        const int64_t total = (int64_t)nvec * S.np;
        k_reduce_partials<<<(int)((total + 255) / 256), 256, 0, stream>>>(partial, (int)nsplit, nvec, S.np, mu);
        e = cudaGetLastError();
    }
    cudaFreeAsync(block, stream);
    return rc != UVC_OK ? rc : status_from_cuda(e);
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
constexpr size_t kNoAllocPartialBytes = kNoAllocScratchBytes - 256;   // after the task counter
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float)];

// Device address of g_noalloc_scratch, resolved once per device and context
// (the host-side name of the array is only a stand-in, not a device address).
// The address belongs to the context the module was loaded into: after a
// cudaDeviceReset a later call runs in a new context, where the module is
// loaded again and the array may sit elsewhere, so the cached address is keyed
// on the context's unique id as well as on the device ordinal.
constexpr int kMaxDevices = 64;
struct NoallocSlot {
    unsigned long long ctx_id = 0;
    float* ptr = nullptr;
};
NoallocSlot g_noalloc_slot[kMaxDevices];
std::mutex g_noalloc_mutex;

// Unique id of the calling thread's current context (cuCtxGetCurrent,
// cuCtxGetId through the runtime's driver entry points, so that the library
// does not link the driver library itself); 0 when there is no current
// context yet or the driver lacks the calls.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

int noalloc_scratch(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return UVC_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocSlot& slot = g_noalloc_slot[dev];
    unsigned long long ctx = current_context_id();
    if (!slot.ptr || ctx == 0 || ctx != slot.ctx_id) {
        void* addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) {
            cudaGetLastError();
            return UVC_E_CUDA;
        }
        if (ctx == 0) ctx = current_context_id();   // the lookup made the primary context current
        slot.ptr = static_cast<float*>(addr);
        slot.ctx_id = ctx;
    }
    *out = slot.ptr;
    return UVC_OK;
}

}  // namespace

int fluence_streamed_noalloc(const uvc_scene* sc, const float* cand, int64_t nc, const LampDev& lamp, const float* t,
                             int32_t nvec, float* mu, cudaStream_t stream) {
    if (sc->np == 0) return UVC_OK;
    const size_t per_split = sizeof(float) * (size_t)nvec * (size_t)sc->np;
    if (per_split > kNoAllocPartialBytes) return UVC_E_SCRATCH;
    float* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != UVC_OK) return rc;
    // the task counter in the first 256 bytes, the partial sums after it
    unsigned long long* next_task = reinterpret_cast<unsigned long long*>(scratch);
    float* partial = scratch + 256 / sizeof(float);
    SceneView S = view_of(sc);
    if (nc == 0) return status_from_cuda(cudaMemsetAsync(mu, 0, per_split, stream));
    const int njb = (S.np + 31) / 32;
    int grid = 0;
    rc = streamed_grid(S, lamp, &grid);
    if (rc != UVC_OK) return rc;
    const int64_t want = 8 * (int64_t)grid * kWarpsPerBlock;
    int64_t nsplit = (want + njb - 1) / njb;
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, (nc + 31) / 32));
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, (int64_t)(kNoAllocPartialBytes / per_split)));
    const int chunk = (int)((nc + nsplit - 1) / nsplit);
    nsplit = (nc + chunk - 1) / chunk;
    const int64_t ntask = nsplit * njb;
    if ((int64_t)grid * kWarpsPerBlock > ntask) grid = (int)((ntask + kWarpsPerBlock - 1) / kWarpsPerBlock);
    // every partial is written before it is read, so the array needs no clearing
    rc = launch_streamed(grid, S, cand, nc, lamp, t, nvec, partial, nsplit, chunk, next_task, stream);
    if (rc != UVC_OK) return rc;
    const int64_t total = (int64_t)nvec * S.np;
    k_reduce_partials<<<(int)((total + 255) / 256), 256, 0, stream>>>(partial, (int)nsplit, nvec, S.np, mu);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
