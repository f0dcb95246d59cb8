// Batched irradiance matrices: many (scene, candidates, lamp) jobs - rooms of
// uneven size crossed with lamp designs - in one persistent launch.
//
// The tasks of all jobs (one task = 32 patches x a chunk of candidates, as in
// k_irradiance) form one flat index space, job after job.  A persistent grid
// walks it round-robin, so every warp sees a mix of big and small jobs and
// the launch ends evenly whatever the job sizes.  The job table lives in
// device memory the caller provides; uvc_batch_launch reads no host data and
// allocates nothing, so it can be captured in a CUDA graph and replayed.
// The autotuner times the tunable launch parameters (candidates per task,
// resident blocks per SM) on a sample of the tasks and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "traverse.cuh"

namespace uvc {
namespace {

struct JobDev {
    SceneView S;
    const float* cand;
    float* A;
    uint32_t* vis;
    int64_t lda;
    int64_t task_begin;   // first task of the job in the flat task space
    int nc, lamp, nchunk, njb;
};

// The lamps and job records of a batch of at most kParamLamps lamps and
// kParamJobs jobs travel in the kernel's parameters (constant memory: the
// sources' heights and powers and the job's scene view, read in the inner
// loops, are warp-uniform broadcasts there, and the compiler re-reads them
// instead of holding them in registers); larger batches read them from the
// device tables.
constexpr int kParamLamps = 12;
constexpr int kParamJobs = 192;
struct LampPack {
    LampDev L[kParamLamps];
    JobDev J[kParamJobs];
};
static_assert(sizeof(LampPack) + 64 <= 32764, "kernel parameters");

// Lamps with the wedge path (LampDev::wedge) use the per-source shared
// arrays, sized for the batch's largest such lamp (wedge_k).  MODE: 0 = no
// lamp of the batch takes the wedge path, 1 = all do, 2 = mixed (chosen per
// job; both paths inlined).  PACK: the lamps and jobs come from `pack`.
template <int MODE, bool PACK>
__global__ void __launch_bounds__(kThreads, UVC_IRR_MIN_BLOCKS)
    k_irradiance_batch(const JobDev* __restrict__ jobs, int njobs, const LampDev* __restrict__ lamps,
                       const __grid_constant__ LampPack pack, int cpt, int64_t task_lo, int64_t task_hi,
                       int stack_cap, int wedge_k) {
    extern __shared__ __align__(16) int smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = smem + warp * stack_cap;
    const WedgeSmem ws = wedge_smem(reinterpret_cast<char*>(smem) + stack_smem_bytes(stack_cap), wedge_k, warp);
    const JobDev* jt = PACK ? pack.J : jobs;
    for (int64_t task = task_lo + (int64_t)blockIdx.x * kWarpsPerBlock + warp; task < task_hi;
         task += (int64_t)gridDim.x * kWarpsPerBlock) {
        int lo = 0, hi = njobs - 1;   // last job starting at or before `task`
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jt[mid].task_begin <= task) lo = mid; else hi = mid - 1;
        }
        const JobDev& J = jt[lo];
        const int64_t local = task - J.task_begin;
        const int jb = (int)(local / J.nchunk), ic = (int)(local % J.nchunk);
        const int j = jb * 32 + lane;
        const PatchLane P = load_patch(J.S, j);
        int cache = -1;
        const int i1 = min(J.nc, (ic + 1) * cpt);
        const LampDev& L = PACK ? pack.L[J.lamp] : lamps[J.lamp];
        for (int i = ic * cpt; i < i1; ++i) {
            const bool wedge = MODE == 1 || (MODE == 2 && L.wedge);
            const float E = wedge ? irradiance_wedge<false>(J.S, J.cand, J.nc, L, i, jb, lane, stack, ws, J.vis,
                                                            J.njb, P, cache)
                                  : irradiance_entry<false>(J.S, J.cand, J.nc, L, i, jb, lane, stack, J.vis,
                                                            J.njb, P, cache);
            if (P.valid) J.A[(size_t)i * J.lda + j] = E;
        }
    }
}

using BatchKernel = void (*)(const JobDev*, int, const LampDev*, const LampPack, int, int64_t, int64_t, int, int);

template <bool PACK>
BatchKernel kernel_for_pack(int mode) {
    return mode == 0 ? k_irradiance_batch<0, PACK> : (mode == 1 ? k_irradiance_batch<1, PACK> : k_irradiance_batch<2, PACK>);
}

BatchKernel kernel_for(int mode, bool pack) { return pack ? kernel_for_pack<true>(mode) : kernel_for_pack<false>(mode); }

bool valid_cpt(int c) { return c == 1 || c == 2 || c == 4 || c == 8 || c == 16; }

}  // namespace
}  // namespace uvc

struct uvc_batch {
    int device = 0;
    int njobs = 0, nlamps = 0;
    std::vector<uvc::JobDev> host_jobs;   // task_begin filled per config
    std::vector<int64_t> pairs;           // nc * np per job
    std::vector<uvc::LampDev> host_lamps;
    uvc::JobDev* dev_jobs = nullptr;      // in the caller's workspace
    uvc::LampDev* dev_lamps = nullptr;
    int stack_cap = 1;
    int wedge_k = 0;                      // largest K among the lamps with the wedge path
    int mode = 0;                         // kernel variant: 0 no wedge lamp, 1 all wedge, 2 mixed
    int64_t total_pairs = 0;
    uvc::LampPack pack{};                 // the lamps and jobs again, for the kernel parameters (small batches)
    int uploaded_cpt = 0;                 // cand_per_task of the uploaded table
    uvc_batch_config tuned{8, 0};        // configuration used by uvc_batch_launch
};

namespace uvc {
namespace {

int64_t fill_task_begin(uvc_batch* b, int cpt) {
    int64_t t = 0;
    for (auto& J : b->host_jobs) {
        J.nchunk = (J.nc + cpt - 1) / cpt;
        J.task_begin = t;
        t += (int64_t)J.nchunk * J.njb;
    }
    return t;
}

int upload(uvc_batch* b, int cpt, cudaStream_t stream, int64_t* total_tasks) {
    *total_tasks = fill_task_begin(b, cpt);
    if (b->njobs <= kParamJobs) std::copy(b->host_jobs.begin(), b->host_jobs.end(), b->pack.J);
    if (b->uploaded_cpt == cpt) return UVC_OK;
    cudaError_t e = cudaMemcpyAsync(b->dev_jobs, b->host_jobs.data(), sizeof(JobDev) * b->njobs,
                                    cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // host table is reused for the next config
    if (e != cudaSuccess) return status_from_cuda(e);
    b->uploaded_cpt = cpt;
    return UVC_OK;
}

int launch_range(const uvc_batch* b, int cpt, int blocks_per_sm, int64_t lo, int64_t hi, cudaStream_t stream) {
    if (hi <= lo) return UVC_OK;
    const bool pack = b->nlamps <= kParamLamps && b->njobs <= kParamJobs;
    BatchKernel k = kernel_for(b->mode, pack);
    const size_t smem = stack_smem_bytes(b->stack_cap) + wedge_smem_bytes(b->wedge_k);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return status_from_cuda(e);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
    int64_t grid = (int64_t)per_sm * sm_count();
    const int64_t warps_needed = (hi - lo + kWarpsPerBlock - 1) / kWarpsPerBlock;
    grid = std::max<int64_t>(1, std::min(grid, warps_needed));
    k<<<(int)grid, kThreads, smem, stream>>>(b->dev_jobs, b->njobs, b->dev_lamps, b->pack, cpt, lo, hi, b->stack_cap,
                                             b->wedge_k);
    return status_from_cuda(cudaGetLastError());
}

// size bucket of a batch for the tuning cache: log2 of its pairs and of its mean sources
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, uvc_batch_config> g_tune_cache;

std::tuple<int, int, int> bucket_of(const uvc_batch* b) {
    double k = 0;
    for (const auto& L : b->host_lamps) k += L.K;
    k /= std::max(1, b->nlamps);
    int dev = 0;
    cudaGetDevice(&dev);
    return {(int)std::log2((double)std::max<int64_t>(1, b->total_pairs)), (int)std::lround(std::log2(k + 1.0)), dev};
}

}  // namespace
}  // namespace uvc

extern "C" {

size_t uvc_batch_workspace_bytes(int32_t njobs, int32_t nlamps) {
    if (njobs < 0 || nlamps < 0) return 0;
    const size_t a = (sizeof(uvc::JobDev) * (size_t)njobs + 255) & ~size_t(255);
    return a + sizeof(uvc::LampDev) * (size_t)nlamps + 256;
}

int uvc_batch_create(const uvc_job* jobs, int32_t njobs, const uvc_lamp* lamps, int32_t nlamps, void* workspace,
                     size_t workspace_bytes, uvc_stream_t stream, uvc_batch** out) {
    if (!out) return UVC_E_INVAL;
    *out = nullptr;
    if (njobs < 1 || nlamps < 1 || !jobs || !lamps || !workspace) return UVC_E_INVAL;
    if (workspace_bytes < uvc_batch_workspace_bytes(njobs, nlamps) || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return UVC_E_INVAL;
    uvc_batch* b = new (std::nothrow) uvc_batch();
    if (!b) return UVC_E_NOMEM;
    cudaGetDevice(&b->device);
    b->njobs = njobs;
    b->nlamps = nlamps;
    b->host_lamps.resize(nlamps);
    float coord_bound = 0.f;   // over every job's scene (a lamp may serve several)
    int64_t max_tris = 0;
    for (int q = 0; q < njobs; ++q)
        if (jobs[q].scene) {
            coord_bound = std::max(coord_bound, jobs[q].scene->coord_bound);
            max_tris = std::max(max_tris, jobs[q].scene->nt);
        }
    for (int l = 0; l < nlamps; ++l) {
        uvc::LampDev& D = b->host_lamps[l];
        if (uvc::lamp_to_device(&lamps[l], &D, coord_bound, max_tris) != UVC_OK) { delete b; return UVC_E_INVAL; }
        if (D.wedge) b->wedge_k = std::max(b->wedge_k, D.K);
        if (l < uvc::kParamLamps) b->pack.L[l] = D;
    }
    int nwedge = 0;
    for (const auto& D : b->host_lamps) nwedge += D.wedge ? 1 : 0;
    b->mode = nwedge == 0 ? 0 : (nwedge == nlamps ? 1 : 2);
    b->host_jobs.resize(njobs);
    b->pairs.resize(njobs);
    int maxcap = 1;
    for (int q = 0; q < njobs; ++q) {
        const uvc_job& J = jobs[q];
        const int64_t lim = int64_t(1) << 31;
        if (!J.scene || J.nc < 0 || J.nc >= lim || J.lamp < 0 || J.lamp >= nlamps || J.lda < J.scene->np ||
            (J.nc > 0 && J.scene->np > 0 && (!J.cand || !J.A))) {
            delete b;
            return UVC_E_INVAL;
        }
        uvc::JobDev& D = b->host_jobs[q];
        D.S = uvc::view_of(J.scene);
        D.cand = J.cand;
        D.A = J.A;
        D.vis = J.vis;
        D.lda = J.lda;
        D.nc = (int)J.nc;
        D.lamp = J.lamp;
        D.njb = (int)((J.scene->np + 31) / 32);
        if (J.nc == 0) D.njb = 0;   // nothing to do for this job
        b->pairs[q] = J.nc * J.scene->np;
        b->total_pairs += b->pairs[q];
        maxcap = std::max(maxcap, D.S.stack_cap);
    }
    b->stack_cap = maxcap;
    char* ws = static_cast<char*>(workspace);
    b->dev_jobs = reinterpret_cast<uvc::JobDev*>(ws);
    b->dev_lamps = reinterpret_cast<uvc::LampDev*>(ws + ((sizeof(uvc::JobDev) * (size_t)njobs + 255) & ~size_t(255)));
    cudaError_t e = cudaMemcpyAsync(b->dev_lamps, b->host_lamps.data(), sizeof(uvc::LampDev) * nlamps,
                                    cudaMemcpyHostToDevice, (cudaStream_t)stream);
    int64_t tasks = 0;
    int rc = e == cudaSuccess ? uvc::upload(b, 8, (cudaStream_t)stream, &tasks) : uvc::status_from_cuda(e);
    if (rc != UVC_OK) { delete b; return rc; }
    *out = b;
    return UVC_OK;
}

int uvc_batch_free(uvc_batch* b) {
    delete b;
    return UVC_OK;
}

int uvc_batch_launch(uvc_batch* b, uvc_stream_t stream) {
    if (!b) return UVC_E_INVAL;
    const int cpt = b->uploaded_cpt;
    const int64_t total = uvc::fill_task_begin(b, cpt);
    return uvc::launch_range(b, cpt, b->tuned.blocks_per_sm, 0, total, (cudaStream_t)stream);
}

int uvc_batch_set_config(uvc_batch* b, const uvc_batch_config* cfg, uvc_stream_t stream) {
    if (!b || !cfg || !uvc::valid_cpt(cfg->cand_per_task) || cfg->blocks_per_sm < 0) return UVC_E_INVAL;
    int64_t tasks = 0;
    int rc = uvc::upload(b, cfg->cand_per_task, (cudaStream_t)stream, &tasks);
    if (rc == UVC_OK) b->tuned = *cfg;
    return rc;
}

int uvc_batch_autotune(uvc_batch* b, double sample_fraction, uvc_batch_config* out, uvc_stream_t stream) {
    if (!b || !out || !(sample_fraction > 0.0) || sample_fraction > 1.0) return UVC_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    {
        std::lock_guard<std::mutex> lock(uvc::g_tune_mutex);
        auto it = uvc::g_tune_cache.find(uvc::bucket_of(b));
        if (it != uvc::g_tune_cache.end()) {
            *out = it->second;
            return uvc_batch_set_config(b, out, stream);
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return UVC_E_CUDA;
    }
    const int cpts[] = {1, 4, 16};
    const int bpss[] = {2, 3};
    float best_ms_per_pair = 3.0e38f;
    uvc_batch_config best{8, 0};
    int rc = UVC_OK;
    for (int cpt : cpts) {
        int64_t total = 0;
        rc = uvc::upload(b, cpt, s, &total);
        if (rc != UVC_OK) break;
        // the sample: a stretch of tasks from the middle of the task space
        const int64_t n = std::max<int64_t>(1, (int64_t)(sample_fraction * (double)total));
        const int64_t lo = std::max<int64_t>(0, total / 2 - n / 2), hi = std::min(total, lo + n);
        for (int bps : bpss) {
            rc = uvc::launch_range(b, cpt, bps, lo, hi, s);   // warm-up
            if (rc != UVC_OK) break;
            cudaEventRecord(e0, s);
            rc = uvc::launch_range(b, cpt, bps, lo, hi, s);
            cudaEventRecord(e1, s);
            if (rc != UVC_OK || cudaEventSynchronize(e1) != cudaSuccess) { rc = rc ? rc : UVC_E_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const float per_task = ms / (float)(hi - lo) / (float)cpt;   // per (task x candidate)
            if (per_task < best_ms_per_pair) {
                best_ms_per_pair = per_task;
                best = uvc_batch_config{cpt, bps};
            }
        }
        if (rc != UVC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != UVC_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(uvc::g_tune_mutex);
        uvc::g_tune_cache[uvc::bucket_of(b)] = best;
    }
    *out = best;
    return uvc_batch_set_config(b, &best, stream);
}

int uvc_batch_info(const uvc_batch* b, int64_t* total_pairs, int32_t* stack_cap, uvc_batch_config* tuned) {
    if (!b) return UVC_E_INVAL;
    if (total_pairs) *total_pairs = b->total_pairs;
    if (stack_cap) *stack_cap = b->stack_cap;
    if (tuned) *tuned = b->tuned;
    return UVC_OK;
}

}  // extern "C"
