/*
 * uvc.h - C ABI of the GB300 irradiance-matrix library (libuvc.so).
 *
 * The library computes the discrete irradiance matrix of the UV coverage
 * planner of Correia Marques, Ramalingam, Pan and Hauser, "Optimized
 * Coverage Planning for UV Surface Disinfection" (arXiv:2103.14137): for
 * candidate lamp positions x_i and
 * surface patches j, the irradiance I_j(x_i) of Eq. (4), evaluated by the
 * inverse-square law of Eq. (7) with its visibility rule, summed over the
 * point sources of a lamp (Sec. IV-C, "Non-Point Light Sources"); the fluence
 * mu_j(t) = sum_i I_j(x_i) t_i of Eq. (5); and the covered surface fraction
 * (the area with mu_j >= mu_min, the constraint of Eq. (8)).
 *
 * Conventions shared by every call
 *   - All array arguments are DEVICE pointers (CUDA global memory of the
 *     current device), C-contiguous, owned by the caller.  The library never
 *     writes an input, never frees a caller buffer and keeps no pointer to a
 *     caller buffer after the call returns (uvc_build_scene copies what it
 *     needs).
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and runs asynchronously; results are valid once the stream has
 *     reached that point.  Argument checks happen synchronously on the host.
 *     uvc_build_scene additionally synchronises `stream` once (it reads the
 *     tree depth and its validation result back to the host).
 *   - Every call returns a status code (UVC_OK = 0).  No C++ exception crosses
 *     the ABI.  Device-side failures (a traversal that exceeded its visit cap)
 *     are recorded in the scene's status word; uvc_scene_status reads it.
 *   - Sizes are int64_t; every count must be >= 0 and < 2^31.
 *   - The GPU path uses FP32 (with error-free transformations where needed);
 *     it contains no FP64 arithmetic and has no CPU fallback.
 */
#ifndef UVC_H
#define UVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* uvc_stream_t; /* same type as cudaStream_t */

/* status codes */
#define UVC_OK 0
#define UVC_E_INVAL 1    /* bad argument: NULL, negative/oversized count, bad index, NaN */
#define UVC_E_NOMEM 2    /* device allocation failed */
#define UVC_E_CUDA 3     /* a CUDA runtime call failed (launch, copy, sync) */
#define UVC_E_STACK 4    /* traversal stack would overflow (tree deeper than supported) */
#define UVC_E_TIMEOUT 5  /* a traversal hit its node-visit cap; affected entries are NaN */
#define UVC_E_SCRATCH 6  /* nvec*np too large for uvc_fluence_streamed_noalloc's fixed scratch */
#define UVC_E_BOUNDS 7   /* checked build only: a traversal met an index out of range (entries NaN) */

#define UVC_MAX_SOURCES 32

/*
 * A lamp as K point sources (Sec. IV-C, "Non-Point Light Sources": a light
 * of any shape is approximated by point sources, each emitting a fraction of
 * the total radiant flux).  Source m of a lamp placed at candidate point c
 * sits at fl32(c + offsets[m]) (one FP32 add per coordinate) and emits
 * weight[m] * power watts.  A point lamp is K = 1, offsets = 0, weight = 1.
 * Host struct, passed by pointer, read during the call only.
 */
typedef struct {
    int32_t K;                            /* 1 <= K <= UVC_MAX_SOURCES */
    float power;                          /* total radiant flux P in watts, finite, >= 0 */
    float offsets[UVC_MAX_SOURCES][3];    /* metres, first K used */
    float weight[UVC_MAX_SOURCES];        /* fractions of P, first K used, finite, >= 0 */
} uvc_lamp;

/*
 * Surface patches (Sec. III-B: the surface is a simplicial complex; each
 * irradiance entry integrates over one patch, Eq. (4)).  The library samples
 * each patch at one point.  Device pointers, np entries each:
 *   centroid  float[np][3]  sample point s_j (metres)
 *   normal    float[np][3]  unit normal n_j pointing INTO the free space
 *   area      float[np]     patch area (m^2), used by uvc_coverage
 *   excl      int32[np][2]  triangles the patch lies on; they never occlude
 *                           their own patch (-1 = unused slot)
 */
typedef struct {
    const float* centroid;
    const float* normal;
    const float* area;
    const int32_t* excl;
} uvc_patches;

typedef struct uvc_scene uvc_scene; /* opaque; owns its device buffers */

/*
 * uvc_build_scene - upload the environment and build its bounding-volume
 * hierarchy (a linear BVH: Morton codes, radix sort, binary radix tree,
 * bottom-up box refit; then a surface-area restructuring pass, see
 * uvc_build_scene_ex).  The paper's environment boundary E is the triangle
 * mesh of Sec. III-B; the hierarchy replaces the paper's rasterised visibility
 * cube (Sec. IV-C, Fig. 2) as the means of answering "does another surface
 * lie closer to the source along the ray" (the visibility rule of Eq. (7)).
 *
 *   verts  float[nv][3] vertex positions (metres), finite
 *   tris   int32[nt][3] vertex indices, each in [0, nv)
 *   patches, np         see uvc_patches; excl entries in [-1, nt)
 *   out                 receives the new scene (freed with uvc_free_scene)
 *
 * All geometry is FP32, and the tolerances of the searches scale with the
 * scene's size D (the diagonal of its bounding box: box widening and
 * clearance slack 1e-5 D, coplanar margin 2^-14 D): they assume coordinates of
 * the order of D, where FP32 resolves 2^-24 |x|.  A scene far from the origin (|x| >> D) should be
 * translated near it, with its candidates, before upload; the library does
 * not move it.
 *
 * nt may be 0 (nothing occludes).  Returns UVC_E_INVAL for NULL pointers,
 * counts out of range, an index out of range or a non-finite coordinate
 * (checked on the device, then reported after one stream synchronisation),
 * UVC_E_NOMEM when device memory runs out.  On error *out is NULL.
 */
int uvc_build_scene(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                    const uvc_patches* patches, int64_t np, uvc_stream_t stream, uvc_scene** out);

/*
 * uvc_build_scene_ex - uvc_build_scene with build options (bit flags):
 *   UVC_BUILD_LBVH_ONLY  keep the plain linear BVH (Morton order + radix tree +
 *                        refit).  Without it, the hierarchy is additionally
 *                        restructured for lower surface-area cost (treelets of
 *                        up to 7 leaves re-wired optimally, bottom-up, one
 *                        pass): the same triangles under the same root, a
 *                        different topology, the same query results, fewer
 *                        nodes visited per query.
 * uvc_build_scene(...) equals uvc_build_scene_ex(..., 0, ...).  Unknown flags:
 * UVC_E_INVAL.
 */
#define UVC_BUILD_LBVH_ONLY 1u
int uvc_build_scene_ex(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const uvc_patches* patches,
                       int64_t np, uint32_t flags, uvc_stream_t stream, uvc_scene** out);

/* uvc_free_scene - release a scene's device buffers (synchronises the device
 * work that may still use them).  NULL is accepted. */
int uvc_free_scene(uvc_scene* scene);

/*
 * uvc_set_fluence_tensor_cores - which kernel uvc_fluence uses for A^T t
 * (Eq. (5)) where the rows of A start on 16-byte boundaries: 1 (the default)
 * the tensor cores (tcgen05 MMAs on split TF32 operands, accumulators in
 * tensor memory), 0 the CUDA cores (FP32 FMAs).  Not in the paper.  Process-
 * wide; read when uvc_fluence enqueues its launch.
 *   enable    0 or 1
 *   previous  HOST int32, may be NULL: receives the setting before the call
 * Returns UVC_OK, or UVC_E_INVAL (setting unchanged) for other values of enable.
 */
int uvc_set_fluence_tensor_cores(int32_t enable, int32_t* previous);

/*
 * uvc_set_wedge_traversal - how the K sources of a vertical line lamp are
 * searched (process-wide; default 1).  Sec. IV-C ("Non-Point Light Sources")
 * approximates a line light by point sources evenly spread along it; when
 * every offset of a lamp is vertical (x = y = 0) and 2 <= K <= 16, all
 * sources of a candidate lie on one vertical line, so the K segments to a
 * patch point lie in one triangle (the wedge).  With 1, the matrix, streamed
 * and batched calls search that wedge once per (candidate, patch) and test
 * each triangle it reaches against every source still searching; with 0,
 * every source is searched on its own.  Both give the visibility of Eq. (7)
 * source by source with the same segment test; they can differ only where a
 * segment grazes a triangle lying in the patch's own plane.  Scenes of more
 * than 2^27 triangles are always searched source by source.  The setting is
 * read when a call (or uvc_batch_create) converts its lamp.
 *   enable    0 or 1
 *   previous  HOST int32, may be NULL: receives the setting before the call
 * Returns UVC_OK, or UVC_E_INVAL (setting unchanged) for other values of enable.
 */
int uvc_set_wedge_traversal(int32_t enable, int32_t* previous);

/*
 * uvc_irradiance_matrix - the irradiance matrix (Sec. IV-C, Eq. (4) and (7)):
 *
 *   A[i][j] = sum_m  w_m P <o_im - s_j, n_j> / (4 pi |o_im - s_j|^3) * V_ijm
 *
 * with o_im = fl32(cand_i + offsets_m), and V_ijm = 1 iff <o_im - s_j, n_j> > 0
 * and no triangle other than the patch's excl triangles meets the open
 * segment between o_im and s_j (watertight FP32 segment/triangle test).
 * The paper prints the two cases of Eq. (7) the other way round; the formula
 * applies to visible patches.  The matrix is the transpose of the paper's
 * I_j(x_i): one row per candidate.
 *
 *   cand  float[nc][3]  candidate lamp positions (the lamp's reference point)
 *   lamp  host struct   K sources, see uvc_lamp
 *   A     float[nc][lda], lda >= np; row i, columns [0, np) are written,
 *         columns >= np untouched
 *   vis   uint32[K][nc][ceil(np/32)] or NULL: bit (j % 32) of word
 *         vis[m][i][j / 32] is V_ijm; bits for j >= np are 0
 *
 * nc = 0 or np = 0 is a no-op.  Errors: UVC_E_INVAL (NULL scene/cand/A with
 * nc*np > 0, K out of range, non-finite lamp data, lda < np), UVC_E_CUDA.
 */
int uvc_irradiance_matrix(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                          float* A, int64_t lda, uint32_t* vis, uvc_stream_t stream);

/*
 * uvc_irradiance_counters - the same computation as uvc_irradiance_matrix
 * (writes A, no visibility words) with traversal instrumentation, for
 * profiling and for the benchmark's algorithmic operation count; slower than
 * the plain call because of the counting atomics.  Synchronises `stream`.
 *   counters  HOST uint64[8]: [0] node visits (per warp packet), [1] leaf
 *             triangle loads (per warp packet; per lane on the wedge path),
 *             [2] packet traversals,
 *             [3] per-segment box tests, [4] per-segment triangle tests,
 *             [5] facing segments that needed a search, [6] per-lane wedge
 *             box tests, [7] per-lane wedge plane tests
 * A packet is one warp: 32 patches and one lamp source (Sec. IV-C: each
 * segment is one source-to-patch visibility query of Eq. (7)), or, for a
 * vertical line lamp on the wedge path, 32 patches and all K sources of one
 * candidate (see uvc_set_wedge_traversal).
 */
int uvc_irradiance_counters(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                            float* A, int64_t lda, uint64_t* counters, uvc_stream_t stream);

/*
 * uvc_irradiance_area_mean - the patch-mean irradiance instead of the centroid
 * sample: the flux each patch receives over its area, which is what the
 * paper's raster estimator measures (Sec. IV-C, mean irradiance = flux /
 * area).  A point source of power w_m P that sees all of a triangle delivers
 * w_m P Omega / (4 pi) to it, Omega the triangle's solid angle (van Oosterom
 * and Strackee, IEEE Trans. Biomed. Eng. 30(2), 1983); so, per source:
 *   - not facing (<n_j, o - s_j> <= 0) or centroid occluded: 0
 *   - centroid and every check point unoccluded: w_m P sum_t Omega_t / (4 pi a_j)
 *     (check points: the patch vertices moved 1e-3 of the way to the centroid,
 *     fl32(q + fl32(1e-3 * fl32(s_j - q))))
 *   - otherwise: the centroid sample w_m P <n_j, v> / (4 pi d^3)
 * The vertex checks are a test of full visibility at 4 (or 7) points, not a
 * proof: an occluder that covers part of a patch but none of its check points
 * is missed.
 *   ptri     float[np][2][3][3] device: each patch as one or two triangles
 *            (vertices in metres; an unused second triangle is all zero)
 *   A, lda   as in uvc_irradiance_matrix (a_j is the area given at build)
 *   nclosed  uint8[nc][np] device or NULL: sources that used the closed form
 * FP32; a failed search writes NaN and records UVC_E_TIMEOUT/UVC_E_STACK in
 * the scene status.  Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
int uvc_irradiance_area_mean(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                             const float* ptri, float* A, int64_t lda, uint8_t* nclosed, uvc_stream_t stream);

/*
 * uvc_irradiance_raster - the paper's own estimator (Sec. IV-C, Fig. 2): per
 * source point a visibility cube of six R x R faces (the paper uses R = 512)
 * holding the nearest triangle seen through each pixel centre (depth test);
 * each pixel's power w_m P Omega_pixel / (4 pi) (the precomputed emission
 * table E) is added to that triangle's flux when the pixel ray meets the
 * triangle's front side (<dir, n_t> < 0) and is absorbed otherwise; the mean
 * irradiance of triangle t is its flux over its area, A[i][t] = F_it / |s_t|
 * (per triangle, not per patch).
 * Cube layout: face f looks along axis a = f / 2 (sign + for even f); pixel
 * (px, py) is the direction with component a = +-1, component (a+1) % 3 =
 * fl32(fl32(2 px + 1) / R) - 1 and component (a+2) % 3 likewise from py, and
 * covers the solid angle of its square on the unit-distance plane.
 *   tri_normal  float[nt][3] device, the front (free) side of each triangle,
 *               by the triangle's index in the build's `tris`
 *   A           float[nc][lda] device, lda >= nt, columns by triangle index
 *   workspace   device scratch; uvc_raster_workspace_bytes(scene, lamp, R, b)
 *               bytes hold batches of b candidates (more bytes, larger
 *               batches; less than b = 1 needs is UVC_E_INVAL)
 * A software rasteriser (setup, prefix-sum balanced fragments, watertight
 * pixel-centre ray tests with a 64-bit atomicMin of (depth, id)); the flux is
 * summed in 2^-40 W fixed point, so results do not depend on thread order.
 * R in [1, 4096].  Enqueued on `stream` (the table copy is synchronous with
 * the host).  Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
size_t uvc_raster_workspace_bytes(const uvc_scene* scene, const uvc_lamp* lamp, int32_t R, int64_t cand_per_batch);
int uvc_irradiance_raster(const uvc_scene* scene, const float* tri_normal, const float* cand, int64_t nc,
                          const uvc_lamp* lamp, int32_t R, float* A, int64_t lda, void* workspace, size_t bytes,
                          uvc_stream_t stream);

/*
 * uvc_fluence - fluence of every patch for nvec dwell-time vectors (Eq. (5)):
 *
 *   mu[v][j] = sum_i t[v][i] * A[i][j]
 *
 *   A   float[nc][lda] as written by uvc_irradiance_matrix (np columns used)
 *   t   float[nvec][nc] dwell times (seconds)
 *   mu  float[nvec][np] output (J/m^2)
 *
 * Where the rows of A start on 16-byte boundaries (lda a multiple of 4, A
 * 16-byte aligned) the product runs on the tensor cores (see
 * uvc_set_fluence_tensor_cores): TF32 operands split in two (x = hi + lo),
 * FP32 accumulation of 32 candidate rows at a time, the stage sums added with
 * Kahan compensation; otherwise, or with the tensor cores switched off, on the
 * CUDA cores in FP32 with blocks of 32 rows summed plainly and the block sums
 * Kahan-compensated.  nvec in [1, 256].  Allocates nothing.  A wait of the
 * tensor-core kernel that runs out records UVC_E_TIMEOUT in the scene's status
 * word (uvc_scene_status).  Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
int uvc_fluence(const uvc_scene* scene, const float* A, int64_t nc, int64_t lda, const float* t,
                int32_t nvec, float* mu, uvc_stream_t stream);

/*
 * uvc_fluence_streamed - the same mu as uvc_fluence of uvc_irradiance_matrix's
 * A, without storing A (Eq. (5) with Eq. (7) evaluated on the fly); for
 * matrices too large to keep.  Candidates are split into chunks whose partial
 * sums go to temporary device memory (stream-ordered allocator) and are then
 * added in a fixed order, so the result is deterministic.
 *   cand, lamp as in uvc_irradiance_matrix; t, nvec, mu as in uvc_fluence.
 */
int uvc_fluence_streamed(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                         const float* t, int32_t nvec, float* mu, uvc_stream_t stream);

/*
 * uvc_fluence_streamed_noalloc - uvc_fluence_streamed for callers that cannot
 * allocate device memory during the call: a host program whose own allocator
 * already holds all the device memory it may use, or a control loop that
 * forbids allocation after start-up because an allocation can block,
 * synchronise the device or fail mid-run.  This call allocates nothing: the
 * warps' task counter (256 bytes) and the per-chunk partial sums go to one
 * fixed device array of 64 MiB that the library defines (every GPU that loads
 * the library holds it until exit).
 * The paper has no counterpart; this is an interface convenience.
 *
 *   Same arguments, result and determinism as uvc_fluence_streamed; fewer
 *   candidate chunks may be used (at most (64 MiB - 256) / (4 * nvec * np) of
 *   them), so the last bits of mu may differ from uvc_fluence_streamed's.
 *   Limit: 4 * nvec * np must not exceed 64 MiB less 256 bytes (67,108,608
 *   bytes), else UVC_E_SCRATCH and nothing is launched.
 *   The first call on a device looks up the array's device address for that
 *   device (cudaGetSymbolAddress) and caches it, keyed on the device and its
 *   current context (after a cudaDeviceReset the first call in the new
 *   context looks it up again); make that first call before any stream
 *   capture.  All calls share the one array, which keeps the last
 *   call's contents (each call writes every partial before reading it), so
 *   calls whose work overlaps on the GPU (e.g. on two streams at once) race
 *   and corrupt each other: serialise them.
 */
int uvc_fluence_streamed_noalloc(const uvc_scene* scene, const float* cand, int64_t nc, const uvc_lamp* lamp,
                                 const float* t, int32_t nvec, float* mu, uvc_stream_t stream);

/*
 * uvc_coverage - covered fraction of the surface for each dwell vector: the
 * patches meeting the dose constraint mu_j >= mu_min of Eq. (8) (inclusive),
 * weighted by area (the "disinfected area" of Sec. V-C) and by count.
 *
 *   mu         float[nvec][np]  fluence (e.g. from uvc_fluence)
 *   cov_area   float[nvec]      sum_j a_j [mu_vj >= mu_min] / sum_j a_j
 *   cov_count  float[nvec] or NULL: fraction of patches meeting it
 *
 * Deterministic FP32 reductions with compensated sums.  nvec in [1, 65535].
 */
int uvc_coverage(const uvc_scene* scene, const float* mu, int32_t nvec, float mu_min, float* cov_area,
                 float* cov_count, uvc_stream_t stream);

/*
 * Batched irradiance matrices: many jobs - (scene, candidates, lamp) triples,
 * e.g. rooms of uneven size crossed with lamp designs (the robot-design
 * comparison of Sec. V-C) - computed by one persistent launch whose warps walk
 * the tasks of all jobs round-robin, so the launch ends evenly whatever the
 * job sizes.  Each job writes its own A (and optional visibility words)
 * exactly as uvc_irradiance_matrix would (bit-identical results).
 *
 *   uvc_job.scene, cand, nc, A, lda, vis  as in uvc_irradiance_matrix
 *   uvc_job.lamp                          index into the `lamps` array
 *
 * uvc_batch_create copies the job table to `workspace` (caller-owned device
 * memory of uvc_batch_workspace_bytes(njobs, nlamps) bytes, 256-byte
 * aligned; it must outlive the batch) and synchronises `stream`.  The caller
 * keeps the scenes and buffers alive while the batch is used.
 * uvc_batch_launch enqueues the whole batch on `stream`; it reads no host
 * data and allocates nothing, so it may be captured in a CUDA graph.
 * uvc_batch_autotune times the tunable launch parameters on a sample of the
 * batch's tasks (sample_fraction of them; the sampled A entries are written,
 * correctly), keeps the fastest for the batch, caches it per size bucket for
 * later batches of this process, and synchronises `stream`.
 * uvc_batch_set_config sets them by hand (cand_per_task in {1, 2, 4, 8, 16};
 * blocks_per_sm 0 = as many as fit).  Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
typedef struct {
    const uvc_scene* scene;
    const float* cand;
    int64_t nc;
    int32_t lamp;
    float* A;
    int64_t lda;
    uint32_t* vis;
} uvc_job;

typedef struct {
    int32_t cand_per_task;   /* candidates a warp handles for its 32 patches */
    int32_t blocks_per_sm;   /* resident blocks per SM, 0 = occupancy limit */
} uvc_batch_config;

typedef struct uvc_batch uvc_batch; /* opaque host-side handle */

size_t uvc_batch_workspace_bytes(int32_t njobs, int32_t nlamps);
int uvc_batch_create(const uvc_job* jobs, int32_t njobs, const uvc_lamp* lamps, int32_t nlamps, void* workspace,
                     size_t workspace_bytes, uvc_stream_t stream, uvc_batch** out);
int uvc_batch_launch(uvc_batch* batch, uvc_stream_t stream);
int uvc_batch_set_config(uvc_batch* batch, const uvc_batch_config* config, uvc_stream_t stream);
int uvc_batch_autotune(uvc_batch* batch, double sample_fraction, uvc_batch_config* chosen, uvc_stream_t stream);
int uvc_batch_info(const uvc_batch* batch, int64_t* total_pairs, int32_t* stack_cap, uvc_batch_config* config);
int uvc_batch_free(uvc_batch* batch);

/*
 * Learned candidate proposal.  The paper samples vantage configurations on a
 * uniform grid and leaves a better choice to future work (Sec. VI); the
 * relaxed LP of Sec. IV-D (Eq. (9)) then keeps only the few configurations
 * with non-zero dwell time.  The proposal scores every candidate with a small
 * perceptron before the irradiance matrix is computed, so the matrix is
 * evaluated for the best-scoring candidates only.  It has no counterpart in
 * the paper's own pipeline.
 *
 * uvc_candidate_features - the scorer's input, per candidate c (row i):
 *   feat[i][b], b = 0..63   fraction of the patch area whose centroid lies at
 *                           squared distance d^2 = |s_j - c|^2 in bin b; the bin
 *                           edges are E_b = fl32((0.1 * 250^(b/64))^2) m^2 for
 *                           b = 1..63 (E_0 = 0, E_64 = infinity), bin b holding
 *                           E_b <= d^2 < E_{b+1}
 *   feat[i][64]             distance from c to the nearest triangle (metres;
 *                           3e38 for a scene without triangles)
 *   feat[i][65]             the height (z) of c
 *   cand  float[nc][3] device;  feat  float rows of ldf >= 66 floats, device
 *   (caller-owned; columns 66..ldf-1 untouched).
 * FP32 arithmetic with fixed-order sums (deterministic).  Errors: UVC_E_INVAL
 * (NULL scene, nc out of range, NULL buffer with nc > 0), UVC_E_STACK (a
 * hierarchy deeper than 126 levels, beyond the nearest-triangle search's
 * fixed stack), UVC_E_CUDA.
 */
int uvc_candidate_features(const uvc_scene* scene, const float* cand, int64_t nc, float* feat, int64_t ldf,
                           uvc_stream_t stream);

/*
 * uvc_probe_features - a visibility sketch of each candidate from the
 * irradiance of all candidates on a small probe sample of the patches (a
 * matrix from uvc_irradiance_matrix on a scene holding only the probe
 * patches).  With E*_j = max_i A[i][j] the best irradiance patch j gets from
 * any candidate, L the lit probe patches (E*_j > 0) and
 * Ebar = sum_L a_j E*_j / sum_L a_j:
 *   hardness  h_j = floor(log2(fl32(E*_j / Ebar))) + 4, clamped to [0, 7]
 *   efficiency bin of fl32(A[i][j] / E*_j): [0, .5) [.5, .7) [.7, .8) [.8, .9)
 *             [.9, .95) [.95, 1] -> 0..5
 *   feat[i][6 h + e] = sum of a_j over L in that (h, e) cell / sum_L a_j
 * In LP terms (Eq. (9)), a candidate that is the most efficient source for
 * hard-to-light patches is the one the optimum spends time at.
 *   A     float[nc][lda] device, lda >= np;  area  float[np] device
 *   work  device scratch of uvc_probe_features_work_bytes(np) bytes (4-aligned)
 *   feat  float rows of ldf >= 48 floats, device (columns 48.. untouched)
 * FP32 with compensated, fixed-order sums; the bins are decided in FP32.
 * Enqueued on `stream`, capturable.  Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
size_t uvc_probe_features_work_bytes(int64_t np);
int uvc_probe_features(const float* A, int64_t nc, int64_t lda, int64_t np, const float* area, void* work,
                       float* feat, int64_t ldf, uvc_stream_t stream);

/*
 * uvc_select_top - the k best-scoring of n candidates (higher score first,
 * equal scores to the lower index, NaN lowest), written in ascending index
 * order: out_idx[r] (int32, may be NULL) and out_cand[r][3] = cand[idx][3]
 * (may be NULL if out_idx is given).  All arrays on the device.
 * n in [0, 16384], k in [0, n].  One block; enqueued on `stream`, capturable.
 * Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
int uvc_select_top(const float* score, int64_t n, int64_t k, const float* cand, float* out_cand, int32_t* out_idx,
                   uvc_stream_t stream);

/*
 * uvc_group_boost - stratified selection: in every group of `group`
 * consecutive candidates (candidates come in spatial grid order, so a group
 * is a neighbourhood) the highest score (lowest index among equal scores, NaN
 * lowest) gets `bonus` added, so that a following uvc_select_top keeps one
 * candidate of every neighbourhood before it ranks the rest globally.
 *   score  float[n] device, updated;  group >= 1
 * Enqueued on `stream`, capturable.  Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
int uvc_group_boost(float* score, int64_t n, int32_t group, float bonus, uvc_stream_t stream);

/*
 * uvc_mark_best - for every probe patch j that some candidate lights, set
 * score[i*] = value where i* = argmax_i A[i][j] (the lowest index among equal
 * maxima), so that a following uvc_select_top keeps the best source of every
 * probe patch whatever the scorer says (value = +inf; if more candidates are
 * marked than kept, the lower indices win).  With rare > 0, every candidate
 * that lights a probe patch lit by at most `rare` candidates is marked too
 * (such patches go dark unless one of their few sources is kept).
 *   A  float[nc][lda] device, lda >= np;  score  float[nc] device, updated
 * Enqueued on `stream`, capturable.  Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
int uvc_mark_best(const float* A, int64_t nc, int64_t lda, int64_t np, float* score, float value, int32_t rare,
                  uvc_stream_t stream);

/*
 * uvc_probe_lost - the fallback check of the proposal: of a probe sample of
 * patches (columns of A), the area fraction that some candidate lights
 * (A[i][j] > 0 for some row i < nc) but none of the selected rows idx[0..k)
 * does:  *out = sum_j a_j [lit by all, dark for the selection] / sum_j a_j.
 *   A     float[nc][lda] device (irradiance of all candidates on the probe)
 *   idx   int32[k] device, rows of A (e.g. from uvc_select_top); rows outside
 *         [0, nc) are ignored
 *   area  float[np] device;  lost  float[np] device scratch;  out  float[1] device
 * Compensated FP32 sums in a fixed order.  Enqueued on `stream`, capturable.
 * Errors: UVC_E_INVAL, UVC_E_CUDA.
 */
int uvc_probe_lost(const float* A, int64_t nc, int64_t lda, int64_t np, const int32_t* idx, int64_t k,
                   const float* area, float* lost, float* out, uvc_stream_t stream);

/*
 * The scorer: logit(x) = w3 . relu(relu(x W1 + b1) W2 + b2) + b3, with x the
 * candidate features (in_dim of them, zero-padded to a multiple of 16),
 * hidden width `hidden`.  W1, W2 and the activations are stored in BF16, the
 * products run on the tensor cores with FP32 accumulation; biases, w3, the
 * head and all gradients are FP32.  Training minimises the weighted binary
 * cross-entropy sum_i w_i (softplus(s_i) - y_i s_i) of the logits s_i against
 * labels y_i in [0, 1] (1 = the LP of Eq. (9) gave the candidate a non-zero
 * dwell time) with Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected).
 *
 * Parameter layout (float[uvc_mlp_param_count]): W1 [in_pad][hidden] (rows
 * in_dim..in_pad-1 unused, keep them 0), b1 [hidden], W2 [hidden][hidden],
 * b2 [hidden], w3 [hidden], b3 [1].  Gradients use the same layout.
 *
 * uvc_mlp_create     in_dim in [1, 4096], hidden a multiple of 8 in [8, 4096],
 *                    max_batch in [1, 2^24]; He-normal initial weights from a
 *                    seeded generator, zero biases; one device allocation,
 *                    freed by uvc_mlp_free.  Synchronises the device.
 * uvc_mlp_params     copies the FP32 parameters to (set = 0) or from (set = 1)
 *                    host memory; n must equal the parameter count.  Synchronous.
 * uvc_mlp_forward    logit float[B] device <- x float[B][in_dim] device, B <=
 *                    max_batch; enqueued on `stream`.
 * uvc_mlp_train_step one forward, backward and Adam update on (x, y, w), each
 *                    device arrays of B rows; *loss (device float, may be NULL)
 *                    receives the batch loss.  lr > 0.  Enqueued on `stream`;
 *                    one model is not used from two streams at once.
 * uvc_mlp_grads      the gradients of the last training step (host copy).
 * Errors: UVC_E_INVAL for NULL handles or out-of-range sizes, UVC_E_NOMEM,
 * UVC_E_CUDA.
 */
typedef struct uvc_mlp uvc_mlp; /* opaque handle */

int uvc_mlp_create(int32_t in_dim, int32_t hidden, int32_t max_batch, uint64_t seed, uvc_mlp** out);
int uvc_mlp_free(uvc_mlp* model);
int64_t uvc_mlp_param_count(const uvc_mlp* model);
int uvc_mlp_params(uvc_mlp* model, float* host, int64_t n, int32_t set);
int uvc_mlp_forward(uvc_mlp* model, const float* x, int32_t B, float* logit, uvc_stream_t stream);
int uvc_mlp_train_step(uvc_mlp* model, const float* x, const float* y, const float* w, int32_t B, float lr,
                       float* loss, uvc_stream_t stream);
int uvc_mlp_grads(const uvc_mlp* model, float* host, int64_t n);

/*
 * uvc_library_flags - how this copy of the library was built: bit
 * UVC_LIB_CHECKED is set for the checked build (compiled with UVC_CHECKED),
 * whose traversals test every node, leaf and cached-triangle index before use
 * and report violations as UVC_E_BOUNDS in the scene's status word (a
 * stand-in for a memory checker; the normal build has no checks).
 */
#define UVC_LIB_CHECKED 1u
uint32_t uvc_library_flags(void);

/* uvc_status_string - static text for a status code (never NULL). */
const char* uvc_status_string(int status);

/*
 * uvc_scene_status - synchronise `stream`, then return and clear the scene's
 * device status word: UVC_OK, or the first device-side error recorded since
 * the last call (UVC_E_TIMEOUT, UVC_E_STACK; in the checked build also
 * UVC_E_BOUNDS, see uvc_library_flags).
 */
int uvc_scene_status(const uvc_scene* scene, uvc_stream_t stream);

/*
 * uvc_scene_set_limits - lower the scene's traversal limits, for tests of the
 * failure handling (a stand-in for a tree too deep for the stack, or a search
 * that does not end).  max_stack: stack entries per warp (the built-in bound
 * is 3 per level of the four-wide tree, plus 4); max_visits: node visits per
 * search (built in: nt + 64); 0 restores the built-in bound, and values above
 * it have no effect.  A search that would exceed a limit stops: its entries
 * become NaN and the status word records UVC_E_STACK or UVC_E_TIMEOUT (first
 * error wins); the other entries are unchanged.  Applies to calls made after
 * it (a batch keeps the limits of its creation); host-only, no device work.
 * Not in the paper.  Errors: UVC_E_INVAL (NULL scene, negative limit).
 */
int uvc_scene_set_limits(uvc_scene* scene, int32_t max_stack, int32_t max_visits);

/*
 * uvc_scene_info - host-side facts about a built scene: triangle and patch
 * counts, depth of the hierarchy (edges from the root to the deepest leaf).
 * Any output pointer may be NULL.
 */
int uvc_scene_info(const uvc_scene* scene, int64_t* nt, int64_t* np, int32_t* depth);

/*
 * uvc_probe_l2_read - bandwidth probe (not in the paper): read the device
 * buffer `buf` (`bytes` bytes, 16-byte aligned, a multiple of 16) `passes`
 * times with 16-byte loads that are cached in L2 only (ld.global.cg), from 4
 * blocks of 512 threads per SM, and write nothing unless the XOR of all words
 * hits one magic value (then one word to `sink`, a device pointer).  Timed by
 * the caller (CUDA events around the call) on a buffer that fits in L2, it
 * gives the L2 read bandwidth that the traversal's bytes are compared with.
 * Asynchronous on `stream`.  Errors: UVC_E_INVAL (NULL pointers, size or
 * alignment, passes < 1), UVC_E_CUDA.
 */
int uvc_probe_l2_read(const void* buf, size_t bytes, int32_t passes, uint32_t* sink, uvc_stream_t stream);

/*
 * uvc_scene_export_traversal - copy the arrays the traversal kernels read to
 * HOST buffers, as they lie in device memory (synchronises the scene's build
 * stream), for inspection and for counting tools that replay the kernels'
 * visit order on the CPU.  Not in the paper.  Any pointer may be NULL.
 *   nodes4     (nt-1) x 128 bytes: the four-wide nodes (valid at the indices
 *              the traversal reaches from the root), each
 *              float q[6][4] (per child pair the x, y, z records
 *              (c0.lo, c1.lo, c0.hi, c1.hi)), int32 r[4] (child refs: >= 0
 *              node, < 0 leaf ~k, 0x7fffffff empty), int32 m[4] (leaf mask,
 *              node mask, 0, 0)
 *   tri        float[nt][3][4]: vertices (x, y, z, w) in sorted order, w of
 *              the first vertex the triangle's input index (int32 bits)
 *   patch_s    float[np][4]: sample point and area
 *   patch_n    float[np][4]: normal and clearance (metres)
 *   patch_excl int32[np][2]: excluded triangles (input indices, -1 = none)
 *   root       the root reference (0, or ~0 for a single triangle)
 *   diameter   diagonal of the triangles' bounding box
 *   coord_bound largest coordinate magnitude of that box
 * Errors: UVC_E_INVAL (NULL scene), UVC_E_CUDA.
 */
int uvc_scene_export_traversal(const uvc_scene* scene, void* nodes4, float* tri, float* patch_s, float* patch_n,
                               int32_t* patch_excl, int32_t* root, float* diameter,
                               float* coord_bound);

/*
 * uvc_irradiance_candidates_per_task - the number of consecutive candidates a
 * warp of uvc_irradiance_matrix (and uvc_irradiance_counters) takes for its 32
 * patches, over which it keeps its occluder cache: the task shape a counting
 * tool needs to replay the kernel's visit order.  Not in the paper.  Always
 * >= 1; no error.
 */
int32_t uvc_irradiance_candidates_per_task(void);

/*
 * uvc_scene_export_bvh - copy the hierarchy to HOST buffers for inspection
 * and testing (synchronises the scene's build stream).  Any pointer may be
 * NULL to skip that array.  For nt >= 2 there are nt-1 internal nodes:
 *   keys      uint64[nt]  sorted Morton keys
 *   order     int32[nt]   triangle index at each sorted position
 *   children  int32[nt-1][2]  child references: >= 0 internal node index,
 *                          < 0 leaf ~k (sorted position k)
 *   boxes     float[nt-1][12] left child lo.xyz, hi.xyz, right child lo.xyz, hi.xyz
 */
int uvc_scene_export_bvh(const uvc_scene* scene, uint64_t* keys, int32_t* order, int32_t* children,
                         float* boxes);

#ifdef __cplusplus
}
#endif

#endif /* UVC_H */
