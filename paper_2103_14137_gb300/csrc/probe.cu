// Bandwidth probe for the memory roofline of the traversal: a streaming read
// of a caller-owned device buffer that fits in L2, through the L2-only load
// path (ld.global.cg), repeated `passes` times.  The traversal's scene (the
// four-wide nodes, the sorted triangles and the patch records) is read from
// L1/L2 in the same way, so bytes per second of this probe are the peak its
// algorithmic bytes are compared against.  Not in the paper.
#include "uvc_internal.cuh"

namespace uvc {
namespace {

constexpr int kProbeThreads = 512;

__global__ void __launch_bounds__(kProbeThreads) k_l2_read(const uint4* __restrict__ buf, int64_t n16, int passes,
                                                           uint32_t* __restrict__ sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (int p = 0; p < passes; ++p) {
        int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc ^= (a.x ^ a.y ^ a.z ^ a.w) ^ (b.x ^ b.y ^ b.z ^ b.w) ^ (c.x ^ c.y ^ c.z ^ c.w) ^ (d.x ^ d.y ^ d.z ^ d.w);
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
        acc = acc * 2654435761u + (uint32_t)p;   // each pass depends on the last: no pass can be dropped
    }
    if (acc == 0x9e3779b9u) *sink = acc;   // keeps the loads alive; practically never written
}

}  // namespace

int probe_l2_read(const void* buf, size_t bytes, int32_t passes, uint32_t* sink, cudaStream_t stream) {
    const int64_t n16 = (int64_t)(bytes / 16);
    const int blocks_per_sm = 4;   // 2,048 threads per SM: enough loads in flight to cover L2 latency
    k_l2_read<<<blocks_per_sm * sm_count(), kProbeThreads, 0, stream>>>(static_cast<const uint4*>(buf), n16, passes,
                                                                        sink);
    return status_from_cuda(cudaGetLastError());
}

}  // namespace uvc
