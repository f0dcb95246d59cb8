// Candidate scorer of the learned proposal: a 3-layer perceptron
//   x (in) -> relu(x W1 + b1) (H) -> relu(. W2 + b2) (H) -> . w3 + b3 (logit)
// with BF16 weights and activations and FP32 accumulation, trained with
// binary cross-entropy on LP dwell-time labels (candidate kept by the relaxed
// LP (9) or not) and Adam.  The dense products run on the tensor cores
// (tcgen05.mma BF16 -> FP32, accumulator in tensor memory) through one GEMM
// kernel whose operands are read with arbitrary strides, so the forward pass,
// the weight gradients (X^T dZ) and the input gradients (dZ W^T) all use it.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "tcgen05.cuh"
#include "uvc_internal.cuh"

struct uvc_mlp {
    int in_dim = 0, in_pad = 0, hidden = 0, max_batch = 0;
    int64_t step = 0;
    void* block = nullptr;
    // fp32 master parameters, gradients, Adam moments: one flat array each
    float *param = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t nparam = 0;
    float *W1, *b1, *W2, *b2, *w3, *b3;         // views into param
    float *gW1, *gb1, *gW2, *gb2, *gw3, *gb3;   // views into grad
    __nv_bfloat16 *W1h, *W2h;                    // bf16 copies used by the GEMMs
    __nv_bfloat16 *Xh, *H1, *H2, *dZ1, *dZ2;     // activations, max_batch rows
    float *dH1, *logit, *dS, *loss;
};

namespace uvc {
namespace {

// The GEMM on the fifth-generation tensor cores: one block per 128 x 64 tile
// of C, accumulated in tensor memory by tcgen05.mma .kind::f16 (BF16 operands,
// FP32 accumulator, M = 128, N = 64, K = 16 per instruction).  Per 32-wide
// slice of K the block's threads gather the A and B tiles with the operands'
// strides (zeros outside the matrices) into shared memory in the tensor
// core's K-major layout (8-row x 16-byte core matrices), one thread issues the
// two MMAs and commits them to an mbarrier, and the block waits for it before
// the next slice overwrites the tiles; the epilogue reads the accumulator back
// with tcgen05.ld (warp w: rows 32w..32w+31), adds the bias, applies the ReLU
// and writes C and/or Ch.  A wait that runs out (bounded: about a second)
// makes the block write NaN.
constexpr int BM = 128, BN = 64, BK = 32, kGemmThreads = 128;
constexpr uint32_t kGemmLbo = 128, kGemmSbo = 256;                  // core matrices along K, 8-row groups
constexpr uint32_t kGemmAStep = (BM / 8) * kGemmSbo;                // one K-step (16 values) of A: 4 KB
constexpr uint32_t kGemmBStep = (BN / 8) * kGemmSbo;                // of B: 2 KB
constexpr uint32_t kGemmIdesc = tc::idesc_f32acc(tc::kFmtBF16, BM, BN);
constexpr uint32_t kGemmTmemCols = BN;                              // FP32 accumulator columns

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]) (relu), A(m,k) = Ap[m*sam + k*sak],
// B(k,n) = Bp[k*sbk + n*sbn]; writes fp32 C (ldc) and/or bf16 Ch (ldh).
__global__ void __launch_bounds__(kGemmThreads) k_gemm(const __nv_bfloat16* __restrict__ Ap, int64_t sam,
                                                       int64_t sak, const __nv_bfloat16* __restrict__ Bp,
                                                       int64_t sbk, int64_t sbn, int M, int N, int K,
                                                       const float* __restrict__ bias, int relu, float* C,
                                                       int64_t ldc, __nv_bfloat16* Ch, int64_t ldh) {
    __shared__ __align__(128) unsigned char As[(BK / 16) * kGemmAStep];
    __shared__ __align__(128) unsigned char Bs[(BK / 16) * kGemmBStep];
    __shared__ uint64_t mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (tid == 0) {
        fail = 0;
        tc::mbar_init(&mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::alloc(&tmem_slot, kGemmTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K; k0 += BK, phase ^= 1u) {
        // A: 128 rows x 4 chunks of 8 K-values, B: 64 rows x 4 chunks; one 16-byte store per chunk
        for (int e = tid; e < (BM + BN) * (BK / 8); e += kGemmThreads) {
            const bool isA = e < BM * (BK / 8);
            const int f = isA ? e : e - BM * (BK / 8);
            const int row = f / (BK / 8), ch = f % (BK / 8);   // row (m or n), chunk of 8 along K
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + ch * 8 + q;
                if (isA) {
                    const int m = m0 + row;
                    v[q] = (m < M && k < K) ? Ap[(int64_t)m * sam + (int64_t)k * sak] : zero;
                } else {
                    const int n = n0 + row;
                    v[q] = (n < N && k < K) ? Bp[(int64_t)k * sbk + (int64_t)n * sbn] : zero;
                }
            }
            const uint32_t off = (uint32_t)(ch >> 1) * (isA ? kGemmAStep : kGemmBStep) + (uint32_t)(row >> 3) * kGemmSbo +
                                 (uint32_t)(ch & 1) * kGemmLbo + (uint32_t)(row & 7) * 16u;
            *reinterpret_cast<uint4*>((isA ? As : Bs) + off) = *reinterpret_cast<const uint4*>(v);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks)
                tc::mma<false>(tmem, tc::smem_desc(tc::smem_u32(As) + ks * kGemmAStep, kGemmLbo, kGemmSbo),
                               tc::smem_desc(tc::smem_u32(Bs) + ks * kGemmBStep, kGemmLbo, kGemmSbo), kGemmIdesc,
                               (k0 > 0 || ks > 0) ? 1u : 0u);
            tc::commit(&mma_done);
        }
        // the MMAs have read the tiles before the next slice overwrites them
        if (!fail && !tc::mbar_wait(&mma_done, phase)) fail = 1;
        __syncthreads();
    }
    tc::fence_after();
    const int m = m0 + 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tc::load16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int n = n0 + c0 + c;
            if (m >= M || n >= N) continue;
            float x = K > 0 ? v[c] : 0.f;
            if (bias) x += bias[n];
            if (relu) x = fmaxf(x, 0.f);
            if (fail) x = __int_as_float(0x7fc00000);
            if (C) C[(int64_t)m * ldc + n] = x;
            if (Ch) Ch[(int64_t)m * ldh + n] = __float2bfloat16(x);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::dealloc(tmem, kGemmTmemCols);
    }
}

void gemm(const __nv_bfloat16* A, int64_t sam, int64_t sak, const __nv_bfloat16* B, int64_t sbk, int64_t sbn, int M,
          int N, int K, const float* bias, bool relu, float* C, int64_t ldc, __nv_bfloat16* Ch, int64_t ldh,
          cudaStream_t s) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<<<grid, kGemmThreads, 0, s>>>(A, sam, sak, B, sbk, sbn, M, N, K, bias, relu ? 1 : 0, C, ldc, Ch, ldh);
}

__global__ void k_to_bf16_pad(const float* __restrict__ x, int B, int in, int pad, __nv_bfloat16* __restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * pad) return;
    const int r = (int)(e / pad), c = (int)(e % pad);
    y[e] = __float2bfloat16(c < in ? x[(int64_t)r * in + c] : 0.f);
}

__global__ void k_cast_bf16(const float* __restrict__ x, int64_t n, __nv_bfloat16* __restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = __float2bfloat16(x[e]);
}

// logit[i] = H2[i] . w3 + b3 (one warp per row)
__global__ void k_head(const __nv_bfloat16* __restrict__ H2, int B, int H, const float* __restrict__ w3,
                       const float* __restrict__ b3, float* __restrict__ logit) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= B) return;
    float s = 0.f;
    for (int n = lane; n < H; n += 32) s += __bfloat162float(H2[(int64_t)row * H + n]) * w3[n];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) logit[row] = s + *b3;
}

// BCE with logits: per row dS = w (sigmoid(s) - y), loss terms; dZ2 = dS w3 [H2 > 0]
__global__ void k_head_back(const float* __restrict__ logit, const float* __restrict__ y,
                            const float* __restrict__ w, const __nv_bfloat16* __restrict__ H2, int B, int H,
                            const float* __restrict__ w3, float* __restrict__ dS, __nv_bfloat16* __restrict__ dZ2,
                            float* __restrict__ loss_terms) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= B) return;
    const float s = logit[row];
    const float p = 1.f / (1.f + expf(-s));
    const float d = w[row] * (p - y[row]);
    if (lane == 0) {
        dS[row] = d;
        const float sp = s > 0.f ? s + log1pf(expf(-s)) : log1pf(expf(s));   // softplus
        loss_terms[row] = w[row] * (sp - y[row] * s);
    }
    for (int n = lane; n < H; n += 32) {
        const float h = __bfloat162float(H2[(int64_t)row * H + n]);
        dZ2[(int64_t)row * H + n] = __float2bfloat16(h > 0.f ? d * w3[n] : 0.f);
    }
}

// out[n] = sum_i (bf16 or fp32) X[i][n] * (wv ? wv[i] : 1), fixed order; one thread per column
__global__ void k_colsum_bf16(const __nv_bfloat16* __restrict__ X, int B, int N, const float* __restrict__ wv,
                              float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int i = 0; i < B; ++i) s += __bfloat162float(X[(int64_t)i * N + n]) * (wv ? wv[i] : 1.f);
    out[n] = s;
}

__global__ void k_sum(const float* __restrict__ x, int n, float* __restrict__ out) {
    __shared__ float part[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// dZ1 = dH1 [H1 > 0] (bf16)
__global__ void k_relu_back(const float* __restrict__ dH, const __nv_bfloat16* __restrict__ Hh, int64_t n,
                            __nv_bfloat16* __restrict__ dZ) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) dZ[e] = __float2bfloat16(__bfloat162float(Hh[e]) > 0.f ? dH[e] : 0.f);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int blocks(int64_t n, int t = 256) { return (int)((n + t - 1) / t); }

void refresh_bf16(uvc_mlp* M, cudaStream_t s) {
    k_cast_bf16<<<blocks((int64_t)M->in_pad * M->hidden), 256, 0, s>>>(M->W1, (int64_t)M->in_pad * M->hidden, M->W1h);
    k_cast_bf16<<<blocks((int64_t)M->hidden * M->hidden), 256, 0, s>>>(M->W2, (int64_t)M->hidden * M->hidden, M->W2h);
}

void forward(uvc_mlp* M, const float* x, int B, float* logit, cudaStream_t s) {
    const int H = M->hidden, P = M->in_pad;
    k_to_bf16_pad<<<blocks((int64_t)B * P), 256, 0, s>>>(x, B, M->in_dim, P, M->Xh);
    gemm(M->Xh, P, 1, M->W1h, H, 1, B, H, P, M->b1, true, nullptr, 0, M->H1, H, s);
    gemm(M->H1, H, 1, M->W2h, H, 1, B, H, H, M->b2, true, nullptr, 0, M->H2, H, s);
    k_head<<<blocks((int64_t)B * 32), 256, 0, s>>>(M->H2, B, H, M->w3, M->b3, logit);
}

}  // namespace
}  // namespace uvc

extern "C" {

int uvc_mlp_create(int32_t in_dim, int32_t hidden, int32_t max_batch, uint64_t seed, uvc_mlp** out) {
    if (!out) return UVC_E_INVAL;
    *out = nullptr;
    if (in_dim < 1 || in_dim > 4096 || hidden < 8 || hidden > 4096 || (hidden % 8) || max_batch < 1 ||
        max_batch > (1 << 24))
        return UVC_E_INVAL;
    uvc_mlp* M = new (std::nothrow) uvc_mlp();
    if (!M) return UVC_E_NOMEM;
    M->in_dim = in_dim;
    M->in_pad = (in_dim + 15) / 16 * 16;
    M->hidden = hidden;
    M->max_batch = max_batch;
    const int64_t P = M->in_pad, H = hidden, Bm = max_batch;
    M->nparam = P * H + H + H * H + H + H + 1;
    const size_t f4 = sizeof(float), h2 = sizeof(__nv_bfloat16);
    size_t bytes = 4 * f4 * M->nparam + h2 * (P * H + H * H) + h2 * (Bm * P + 4 * Bm * H) + f4 * (Bm * H + 3 * Bm + 64) +
                   16 * 256;
    if (cudaMalloc(&M->block, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete M;
        return UVC_E_NOMEM;
    }
    char* p = static_cast<char*>(M->block);
    auto take = [&](size_t n) {
        char* q = p;
        p += (n + 255) & ~size_t(255);
        return q;
    };
    M->param = (float*)take(f4 * M->nparam);
    M->grad = (float*)take(f4 * M->nparam);
    M->m1 = (float*)take(f4 * M->nparam);
    M->m2 = (float*)take(f4 * M->nparam);
    M->W1h = (__nv_bfloat16*)take(h2 * P * H);
    M->W2h = (__nv_bfloat16*)take(h2 * H * H);
    M->Xh = (__nv_bfloat16*)take(h2 * Bm * P);
    M->H1 = (__nv_bfloat16*)take(h2 * Bm * H);
    M->H2 = (__nv_bfloat16*)take(h2 * Bm * H);
    M->dZ1 = (__nv_bfloat16*)take(h2 * Bm * H);
    M->dZ2 = (__nv_bfloat16*)take(h2 * Bm * H);
    M->dH1 = (float*)take(f4 * Bm * H);
    M->logit = (float*)take(f4 * Bm);
    M->dS = (float*)take(f4 * Bm);
    M->loss = (float*)take(f4 * (Bm + 1));
    float* q = M->param;
    M->W1 = q; q += P * H; M->b1 = q; q += H; M->W2 = q; q += H * H; M->b2 = q; q += H; M->w3 = q; q += H; M->b3 = q;
    q = M->grad;
    M->gW1 = q; q += P * H; M->gb1 = q; q += H; M->gW2 = q; q += H * H; M->gb2 = q; q += H; M->gw3 = q; q += H; M->gb3 = q;
    // He initialisation (padded input rows stay zero), zero biases
    std::vector<float> h(M->nparam, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> n1(0.f, std::sqrt(2.f / in_dim)), n2(0.f, std::sqrt(2.f / hidden));
    for (int r = 0; r < in_dim; ++r)
        for (int c = 0; c < H; ++c) h[r * H + c] = n1(rng);
    for (int64_t e = 0; e < H * H; ++e) h[P * H + H + e] = n2(rng);
    for (int64_t e = 0; e < H; ++e) h[P * H + H + H * H + H + e] = n2(rng) * 0.5f;
    cudaError_t e = cudaMemcpy(M->param, h.data(), f4 * M->nparam, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->m1, 0, f4 * M->nparam);
    if (e == cudaSuccess) e = cudaMemset(M->m2, 0, f4 * M->nparam);
    if (e != cudaSuccess) {
        cudaFree(M->block);
        delete M;
        return uvc::status_from_cuda(e);
    }
    uvc::refresh_bf16(M, nullptr);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(M->block);
        delete M;
        return uvc::status_from_cuda(e);
    }
    *out = M;
    return UVC_OK;
}

int uvc_mlp_free(uvc_mlp* M) {
    if (!M) return UVC_OK;
    cudaDeviceSynchronize();
    cudaFree(M->block);
    delete M;
    return UVC_OK;
}

int64_t uvc_mlp_param_count(const uvc_mlp* M) { return M ? M->nparam : -1; }

int uvc_mlp_params(uvc_mlp* M, float* host, int64_t n, int32_t set) {
    if (!M || !host || n != M->nparam) return UVC_E_INVAL;
    cudaError_t e = set ? cudaMemcpy(M->param, host, sizeof(float) * n, cudaMemcpyHostToDevice)
                        : cudaMemcpy(host, M->param, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && set) {
        uvc::refresh_bf16(M, nullptr);
        e = cudaDeviceSynchronize();
    }
    return uvc::status_from_cuda(e);
}

int uvc_mlp_forward(uvc_mlp* M, const float* x, int32_t B, float* logit, uvc_stream_t stream) {
    if (!M || B < 0 || B > M->max_batch || (B > 0 && (!x || !logit))) return UVC_E_INVAL;
    if (B == 0) return UVC_OK;
    uvc::forward(M, x, B, logit, (cudaStream_t)stream);
    return uvc::status_from_cuda(cudaGetLastError());
}

int uvc_mlp_train_step(uvc_mlp* M, const float* x, const float* y, const float* w, int32_t B, float lr,
                       float* loss, uvc_stream_t stream) {
    if (!M || B < 1 || B > M->max_batch || !x || !y || !w || !(lr > 0.f)) return UVC_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int H = M->hidden, P = M->in_pad;
    uvc::forward(M, x, B, M->logit, s);
    uvc::k_head_back<<<uvc::blocks((int64_t)B * 32), 256, 0, s>>>(M->logit, y, w, M->H2, B, H, M->w3, M->dS, M->dZ2,
                                                                  M->loss + 1);
    uvc::k_sum<<<1, 256, 0, s>>>(M->loss + 1, B, M->loss);
    // head: gw3 = H2^T dS, gb3 = sum dS
    uvc::k_colsum_bf16<<<uvc::blocks(H), 256, 0, s>>>(M->H2, B, H, M->dS, M->gw3);
    uvc::k_sum<<<1, 256, 0, s>>>(M->dS, B, M->gb3);
    // layer 2: gW2 = H1^T dZ2, gb2 = colsum dZ2, dH1 = dZ2 W2^T
    uvc::gemm(M->H1, 1, H, M->dZ2, H, 1, H, H, B, nullptr, false, M->gW2, H, nullptr, 0, s);
    uvc::k_colsum_bf16<<<uvc::blocks(H), 256, 0, s>>>(M->dZ2, B, H, nullptr, M->gb2);
    uvc::gemm(M->dZ2, H, 1, M->W2h, 1, H, B, H, H, nullptr, false, M->dH1, H, nullptr, 0, s);
    uvc::k_relu_back<<<uvc::blocks((int64_t)B * H), 256, 0, s>>>(M->dH1, M->H1, (int64_t)B * H, M->dZ1);
    // layer 1: gW1 = X^T dZ1, gb1 = colsum dZ1
    uvc::gemm(M->Xh, 1, P, M->dZ1, H, 1, P, H, B, nullptr, false, M->gW1, H, nullptr, 0, s);
    uvc::k_colsum_bf16<<<uvc::blocks(H), 256, 0, s>>>(M->dZ1, B, H, nullptr, M->gb1);
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
    uvc::k_adam<<<uvc::blocks(M->nparam), 256, 0, s>>>(M->param, M->grad, M->m1, M->m2, M->nparam, lr, b1, b2, 1e-8f,
                                                       c1, c2);
    uvc::refresh_bf16(M, s);
    if (loss) cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return uvc::status_from_cuda(cudaGetLastError());
}

int uvc_mlp_grads(const uvc_mlp* M, float* host, int64_t n) {
    if (!M || !host || n != M->nparam) return UVC_E_INVAL;
    return uvc::status_from_cuda(cudaMemcpy(host, M->grad, sizeof(float) * n, cudaMemcpyDeviceToHost));
}

}  // extern "C"
