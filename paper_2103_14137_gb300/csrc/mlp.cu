// Candidate scorer of the learned proposal: a 3-layer perceptron
//   x (in) -> relu(x W1 + b1) (H) -> relu(. W2 + b2) (H) -> . w3 + b3 (logit)
// with BF16 weights and activations and FP32 accumulation, trained with
// binary cross-entropy on LP dwell-time labels (candidate kept by the relaxed
// LP (9) or not) and Adam.  The dense products run on the tensor cores
// (mma.sync m16n8k16 BF16 -> FP32) through one GEMM kernel whose operands are
// read with arbitrary strides, so the forward pass, the weight gradients
// (X^T dZ) and the input gradients (dZ W^T) all use it.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

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

constexpr int BM = 64, BN = 64, BK = 32, kGemmThreads = 128;

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]) (relu), A(m,k) = Ap[m*sam + k*sak],
// B(k,n) = Bp[k*sbk + n*sbn]; writes fp32 C (ldc) and/or bf16 Ch (ldh).
__global__ void __launch_bounds__(kGemmThreads) k_gemm(const __nv_bfloat16* __restrict__ Ap, int64_t sam,
                                                       int64_t sak, const __nv_bfloat16* __restrict__ Bp,
                                                       int64_t sbk, int64_t sbn, int M, int N, int K,
                                                       const float* __restrict__ bias, int relu, float* C,
                                                       int64_t ldc, __nv_bfloat16* Ch, int64_t ldh) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + 8];
    __shared__ __align__(16) __nv_bfloat16 Bt[BN][BK + 8];   // B transposed: Bt[n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, t4 = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += kGemmThreads) {
            const int r = e / BK, c = e % BK;
            const int m = m0 + r, k = k0 + c;
            As[r][c] = (m < M && k < K) ? Ap[(int64_t)m * sam + (int64_t)k * sak] : zero;
        }
        for (int e = tid; e < BN * BK; e += kGemmThreads) {
            const int r = e / BK, c = e % BK;   // r = n, c = k
            const int n = n0 + r, k = k0 + c;
            Bt[r][c] = (n < N && k < K) ? Bp[(int64_t)k * sbk + (int64_t)n * sbn] : zero;
        }
        __syncthreads();
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm * 32 + mi * 16 + g, c = kk + t4 * 2;
                af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r][c]);
                af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c]);
                af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r][c + 8]);
                af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c + 8]);
            }
            for (int ni = 0; ni < 4; ++ni) {
                const int n = wn * 32 + ni * 8 + g, c = kk + t4 * 2;
                bf[ni][0] = *reinterpret_cast<const uint32_t*>(&Bt[n][c]);
                bf[ni][1] = *reinterpret_cast<const uint32_t*>(&Bt[n][c + 8]);
            }
            for (int mi = 0; mi < 2; ++mi)
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bf[ni]);
        }
        __syncthreads();
    }
    for (int mi = 0; mi < 2; ++mi)
        for (int ni = 0; ni < 4; ++ni)
            for (int h = 0; h < 2; ++h)
                for (int q = 0; q < 2; ++q) {
                    const int m = m0 + wm * 32 + mi * 16 + g + 8 * h;
                    const int n = n0 + wn * 32 + ni * 8 + t4 * 2 + q;
                    if (m >= M || n >= N) continue;
                    float v = acc[mi][ni][2 * h + q];
                    if (bias) v += bias[n];
                    if (relu) v = fmaxf(v, 0.f);
                    if (C) C[(int64_t)m * ldc + n] = v;
                    if (Ch) Ch[(int64_t)m * ldh + n] = __float2bfloat16(v);
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
