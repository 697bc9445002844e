// sph_mlp_train.cu -- training of the warm-start network on the GPU: forward and backward
// of the mean-squared error on tcgen05 tensor cores (BF16 operands, FP32 accumulation in
// tensor memory), Adam updates of the FP32 master weights, and the feature / label
// standardisation statistics.  Per CTA, 128 samples:
//   forward   D1 = F W1^T, a1 = gelu(z1);  D2 = a1 W2^T, a2 = gelu(z2);  y = a2 . W3 + b3
//   backward  dy = 2 (y - t) / B;  delta2 = dy W3 gelu'(z2);  D3 = delta2 W2 (-> delta1)
//             dW2 = delta2^T a1 and dW1 = delta1^T F as MMAs over the sample dimension
//             (the 64 weight rows padded to the 128-row MMA shape)
// Gradients are accumulated across CTAs with FP32 atomics (training does not need a
// bit-reproducible order); the loss sum in FP64.
#include <cuda_bf16.h>

#include <algorithm>

#include "sph.h"
#include "sph_internal.cuh"
#include "sph_tc.cuh"

namespace sph {

namespace {

constexpr int kH = 64;
constexpr int kF = 4;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH * kF;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
constexpr int kNW = kOffB3 + 1;
constexpr int kOffMuF = kNW;
constexpr int kOffSdF = kOffMuF + kF;
constexpr int kOffMuY = kOffSdF + kF;
constexpr int kOffSdY = kOffMuY + 1;
static_assert(kOffSdY + 1 == SPH_MLP_PARAMS, "parameter block layout");
static_assert(kNW == SPH_MLP_WEIGHTS, "weight count");

// shared-memory map (bytes); every operand tile starts on a 1 KB boundary
constexpr uint32_t kA1 = 0;          // 128 x 16   features (samples x k)
constexpr uint32_t kB1 = 4096;       // 64 x 16    W1
constexpr uint32_t kA2 = 8192;       // 128 x 64   a1 (samples x k)
constexpr uint32_t kB2 = 24576;      // 64 x 64    W2 (o x k)
constexpr uint32_t kB2T = 32768;     // 64 x 64    W2^T (k x o)
constexpr uint32_t kAD2 = 40960;     // 128 x 64   delta2 (samples x o)
constexpr uint32_t kAD2T = 57344;    // 128 x 128  delta2^T (o x samples), rows 64.. zero
constexpr uint32_t kBA1T = 90112;    // 64 x 128   a1^T (k x samples)
constexpr uint32_t kAD1T = 106496;   // 128 x 128  delta1^T (k x samples), rows 64.. zero
constexpr uint32_t kBFT = 139264;    // 16 x 128   F^T (k x samples), rows 4.. zero
constexpr uint32_t kVec = 143360;    // b1, b2, w3 (float[64] each)
constexpr uint32_t kRed = 144128;    // reductions: dW3[64], db2[64], db1[64], db3, loss
constexpr uint32_t kBar = 145152;
constexpr uint32_t kTmemSlot = 145160;
constexpr uint32_t kSmem = 146 * 1024;
constexpr uint32_t kCols = 256;
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ void store8(unsigned char *tile, uint32_t r, uint32_t k0, uint32_t K, const float *v)
{
    *reinterpret_cast<uint4 *>(tile + tc::tile_offset(r, k0, K)) =
        make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}
__device__ __forceinline__ void store1(unsigned char *tile, uint32_t r, uint32_t k, uint32_t K, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(tile + tc::tile_offset(r, k, K)) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ void sync_for_mma()
{
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Index of the sample in row r of batch position p: a bijection of [0, n) per epoch.
__device__ __forceinline__ int64_t permute(int64_t p, int64_t n, uint64_t a, uint64_t c)
{
    return (int64_t)(((uint64_t)p * a + c) % (uint64_t)n);
}

// Gradient of the batch's mean squared error (standardised features and labels).
__global__ void __launch_bounds__(128) k_mlp_grad(const float *__restrict__ w, const float4 *__restrict__ F,
                                                  const float *__restrict__ T, int64_t n, int64_t batch_begin,
                                                  int64_t batch_size, uint64_t pa, uint64_t pc, float *grad,
                                                  double *loss, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int t = threadIdx.x, warp = t >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kBar);
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kTmemSlot);
    float *vb1 = reinterpret_cast<float *>(sm + kVec), *vb2 = vb1 + kH, *vw3 = vb2 + kH;
    float *rw3 = reinterpret_cast<float *>(sm + kRed), *rb2 = rw3 + kH, *rb1 = rb2 + kH, *rb3 = rb1 + kH;
    float *rloss = rb3 + 1;

    const int64_t pos = (int64_t)blockIdx.x * 128 + t;
    const bool valid = pos < batch_size && batch_begin + pos < n;
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    float target = 0.0f;
    if (valid) {
        const int64_t s = permute(batch_begin + pos, n, pa, pc);
        const float4 q = F[s];
        f[0] = q.x; f[1] = q.y; f[2] = q.z; f[3] = q.w;
        target = T[s];
    }
    if (warp == 0) tc::tmem_alloc(slot, kCols);
    if (t == 0) tc::mbar_init(bar, 1);
    // zero the padded halves and stage the operands
    for (uint32_t o = t * 16; o < 16384; o += 128 * 16) {
        *reinterpret_cast<uint4 *>(sm + kAD2T + 16384 + o) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4 *>(sm + kAD1T + 16384 + o) = make_uint4(0, 0, 0, 0);
    }
    for (uint32_t o = t * 16; o < 4096; o += 128 * 16) *reinterpret_cast<uint4 *>(sm + kBFT + o) = make_uint4(0, 0, 0, 0);
    for (int k = t; k < 3 * kH + 2; k += 128) rw3[k] = 0.0f;
    __syncthreads();
    {
        const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float v[8] = {f[0], f[1], f[2], f[3], 0.f, 0.f, 0.f, 0.f};
        store8(sm + kA1, t, 0, 16, v);
        store8(sm + kA1, t, 8, 16, z8);
        for (int k = 0; k < 4; ++k) store1(sm + kBFT, k, t, 128, f[k]);
        if (t < kH) {
            float u[8] = {w[kOffW1 + 4 * t], w[kOffW1 + 4 * t + 1], w[kOffW1 + 4 * t + 2], w[kOffW1 + 4 * t + 3],
                          0.f, 0.f, 0.f, 0.f};
            store8(sm + kB1, t, 0, 16, u);
            store8(sm + kB1, t, 8, 16, z8);
            vb1[t] = w[kOffB1 + t];
            vb2[t] = w[kOffB2 + t];
            vw3[t] = w[kOffW3 + t];
        }
        for (int idx = t; idx < kH * 8; idx += 128) {
            const int r = idx >> 3, kc = (idx & 7) * 8;
            float u[8], ut[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                u[q] = w[kOffW2 + r * kH + kc + q];          // W2[r][kc+q]
                ut[q] = w[kOffW2 + (kc + q) * kH + r];       // W2^T[r][kc+q] = W2[kc+q][r]
            }
            store8(sm + kB2, r, kc, kH, u);
            store8(sm + kB2T, r, kc, kH, ut);
        }
    }
    sync_for_mma();
    const uint32_t tmem = *slot;
    const uint32_t sb = tc::smem_addr(sm);
    const uint32_t id64 = tc::idesc_bf16_f32(128, 64), id16 = tc::idesc_bf16_f32(128, 16);
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    bool good = true;
    uint32_t phase = 0;
    auto wait_mma = [&]() {
        good = tc::mbar_wait_bounded(bar, phase & 1u, kWaitLimit) && good;
        ++phase;
        tc::fence_after_sync();
    };
    // layer 1 -> tensor-memory columns [0, 64)
    if (t == 0) {
        tc::mma_bf16(tmem, tc::smem_desc(sb + kA1, 128, 256), tc::smem_desc(sb + kB1, 128, 256), id64, 0);
        tc::mma_commit(bar);
    }
    wait_mma();
    for (int c = 0; c < 4; ++c) {
        float v[16];
        tc::tmem_ld16(tmem + lanes + c * 16, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[k] = gelu(v[k] + vb1[c * 16 + k]);
            store1(sm + kBA1T, c * 16 + k, t, 128, v[k]);
        }
        store8(sm + kA2, t, c * 16, kH, v);
        store8(sm + kA2, t, c * 16 + 8, kH, v + 8);
    }
    sync_for_mma();
    // layer 2 -> columns [64, 128)
    if (t == 0) {
        for (int k = 0; k < 4; ++k)
            tc::mma_bf16(tmem + 64, tc::smem_desc(sb + kA2 + k * 256, 128, 1024),
                         tc::smem_desc(sb + kB2 + k * 256, 128, 1024), id64, k > 0);
        tc::mma_commit(bar);
    }
    wait_mma();
    float y = w[kOffB3];
    for (int c = 0; c < 4; ++c) {
        float v[16];
        tc::tmem_ld16(tmem + lanes + 64 + c * 16, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) y = fmaf(vw3[c * 16 + k], gelu(v[k] + vb2[c * 16 + k]), y);
    }
    const float inv_b = 1.0f / (float)batch_size;
    const float e = valid ? (y - target) : 0.0f;
    const float dy = 2.0f * e * inv_b;
    atomicAdd(rloss, e * e);
    atomicAdd(rb3, dy);
    for (int c = 0; c < 4; ++c) {
        float v[16], d[16];
        tc::tmem_ld16(tmem + lanes + 64 + c * 16, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int o = c * 16 + k;
            const float z = v[k] + vb2[o];
            d[k] = dy * vw3[o] * gelu_d(z);
            atomicAdd(&rw3[o], dy * gelu(z));
            atomicAdd(&rb2[o], d[k]);
            store1(sm + kAD2T, o, t, 128, d[k]);
        }
        store8(sm + kAD2, t, c * 16, kH, d);
        store8(sm + kAD2, t, c * 16 + 8, kH, d + 8);
    }
    sync_for_mma();
    // delta2 W2 -> columns [128, 192)
    if (t == 0) {
        for (int k = 0; k < 4; ++k)
            tc::mma_bf16(tmem + 128, tc::smem_desc(sb + kAD2 + k * 256, 128, 1024),
                         tc::smem_desc(sb + kB2T + k * 256, 128, 1024), id64, k > 0);
        tc::mma_commit(bar);
    }
    wait_mma();
    for (int c = 0; c < 4; ++c) {
        float g[16], z[16];
        tc::tmem_ld16(tmem + lanes + 128 + c * 16, g);
        tc::tmem_ld16(tmem + lanes + c * 16, z);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int o = c * 16 + k;
            const float d1 = g[k] * gelu_d(z[k] + vb1[o]);
            atomicAdd(&rb1[o], d1);
            store1(sm + kAD1T, o, t, 128, d1);
        }
    }
    sync_for_mma();
    // dW2 = delta2^T a1 -> columns [192, 256); dW1 = delta1^T F -> columns [0, 16)
    if (t == 0) {
        for (int k = 0; k < 8; ++k)
            tc::mma_bf16(tmem + 192, tc::smem_desc(sb + kAD2T + k * 256, 128, 2048),
                         tc::smem_desc(sb + kBA1T + k * 256, 128, 2048), id64, k > 0);
        for (int k = 0; k < 8; ++k)
            tc::mma_bf16(tmem, tc::smem_desc(sb + kAD1T + k * 256, 128, 2048),
                         tc::smem_desc(sb + kBFT + k * 256, 128, 2048), id16, k > 0);
        tc::mma_commit(bar);
    }
    wait_mma();
    if (warp < 2) {                                   // rows 0..63 hold the 64 weight rows
        const int o = t;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tc::tmem_ld16(tmem + lanes + 192 + c * 16, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) atomicAdd(&grad[kOffW2 + o * kH + c * 16 + k], v[k]);
        }
        float v[16];
        tc::tmem_ld16(tmem + lanes, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(&grad[kOffW1 + o * kF + k], v[k]);
    }
    __syncthreads();
    if (t < kH) {
        atomicAdd(&grad[kOffW3 + t], rw3[t]);
        atomicAdd(&grad[kOffB2 + t], rb2[t]);
        atomicAdd(&grad[kOffB1 + t], rb1[t]);
    }
    if (t == 0) {
        atomicAdd(&grad[kOffB3], *rb3);
        atomicAdd(loss, (double)*rloss);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (!good && t == 0) {
        tc::mbar_wait_bounded(bar, (phase - 1) & 1u, kWaitLimit);
        atomicExch(err, 1);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// Adam (Kingma & Ba) on the FP32 master weights; clears the gradient.
__global__ void k_mlp_adam(float *w, float *m, float *v, float *grad, int64_t step, float lr, float b1, float b2,
                           float eps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNW) return;
    const float g = grad[k];
    grad[k] = 0.0f;
    const float mk = b1 * m[k] + (1.0f - b1) * g;
    const float vk = b2 * v[k] + (1.0f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Mean and standard deviation of the raw features and labels (FP64 sums).
__global__ void k_mlp_moments(const float4 *__restrict__ F, const float *__restrict__ T, int64_t n, double *acc)
{
    double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = F[i];
        const double x[5] = {q.x, q.y, q.z, q.w, T[i]};
        for (int a = 0; a < 5; ++a) {
            s[a] += x[a];
            s[5 + a] += x[a] * x[a];
        }
    }
    for (int a = 0; a < 10; ++a) {
        double r = s[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc[a], r);
    }
}

__global__ void k_mlp_standardise(const float4 *__restrict__ F, const float *__restrict__ T, int64_t n,
                                  const double *acc, float *params, float4 *Fs, float *Ts)
{
    __shared__ float mu[5], sd[5];
    if (threadIdx.x < 5) {
        const double m = acc[threadIdx.x] / (double)n;
        double var = acc[5 + threadIdx.x] / (double)n - m * m;
        double s = var > 0.0 ? sqrt(var) : 0.0;
        if (!(s > 1e-12 * (fabs(m) + 1.0))) s = 1.0;   // a constant column is left unscaled
        mu[threadIdx.x] = (float)m;
        sd[threadIdx.x] = (float)s;
        if (blockIdx.x == 0) {
            if (threadIdx.x < 4) {
                params[kOffMuF + threadIdx.x] = (float)m;
                params[kOffSdF + threadIdx.x] = (float)s;
            } else {
                params[kOffMuY] = (float)m;
                params[kOffSdY] = (float)s;
            }
        }
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = F[i];
        Fs[i] = make_float4((q.x - mu[0]) / sd[0], (q.y - mu[1]) / sd[1], (q.z - mu[2]) / sd[2], (q.w - mu[3]) / sd[3]);
        Ts[i] = (T[i] - mu[4]) / sd[4];
    }
}

__global__ void k_epoch_loss(double *acc, float *out, int64_t n)
{
    *out = (float)(*acc / (double)n);
    *acc = 0.0;
}

uint64_t mix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) {
        uint64_t r = a % b;
        a = b;
        b = r;
    }
    return a;
}

cudaError_t set_attr()
{
    return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

}  // namespace

}  // namespace sph

using namespace sph;

extern "C" sph_status sph_mlp_grad(const float *params, const float *features, const float *labels, int64_t n,
                                   float *grad, double *loss, int32_t *error, void *stream)
{
    if (n <= 0 || !params || !features || !labels || !grad || !loss || !error) return SPH_EINVAL;
    if ((n + 127) / 128 > 0x7fffffff) return SPH_EINVAL;
    if (set_attr() != cudaSuccess) return SPH_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * kNW, s) != cudaSuccess) return SPH_ECUDA;
    if (cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return SPH_ECUDA;
    k_mlp_grad<<<(unsigned)((n + 127) / 128), 128, kSmem, s>>>(params, reinterpret_cast<const float4 *>(features),
                                                               labels, n, 0, n, 1, 0, grad, loss,
                                                               reinterpret_cast<int *>(error));
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
}

extern "C" sph_status sph_mlp_train(const float *features, const float *labels, int64_t n, float *params,
                                    float *adam_state, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                    float *loss_history, int32_t *error, void *stream)
{
    if (n < 2 || !features || !labels || !params || !adam_state || !error || epochs < 0 || batch < 1 ||
        !(lr > 0.0f))
        return SPH_EINVAL;
    if (set_attr() != cudaSuccess) return SPH_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    float4 *Fs = nullptr;
    float *Ts = nullptr, *grad = nullptr;
    double *acc = nullptr;
    auto cleanup = [&]() {
        if (Fs) cudaFreeAsync(Fs, s);
        if (Ts) cudaFreeAsync(Ts, s);
        if (grad) cudaFreeAsync(grad, s);
        if (acc) cudaFreeAsync(acc, s);
    };
    if (cudaMallocAsync(&Fs, sizeof(float4) * n, s) != cudaSuccess || cudaMallocAsync(&Ts, sizeof(float) * n, s) != cudaSuccess ||
        cudaMallocAsync(&grad, sizeof(float) * kNW, s) != cudaSuccess ||
        cudaMallocAsync(&acc, sizeof(double) * 12, s) != cudaSuccess) {
        cleanup();
        return SPH_ENOMEM;
    }
    bool ok = cudaMemsetAsync(acc, 0, sizeof(double) * 12, s) == cudaSuccess &&
              cudaMemsetAsync(grad, 0, sizeof(float) * kNW, s) == cudaSuccess;
    const float4 *F = reinterpret_cast<const float4 *>(features);
    k_mlp_moments<<<304, 256, 0, s>>>(F, labels, n, acc);
    k_mlp_standardise<<<304, 256, 0, s>>>(F, labels, n, acc, params, Fs, Ts);
    cudaMemsetAsync(acc, 0, sizeof(double) * 12, s);
    float *m = adam_state, *v = adam_state + kNW;
    int64_t step = 0;
    const int64_t B = batch;
    for (int32_t e = 0; e < epochs && ok; ++e) {
        // a fresh bijection of the samples for this epoch
        uint64_t a = mix64(seed * 0x100000001B3ull + (uint64_t)e) % (uint64_t)(n - 1) + 1;
        while (gcd64(a, (uint64_t)n) != 1) a = a % (uint64_t)(n - 1) + 1;
        const uint64_t c = mix64(seed ^ (0xA5A5A5A5ull + (uint64_t)e)) % (uint64_t)n;
        for (int64_t b0 = 0; b0 < n; b0 += B) {
            const int64_t bs = std::min<int64_t>(B, n - b0);
            k_mlp_grad<<<(unsigned)((bs + 127) / 128), 128, kSmem, s>>>(params, Fs, Ts, n, b0, bs, a, c, grad, acc,
                                                                        reinterpret_cast<int *>(error));
            ++step;
            k_mlp_adam<<<(kNW + 255) / 256, 256, 0, s>>>(params, m, v, grad, step, lr, 0.9f, 0.999f, 1e-8f);
        }
        if (loss_history) k_epoch_loss<<<1, 1, 0, s>>>(acc, loss_history + e, n);
        ok = cudaGetLastError() == cudaSuccess;
    }
    cleanup();
    return ok && cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
}
