// sph_mlp.cu -- learned warm start of the constant-density solve (this library's
// addition; the paper has no learned component): a per-particle network
//   y = W3 gelu(W2 gelu(W1 f + b1) + b2) + b3,   f in R^4, hidden 64, exact-erf GELU,
// on standardised features f = (raw - mean) / std; a fraction of the prediction,
// kappa0 = frac max((y std_y + mean_y) 9.81 h, 0), applies where the fluid compresses.
// Both hidden layers run on the tcgen05 tensor cores (BF16 operands, FP32 accumulation
// in tensor memory) for tiles of 128 rows; the 64-wide output dot product runs on the
// CUDA cores while the second layer's accumulators are read back.  The kernels are
// persistent: a CTA allocates its tensor memory and stages the weights once, then walks
// its tiles.  Inside a step only the particles whose gate is open are rows.
//
// Parameter block (float, length kMlpParams): W1[64][4], b1[64], W2[64][64], b2[64],
// W3[64], b3, feature mean[4], feature std[4], label mean, label std.
#include <cuda_bf16.h>

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
constexpr int kMlpParams = kOffSdY + 1;
static_assert(kMlpParams == SPH_MLP_PARAMS, "parameter block layout");

// shared-memory map of one CTA (bytes)
constexpr uint32_t kSmA1 = 0;          // 128 x 16 bf16
constexpr uint32_t kSmB1 = 4096;       // 64 x 16 bf16
constexpr uint32_t kSmA2 = 8192;       // 128 x 64 bf16
constexpr uint32_t kSmB2 = 24576;      // 64 x 64 bf16
constexpr uint32_t kSmVec = 32768;     // b1, b2, w3 (float[64] each)
constexpr uint32_t kSmBar = 33536;     // mbarrier
constexpr uint32_t kSmTmem = 33544;    // tensor-memory address
constexpr uint32_t kSmUsed = 33600;
// requested dynamic shared memory: caps residency at 4 CTAs per SM (4 x (52 + 1) KB of the
// SM's 228 KB; a fifth would need 265), so 4 x 128 tensor-memory columns never exceed 512
constexpr uint32_t kSmRequest = 52 * 1024;
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Store 8 bf16 (one core-matrix row) at tile element (r, k0) of an R x K K-major tile.
__device__ __forceinline__ void store8(unsigned char *tile, uint32_t r, uint32_t k0, uint32_t K, const float *v)
{
    uint4 q = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
    *reinterpret_cast<uint4 *>(tile + tc::tile_offset(r, k0, K)) = q;
}

// One CTA runs the network over 128-row tiles: it allocates its tensor memory and stages
// the weights once, then walks tiles tile0, tile0 + stride, ... < ntiles.  Thread t owns
// row t of a tile; rows.load(tile, t, f) fills the standardised features of that row
// (false: padding, features zero) and rows.store(tile, t, y) receives the standardised
// output y of every valid row.  Returns false if a tensor-core wait gave up (the caller
// flags the error).
template <class Rows>
__device__ bool mlp_tiles(const float *__restrict__ w, unsigned char *sm, int64_t tile0, int64_t ntiles,
                          int64_t stride, Rows &rows)
{
    const int t = threadIdx.x, warp = t >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kSmBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kSmTmem);
    float *b1 = reinterpret_cast<float *>(sm + kSmVec);
    float *b2 = b1 + kH;
    float *w3 = b2 + kH;
    if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
    if (t == 0) tc::mbar_init(bar, 1);
    // layer-1 operand A: row t = (f0..f3, 0 x 12), the zero half written once; B1 row n =
    // W1[n][0..3], 0 x 12; W2 as the layer-2 operand B
    {
        const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        store8(sm + kSmA1, t, 8, 16, z);
        if (t < kH) {
            float u[8] = {w[kOffW1 + t * kF + 0], w[kOffW1 + t * kF + 1], w[kOffW1 + t * kF + 2],
                          w[kOffW1 + t * kF + 3], 0.f, 0.f, 0.f, 0.f};
            store8(sm + kSmB1, t, 0, 16, u);
            store8(sm + kSmB1, t, 8, 16, z);
            b1[t] = w[kOffB1 + t];
            b2[t] = w[kOffB2 + t];
            w3[t] = w[kOffW3 + t];
        }
        for (int idx = t; idx < kH * 8; idx += blockDim.x) {
            const int n = idx >> 3, kc = (idx & 7) * 8;
            float u[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) u[q] = w[kOffW2 + n * kH + kc + q];
            store8(sm + kSmB2, n, kc, kH, u);
        }
    }
    const float b3 = w[kOffB3];
    const uint32_t idesc = tc::idesc_bf16_f32(128, kH);
    const uint32_t sbase = tc::smem_addr(sm);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    bool good = true;
    uint32_t failed_parity = 1;
    uint32_t tmem = 0;
    for (int64_t tile = tile0; tile < ntiles; tile += stride) {
        float f[4];
        const bool valid = rows.load(tile, t, f);
        {
            const float v[8] = {f[0], f[1], f[2], f[3], 0.f, 0.f, 0.f, 0.f};
            store8(sm + kSmA1, t, 0, 16, v);
        }
        // orders this tile's operand writes before the MMA and the previous tile's
        // tensor-memory reads before the accumulators are overwritten; a failed wait of the
        // previous tile ends the walk on every thread
        tc::fence_proxy_async();
        tc::fence_before_sync();
        if (!__syncthreads_and(good)) { failed_parity = 1; break; }
        tc::fence_after_sync();
        tmem = *tmem_slot;
        if (t == 0) {
            // D1[128 x 64] = A1[128 x 16] B1[64 x 16]^T: one K = 16 step
            tc::mma_bf16(tmem, tc::smem_desc(sbase + kSmA1, 128, 256), tc::smem_desc(sbase + kSmB1, 128, 256),
                         idesc, 0);
            tc::mma_commit(bar);
        }
        good = tc::mbar_wait_bounded(bar, 0, kWaitLimit);
        tc::fence_after_sync();
        // hidden layer 1: bias, GELU, BF16 -> layer-2 operand A (row t)
#pragma unroll
        for (int c = 0; c < kH / 16; ++c) {
            float v[16];
            tc::tmem_ld16(tmem + lane_base + c * 16, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = gelu(v[k] + b1[c * 16 + k]);
            store8(sm + kSmA2, t, c * 16, kH, v);
            store8(sm + kSmA2, t, c * 16 + 8, kH, v + 8);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        if (!__syncthreads_and(good)) { failed_parity = 0; break; }
        tc::fence_after_sync();
        if (t == 0) {
            // D2[128 x 64] = A2[128 x 64] W2^T in four K = 16 steps (two core matrices each)
#pragma unroll
            for (int k = 0; k < kH / 16; ++k)
                tc::mma_bf16(tmem + kH, tc::smem_desc(sbase + kSmA2 + k * 256, 128, 1024),
                             tc::smem_desc(sbase + kSmB2 + k * 256, 128, 1024), idesc, k > 0 ? 1u : 0u);
            tc::mma_commit(bar);
        }
        good = tc::mbar_wait_bounded(bar, 1, kWaitLimit);
        tc::fence_after_sync();
        float y = b3;
#pragma unroll
        for (int c = 0; c < kH / 16; ++c) {
            float v[16];
            tc::tmem_ld16(tmem + lane_base + kH + c * 16, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) y = fmaf(w3[c * 16 + k], gelu(v[k] + b2[c * 16 + k]), y);
        }
        if (valid) rows.store(tile, t, y);
    }
    tc::fence_before_sync();
    good = __syncthreads_and(good);
    if (!good && t == 0) {
        // an MMA did not report completion: give it one more bounded wait before the
        // tensor memory is released
        tc::mbar_wait_bounded(bar, failed_parity, kWaitLimit);
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(*tmem_slot, kTmemCols);
    return good;
}

// Rows of the standalone forward: standardised features [n][4] -> y [n].
struct DenseRows {
    const float4 *feat;
    float *y;
    int64_t n;
    __device__ bool load(int64_t tile, int t, float f[4]) const
    {
        const int64_t i = tile * 128 + t;
        if (i >= n) {
            f[0] = f[1] = f[2] = f[3] = 0.f;
            return false;
        }
        const float4 q = feat[i];
        f[0] = q.x; f[1] = q.y; f[2] = q.z; f[3] = q.w;
        return true;
    }
    __device__ void store(int64_t tile, int t, float out) const { y[tile * 128 + t] = out; }
};

__global__ void __launch_bounds__(128) k_mlp_forward(const float *__restrict__ w, const float4 *__restrict__ feat,
                                                     int64_t n, float *__restrict__ y, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    DenseRows rows{feat, y, n};
    const int64_t ntiles = (n + 127) / 128;
    if (!mlp_tiles(w, sm, blockIdx.x, ntiles, gridDim.x, rows) && threadIdx.x == 0) atomicExch(err, 1);
}

// Rows of the learned warm start: the compact list of gated particles (particle, scene)
// that k_warm_density appended; raw features standardised here, the output scaled to
// kappa0 = f max((y std_y + mean_y) 9.81 h, 0) with the scene's fraction f, and written
// with its pressure slot.
struct GatedRows {
    const int2 *list;
    const float4 *feat;
    const SceneDev *scenes;
    float *k0, *ksum;
    float4 *pos_s;
    const float4 *vel_c;
    const float *w;
    int32_t n;
    int32_t i, s;   // the row's particle and scene
    __device__ bool load(int64_t tile, int t, float f[4])
    {
        const int64_t r = tile * 128 + t;
        if (r >= n) {
            f[0] = f[1] = f[2] = f[3] = 0.f;
            return false;
        }
        const int2 e = list[r];
        i = e.x;
        s = e.y;
        const float4 q = feat[i];
        f[0] = (q.x - w[kOffMuF + 0]) / w[kOffSdF + 0];
        f[1] = (q.y - w[kOffMuF + 1]) / w[kOffSdF + 1];
        f[2] = (q.z - w[kOffMuF + 2]) / w[kOffSdF + 2];
        f[3] = (q.w - w[kOffMuF + 3]) / w[kOffSdF + 3];
        return true;
    }
    __device__ void store(int64_t, int, float y) const
    {
        const SceneDev &sc = scenes[s];
        const float k = sc.learned_frac * fmaxf((y * w[kOffSdY] + w[kOffMuY]) * 9.81f * sc.h, 0.0f);
        k0[i] = k;
        ksum[i] = k;
        reinterpret_cast<float *>(pos_s + i)[3] = k / vel_c[i].w;
    }
};

// Learned warm start inside a step: a persistent grid over the gated rows (their count
// is known only on the device).
__global__ void __launch_bounds__(128) k_mlp_warm(Ptrs P)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    kernel_enter(P.ctl, KID_MLP_WARM);
    const int32_t n = P.ctl->mlp_n;
    const int64_t ntiles = (n + 127) / 128;
    if (!P.ctl->have_mlp || (int64_t)blockIdx.x >= ntiles) return;  // uniform per block
    GatedRows rows{P.mlp_rows, reinterpret_cast<const float4 *>(P.feat), P.scenes, P.k0, P.ksum, P.pos_s, P.vel_c,
                   P.mlp_w, n, 0, 0};
    if (!mlp_tiles(P.mlp_w, sm, blockIdx.x, ntiles, gridDim.x, rows) && threadIdx.x == 0)
        atomicExch(&P.ctl->error, 4);
}

// Resident CTAs of the network kernels per SM: the shared-memory request caps it, so that
// their tensor-memory columns (128 each) never exceed the SM's 512.
constexpr int kMlpCtasPerSm = 4;

int mlp_grid(int64_t tiles)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
            nsm = 1;
    }
    const int64_t g = (int64_t)nsm * kMlpCtasPerSm;
    return (int)(tiles < g ? (tiles > 0 ? tiles : 1) : g);
}

}  // namespace

void launch_mlp_warm(const Ptrs &P, cudaStream_t s)
{
    k_mlp_warm<<<mlp_grid((P.nlearned + 127) / 128), 128, kSmRequest, s>>>(P);
}

cudaError_t mlp_prepare_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_mlp_warm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmRequest);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmRequest);
}

}  // namespace sph

using namespace sph;

extern "C" sph_status sph_mlp_forward(const float *params, const float *features, int64_t n, float *y, int32_t *error,
                                      void *stream)
{
    if (n < 0 || (n > 0 && (!params || !features || !y || !error))) return SPH_EINVAL;
    if (n == 0) return SPH_OK;
    if (mlp_prepare_kernels() != cudaSuccess) return SPH_ECUDA;
    k_mlp_forward<<<mlp_grid((n + 127) / 128), 128, kSmRequest, (cudaStream_t)stream>>>(
        params, reinterpret_cast<const float4 *>(features), n, y, reinterpret_cast<int *>(error));
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
}
