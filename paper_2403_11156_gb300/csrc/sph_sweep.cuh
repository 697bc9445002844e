// sph_sweep.cuh -- shared pieces of the neighbour sweeps: the cubic-spline kernel, the
// mapping of T threads ("lanes") onto one particle, and the layout of the per-step
// neighbour lists.
//
// With T lanes per particle, the particle's neighbours are split into T sub-lists: lane s
// records the candidates jb + s, jb + s + T, ... of every stencil row, and every later
// sweep has lane s visit sub-list s, the T partial sums being combined with warp
// shuffles.  A warp then holds 32/T consecutive particles (one or two grid cells), whose
// k-th neighbours are nearly the same particles, so each warp-wide gather touches one or
// two cache lines; small scenes also get T times more threads.
// Entry k of sub-list s of particle i is at ((k NF) + i) T + s (coalesced across a warp
// for fixed k); the T sub-list lengths are packed in one uint32 per particle, 8 bits each.
#pragma once

#include "sph_internal.cuh"

namespace sph {

// Cubic spline (Sec. 3.2 with h = 4r, Sec. 5): W = sigma w(q), grad W = kgrad g(q) x/|x|.
__device__ __forceinline__ float spline_w(float q)
{
    if (q <= 0.5f) return fmaf(6.0f * q, q * q, fmaf(-6.0f * q, q, 1.0f));
    float t = fmaxf(1.0f - q, 0.0f);
    return 2.0f * t * t * t;
}

// grad W_ij = factor * x_ij; zero for coincident particles.
__device__ __forceinline__ float grad_factor(const SceneDev &sc, float r2)
{
    if (!(r2 > 0.0f)) return 0.0f;
    float rinv = rsqrtf(r2);
    float q = r2 * rinv * sc.inv_h;
    float g = (q <= 0.5f) ? q * fmaf(3.0f, q, -2.0f) : -(fmaxf(1.0f - q, 0.0f) * fmaxf(1.0f - q, 0.0f));
    return sc.kgrad * g * rinv;
}

template <int T>
struct Lane {
    const SceneDev *sc;
    SceneState *st;
    int64_t i;    // particle (global index)
    int s;        // lane within the particle's group
    bool valid;
};

// Particle and lane of this thread in a sweep launched over the sweep-block table.
template <int T>
__device__ __forceinline__ Lane<T> lane_ctx(const Ptrs &P)
{
    Lane<T> c;
    const int32_t sidx = P.tblk_scene[blockIdx.x];
    c.sc = &P.scenes[sidx];
    c.st = &P.st[sidx];
    const int64_t local = (int64_t)(blockIdx.x - c.sc->tblk_first) * (kBlock / T) + threadIdx.x / T;
    c.s = (int)(threadIdx.x % T);
    c.valid = local < c.sc->nf;
    c.i = c.sc->f_off + local;
    return c;
}

// Sum over the T lanes of a particle; every thread of the warp must call it.
template <int T, typename V>
__device__ __forceinline__ V group_sum(V v)
{
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sub-list lengths are packed 32/T bits each (T = 1: the plain count).
template <int T>
__device__ __forceinline__ uint32_t lane_mask()
{
    return T == 1 ? 0xFFFFFFFFu : ((1u << (32 / T)) - 1u);
}
template <int T>
__device__ __forceinline__ int lane_count(int32_t packed, int s)
{
    return (int)(((uint32_t)packed >> ((32 / T) * s)) & lane_mask<T>());
}
template <int T>
__device__ __forceinline__ uint32_t lane_pack(int n, int s)
{
    return (uint32_t)n << ((32 / T) * s);
}

template <int T>
__device__ __forceinline__ int64_t list_at(int64_t NF, int64_t i, int k, int s)
{
    return ((int64_t)k * NF + i) * T + s;
}

// Visit entries [0, n) of sub-list s of particle i, software-pipelined in batches of U:
// the indices of batch b + 1 are loaded before the visits of batch b, whose U gathers the
// compiler issues together (the visits only accumulate in registers), so each batch costs
// one memory latency instead of two.  Prefetches past the end re-read entry n - 1.  NC:
// the list is read-only for the kernel (read-only data path); otherwise plain loads, for
// a list this thread has just written.  Visiting order = list order.
template <int U, int T, bool NC = true, typename F>
__device__ __forceinline__ void for_list(const int32_t *__restrict__ list, int64_t NF, int64_t i, int s, int n,
                                         F &&visit)
{
    if (n <= 0) return;
    auto ld = [&](int k) {
        const int64_t a = list_at<T>(NF, i, min(k, n - 1), s);
        return NC ? __ldg(list + a) : list[a];
    };
    int32_t j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = ld(u);
    int k = 0;
    for (; k + U <= n; k += U) {
        int32_t jn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) jn[u] = ld(k + U + u);
#pragma unroll
        for (int u = 0; u < U; ++u) visit(j[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) j[u] = jn[u];
    }
#pragma unroll
    for (int u = 0; u < U - 1; ++u)
        if (k + u < n) visit(j[u]);
}

// Visit the candidates j0, j0 + T, ... below je of a grid row in batches of U: the U
// position loads of a batch are issued before any visit, in index order.
template <int U, int T, typename F>
__device__ __forceinline__ void for_range(const float4 *__restrict__ pos, uint32_t j0, uint32_t je, F &&visit)
{
    uint32_t j = j0;
    for (; j + (uint32_t)((U - 1) * T) < je; j += (uint32_t)(U * T)) {
        float4 p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) p[u] = __ldg(pos + j + u * T);
#pragma unroll
        for (int u = 0; u < U; ++u) visit(j + (uint32_t)(u * T), p[u]);
    }
    for (; j < je; j += (uint32_t)T) visit(j, __ldg(pos + j));
}

}  // namespace sph

// Instantiate CALL(T) for the context's threads per particle.
#define SPH_BY_LANES(P, CALL)                  \
    do {                                       \
        if ((P).lanes == 4) { CALL(4); }       \
        else if ((P).lanes == 2) { CALL(2); }  \
        else { CALL(1); }                      \
    } while (0)
