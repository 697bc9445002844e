// sph_sweep.cuh -- shared pieces of the neighbour sweeps: the cubic-spline kernel, the
// mapping of T threads ("lanes") onto one particle, and the layout of the per-step
// neighbour lists.
//
// Entry k of particle i's list is at k NF + i (k-major: coalesced across a warp for fixed
// k).  The T lanes of a particle share its list: lane s visits entries s, s + T, s + 2T,
// ..., and the T partial sums are combined with warp shuffles.  A warp then holds 32/T
// consecutive particles (about one grid cell at T = 4), whose lists are nearly the same
// particles in the same order, so a warp-wide gather touches one or two cache lines
// instead of four or five, and the lanes' shares differ by at most one entry.  The
// density sweep builds each list cooperatively: the T lanes test T consecutive candidates
// at a time and append the hits in candidate order, so the list is the same for every T.
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

// The two constants of the spline gradient, copied into registers before a list walk (a
// reference into the scene record would let the compiler reload them per pair).
struct Spline {
    float inv_h, kgrad;
    __device__ __forceinline__ explicit Spline(const SceneDev &sc) : inv_h(sc.inv_h), kgrad(sc.kgrad) {}
};

// grad W_ij = factor * x_ij; zero for coincident particles.
__device__ __forceinline__ float grad_factor(const Spline &k, float r2)
{
    if (!(r2 > 0.0f)) return 0.0f;
    float rinv = rsqrtf(r2);
    float q = r2 * rinv * k.inv_h;
    float g = (q <= 0.5f) ? q * fmaf(3.0f, q, -2.0f) : -(fmaxf(1.0f - q, 0.0f) * fmaxf(1.0f - q, 0.0f));
    return k.kgrad * g * rinv;
}
__device__ __forceinline__ float grad_factor(const SceneDev &sc, float r2) { return grad_factor(Spline(sc), r2); }

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

// Mask of the T lanes of this thread's particle within its warp.
template <int T>
__device__ __forceinline__ unsigned group_mask()
{
    return T == 32 ? 0xffffffffu : (((1u << T) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(T - 1)));
}

// Visit this lane's entries s, s + T, ... below n of particle i's list, software-
// pipelined in batches of U: the entries of batch b + 1 are loaded before the visits of
// batch b, whose U gathers the compiler issues together (the visits only accumulate in
// registers), so each batch costs one memory latency.  Prefetches past the end re-read the
// lane's last entry.  NC: the list is read-only for the kernel (read-only data path);
// otherwise plain loads, for a list this warp has just written.  Visiting order = list
// order.
// A read-only list is streamed once per sweep: its loads bypass L1 and are marked first for
// eviction in L2, so that they do not displace the particles' positions and velocities
// (the gathered data, which the sweeps reuse from L2).
__device__ __forceinline__ uint64_t stream_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t *p, uint64_t pol)
{
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

template <int U, int T, bool NC = true, typename F>
__device__ __forceinline__ void for_list(const int32_t *__restrict__ list, int64_t NF, int64_t i, int s, int n,
                                         F &&visit)
{
    const int m = n > s ? (n - s + T - 1) / T : 0;   // this lane's entries
    if (m <= 0) return;
    const uint64_t pol = NC ? stream_policy() : 0ull;
    auto ld = [&](int k) {
        const int64_t a = (int64_t)(s + T * min(k, m - 1)) * NF + i;
        return NC ? ld_stream(list + a, pol) : list[a];
    };
    int32_t j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = ld(u);
    int k = 0;
    for (; k + U <= m; k += U) {
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
        if (k + u < m) visit(j[u]);
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
        else if ((P).lanes == 8) { CALL(8); }  \
        else if ((P).lanes == 2) { CALL(2); }  \
        else { CALL(1); }                      \
    } while (0)
