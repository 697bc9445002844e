// sph_visc.cu -- implicit viscosity (Sec. 3.6.2): (I - dt A) v* = v~ solved by a
// matrix-free conjugate gradient (Sec. 4.2 "conjugate gradient (matrix free)").
//
//   (A v)_i = sum_j A_ij (v_j - v_i),
//   A_ij = -2(d+2) mu mbar_ij / (rho_i rho_j) grad W_ij x_ij^T / (|x_ij|^2 + 0.01 h^2),
// d = 3, mbar = m (one particle mass per scene), mu = nu rho0.  The operator is applied
// on the fly from the neighbour lists; the CG vectors live in float4 arrays whose w lane
// keeps rho so that one gather serves both.  Dot products are accumulated per block in
// FP64 and summed per scene in a fixed order: the initial residual by the last block of
// each scene, the two products of an iteration by one-block kernels (alpha after the
// matrix sweep, beta and the stopping test after the update), so the wide kernels of the
// loop only write partials.  The loop runs on the device (CUDA graph while node) until
// |r| <= tol |b| or cg_max_iter.
#include "sph_sweep.cuh"

namespace sph {

namespace {

struct Ctx {
    const SceneDev *sc;
    SceneState *st;
    int64_t i;
    bool valid;
};

__device__ __forceinline__ Ctx ctx(const Ptrs &P)
{
    Ctx c;
    int32_t s = P.fblk_scene[blockIdx.x];
    c.sc = &P.scenes[s];
    c.st = &P.st[s];
    int64_t local = (int64_t)(blockIdx.x - c.sc->fblk_first) * kBlock + threadIdx.x;
    c.valid = local < c.sc->nf;
    c.i = c.sc->f_off + local;
    return c;
}

// y = (I - dt A) x at particle i from T lanes (every thread of the warp calls it; the
// result is valid in lanes of valid particles); X holds x in xyz and rho in w.
template <int T>
__device__ __forceinline__ float3 apply_m(const Ptrs &P, const SceneDev &sc, const Lane<T> &c, float4 pi,
                                          float4 xi, const float4 *__restrict__ X, float dt)
{
    const int64_t NF = P.NF, i = c.i;
    const float reg = 0.01f * sc.h2;
    const Spline sp(sc);
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    if (c.valid) {
        for_list<4, T>(P.nbr, NF, i, c.s, P.nnf[i], [&](int32_t j) {
            const float4 pj = __ldg(P.pos_s + j);
            const float4 xj = __ldg(X + j);
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            // grad W_ij (x_ij . (x_j - x_i)) / (rho_j (r^2 + reg))
            const float q = grad_factor(sp, r2) * (dx * (xj.x - xi.x) + dy * (xj.y - xi.y) + dz * (xj.z - xi.z)) /
                            (xj.w * (r2 + reg));
            ax = fmaf(q, dx, ax); ay = fmaf(q, dy, ay); az = fmaf(q, dz, az);
        });
    }
    ax = group_sum<T>(ax); ay = group_sum<T>(ay); az = group_sum<T>(az);
    // (A x)_i = -10 mu m / rho_i * acc, so (I - dt A) x = x + dt 10 mu m / rho_i * acc
    const float k = c.valid ? dt * 10.0f * sc.mu * sc.m / xi.w : 0.0f;
    return make_float3(fmaf(k, ax, xi.x), fmaf(k, ay, xi.y), fmaf(k, az, xi.z));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sums of two doubles (result in thread 0).
__device__ void block_sum2(double &a, double &b, double *sh)
{
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[2 * w] = a;
        sh[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) {
            a += sh[2 * k];
            b += sh[2 * k + 1];
        }
    }
}

// Per-block partial sums, then the scene's last block sums them in block order (the
// scene's blocks are [first, first + count) of the launch).  Returns true in thread 0 of
// the last block, with the totals in a and b.
__device__ bool scene_reduce2(const Ptrs &P, int32_t first, int32_t count, SceneState &st, double &a, double &b,
                              double *sh, int *s_last)
{
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) {
        P.cg_dots[2 * blockIdx.x] = a;
        P.cg_dots[2 * blockIdx.x + 1] = b;
        __threadfence();
        uint32_t prev = atomicAdd(&st.counter, 1u);
        *s_last = (prev == (uint32_t)count - 1u);
    }
    __syncthreads();
    if (!*s_last) return false;
    __threadfence();
    const double2 *d = reinterpret_cast<const double2 *>(P.cg_dots) + first;
    double ta = 0.0, tb = 0.0;
#pragma unroll 8
    for (int k = threadIdx.x; k < count; k += kBlock) {
        const double2 v = __ldcg(d + k);
        ta += v.x;
        tb += v.y;
    }
    block_sum2(ta, tb, sh);
    a = ta;
    b = tb;
    if (threadIdx.x == 0) st.counter = 0;
    return threadIdx.x == 0;
}

__device__ __forceinline__ bool cg_active(const SceneDev &sc, const SceneState &st)
{
    return sc.visc_mode == 3 && st.cg_active != 0;
}

// Per-block partial sums of two doubles, written for a later one-block reduction.
__device__ __forceinline__ void block_partials2(const Ptrs &P, double a, double b, double *sh)
{
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) {
        P.cg_dots[2 * blockIdx.x] = a;
        P.cg_dots[2 * blockIdx.x + 1] = b;
    }
}

constexpr int kReduceThreads = 1024;

// One block (kReduceThreads threads) sums, per scene with an active CG, the block partials
// of the preceding launch over the scene's sweep blocks (SWEEP) or fluid blocks, in a fixed
// order that depends only on the scene (thread t takes partials t, t + 1024, ..., then a
// fixed tree), so a scene reduces the same way alone and in any batch; the scenes go in
// turn.  done(scene, a, b) runs in one thread per scene.
template <bool SWEEP, typename F>
__device__ void reduce_scenes(const Ptrs &P, double *sh, F &&done)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double2 *d = reinterpret_cast<const double2 *>(P.cg_dots);
    for (int q = 0; q < P.nscenes; ++q) {
        const SceneDev &qd = P.scenes[q];
        if (!cg_active(qd, P.st[q])) continue;   // uniform: nothing wrote the state yet
        const int32_t first = SWEEP ? qd.tblk_first : qd.fblk_first;
        const int32_t count = SWEEP ? qd.tblk_count : qd.fblk_count;
        double a = 0.0, b = 0.0;
        for (int k = threadIdx.x; k < count; k += kReduceThreads) {
            const double2 v = __ldcg(d + first + k);
            a += v.x;
            b += v.y;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) {
            sh[2 * warp] = a;
            sh[2 * warp + 1] = b;
        }
        __syncthreads();
        if (warp == 0) {
            double u = sh[2 * lane], w = sh[2 * lane + 1];
            u = warp_sum(u);
            w = warp_sum(w);
            if (lane == 0) done(q, u, w);
        }
        __syncthreads();
    }
}

// x0 = v~ (already in vel_c), r0 = b - (I - dt A) x0, p0 = r0; |r0|^2 and |b|^2.
template <int T>
__global__ void __launch_bounds__(kBlock) k_cg_init(Ptrs P)
{
    __shared__ double sh[2 * kBlock / 32];
    __shared__ int s_last;
    kernel_enter(P.ctl, KID_CG_INIT);
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    SceneState &st = *c.st;
    if (sc.visc_mode != 3) return;  // uniform per block
    double rr = 0.0, bb = 0.0;
    const int64_t i = c.i;
    const float4 pi = c.valid ? P.pos_s[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 xi = c.valid ? P.vel_c[i] : make_float4(0.f, 0.f, 0.f, 1.f);
    const float3 mx = apply_m<T>(P, sc, c, pi, xi, P.vel_c, st.dt);
    if (c.valid && c.s == 0) {
        const float4 r = make_float4(xi.x - mx.x, xi.y - mx.y, xi.z - mx.z, xi.w);
        P.cg_r[i] = r;
        P.cg_p[i] = r;
        rr = (double)r.x * r.x + (double)r.y * r.y + (double)r.z * r.z;
        bb = (double)xi.x * xi.x + (double)xi.y * xi.y + (double)xi.z * xi.z;
    }
    if (scene_reduce2(P, sc.tblk_first, sc.tblk_count, st, rr, bb, sh, &s_last)) {
        st.cg_rr = rr;
        st.cg_bb = bb;
        st.cg_it = 0;
        const double tol = (double)sc.cg_tol;
        st.cg_active = (sc.cg_max > 0 && rr > tol * tol * bb) ? 1 : 0;
        st.cg_res = bb > 0.0 ? (float)sqrt(rr / bb) : 0.0f;
    }
}

// Ap = (I - dt A) p and the block partials of p.Ap.
template <int T>
__global__ void __launch_bounds__(kBlock) k_cg_ap(Ptrs P)
{
    __shared__ double sh[2 * kBlock / 32];
    kernel_enter(P.ctl, KID_CG_AP);
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    SceneState &st = *c.st;
    if (!cg_active(sc, st)) return;  // uniform per block
    double pap = 0.0, unused = 0.0;
    const int64_t i = c.i;
    const float4 pi = c.valid ? P.pos_s[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 p = c.valid ? P.cg_p[i] : make_float4(0.f, 0.f, 0.f, 1.f);
    const float3 ap = apply_m<T>(P, sc, c, pi, p, P.cg_p, st.dt);
    if (c.valid && c.s == 0) {
        P.cg_ap[i] = make_float4(ap.x, ap.y, ap.z, 0.0f);
        pap = (double)p.x * ap.x + (double)p.y * ap.y + (double)p.z * ap.z;
    }
    block_partials2(P, pap, unused, sh);
}

// alpha = |r|^2 / p.Ap per scene (one block).
__global__ void __launch_bounds__(kReduceThreads) k_cg_alpha(Ptrs P)
{
    __shared__ double sh[2 * kReduceThreads / 32];
    kernel_enter(P.ctl, KID_CG_ALPHA);
    reduce_scenes<true>(P, sh, [&](int q, double pap, double) {
        SceneState &qs = P.st[q];
        qs.cg_alpha = pap > 0.0 ? qs.cg_rr / pap : 0.0;
    });
}

// x += alpha p, r -= alpha Ap and the block partials of |r_new|^2.
__global__ void __launch_bounds__(kBlock) k_cg_xr(Ptrs P)
{
    __shared__ double sh[2 * kBlock / 32];
    kernel_enter(P.ctl, KID_CG_XR);
    Ctx c = ctx(P);
    const SceneDev &sc = *c.sc;
    SceneState &st = *c.st;
    if (!cg_active(sc, st)) return;
    double rr = 0.0, unused = 0.0;
    if (c.valid) {
        const int64_t i = c.i;
        const float a = (float)st.cg_alpha;
        const float4 p = P.cg_p[i];
        const float4 ap = P.cg_ap[i];
        float4 x = P.vel_c[i];
        float4 r = P.cg_r[i];
        x.x = fmaf(a, p.x, x.x); x.y = fmaf(a, p.y, x.y); x.z = fmaf(a, p.z, x.z);
        r.x = fmaf(-a, ap.x, r.x); r.y = fmaf(-a, ap.y, r.y); r.z = fmaf(-a, ap.z, r.z);
        P.vel_c[i] = x;
        P.cg_r[i] = r;
        rr = (double)r.x * r.x + (double)r.y * r.y + (double)r.z * r.z;
    }
    block_partials2(P, rr, unused, sh);
}

// beta = |r_new|^2 / |r|^2 per scene, the iteration count and the residual; a scene stops
// at |r| <= tol |b| or cg_max_iter, and the loop goes on while any scene continues (one
// block; sets the CUDA graph's while condition).
__global__ void __launch_bounds__(kReduceThreads) k_cg_beta(Ptrs P, cudaGraphConditionalHandle handle,
                                                           int use_handle)
{
    __shared__ double sh[2 * kReduceThreads / 32];
    __shared__ int s_any;
    kernel_enter(P.ctl, KID_CG_BETA);
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    reduce_scenes<false>(P, sh, [&](int q, double rr, double) {
        const SceneDev &qd = P.scenes[q];
        SceneState &qs = P.st[q];
        qs.cg_beta = qs.cg_rr > 0.0 ? rr / qs.cg_rr : 0.0;
        qs.cg_rr = rr;
        qs.cg_it += 1;
        qs.cg_res = qs.cg_bb > 0.0 ? (float)sqrt(rr / qs.cg_bb) : 0.0f;
        const double tol = (double)qd.cg_tol;
        if (qs.cg_it >= qd.cg_max || !(qs.cg_rr > tol * tol * qs.cg_bb)) qs.cg_active = 0;
        else atomicOr(&s_any, 1);
    });
    __syncthreads();
    if (threadIdx.x != 0) return;
    uint32_t any = s_any;
    uint32_t guard = ++P.ctl->loop_guard;
    if (guard > 100000u) {
        any = 0;
        P.ctl->error = 3;
    }
    if (!any) P.ctl->loop_guard = 0;
    P.ctl->loop_flag = any;
    if (use_handle) cudaGraphSetConditional(handle, any);
}

// p = r + beta p for the scenes whose CG goes on.
__global__ void __launch_bounds__(kBlock) k_cg_p(Ptrs P)
{
    kernel_enter(P.ctl, KID_CG_P);
    Ctx c = ctx(P);
    const SceneDev &sc = *c.sc;
    SceneState &st = *c.st;
    if (cg_active(sc, st) && c.valid) {
        const int64_t i = c.i;
        const float b = (float)st.cg_beta;
        const float4 r = P.cg_r[i];
        float4 p = P.cg_p[i];
        p.x = fmaf(b, p.x, r.x); p.y = fmaf(b, p.y, r.y); p.z = fmaf(b, p.z, r.z);
        P.cg_p[i] = p;
    }
}

}  // namespace

void launch_cg_init(const Ptrs &P, cudaStream_t s)
{
#define SPH_L(T) k_cg_init<T><<<P.ntblk, kBlock, 0, s>>>(P)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
}
void launch_cg_ap(const Ptrs &P, cudaStream_t s)
{
#define SPH_L(T) k_cg_ap<T><<<P.ntblk, kBlock, 0, s>>>(P)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
}
void launch_cg_alpha(const Ptrs &P, cudaStream_t s) { k_cg_alpha<<<1, kReduceThreads, 0, s>>>(P); }
void launch_cg_xr(const Ptrs &P, cudaStream_t s) { k_cg_xr<<<P.nfblk, kBlock, 0, s>>>(P); }
void launch_cg_beta(const Ptrs &P, cudaGraphConditionalHandle h, int use_handle, cudaStream_t s)
{
    k_cg_beta<<<1, kReduceThreads, 0, s>>>(P, h, use_handle);
}
void launch_cg_p(const Ptrs &P, cudaStream_t s) { k_cg_p<<<P.nfblk, kBlock, 0, s>>>(P); }

}  // namespace sph
