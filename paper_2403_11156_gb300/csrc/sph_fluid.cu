// sph_fluid.cu -- per-particle sweeps of the DFSPH step.
//
// T threads (lanes, T = 1, 2, 4 or 8) own one fluid particle in grid order.  The density
// sweep walks the (2R+1)^3-cell neighbourhood ((2R+1)^2 contiguous index ranges) once
// per step and records the particle's neighbours in one k-major list, in candidate order
// (with T > 1 the lanes test T consecutive candidates at a time and append the hits by a
// ballot over the group, so the list is the same for every T).  Every later sweep of the
// step (divergence and density Jacobi passes, non-pressure forces, warm starts) gathers
// through that list, lane s taking entries s, s + T, ..., and combines the T partial sums
// with warp shuffles.  The solvers' error sums are accumulated per block in FP64 by pass A,
// folded by pass B and summed in a fixed order by a one-block check kernel, which also
// decides the loop condition on the device (CUDA graph conditional node).
#include <math_constants.h>

#include <type_traits>

#include "sph_sweep.cuh"

namespace sph {

namespace {

__device__ __forceinline__ void set_w(float4 *p, int64_t i, float w)
{
    reinterpret_cast<float *>(p + i)[3] = w;
}

struct BlockCtx {
    const SceneDev *sc;
    SceneState *st;
    int64_t i;
    bool valid;
};

__device__ __forceinline__ BlockCtx fluid_ctx(const Ptrs &P)
{
    BlockCtx c;
    int32_t s = P.fblk_scene[blockIdx.x];
    c.sc = &P.scenes[s];
    c.st = &P.st[s];
    int64_t local = (int64_t)(blockIdx.x - c.sc->fblk_first) * kBlock + threadIdx.x;
    c.valid = local < c.sc->nf;
    c.i = c.sc->f_off + local;
    return c;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_max(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Pass A's error partials are folded by pass B's blocks, fold_size(count) consecutive ones
// per fold (at least 8, and at most 256 folds per scene), and the check kernel sums a
// scene's folds with one warp.  The order depends only on the scene's own block count, so
// a scene reduces the same way alone and in any batch.
__device__ __forceinline__ int32_t fold_size(int32_t count) { return max(8, (count + 255) / 256); }

// Fixed-order block sum of one double per thread (deterministic).
__device__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kBlock / 32; ++k) t += sh[k];
    return t;  // valid in thread 0
}

// ------------------------------------------------------------------------------------
// Step begin: per-scene counters and the step size.
__global__ void k_step_begin(Ptrs P)
{
    kernel_enter(P.ctl, KID_STEP_BEGIN);
    int s = threadIdx.x + blockIdx.x * blockDim.x;
    if (s == 0) {
        P.ctl->loop_guard = 0;
        P.ctl->mlp_n = 0;
    }
    if (s >= P.nscenes) return;
    const SceneDev &sc = P.scenes[s];
    SceneState &st = P.st[s];
    float od = P.ctl->dt_override;
    st.dt = od > 0.0f ? od : (sc.cfl > 0.0f ? st.dt_next : sc.dt_max);
    for (int k = 0; k < 2; ++k) {
        st.last_it[k] = st.it[k];
        st.it[k] = 0;
        st.err[k] = CUDART_INF;
        st.err0[k] = 0.0;
    }
    st.counter = 0;
    st.max_nn_f = 0;
    st.max_nn_b = 0;
    st.maxv2 = 0.0f;
    if (sc.strong)   // strongly coupled bodies accumulate the step's force during the solves
        for (int k = 0; k < sc.nbody; ++k) {
            BodyDev &B = P.bodies[sc.body_off + k];
            for (int a = 0; a < 3; ++a) {
                B.force[a] = 0.0;
                B.torque[a] = 0.0;
            }
        }
}

// ------------------------------------------------------------------------------------
// Density (Eq. density + Sec. 3.5 boundary term), DFSPH alpha, neighbour lists, and the
// gate of the divergence warm start (D rho/Dt with the velocities at step start).
// Nine resident blocks per SM with one lane (56 registers; left to itself the compiler picks
// 48 and spills, measured 4 % slower on the 1.2M scene), eight with several (64 registers
// for the batched cooperative append).
template <int T>
__global__ void __launch_bounds__(kBlock, T == 1 ? 9 : 8) k_density_alpha(Ptrs P)
{
    kernel_enter(P.ctl, KID_DENSITY);
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    const int64_t i = c.i, NF = P.NF;
    const int s = c.s;
    const bool gate = sc.warm != 0 && sc.div_on;
    int nn_f = 0, nn_b = 0;  // this lane's neighbours (may exceed its capacity)
    // this lane's shares of rho - m W(0), sum grad W, sum |grad W|^2 and D rho/Dt
    float rho_l = 0.0f, s1x = 0.0f, s1y = 0.0f, s1z = 0.0f, s2 = 0.0f, div_l = 0.0f;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c.valid) {
        pi = P.pos_s[i];
        const float4 vi = P.vel_s[i];
        const int32_t cx = cell_coord(pi.x, sc.origin[0], sc.cell, sc.dims[0]);
        const int32_t cy = cell_coord(pi.y, sc.origin[1], sc.cell, sc.dims[1]);
        const int32_t cz = cell_coord(pi.z, sc.origin[2], sc.cell, sc.dims[2]);
        const int32_t R = sc.R;
        const float h2 = sc.h2, cull2 = sc.cull2, cs = sc.cell;
        const unsigned long long pixy = pack_xy(pi.x, pi.y);   // for the packed candidate test
        // offset of the particle inside its cell, per axis: the distance from the particle
        // to a stencil cell d cells away is at least gap(d) (zero for d = 0)
        const float ox = pi.x - fmaf((float)cx, cs, sc.origin[0]);
        const float oy = pi.y - fmaf((float)cy, cs, sc.origin[1]);
        const float oz = pi.z - fmaf((float)cz, cs, sc.origin[2]);
        auto gap = [&](float o, int32_t d) {
            const float g = d < 0 ? fmaf((float)(-d - 1), cs, o) : (d > 0 ? fmaf((float)d, cs, -o) : 0.0f);
            return fmaxf(g, 0.0f);
        };
        const int cap_f = sc.cap_f, cap_b = sc.cap_b;
        const uint32_t self = (uint32_t)i;
        int32_t *slot_f = P.nbr + i;   // this particle's next list entry (one lane per particle)
        // the group's lanes relative to this one (cooperative append for T > 1)
        const unsigned gmask = group_mask<T>();
        const int gshift = (int)(threadIdx.x & 31u) & ~(T - 1);
        const unsigned below = (1u << s) - 1u;
        // phase 1: the float predicate over the stencil's index ranges only records
        // neighbours; keeping the per-pair work out of this loop keeps the warp converged
        // while most candidates are rejected.  Rows and end cells whose nearest point is
        // farther than h (plus a margin above the rounding of these bounds) are skipped:
        // they hold no particle that passes the predicate, so the lists are unchanged.
        // With T > 1 the lanes test T consecutive candidates at a time and append the hits
        // in candidate order (ballot over the group), so every T builds the same list.
        for (int32_t dz = -R; dz <= R; ++dz) {
            const int32_t z = cz + dz;
            if (z < 0 || z >= sc.dims[2]) continue;
            const float gz = T > 1 ? gap(oz, dz) : 0.0f;
            for (int32_t dy = -R; dy <= R; ++dy) {
                const int32_t y = cy + dy;
                if (y < 0 || y >= sc.dims[1]) continue;
                int32_t x0 = cx - R, x1 = cx + R;
                if (T > 1) {   // with one lane the culling's registers cost more than it saves
                    const float gy = gap(oy, dy);
                    const float g2 = fmaf(gy, gy, gz * gz);
                    if (g2 > cull2) continue;
                    while (x0 < cx && fmaf(gap(ox, x0 - cx), gap(ox, x0 - cx), g2) > cull2) ++x0;
                    while (x1 > cx && fmaf(gap(ox, x1 - cx), gap(ox, x1 - cx), g2) > cull2) --x1;
                }
                x0 = max(x0, 0);
                x1 = min(x1, sc.dims[0] - 1);
                const int64_t row = sc.c_off + (int64_t)sc.dims[0] * (y + (int64_t)sc.dims[1] * z);
                const uint32_t jb = P.cell_start[row + x0], je = P.cell_start[row + x1 + 1];
                if constexpr (T == 1) {
                    if (je - jb <= 64u) {
                        // a row of up to 64 candidates: the predicate only sets bits of a
                        // mask (no store or counter per candidate, most are rejected), and
                        // the hits are appended in candidate order from the mask
                        auto bits = [&](uint32_t b0, uint32_t b1) {
                            // four candidates per batch: their loads issue together, and their
                            // hits are combined at fixed shifts before one shift into place
                            uint32_t mk = 0u;
                            uint32_t j = b0;
                            for (; j + 3u < b1; j += 4u) {
                                float4 pc[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) pc[u] = __ldg(P.pos_s + j + u);
                                uint32_t q = 0u;
#pragma unroll
                                for (int u = 0; u < 4; ++u) q |= (uint32_t)(pred_d2_xy2(pixy, pi.z, pc[u]) < h2) << u;
                                mk |= q << (j - b0);
                            }
                            for (; j < b1; ++j) mk |= (uint32_t)(pred_d2_xy2(pixy, pi.z, __ldg(P.pos_s + j)) < h2) << (j - b0);
                            return mk;
                        };
                        uint64_t m = bits(jb, min(je, jb + 32u));
                        if (je > jb + 32u) m |= (uint64_t)bits(jb + 32u, je) << 32;
                        // only the stencil's centre row holds the particle itself
                        if (dz == 0 && dy == 0) m &= ~(1ull << (self - jb));
                        for (; m != 0ull; m &= m - 1ull) {
                            if (nn_f < cap_f) *slot_f = (int32_t)(jb + (uint32_t)(__ffsll((long long)m) - 1));
                            slot_f += NF;
                            ++nn_f;
                        }
                    } else {
                        // longer rows: a predicated store through a running slot pointer
                        auto scan = [&](auto check_self) {
                            for_range<4, 1>(P.pos_s, jb, je, [&](uint32_t j, float4 pj) {
                                float dx, dy2, dz2;
                                const float d2 = pred_d2(pi, pj, dx, dy2, dz2);
                                const bool hit = d2 < h2 && (!decltype(check_self)::value || j != self);
                                if (hit && nn_f < cap_f) *slot_f = (int32_t)j;
                                slot_f += hit ? NF : 0;
                                nn_f += hit;
                            });
                        };
                        if (dz == 0 && dy == 0) scan(std::true_type{});
                        else scan(std::false_type{});
                    }
                } else {
                    // the group's lanes test T consecutive candidates at a time and append the
                    // hits in candidate order; full batches of kCand groups load all their
                    // candidates before the first test (one memory latency per batch)
                    auto append = [&](uint32_t j, bool hit) {
                        const unsigned bits = __ballot_sync(gmask, hit) >> gshift;
                        const int slot = nn_f + __popc(bits & below);
                        if (hit && slot < cap_f) P.nbr[(int64_t)slot * NF + i] = (int32_t)j;
                        nn_f += __popc(bits);
                    };
                    constexpr int kCand = 4;
                    uint32_t j0 = jb;
                    for (; j0 + (uint32_t)(kCand * T) <= je; j0 += (uint32_t)(kCand * T)) {   // uniform in the group
                        float4 pc[kCand];
#pragma unroll
                        for (int u = 0; u < kCand; ++u) pc[u] = __ldg(P.pos_s + j0 + (uint32_t)(u * T + s));
#pragma unroll
                        for (int u = 0; u < kCand; ++u) {
                            const uint32_t j = j0 + (uint32_t)(u * T + s);
                            float dx, dy2, dz2;
                            append(j, pred_d2(pi, pc[u], dx, dy2, dz2) < h2 && j != self);
                        }
                    }
                    for (; j0 < je; j0 += (uint32_t)T) {   // uniform in the group
                        const uint32_t j = j0 + (uint32_t)s;
                        bool hit = false;
                        if (j < je) {
                            float dx, dy2, dz2;
                            hit = pred_d2(pi, __ldg(P.pos_s + j), dx, dy2, dz2) < h2 && j != self;
                        }
                        append(j, hit);
                    }
                }
                if (sc.nb > 0) {
                    const uint32_t bb = P.bcell_start[row + x0], be = P.bcell_start[row + x1 + 1];
                    for (uint32_t b0 = bb; b0 < be; b0 += (uint32_t)T) {
                        const uint32_t b = b0 + (uint32_t)s;
                        bool hit = false;
                        if (b < be) {
                            float dx, dy2, dz2;
                            hit = pred_d2(pi, __ldg(P.bpos_s + b), dx, dy2, dz2) < h2;
                        }
                        const unsigned bits = T == 1 ? (unsigned)hit : (__ballot_sync(gmask, hit) >> gshift);
                        const int slot = nn_b + __popc(bits & below);
                        if (hit && slot < cap_b) P.bnbr[(int64_t)slot * NF + i] = (int32_t)b;
                        nn_b += __popc(bits);
                    }
                }
            }
        }
        // the lists were written by the group's lanes: order them before the reads below
        if (T > 1) __syncwarp(gmask);
        const int32_t *__restrict__ nbr = P.nbr;
        const int32_t *__restrict__ bnbr = P.bnbr;
        // phase 2: density, alpha and the warm-start gate over the recorded list (this
        // lane's share of its entries)
        float w_sum = 0.0f, fx = 0.0f, fy = 0.0f, fz = 0.0f, div_f = 0.0f;
        const Spline sp(sc);
        for_list<2, T, false>(nbr, NF, i, s, min(nn_f, cap_f), [&](int32_t j) {
            const float4 pj = __ldg(P.pos_s + j);
            float dx, dy2, dz2;
            const float d2 = pred_d2(pi, pj, dx, dy2, dz2);
            w_sum += spline_w(sqrtf(d2) * sp.inv_h);
            const float f = grad_factor(sp, d2);
            const float gx = f * dx, gy = f * dy2, gz = f * dz2;
            fx += gx; fy += gy; fz += gz;
            s2 = fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, s2)));
            if (gate) {
                const float4 vj = __ldg(P.vel_s + j);
                div_f += (vi.x - vj.x) * gx + (vi.y - vj.y) * gy + (vi.z - vj.z) * gz;
            }
        });
        rho_l = sc.m * sc.sigma * w_sum;
        s1x = sc.m * fx; s1y = sc.m * fy; s1z = sc.m * fz;
        s2 *= sc.m * sc.m;
        div_l = sc.m * div_f;
        const int nb = min(nn_b, cap_b);
        if (nb > 0) {
            float wb = 0.0f, divb = 0.0f;
            const bool moving = sc.has_moving != 0;
            for_list<1, T, false>(bnbr, NF, i, s, nb, [&](int32_t b) {
                const float4 pb = __ldg(P.bpos_s + b);
                float dx, dy2, dz2;
                const float d2 = pred_d2(pi, pb, dx, dy2, dz2);
                const float psi = pb.w;
                wb += psi * spline_w(sqrtf(d2) * sp.inv_h);
                const float f = psi * grad_factor(sp, d2);
                const float gx = f * dx, gy = f * dy2, gz = f * dz2;
                s1x += gx; s1y += gy; s1z += gz;
                if (gate) {
                    float4 vb = moving ? __ldg(P.bvel_s + b) : make_float4(0.f, 0.f, 0.f, 0.f);
                    divb += (vi.x - vb.x) * gx + (vi.y - vb.y) * gy + (vi.z - vb.z) * gz;
                }
            });
            rho_l += sc.sigma * wb;
            div_l += divb;
        }
    }
    // combine the lanes (all threads of the warp take part)
    rho_l = group_sum<T>(rho_l);
    s1x = group_sum<T>(s1x); s1y = group_sum<T>(s1y); s1z = group_sum<T>(s1z);
    s2 = group_sum<T>(s2);
    div_l = group_sum<T>(div_l);
    if (c.valid && s == 0) {
        const float rho = fmaf(sc.m, sc.sigma, rho_l);
        const float den = fmaf(s1x, s1x, fmaf(s1y, s1y, fmaf(s1z, s1z, s2)));
        const float alpha = den > sc.eps_alpha ? rho / den : 0.0f;
        P.alpha[i] = alpha;
        set_w(P.vel_s, i, rho);
        P.nnf[i] = min(nn_f, sc.cap_f);
        P.nnb[i] = min(nn_b, sc.cap_b);
        float kv0 = 0.0f;
        if (gate && div_l > 0.0f) kv0 = sc.warm_frac * P.kvprev_s[i] / c.st->dt;
        P.kvsum[i] = kv0;
        set_w(P.pos_s, i, kv0 / rho);
    }
    // the counts are the same in all lanes of a particle (one atomic per warp: spread over
    // this long sweep they cost less than a block barrier would)
    const int mf = warp_max(nn_f), mb = warp_max(nn_b);
    if ((threadIdx.x & 31) == 0) {
        if (mf > 0) atomicMax(&c.st->max_nn_f, mf);
        if (mb > 0) atomicMax(&c.st->max_nn_b, mb);
        if (mf > sc.cap_f || mb > sc.cap_b) atomicOr(&c.st->flags, 1);
    }
}

// ------------------------------------------------------------------------------------
// This lane's share of D rho_i/Dt = sum_j m (v_i - v_j).grad W_ij + sum_b Psi_b (v_i -
// v_b).grad W_ib (SPH divergence of Sec. 3.2 in the continuity equation, boundary per
// Sec. 3.5); group_sum of the shares is the full sum.
constexpr int kBatch = 4;

template <int B, int T>
__device__ __forceinline__ float drho_dt_lane(const Ptrs &P, const SceneDev &sc, int64_t i, int s, float4 pi,
                                              float4 vi, const float4 *__restrict__ V)
{
    const int64_t NF = P.NF;
    const Spline sp(sc);
    float acc = 0.0f;
    for_list<B, T>(P.nbr, NF, i, s, P.nnf[i], [&](int32_t j) {
        const float4 pj = __ldg(P.pos_s + j);
        const float4 vj = __ldg(V + j);
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const float f = grad_factor(sp, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        acc = fmaf(f, (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz, acc);
    });
    float accb = 0.0f;
    const bool moving = sc.has_moving != 0;
    for_list<4, T>(P.bnbr, NF, i, s, P.nnb[i], [&](int32_t b) {
        const float4 pb = __ldg(P.bpos_s + b);
        const float dx = pi.x - pb.x, dy = pi.y - pb.y, dz = pi.z - pb.z;
        const float f = pb.w * grad_factor(sp, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        float ux = vi.x, uy = vi.y, uz = vi.z;
        if (moving) {
            const float4 vb = __ldg(P.bvel_s + b);
            ux -= vb.x; uy -= vb.y; uz -= vb.z;
        }
        accb = fmaf(f, ux * dx + uy * dy + uz * dz, accb);
    });
    return fmaf(sc.m, acc, accb);
}

// Pass A of a Jacobi iteration (Alg. ppe_solver "refine p"): the source term of
// Eq. velocity_source (solver 0) or Eq. density_source with rho* (solver 1), the
// stiffness kappa_i = alpha_i e_i / dt^(1 or 2), and the block's FP64 error partial.
template <int S, int B, int T>
__global__ void __launch_bounds__(kBlock) k_pass_a(Ptrs P)
{
    __shared__ double sh[kBlock / 32];
    kernel_enter(P.ctl, (KID_PASS_A0 + S));
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    SceneState &st = *c.st;
    if (!solver_active(sc, st, S)) return;  // uniform per block
    const float dt = st.dt;
    const float4 *V = S == 0 ? P.vel_s : P.vel_c;
    const int64_t i = c.i;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = pi;
    float D = 0.0f;
    if (c.valid) {
        pi = P.pos_s[i];
        vi = V[i];
        D = drho_dt_lane<B, T>(P, sc, i, c.s, pi, vi, V);
    }
    D = group_sum<T>(D);
    double e = 0.0;
    if (c.valid && c.s == 0) {
        const float rho = vi.w;
        float ei, kappa;
        if (S == 0) {
            ei = fmaxf(D, 0.0f);
            kappa = P.alpha[i] * ei / dt;
            P.kvsum[i] += kappa;
        } else if (sc.solver == 2) {
            // PCISPH: refine the total pressure p <- max(p + delta (rho* - rho0), 0) with
            // the prototype's delta; the pass B applies the change (kept as p/rho)
            const float dev = fmaf(dt, D, rho - sc.rho0);
            ei = fmaxf(dev, 0.0f);
            const float p_old = P.ksum[i] * rho;
            const float p_new = fmaxf(fmaf(sc.pci_c / (dt * dt), dev, p_old), 0.0f);
            kappa = (p_new - p_old) / rho;
            P.ksum[i] = p_new / rho;
        } else {
            ei = fmaxf(fmaf(dt, D, rho - sc.rho0), 0.0f);
            kappa = P.alpha[i] * ei / (dt * dt);
            P.ksum[i] += kappa;
        }
        set_w(P.pos_s, i, kappa / rho);
        e = (double)ei;
    }
    // the block's FP64 error partial; pass B folds the partials and the check kernel sums
    // the folds in a fixed order (no last-block step here: pass A only has to finish)
    const double bsum = block_sum(e, sh);
    if (threadIdx.x == 0) P.partial[blockIdx.x] = bsum;
}

// Pass B (Alg. ppe_solver "update v*"): pressure acceleration of Sec. 3.3 Eq.
// pressure_acceleration with p/rho^2 = kappa/rho, plus the boundary term of Sec. 3.5
// Eq. rigid_pressure per unit fluid mass:
//   v_i -= dt [ sum_j m (k_i/rho_i + k_j/rho_j) grad W_ij + sum_b Psi_b (k_i/rho_i) grad W_ib ]
// WARM = 1 applies the warm-start kappas (no loop bookkeeping).  With one lane and gather
// batch 4 the loop's pass B is held to 40 registers (12 resident blocks per SM instead of
// 10): it is bound by the gathers' latency, and the extra warps outweigh a few spilled words
// (measured on the 1.2M scene: 84 -> 80 us per density launch, 90 -> 81 per divergence
// launch).  Every other variant keeps the compiler's choice (a minimum of 0 blocks): the warm
// pass already fits in 40 registers, and batch 8 would spill 152 bytes.
template <int S, int WARM, int B, int T>
__global__ void __launch_bounds__(kBlock, (T == 1 && WARM == 0 && B == 4) ? 11 : 0) k_pass_b(Ptrs P)
{
    kernel_enter(P.ctl, (WARM ? KID_PASS_B0W + S : KID_PASS_B0 + S));
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    SceneState &st = *c.st;
    // uniform per block; WCSPH scenes apply their equation-of-state pressure here.  In the
    // loop, a scene's pass B runs exactly when its pass A did: the solver state only
    // changes in the check kernel that follows.
    const bool run = WARM ? warm_pass_runs(sc, S) : solver_active(sc, st, S);
    if (run) {
        const int64_t i = c.i, NF = P.NF;
        const int s = c.s;
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
        if (c.valid) {
            const float4 pi = P.pos_s[i];
            const float ki = pi.w;
            const Spline sp(sc);
            for_list<B, T>(P.nbr, NF, i, s, P.nnf[i], [&](int32_t j) {
                const float4 pj = __ldg(P.pos_s + j);
                const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                const float f = grad_factor(sp, fmaf(dx, dx, fmaf(dy, dy, dz * dz))) * (ki + pj.w);
                ax = fmaf(f, dx, ax); ay = fmaf(f, dy, ay); az = fmaf(f, dz, az);
            });
            ax *= sc.m; ay *= sc.m; az *= sc.m;
            if (ki != 0.0f) {
                float bx = 0.0f, by = 0.0f, bz = 0.0f;
                for_list<4, T>(P.bnbr, NF, i, s, P.nnb[i], [&](int32_t b) {
                    const float4 pb = __ldg(P.bpos_s + b);
                    const float dx = pi.x - pb.x, dy = pi.y - pb.y, dz = pi.z - pb.z;
                    const float f = pb.w * grad_factor(sp, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    bx = fmaf(f, dx, bx); by = fmaf(f, dy, by); bz = fmaf(f, dz, bz);
                });
                ax = fmaf(ki, bx, ax); ay = fmaf(ki, by, ay); az = fmaf(ki, bz, az);
            }
        }
        ax = group_sum<T>(ax); ay = group_sum<T>(ay); az = group_sum<T>(az);
        if (c.valid && s == 0) {
            float4 *V = S == 0 ? P.vel_s : P.vel_c;
            const float dt = st.dt;
            float4 v = V[i];
            v.x -= dt * ax; v.y -= dt * ay; v.z -= dt * az;
            V[i] = v;
        }
    }
    if (WARM) return;
    // fold pass A's error partials: the scene's first ceil(count / F) blocks each sum F
    // consecutive ones in block order (the check kernel, a later launch, sums the folds)
    if (run && threadIdx.x == 0) {
        const int32_t lb = (int32_t)blockIdx.x - sc.tblk_first;
        const int32_t F = fold_size(sc.tblk_count);
        if (lb < (sc.tblk_count + F - 1) / F) {
            const int32_t k0 = lb * F, k1 = min(k0 + F, sc.tblk_count);
            double t = 0.0;
            for (int32_t k = k0; k < k1; ++k) t += __ldcg(P.partial + sc.tblk_first + k);
            P.partial2[blockIdx.x] = t;
        }
    }
}

// Convergence test of one Jacobi iteration (Alg. ppe_solver's loop condition), one block
// after pass B: one warp per scene (32 scenes at a time) sums the scene's folds in a fixed
// order (lane l takes folds l, l + 32, ..., then a butterfly), which gives the mean error;
// the iteration counters advance and the loop condition is set for the host and for the
// CUDA graph's while node.
constexpr int kCheckThreads = 1024;

template <int S>
__global__ void __launch_bounds__(kCheckThreads) k_solver_check(Ptrs P, cudaGraphConditionalHandle handle,
                                                               int use_handle)
{
    __shared__ int s_any;
    kernel_enter(P.ctl, KID_CHECK0 + S);
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q < P.nscenes; q += kCheckThreads / 32) {
        const SceneDev &qd = P.scenes[q];
        SceneState &qs = P.st[q];
        if (!solver_active(qd, qs, S)) continue;   // its pass A and B did not run
        const int32_t F = fold_size(qd.tblk_count);
        const int32_t nfold = (qd.tblk_count + F - 1) / F;
        double t = 0.0;
#pragma unroll 8
        for (int k = lane; k < nfold; k += 32) t += __ldcg(P.partial2 + qd.tblk_first + k);
        t = warp_sum(t);
        if (lane == 0) {
            double err = t * qd.err_scale;   // FP64 division is a long sequence here
            if (S == 0) err *= (double)qs.dt;
            if (qs.it[S] == 0) qs.err0[S] = err;
            qs.err[S] = err;
            qs.it[S] += 1;
            qs.total_it[S] += 1;
            if (!solver_active(qd, qs, S) && qs.err[S] > (double)qd.eta[S]) qs.flags |= 2;
            if (solver_active(qd, qs, S)) atomicOr(&s_any, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    uint32_t any = s_any;
    uint32_t guard = ++P.ctl->loop_guard;
    if (guard > 100000u) {
        any = 0;
        P.ctl->error = 2;
    }
    if (!any) P.ctl->loop_guard = 0;
    P.ctl->loop_flag = any;
    if (use_handle) cudaGraphSetConditional(handle, any);
}

// ------------------------------------------------------------------------------------
// Non-pressure forces (Sec. 3.3 Alg. general_algorithm, Sec. 4.2: gravity, then
// viscosity): v* = v + dt (g + (mu/rho_i) lap v_i) with Eq. lap
//   lap v_i = 2(d+2) sum_j (m/rho_j) (v_ij . x_ij)/(|x_ij|^2 + 0.01 h^2) grad W_ij,
// or XSPH smoothing c sum_j (m/rho_j)(v_j - v_i) W_ij.  Writes v* to the canonical
// velocity array and clears the density-solve stiffness sum.
template <int T>
__global__ void __launch_bounds__(kBlock) k_nonpressure(Ptrs P)
{
    kernel_enter(P.ctl, KID_NONP);
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    const int64_t i = c.i, NF = P.NF;
    const int s = c.s;
    float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    const bool visc = sc.visc_mode == 1 || sc.visc_mode == 2;  // uniform per block
    if (c.valid) {
        vi = P.vel_s[i];
        if (visc) {
            const float4 pi = P.pos_s[i];
            const float reg = 0.01f * sc.h2;
            const bool lap = sc.visc_mode == 1;
            const Spline sp(sc);
            for_list<kBatch, T>(P.nbr, NF, i, s, P.nnf[i], [&](int32_t j) {
                const float4 pj = __ldg(P.pos_s + j);
                const float4 vj = __ldg(P.vel_s + j);
                const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                const float ux = vi.x - vj.x, uy = vi.y - vj.y, uz = vi.z - vj.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (lap) {
                    const float f = grad_factor(sp, r2);
                    const float q = f * (ux * dx + uy * dy + uz * dz) / ((r2 + reg) * vj.w);
                    sx = fmaf(q, dx, sx); sy = fmaf(q, dy, sy); sz = fmaf(q, dz, sz);
                } else {
                    const float w = spline_w(sqrtf(r2) * sp.inv_h) / vj.w;
                    sx = fmaf(-w, ux, sx); sy = fmaf(-w, uy, sy); sz = fmaf(-w, uz, sz);
                }
            });
        }
    }
    if (visc) {
        sx = group_sum<T>(sx); sy = group_sum<T>(sy); sz = group_sum<T>(sz);
    }
    if (!c.valid || s != 0) return;
    const float dt = c.st->dt;
    const float rho_i = vi.w;
    const float ax = sc.g[0], ay = sc.g[1], az = sc.g[2];
    float4 v = vi;
    if (sc.visc_mode == 1) {
        const float k = 10.0f * sc.mu * sc.m / rho_i;
        v.x += dt * fmaf(k, sx, ax); v.y += dt * fmaf(k, sy, ay); v.z += dt * fmaf(k, sz, az);
    } else if (sc.visc_mode == 2) {
        const float k = sc.xsph * sc.m * sc.sigma;
        v.x += fmaf(dt, ax, k * sx); v.y += fmaf(dt, ay, k * sy); v.z += fmaf(dt, az, k * sz);
    } else {
        v.x += dt * ax; v.y += dt * ay; v.z += dt * az;
    }
    v.w = rho_i;
    P.vel_c[i] = v;
    // WCSPH: the equation of state of Sec. 3.4.1, p = k ((rho/rho0)^gamma - 1) clamped at
    // zero, evaluated as k expm1(gamma log1p(rho/rho0 - 1)) for accuracy near rho0; the
    // pressure pass then uses p/rho^2 (the kappa/rho slot) and the stiffness sum keeps
    // p/rho (so that p = kappa_sum rho for output and for the rigid reaction)
    float w = 0.0f, ks = 0.0f;
    if (sc.solver == 1) {
        const float p = fmaxf(sc.eos_k * expm1f(sc.eos_gamma * log1pf((rho_i - sc.rho0) / sc.rho0)), 0.0f);
        ks = p / rho_i;
        w = ks / rho_i;
    }
    P.ksum[i] = ks;
    P.k0[i] = 0.0f;
    set_w(P.pos_s, i, w);
}

// Warm start of the constant-density solve: the predicted deviation rho* - rho0 with
// v* gates a fraction (default half) of the previous step's stiffness (kept as kappa
// dt^2); the learned mode
// stores the network's input features instead (rho/rho0 - 1, dt Drho/Dt/rho0,
// (n_f + n_b)/33, kappa_prev/(9.81 h)) and a separate kernel fills kappa0.  With a
// learned gate g > 0 a scene whose previous density solve took g iterations or fewer
// takes the previous-step start in this step (the network would run for nothing at the
// solve's floor).
template <int T>
__global__ void __launch_bounds__(kBlock) k_warm_density(Ptrs P)
{
    kernel_enter(P.ctl, KID_WARM);
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    if (sc.warm == 0) return;  // uniform per block
    const int64_t i = c.i;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = pi;
    float D = 0.0f;
    if (c.valid) {
        pi = P.pos_s[i];
        vi = P.vel_c[i];
        D = drho_dt_lane<kBatch, T>(P, sc, i, c.s, pi, vi, P.vel_c);
    }
    D = group_sum<T>(D);
    const bool own = c.valid && c.s == 0;
    const float dt = c.st->dt;
    const float rho = vi.w;
    const float dev = fmaf(dt, D, rho - sc.rho0);
    // learned mode (uniform per block): the network runs unless the gate holds it back
    const bool net = sc.warm == 2 && (sc.learned_gate == 0 || c.st->last_it[1] > sc.learned_gate);
    // learned mode: the gated particles (predicted compression) are appended to the rows
    // of the network kernel, one atomic per warp (the whole warp is converged here)
    if (net) {
        const bool gated = own && dev > 0.0f && P.ctl->have_mlp;
        const unsigned m = __ballot_sync(0xffffffffu, gated);
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (m != 0) {
            const int lead = __ffs(m) - 1;
            if (lane == lead) base = atomicAdd(&P.ctl->mlp_n, __popc(m));
            base = __shfl_sync(0xffffffffu, base, lead);
        }
        if (gated) P.mlp_rows[base + __popc(m & ((1u << lane) - 1u))] = make_int2((int)i, P.tblk_scene[blockIdx.x]);
    }
    if (!own) return;
    // the network's inputs are recorded in both warm-start modes (the previous-step mode
    // produces the training data)
    const float kref = 9.81f * sc.h;
    float4 f;
    f.x = rho / sc.rho0 - 1.0f;
    f.y = dt * D / sc.rho0;
    f.z = (float)(P.nnf[i] + P.nnb[i]) / 33.0f;
    f.w = P.kprev_s[i] / (dt * dt) / kref;
    reinterpret_cast<float4 *>(P.feat)[i] = f;
    float k0 = 0.0f;
    if (!net && dev > 0.0f) k0 = sc.warm_frac * P.kprev_s[i] / (dt * dt);
    // learned mode: zero here, the network kernel fills the gated rows
    P.k0[i] = k0;
    P.ksum[i] = k0;
    set_w(P.pos_s, i, k0 / rho);
}

// Advect (Sec. 3.3 Alg. general_algorithm, symplectic Euler): x = x + dt v*, written
// back in grid order as the next step's canonical state, with the warm-start memory.
__global__ void __launch_bounds__(kBlock) k_advect(Ptrs P)
{
    kernel_enter(P.ctl, KID_ADVECT);
    BlockCtx c = fluid_ctx(P);
    float v2 = 0.0f;
    bool bad = false;
    if (c.valid) {
        const int64_t i = c.i;
        const float dt = c.st->dt;
        const float4 v = P.vel_c[i];
        float4 p = P.pos_s[i];
        p.x = fmaf(dt, v.x, p.x);
        p.y = fmaf(dt, v.y, p.y);
        p.z = fmaf(dt, v.z, p.z);
        p.w = 0.0f;
        P.pos_c[i] = p;
        P.id_c[i] = P.id_s[i];
        P.kprev_c[i] = P.ksum[i] * dt * dt;
        P.kvprev_c[i] = P.kvsum[i] * dt;
        v2 = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
        bad = !isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z) || !isfinite(v2);
    }
    float m = v2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const unsigned anybad = __ballot_sync(0xffffffffu, bad);
    // the block's largest finite |v|^2 and its bad flag reach the scene with one atomic each
    // (one per warp, on a single word, serialises in L2 and bounded this kernel)
    __shared__ float s_m[kBlock / 32];
    __shared__ unsigned s_bad[kBlock / 32];
    if ((threadIdx.x & 31) == 0) {
        s_m[threadIdx.x >> 5] = (m > 0.0f && isfinite(m)) ? m : 0.0f;
        s_bad[threadIdx.x >> 5] = anybad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bm = s_m[0];
        unsigned bb = s_bad[0];
        for (int w = 1; w < kBlock / 32; ++w) {
            bm = fmaxf(bm, s_m[w]);
            bb |= s_bad[w];
        }
        if (bm > 0.0f) atomicMax(reinterpret_cast<int *>(&c.st->maxv2), __float_as_int(bm));
        if (bb) atomicOr(&c.st->flags, 4);
    }
}

// Step end: CFL step for the next step (not in the paper: dt = min(dt_max, cfl 2r /
// max|v|)), counters, and the rigid bodies (symplectic Euler with a renormalised
// quaternion; weak coupling: bodies move only between fluid steps, Sec. 2.2 / 6).
__global__ void k_step_end(Ptrs P)
{
    kernel_enter(P.ctl, KID_STEP_END);
    int t = threadIdx.x;
    for (int s = t; s < P.nscenes; s += blockDim.x) {
        const SceneDev &sc = P.scenes[s];
        SceneState &st = P.st[s];
        float vm = sqrtf(st.maxv2);
        float dt = sc.dt_max;
        if (sc.cfl > 0.0f && vm > 0.0f) dt = fminf(dt, sc.cfl * sc.two_r / vm);
        st.dt_next = dt;
        st.steps += 1;
    }
    for (int k = t; k < P.nbodies_total; k += blockDim.x) {
        BodyDev &B = P.bodies[k];
        const SceneDev &sc = P.scenes[B.scene];
        const double dt = (double)P.st[B.scene].dt;
        const double fs = sc.strong ? 0.0 : 1.0;   // strong coupling applied the fluid's impulses already
        // FP64 division is a long dependent sequence on this GPU: the body record carries
        // 1/m and 1/I, and the quaternion is renormalised with one reciprocal square root
        const double inv_m = B.inv_mass;
        const double inv_i[3] = {B.inv_inertia[0], B.inv_inertia[1], B.inv_inertia[2]};
        for (int a = 0; a < 3; ++a) B.vel[a] += dt * (fs * B.force[a] * inv_m + (double)sc.g[a]);
        for (int a = 0; a < 3; ++a) B.com[a] += dt * B.vel[a];
        double w = B.quat[0], x = B.quat[1], y = B.quat[2], z = B.quat[3];
        double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                          {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                          {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        double Iw[3][3], Ii[3][3];
        for (int a = 0; a < 3; ++a)
            for (int e = 0; e < 3; ++e) {
                Iw[a][e] = 0.0;
                Ii[a][e] = 0.0;
                for (int q = 0; q < 3; ++q) {
                    Iw[a][e] += R[a][q] * B.inertia[q] * R[e][q];
                    Ii[a][e] += R[a][q] * inv_i[q] * R[e][q];
                }
            }
        double o[3] = {B.omega[0], B.omega[1], B.omega[2]};
        double L[3];
        for (int a = 0; a < 3; ++a) L[a] = Iw[a][0] * o[0] + Iw[a][1] * o[1] + Iw[a][2] * o[2];
        double rhs[3] = {fs * B.torque[0] - (o[1] * L[2] - o[2] * L[1]),
                         fs * B.torque[1] - (o[2] * L[0] - o[0] * L[2]),
                         fs * B.torque[2] - (o[0] * L[1] - o[1] * L[0])};
        for (int a = 0; a < 3; ++a) B.omega[a] += dt * (Ii[a][0] * rhs[0] + Ii[a][1] * rhs[1] + Ii[a][2] * rhs[2]);
        double ox = B.omega[0], oy = B.omega[1], oz = B.omega[2];
        double dw = 0.5 * (-ox * x - oy * y - oz * z);
        double dx = 0.5 * (ox * w + oy * z - oz * y);
        double dy = 0.5 * (oy * w + oz * x - ox * z);
        double dz = 0.5 * (oz * w + ox * y - oy * x);
        w += dt * dw; x += dt * dx; y += dt * dy; z += dt * dz;
        const double inv_nq = rsqrt(w * w + x * x + y * y + z * z);
        B.quat[0] = w * inv_nq; B.quat[1] = x * inv_nq; B.quat[2] = y * inv_nq; B.quat[3] = z * inv_nq;
        // no contact model (the paper delegates contact to PyBullet): the bounding sphere
        // is clamped inside the domain, and each clamp is counted
        for (int a = 0; a < 3; ++a) {
            if (B.com[a] < B.lo[a]) {
                B.com[a] = B.lo[a];
                if (B.vel[a] < 0.0) B.vel[a] = 0.0;
                atomicAdd(&P.st[B.scene].clamps, 1);
            }
            if (B.com[a] > B.hi[a]) {
                B.com[a] = B.hi[a];
                if (B.vel[a] > 0.0) B.vel[a] = 0.0;
                atomicAdd(&P.st[B.scene].clamps, 1);
            }
        }
    }
}

__global__ void k_set_dt(Control *ctl, float dt)
{
    kernel_enter(ctl, KID_SET_DT);
    ctl->dt_override = dt;
}

}  // namespace

void launch_step_begin(const Ptrs &P, cudaStream_t s)
{
    int t = P.nscenes < 1024 ? ((P.nscenes + 31) / 32) * 32 : 1024;
    int b = (P.nscenes + t - 1) / t;
    k_step_begin<<<b, t, 0, s>>>(P);
}
// Sweep kernels take T from the context (threads per particle) and the gather batch B
// of the Jacobi passes from its tuning: (T, B) in {(1, 4), (1, 8), (2, 4), (4, 4)}.
void launch_density_alpha(const Ptrs &P, cudaStream_t s)
{
#define SPH_L(T) k_density_alpha<T><<<P.ntblk, kBlock, 0, s>>>(P)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
}
void launch_pass_a(const Ptrs &P, int solver, int batch, cudaStream_t s)
{
#define SPH_A(S, B, T) k_pass_a<S, B, T><<<P.ntblk, kBlock, 0, s>>>(P)
    if (P.lanes == 4) { if (solver == 0) SPH_A(0, 4, 4); else SPH_A(1, 4, 4); }
    else if (P.lanes == 8) { if (solver == 0) SPH_A(0, 4, 8); else SPH_A(1, 4, 8); }
    else if (P.lanes == 2) { if (solver == 0) SPH_A(0, 4, 2); else SPH_A(1, 4, 2); }
    else if (batch == 8) { if (solver == 0) SPH_A(0, 8, 1); else SPH_A(1, 8, 1); }
    else { if (solver == 0) SPH_A(0, 4, 1); else SPH_A(1, 4, 1); }
#undef SPH_A
}
void launch_pass_b(const Ptrs &P, int solver, int warm, int batch, cudaStream_t s)
{
#define SPH_B(S, W, B, T) k_pass_b<S, W, B, T><<<P.ntblk, kBlock, 0, s>>>(P)
#define SPH_BW(B, T)                                                 \
    do {                                                             \
        if (solver == 0) { if (warm) SPH_B(0, 1, B, T); else SPH_B(0, 0, B, T); } \
        else { if (warm) SPH_B(1, 1, B, T); else SPH_B(1, 0, B, T); }             \
    } while (0)
    if (P.lanes == 4) SPH_BW(4, 4);
    else if (P.lanes == 8) SPH_BW(4, 8);
    else if (P.lanes == 2) SPH_BW(4, 2);
    else if (batch == 8) SPH_BW(8, 1);
    else SPH_BW(4, 1);
#undef SPH_BW
#undef SPH_B
}
void launch_solver_check(const Ptrs &P, int solver, cudaGraphConditionalHandle h, int use_handle, cudaStream_t s)
{
    if (solver == 0) k_solver_check<0><<<1, kCheckThreads, 0, s>>>(P, h, use_handle);
    else k_solver_check<1><<<1, kCheckThreads, 0, s>>>(P, h, use_handle);
}
void launch_nonpressure(const Ptrs &P, cudaStream_t s)
{
#define SPH_L(T) k_nonpressure<T><<<P.ntblk, kBlock, 0, s>>>(P)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
}
void launch_warm_density(const Ptrs &P, cudaStream_t s)
{
#define SPH_L(T) k_warm_density<T><<<P.ntblk, kBlock, 0, s>>>(P)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
}
void launch_advect(const Ptrs &P, cudaStream_t s) { k_advect<<<P.nfblk, kBlock, 0, s>>>(P); }
void launch_step_end(const Ptrs &P, cudaStream_t s) { k_step_end<<<1, 128, 0, s>>>(P); }
void launch_set_dt(const Ptrs &P, float dt, cudaStream_t s) { k_set_dt<<<1, 1, 0, s>>>(P.ctl, dt); }

}  // namespace sph
