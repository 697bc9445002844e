// sph_rigid.cu -- Akinci boundary handling and two-way rigid coupling (Sec. 3.5).
//
//  * boundary pseudo-mass Psi_b = rho0 / sum_k W_bk over boundary neighbours, the
//    particle itself included (all walls and bodies count);
//  * moving-body boundary particles follow their body: x_b = com + R r0_b,
//    v_b = v + omega x (R r0_b);
//  * the reaction of Eq. rigid_pressure_symmetric: F_{b<-i} = m Psi_b (kappa_i/rho_i)
//    grad W_ib with the step's total applied kappa (divergence + density solves), summed
//    per body with its torque in FP64 and reduced in a fixed order.
#include "sph_sweep.cuh"

namespace sph {

namespace {

// Boundary particles of moving bodies follow their body (original order).
__global__ void __launch_bounds__(kBlock) k_boundary_update(Ptrs P)
{
    kernel_enter(P.ctl, KID_BUPDATE);
    const SceneDev &sc = P.scenes[P.bblk_scene[blockIdx.x]];
    if (!sc.has_moving) return;
    int64_t local = (int64_t)(blockIdx.x - sc.bblk_first) * kBlock + threadIdx.x;
    if (local >= sc.nb) return;
    int64_t b = sc.b_off + local;
    int32_t k = P.bbody[b];
    if (k < 0) return;
    const BodyDev &B = P.bodies[sc.body_off + k];
    double w = B.quat[0], x = B.quat[1], y = B.quat[2], z = B.quat[3];
    float4 r0 = P.br0[b];
    double rx = r0.x, ry = r0.y, rz = r0.z;
    double wx = (1 - 2 * (y * y + z * z)) * rx + 2 * (x * y - w * z) * ry + 2 * (x * z + w * y) * rz;
    double wy = 2 * (x * y + w * z) * rx + (1 - 2 * (x * x + z * z)) * ry + 2 * (y * z - w * x) * rz;
    double wz = 2 * (x * z - w * y) * rx + 2 * (y * z + w * x) * ry + (1 - 2 * (x * x + y * y)) * rz;
    P.bx_o[b] = make_float4((float)(B.com[0] + wx), (float)(B.com[1] + wy), (float)(B.com[2] + wz), 0.0f);
    P.bv_o[b] = make_float4((float)(B.vel[0] + (B.omega[1] * wz - B.omega[2] * wy)),
                            (float)(B.vel[1] + (B.omega[2] * wx - B.omega[0] * wz)),
                            (float)(B.vel[2] + (B.omega[0] * wy - B.omega[1] * wx)), 0.0f);
}

// Psi_b = rho0 / (sigma (1 + sum_k w(q_bk)))  (grid order; stored in bpos_s.w).  Every
// scene's: a per-step boundary sort (any moving body in the context) rebuilds the grid
// order, and with it the w slot, of every scene's boundary, static walls included.
__global__ void __launch_bounds__(kBlock) k_boundary_psi(Ptrs P)
{
    kernel_enter(P.ctl, KID_PSI);
    const SceneDev &sc = P.scenes[P.bblk_scene[blockIdx.x]];
    int64_t local = (int64_t)(blockIdx.x - sc.bblk_first) * kBlock + threadIdx.x;
    if (local >= sc.nb) return;
    int64_t b = sc.b_off + local;
    const float4 pb = P.bpos_s[b];
    const int32_t cx = cell_coord(pb.x, sc.origin[0], sc.cell, sc.dims[0]);
    const int32_t cy = cell_coord(pb.y, sc.origin[1], sc.cell, sc.dims[1]);
    const int32_t cz = cell_coord(pb.z, sc.origin[2], sc.cell, sc.dims[2]);
    const int32_t R = sc.R;
    const int32_t x0 = max(cx - R, 0), x1 = min(cx + R, sc.dims[0] - 1);
    const float h2 = sc.h2, inv_h = sc.inv_h;
    float ws = 0.0f;
    for (int32_t dz = -R; dz <= R; ++dz) {
        const int32_t z = cz + dz;
        if (z < 0 || z >= sc.dims[2]) continue;
        for (int32_t dy = -R; dy <= R; ++dy) {
            const int32_t y = cy + dy;
            if (y < 0 || y >= sc.dims[1]) continue;
            const int64_t row = sc.c_off + (int64_t)sc.dims[0] * (y + (int64_t)sc.dims[1] * z);
            const uint32_t jb = P.bcell_start[row + x0], je = P.bcell_start[row + x1 + 1];
            for (uint32_t k = jb; k < je; ++k) {
                if ((int64_t)k == b) continue;
                float dx, dy2, dz2;
                const float d2 = pred_d2(pb, P.bpos_s[k], dx, dy2, dz2);
                if (!(d2 < h2)) continue;
                ws += spline_w(sqrtf(d2) * inv_h);
            }
        }
    }
    reinterpret_cast<float *>(P.bpos_s + b)[3] = sc.rho0 / (sc.sigma * (1.0f + ws));
}

// Force and torque of the fluid on each body of the scene (the T lanes of a particle share
// its boundary list; the block sums add all lanes), as per-block partials.  INC = false:
// weakly coupled scenes, from the step's total applied stiffness after the solves;
// INC = true: strongly coupled scenes, from the stiffness just applied (kappa/rho of the
// current sweep).
template <int T, bool INC>
__global__ void __launch_bounds__(kBlock) k_body_force(Ptrs P, int phase)
{
    __shared__ double sh6[kBlock / 32][6];
    kernel_enter(P.ctl, INC ? KID_BFORCE_INC : KID_BFORCE);
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    if (sc.nbody == 0 || (sc.strong != 0) != INC) return;  // uniform per block
    // in a batch, a scene whose pass B did not run (its solve has stopped, or it has no warm
    // start) applied no stiffness here: its bodies and their boundary velocities stay as they
    // would alone
    if (INC && !strong_update_applies(sc, *c.st, phase)) return;
    const int64_t i = c.i, NF = P.NF;
    const int nb = c.valid ? P.nnb[i] : 0;
    // which bodies this block's particles touch (most blocks touch none, or only walls).
    // Strong coupling reads the step's mask (k_body_touch) and leaves untouched blocks
    // at once, writing nothing: the apply kernel skips their partials.  The weak path
    // finds the mask here and writes zero partials for untouched bodies.
    unsigned long long touched;
    if (INC) {
        touched = P.blk_touch[blockIdx.x];
        if (touched == 0ull) return;  // uniform per block
    } else {
        __shared__ unsigned long long s_mask;
        if (threadIdx.x == 0) s_mask = 0ull;
        __syncthreads();
        unsigned long long mine = 0ull;
        for (int t = c.s; t < nb; t += T) {
            const int32_t k = P.bbody_s[P.bnbr[(int64_t)t * NF + i]];
            if (k >= 0) mine |= 1ull << k;
        }
        if (mine) atomicOr(&s_mask, mine);
        __syncthreads();
        touched = s_mask;
    }
    // the particle's own state is needed only in blocks that touch a body, and there only
    // by particles with boundary neighbours
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    float kt = 0.0f;
    if (touched && nb > 0) {
        pi = P.pos_s[i];
        kt = INC ? pi.w : (P.ksum[i] + P.kvsum[i]) / P.vel_c[i].w;
    }
    for (int k = 0; k < sc.nbody; ++k) {
        double f[6] = {0, 0, 0, 0, 0, 0};
        const bool any = (touched >> k) & 1ull;
        if (any) {
            const BodyDev &B = P.bodies[sc.body_off + k];
            const Spline sp(sc);
            for (int t = c.s; t < nb; t += T) {
                const int32_t b = P.bnbr[(int64_t)t * NF + i];
                if (P.bbody_s[b] != k) continue;
                const float4 pb = P.bpos_s[b];
                const float dx = pi.x - pb.x, dy = pi.y - pb.y, dz = pi.z - pb.z;
                const float g = grad_factor(sp, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                const double s = (double)sc.m * (double)pb.w * (double)kt * (double)g;
                const double Fx = s * dx, Fy = s * dy, Fz = s * dz;
                const double rx = (double)pb.x - B.com[0], ry = (double)pb.y - B.com[1], rz = (double)pb.z - B.com[2];
                f[0] += Fx; f[1] += Fy; f[2] += Fz;
                f[3] += ry * Fz - rz * Fy;
                f[4] += rz * Fx - rx * Fz;
                f[5] += rx * Fy - ry * Fx;
            }
        }
        if (INC && !any) continue;   // the apply kernel skips this block for body k
        double *part = P.body_partial + (int64_t)(sc.body_off + k) * 6 * P.ntblk + blockIdx.x;
        if (!any) {
            if (threadIdx.x < 6) part[(int64_t)threadIdx.x * P.ntblk] = 0.0;
            continue;
        }
        // the six components in one pass (each the same butterfly and the same fold over the
        // warps, in the same order, as a sum of its own): two barriers instead of twelve
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) f[a] += __shfl_xor_sync(0xffffffffu, f[a], o);
        __syncthreads();   // the previous body's reads of sh6 are done
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int a = 0; a < 6; ++a) sh6[threadIdx.x >> 5][a] = f[a];
        __syncthreads();
        if (threadIdx.x < 6) {
            double t = 0.0;
            for (int w = 0; w < kBlock / 32; ++w) t += sh6[w][threadIdx.x];
            part[(int64_t)threadIdx.x * P.ntblk] = t;
        }
    }
}

// Strong coupling: the bodies each sweep block's particles touch, once per step (positions
// and neighbour lists are fixed from the density sweep to the advection), as a bit mask of
// the scene's bodies; blocks of other scenes get 0.
template <int T>
__global__ void __launch_bounds__(kBlock) k_body_touch(Ptrs P)
{
    __shared__ unsigned long long s_mask;
    kernel_enter(P.ctl, KID_BTOUCH);
    const Lane<T> c = lane_ctx<T>(P);
    const SceneDev &sc = *c.sc;
    if (threadIdx.x == 0) s_mask = 0ull;
    __syncthreads();
    if (sc.strong && sc.nbody > 0) {   // uniform per block
        const int64_t NF = P.NF;
        const int nb = c.valid ? P.nnb[c.i] : 0;
        unsigned long long mine = 0ull;
        for (int t = c.s; t < nb; t += T) {
            const int32_t k = P.bbody_s[P.bnbr[(int64_t)t * NF + c.i]];
            if (k >= 0) mine |= 1ull << k;
        }
        if (mine) atomicOr(&s_mask, mine);
    }
    __syncthreads();
    if (threadIdx.x == 0) P.blk_touch[blockIdx.x] = s_mask;
}

// Sum of one body's force or torque component over its scene's sweep blocks, in block
// order (one CUDA block per body and component).
__global__ void __launch_bounds__(256) k_body_reduce(Ptrs P)
{
    __shared__ double sh[8];
    kernel_enter(P.ctl, KID_BREDUCE);
    const int body = blockIdx.x / 6, a = blockIdx.x % 6;
    BodyDev &B = P.bodies[body];
    const SceneDev &sc = P.scenes[B.scene];
    if (sc.strong) return;   // strongly coupled bodies take their forces during the solves
    const double *part = P.body_partial + ((int64_t)body * 6 + a) * P.ntblk + sc.tblk_first;
    double t = 0.0;
#pragma unroll 4
    for (int q = threadIdx.x; q < sc.tblk_count; q += 256) t += part[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += sh[w];
        if (a < 3) B.force[a] = tot;
        else B.torque[a - 3] = tot;
    }
}

// Strong coupling: one block per body sums the partials of the stiffness just applied (in
// block order), adds them to the step's force and torque and applies the impulse,
// v += dt F / M, omega += dt I^-1 tau (world inertia of the step's orientation).
__global__ void __launch_bounds__(256) k_body_apply(Ptrs P, int phase)
{
    __shared__ double sh6[8][6];
    __shared__ double s_f[6];
    kernel_enter(P.ctl, KID_BAPPLY);
    const int body = blockIdx.x;
    BodyDev &B = P.bodies[body];
    const SceneDev &sc = P.scenes[B.scene];
    if (!sc.strong) return;
    if (!strong_update_applies(sc, P.st[B.scene], phase)) return;   // as k_body_force
    // the partials of the blocks that touch this body, in block order (thread t takes
    // blocks t, t + 256, ...; the other blocks contribute nothing)
    const int k = body - sc.body_off;
    double f[6] = {0, 0, 0, 0, 0, 0};
    for (int q = threadIdx.x; q < sc.tblk_count; q += 256) {
        if (!((P.blk_touch[sc.tblk_first + q] >> k) & 1ull)) continue;
        for (int a = 0; a < 6; ++a) f[a] += P.body_partial[((int64_t)body * 6 + a) * P.ntblk + sc.tblk_first + q];
    }
    // the six components in one pass (each the same butterfly and fold over the warps as a
    // sum of its own)
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f[a] += __shfl_xor_sync(0xffffffffu, f[a], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int a = 0; a < 6; ++a) sh6[threadIdx.x >> 5][a] = f[a];
    __syncthreads();
    if (threadIdx.x < 6) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += sh6[w][threadIdx.x];
        s_f[threadIdx.x] = tot;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double dt = (double)P.st[B.scene].dt;
    const double w = B.quat[0], x = B.quat[1], y = B.quat[2], z = B.quat[3];
    const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    // the body record's reciprocals (FP64 division is a long dependent sequence here)
    const double inv_m = B.inv_mass;
    const double inv_i[3] = {B.inv_inertia[0], B.inv_inertia[1], B.inv_inertia[2]};
    for (int a = 0; a < 3; ++a) {
        B.force[a] += s_f[a];
        B.torque[a] += s_f[3 + a];
        B.vel[a] += dt * s_f[a] * inv_m;
    }
    for (int a = 0; a < 3; ++a) {
        double d = 0.0;
        for (int e = 0; e < 3; ++e) {
            double ii = 0.0;
            for (int q = 0; q < 3; ++q) ii += R[a][q] * inv_i[q] * R[e][q];
            d += ii * s_f[3 + e];
        }
        B.omega[a] += dt * d;
    }
}

// Strong coupling: the boundary particles of strongly coupled bodies follow the updated
// body velocities, v_b = v + omega x (x_b - com) (grid order).  Only where the body update
// applied: the step-start values come from the body-frame offsets, these from the float
// boundary positions, and the two differ in the last bit, so a scene must see this kernel
// exactly where it would alone.
__global__ void __launch_bounds__(kBlock) k_boundary_vel(Ptrs P, int phase)
{
    kernel_enter(P.ctl, KID_BVEL);
    const int32_t scene = P.bblk_scene[blockIdx.x];
    const SceneDev &sc = P.scenes[scene];
    if (!sc.strong || sc.nbody == 0) return;
    if (!strong_update_applies(sc, P.st[scene], phase)) return;
    const int64_t local = (int64_t)(blockIdx.x - sc.bblk_first) * kBlock + threadIdx.x;
    if (local >= sc.nb) return;
    const int64_t b = sc.b_off + local;
    const int32_t k = P.bbody_s[b];
    if (k < 0) return;
    const BodyDev &B = P.bodies[sc.body_off + k];
    const float4 pb = P.bpos_s[b];
    const double rx = (double)pb.x - B.com[0], ry = (double)pb.y - B.com[1], rz = (double)pb.z - B.com[2];
    P.bvel_s[b] = make_float4((float)(B.vel[0] + (B.omega[1] * rz - B.omega[2] * ry)),
                              (float)(B.vel[1] + (B.omega[2] * rx - B.omega[0] * rz)),
                              (float)(B.vel[2] + (B.omega[0] * ry - B.omega[1] * rx)), 0.0f);
}

}  // namespace

void launch_body_touch(const Ptrs &P, cudaStream_t s)
{
    if (!P.ntblk || !P.nbodies_total) return;
#define SPH_L(T) k_body_touch<T><<<P.ntblk, kBlock, 0, s>>>(P)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
}

void launch_strong_update(const Ptrs &P, int phase, cudaStream_t s)
{
    if (!P.ntblk || !P.nbodies_total) return;
#define SPH_L(T) k_body_force<T, true><<<P.ntblk, kBlock, 0, s>>>(P, phase)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
    k_body_apply<<<P.nbodies_total, 256, 0, s>>>(P, phase);
    if (P.nbblk) k_boundary_vel<<<P.nbblk, kBlock, 0, s>>>(P, phase);
}

void launch_boundary_update(const Ptrs &P, cudaStream_t s)
{
    if (P.nbblk) k_boundary_update<<<P.nbblk, kBlock, 0, s>>>(P);
}
void launch_boundary_psi(const Ptrs &P, cudaStream_t s)
{
    if (P.nbblk) k_boundary_psi<<<P.nbblk, kBlock, 0, s>>>(P);
}
void launch_body_force(const Ptrs &P, cudaStream_t s)
{
    if (!P.ntblk) return;
#define SPH_L(T) k_body_force<T, false><<<P.ntblk, kBlock, 0, s>>>(P, -1)
    SPH_BY_LANES(P, SPH_L);
#undef SPH_L
}
void launch_body_reduce(const Ptrs &P, cudaStream_t s)
{
    if (P.nbodies_total) k_body_reduce<<<P.nbodies_total * 6, 256, 0, s>>>(P);
}

}  // namespace sph
