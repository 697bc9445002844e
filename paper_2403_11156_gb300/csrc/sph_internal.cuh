// sph_internal.cuh -- device-side data layout and kernel launchers of the DFSPH pipeline.
//
// Layout in HBM (all scenes of a context concatenated; a scene is a contiguous range):
//   fluid, current sorted order  pos_s  float4 (x, y, z, kappa/rho of the current sweep)
//                                vel_s  float4 (v, rho)
//   fluid, canonical order       pos_c, vel_c (same packing), kprev_c, kvprev_c, id_c
//   neighbour lists              nbr[k * NF + i], bnbr[k * NF + i]  (k-major: coalesced)
//   boundary, original order     bx_o float4 (x, 0), bv_o float4, br0 float4, bbody int32
//   boundary, sorted order       bpos_s float4 (x, Psi), bvel_s float4 (v_b, 0)
// "Canonical" is the sorted order of the previous step: the reorder gathers canonical ->
// sorted, the step ends by writing the advected state back into the canonical arrays.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "sph.h"

namespace sph {

constexpr int kBlock = 128;           // threads per particle block
constexpr int kMaxBodies = 64;

// Per-scene constants (device, read-only during a step).
struct SceneDev {
    int64_t f_off, nf;                // fluid range
    int64_t b_off, nb;                // boundary range
    int64_t c_off;                    // first global cell of this scene's grid
    int32_t dims[3];
    int32_t ncell;
    float origin[3];
    float cell;
    float h, h2, inv_h;
    float m;                          // particle mass rho0 (2r)^3
    float rho0;
    float sigma;                      // W(0) = 8/(pi h^3)
    float kgrad;                      // 48/(pi h^4): grad W = kgrad g(q) x/|x|
    float eps_alpha;                  // alpha guard on the denominator
    float mu;                         // nu rho0
    float xsph;
    float g[3];
    float eta[2];                     // [0] divergence, [1] density
    float dt_max, cfl, two_r;
    int32_t min_it[2], max_it[2];
    int32_t visc_mode, warm, div_on, has_moving;
    int32_t body_off, nbody;
    int32_t fblk_first, fblk_count;   // fluid particle blocks of this scene
    int32_t bblk_first, bblk_count;   // boundary particle blocks
    int32_t tblk_first, tblk_count;   // sweep blocks (kBlock / lanes particles each)
    int32_t cap_f, cap_b;             // neighbour list capacities (per particle)
    int32_t R;                        // stencil radius in cells: 1 (cell >= h), 2 (cell >= h/2)
    float cg_tol;
    int32_t cg_max;
    float cull2;                      // (h + margin)^2: stencil cells farther are skipped
    int32_t solver;                   // 0 DFSPH, 1 WCSPH, 2 PCISPH
    float eos_k, eos_gamma;           // WCSPH equation of state
    float pci_c;                      // PCISPH prototype stiffness times dt^2
    float warm_frac;                  // fraction of the previous stiffness warm-starting a solve
    int32_t strong;                   // strong rigid coupling: bodies pushed during the solves
    float learned_frac;               // fraction of the network's stiffness warm-starting it
    int32_t learned_gate;             // the network runs only above this many density iterations
    double err_scale;                 // 1 / (nf rho0): a solve's error sum to its mean per rho0
};

// Per-scene mutable state (device).
struct SceneState {
    float dt, dt_next;
    float maxv2;                      // written via atomicMax on the bit pattern
    int32_t flags;
    int32_t it[2];                    // iterations of the current step
    double err[2], err0[2];
    uint32_t counter;                 // last-block counter of the CG's initial residual
    int32_t max_nn_f, max_nn_b;
    int32_t cg_it;
    float cg_res;
    int32_t cg_active;
    int32_t clamps;
    double cg_rr, cg_bb, cg_alpha, cg_beta;
    int64_t steps;
    int64_t total_it[2];
    int32_t last_it[2];               // iterations of the previous step
    int32_t pad_s[2];
};

// Rigid body state (device, FP64).
struct BodyDev {
    double mass, inertia[3];
    double inv_mass, inv_inertia[3];  // reciprocals, set with the mass (FP64 division is slow)
    double com[3], quat[4], vel[3], omega[3];
    double force[3], torque[3];
    double radius;                    // bounding sphere of its boundary particles
    double lo[3], hi[3];              // clamp box of the centre of mass
    int32_t scene;
    int32_t pad;
};

// State of one decoupled look-back scan: tile ticket, finished tiles, epoch of the tile
// words (the fluid and the boundary sort each own one, so the two can run concurrently).
struct ScanCtl {
    int32_t tile_counter;
    int32_t done;
    uint32_t epoch;
    int32_t pad;
};

// Context-wide control words (device).
struct Control {
    uint32_t probe_flag;              // never set: the wait of sph_probe_wait_timeout
    uint32_t loop_flag;               // host-readable copy of the loop condition
    uint32_t loop_guard;              // iterations of the current loop
    uint32_t pad0;
    int64_t launches;                 // kernel launches counted on the device
    float dt_override;                // > 0: fixed step for all scenes
    int32_t nscenes;
    ScanCtl scan[2];                  // look-back state of the fluid (0) and boundary (1) sorts
    int32_t error;                    // bounded-wait failures
    int32_t have_mlp;                 // warm-start network loaded
    uint32_t trace_n, trace_cap;      // device trace: stamps written / capacity
    unsigned long long *trace;        // (globaltimer << 8 | kernel id) per launch, or null
    int32_t mlp_n;                    // rows the warm-start network runs on this step
    int32_t pad1;
    int32_t nlarge[2];                // crowded cells of the fluid (0) / boundary (1) sort
};

// Kernel identifiers of the device trace.
enum KernelId : uint32_t {
    KID_STEP_BEGIN = 1,
    KID_KEY_HIST_F = 2,
    KID_KEY_HIST_B = 3,
    KID_SCAN = 4,
    KID_SCATTER_F = 5,
    KID_SCATTER_B = 6,
    KID_RANK_F = 7,
    KID_RANK_B = 8,
    KID_DENSITY = 9,
    KID_PASS_A0 = 10,
    KID_PASS_A1 = 11,
    KID_PASS_B0 = 12,
    KID_PASS_B1 = 13,
    KID_PASS_B0W = 14,
    KID_PASS_B1W = 15,
    KID_NONP = 16,
    KID_WARM = 17,
    KID_ADVECT = 18,
    KID_STEP_END = 19,
    KID_SET_DT = 20,
    KID_BUPDATE = 21,
    KID_PSI = 22,
    KID_BFORCE = 23,
    KID_BREDUCE = 24,
    KID_CG_INIT = 25,
    KID_CG_AP = 26,
    KID_CG_XR = 27,
    KID_CG_P = 28,
    KID_MLP_WARM = 29,
    KID_BFORCE_INC = 30,
    KID_BAPPLY = 31,
    KID_BVEL = 32,
    KID_CHECK0 = 33,
    KID_CHECK1 = 34,
    KID_CG_ALPHA = 35,
    KID_CG_BETA = 36,
    KID_BTOUCH = 37,
    KID_RANK_LARGE_F = 38,
    KID_RANK_LARGE_B = 39
};

static_assert(KID_STEP_BEGIN == SPH_KID_STEP_BEGIN, "trace id");
static_assert(KID_KEY_HIST_F == SPH_KID_KEY_HIST_F, "trace id");
static_assert(KID_KEY_HIST_B == SPH_KID_KEY_HIST_B, "trace id");
static_assert(KID_SCAN == SPH_KID_SCAN, "trace id");
static_assert(KID_SCATTER_F == SPH_KID_SCATTER_F, "trace id");
static_assert(KID_SCATTER_B == SPH_KID_SCATTER_B, "trace id");
static_assert(KID_RANK_F == SPH_KID_RANK_F, "trace id");
static_assert(KID_RANK_B == SPH_KID_RANK_B, "trace id");
static_assert(KID_DENSITY == SPH_KID_DENSITY, "trace id");
static_assert(KID_PASS_A0 == SPH_KID_PASS_A0, "trace id");
static_assert(KID_PASS_A1 == SPH_KID_PASS_A1, "trace id");
static_assert(KID_PASS_B0 == SPH_KID_PASS_B0, "trace id");
static_assert(KID_PASS_B1 == SPH_KID_PASS_B1, "trace id");
static_assert(KID_PASS_B0W == SPH_KID_PASS_B0W, "trace id");
static_assert(KID_PASS_B1W == SPH_KID_PASS_B1W, "trace id");
static_assert(KID_NONP == SPH_KID_NONP, "trace id");
static_assert(KID_WARM == SPH_KID_WARM, "trace id");
static_assert(KID_ADVECT == SPH_KID_ADVECT, "trace id");
static_assert(KID_STEP_END == SPH_KID_STEP_END, "trace id");
static_assert(KID_SET_DT == SPH_KID_SET_DT, "trace id");
static_assert(KID_BUPDATE == SPH_KID_BUPDATE, "trace id");
static_assert(KID_PSI == SPH_KID_PSI, "trace id");
static_assert(KID_BFORCE == SPH_KID_BFORCE, "trace id");
static_assert(KID_BREDUCE == SPH_KID_BREDUCE, "trace id");
static_assert(KID_CG_INIT == SPH_KID_CG_INIT, "trace id");
static_assert(KID_CG_AP == SPH_KID_CG_AP, "trace id");
static_assert(KID_CG_XR == SPH_KID_CG_XR, "trace id");
static_assert(KID_CG_P == SPH_KID_CG_P, "trace id");
static_assert(KID_MLP_WARM == SPH_KID_MLP_WARM, "trace id");
static_assert(KID_BFORCE_INC == SPH_KID_BFORCE_INC, "trace id");
static_assert(KID_BAPPLY == SPH_KID_BAPPLY, "trace id");
static_assert(KID_BVEL == SPH_KID_BVEL, "trace id");
static_assert(KID_CHECK0 == SPH_KID_CHECK0, "trace id");
static_assert(KID_CHECK1 == SPH_KID_CHECK1, "trace id");
static_assert(KID_CG_ALPHA == SPH_KID_CG_ALPHA, "trace id");
static_assert(KID_CG_BETA == SPH_KID_CG_BETA, "trace id");
static_assert(KID_BTOUCH == SPH_KID_BTOUCH, "trace id");
static_assert(KID_RANK_LARGE_F == SPH_KID_RANK_LARGE_F, "trace id");
static_assert(KID_RANK_LARGE_B == SPH_KID_RANK_LARGE_B, "trace id");

// First thread of every kernel: count the launch and, when tracing, stamp its start.
__device__ __forceinline__ void kernel_enter(Control *ctl, uint32_t id)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->launches), 1ull);
        unsigned long long *tr = ctl->trace;
        if (tr) {
            const uint32_t k = atomicAdd(&ctl->trace_n, 1u);
            if (k < ctl->trace_cap) {
                unsigned long long t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                tr[k] = (t << 8) | id;
            }
        }
    }
}

struct Ptrs {
    const SceneDev *scenes;
    SceneState *st;
    Control *ctl;
    BodyDev *bodies;
    const int32_t *fblk_scene;        // scene of each fluid block
    const int32_t *bblk_scene;        // scene of each boundary block
    const int32_t *tblk_scene;        // scene of each sweep block
    int32_t nfblk, nbblk, nscenes, nbodies_total;
    int32_t ntblk;                    // sweep blocks
    int32_t lanes;                    // threads per fluid particle in the sweeps: 1, 2, 4, 8
    int64_t NF, NB, NC;               // totals: fluid, boundary, cells
    // fluid
    float4 *pos_s, *vel_s, *pos_c, *vel_c;
    float *kprev_c, *kvprev_c, *kprev_s, *kvprev_s;
    float *ksum, *kvsum, *alpha, *k0;
    int32_t *id_c, *id_s;
    int32_t *nnf, *nnb;               // neighbour counts (capped at the list capacity)
    int32_t *nbr, *bnbr;
    float *feat;                      // [NF][4]
    // grid scratch (fluid)
    uint32_t *cell_count, *cell_start;
    uint32_t *key_tmp, *slot_tmp;
    uint32_t *sid_tmp, *src_tmp, *cell_tmp;
    // boundary
    float4 *bx_o, *bv_o, *br0;
    int32_t *bbody;
    float4 *bpos_s, *bvel_s;
    int32_t *bid_s;
    int32_t *bbody_s;
    uint32_t *bcell_count, *bcell_start;
    uint32_t *bkey_tmp, *bslot_tmp, *bsid_tmp, *bsrc_tmp, *bcell_tmp;
    uint32_t *large_f, *large_b;      // crowded cells of the fluid / boundary sort (lists)
    // reductions
    double *partial;                  // [ntblk] pass A's FP64 error partial per block
    double *partial2;                 // [ntblk] pass B's folds of kFold partials
    double *body_partial;             // [body][6][ntblk] per-block force/torque partials
    unsigned long long *blk_touch;    // [ntblk] bodies each sweep block touches (strong coupling)
    uint64_t *scan_status;            // [tiles] look-back words of the fluid sort
    uint64_t *bscan_status;           // [tiles] and of the boundary sort
    int32_t scan_tiles;
    // implicit viscosity CG
    float4 *cg_r, *cg_p, *cg_ap;
    double *cg_dots;                  // per-block partials [max(nfblk, ntblk)][2]
    // network
    float *mlp_w;                     // device parameter block (float)
    int2 *mlp_rows;                   // [nlearned] gated (particle, scene) rows of the step
    int64_t nlearned;                 // fluid particles of learned-warm-start scenes
};

// ------------------------------------------------------------------ grid (sph_grid.cu)
// Cell coordinate under the float contract: clamp(floor((x - o)/c), 0, n-1).
__device__ __forceinline__ int32_t cell_coord(float x, float o, float c, int32_t n)
{
    float t = __fdiv_rn(__fsub_rn(x, o), c);
    if (!(t > 0.0f)) return 0;
    if (t >= (float)(n - 1)) return n - 1;
    return (int32_t)floorf(t);
}

// Neighbour predicate contract: d2 = ((dx*dx)+(dy*dy))+(dz*dz) in float, no FMA, d2 < h2.
// Whether a scene's Jacobi solve s (0 divergence, 1 density) takes another iteration: its
// pass A and B run, and so does the strong-coupling body update after them, exactly when
// this holds (the state only changes in the check kernel that ends the iteration).
__device__ __forceinline__ bool solver_active(const SceneDev &sc, const SceneState &st, int s)
{
    if (s == 0 && !sc.div_on) return false;
    int it = st.it[s];
    if (it >= sc.max_it[s]) return false;
    return it < sc.min_it[s] || st.err[s] > (double)sc.eta[s];
}

// Whether a scene's warm-start pass of solve s applies a pressure: its warm start (the
// divergence solve's only where that solve runs), or for a WCSPH scene the equation-of-state
// pressure, which the density solve's warm pass applies once.
__device__ __forceinline__ bool warm_pass_runs(const SceneDev &sc, int s)
{
    return (sc.warm != 0 && (s == 1 || sc.div_on)) || (s == 1 && sc.solver == 1);
}

// The strong-coupling body update applies where its scene's pass B just ran: phase s (0
// divergence, 1 density) inside that solve's Jacobi loop, 2 + s after its warm-start pass
// (a negative phase: unconditionally).
__device__ __forceinline__ bool strong_update_applies(const SceneDev &sc, const SceneState &st, int phase)
{
    if (phase < 0) return true;
    return phase >= 2 ? warm_pass_runs(sc, phase - 2) : solver_active(sc, st, phase);
}

__device__ __forceinline__ float pred_d2(float4 a, float4 b, float &dx, float &dy, float &dz)
{
    dx = __fsub_rn(a.x, b.x);
    dy = __fsub_rn(a.y, b.y);
    dz = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// The same d2 with the x and y differences and squares as packed FP32 pairs (axy holds a.x in
// its low half, a.y in its high half): each half rounds like the scalar operation, and the
// sums keep the order above, so the value is identical, in fewer instructions.
__device__ __forceinline__ unsigned long long pack_xy(float x, float y)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float pred_d2_xy2(unsigned long long axy, float az, float4 b)
{
    unsigned long long d, q;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(axy), "l"(pack_xy(b.x, b.y)));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(q) : "l"(d));
    float qx, qy;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(qx), "=f"(qy) : "l"(q));
    const float dz = __fsub_rn(az, b.z);
    return __fadd_rn(__fadd_rn(qx, qy), __fmul_rn(dz, dz));
}

enum SortWhat { SORT_FLUID = 0, SORT_BOUNDARY = 1 };

void launch_key_hist(const Ptrs &P, SortWhat what, cudaStream_t s);
void launch_scan_cells(const Ptrs &P, SortWhat what, cudaStream_t s);
void launch_scatter(const Ptrs &P, SortWhat what, cudaStream_t s);
void launch_rank_gather(const Ptrs &P, SortWhat what, cudaStream_t s);
void launch_scan(uint32_t *count, uint32_t *start, int64_t n, uint64_t *status, int32_t tiles,
                 ScanCtl *sc, Control *ctl, cudaStream_t s);
int32_t scan_tiles_for(int64_t n);

// In-cell ranking: a cell of at most kRankSmall particles ranks each one by counting the
// cell's smaller ids (O(occupancy) per particle); a more crowded cell is queued and sorted
// by one block with a stable radix sort (O(occupancy) per pass), so no input makes the
// grid order quadratic.
constexpr uint32_t kRankSmall = 64;
int64_t large_capacity(int64_t n);   // queue entries a sort of n particles can need

// ------------------------------------------------------------------ fluid (sph_fluid.cu)
void launch_step_begin(const Ptrs &P, cudaStream_t s);
void launch_density_alpha(const Ptrs &P, cudaStream_t s);
void launch_pass_a(const Ptrs &P, int solver, int batch, cudaStream_t s);
void launch_pass_b(const Ptrs &P, int solver, int warm, int batch, cudaStream_t s);
void launch_solver_check(const Ptrs &P, int solver, cudaGraphConditionalHandle h, int use_handle, cudaStream_t s);
void launch_nonpressure(const Ptrs &P, cudaStream_t s);
void launch_warm_density(const Ptrs &P, cudaStream_t s);
void launch_advect(const Ptrs &P, cudaStream_t s);
void launch_step_end(const Ptrs &P, cudaStream_t s);
void launch_set_dt(const Ptrs &P, float dt, cudaStream_t s);

// ------------------------------------------------------------------ network (sph_mlp.cu)
void launch_mlp_warm(const Ptrs &P, cudaStream_t s);
cudaError_t mlp_prepare_kernels();

// ------------------------------------------------------------------ implicit viscosity (sph_visc.cu)
void launch_cg_init(const Ptrs &P, cudaStream_t s);
void launch_cg_ap(const Ptrs &P, cudaStream_t s);
void launch_cg_alpha(const Ptrs &P, cudaStream_t s);
void launch_cg_xr(const Ptrs &P, cudaStream_t s);
void launch_cg_beta(const Ptrs &P, cudaGraphConditionalHandle h, int use_handle, cudaStream_t s);
void launch_cg_p(const Ptrs &P, cudaStream_t s);

// ------------------------------------------------------------------ post-processing (sph_post.cu)
cudaError_t post_surface_field(const SceneDev &sc, const float4 *pos, const float4 *vel, const float origin[3],
                               float spacing, const int32_t dims[3], float *out, cudaStream_t s);
cudaError_t post_height_map(const float4 *pos, int64_t n, const float lo[2], const float hi[2], int32_t w,
                            int32_t h, float radius, float *out, cudaStream_t s);

// ------------------------------------------------------------------ rigid (sph_rigid.cu)
void launch_boundary_update(const Ptrs &P, cudaStream_t s);
void launch_boundary_psi(const Ptrs &P, cudaStream_t s);
void launch_body_force(const Ptrs &P, cudaStream_t s);
void launch_body_reduce(const Ptrs &P, cudaStream_t s);
void launch_body_touch(const Ptrs &P, cudaStream_t s);
// Strong coupling: the body update from the stiffness just applied, in the scenes whose pass
// B just ran (phase as for strong_update_applies: 0 or 1 in that solve's Jacobi loop, 2 + s
// after solve s's warm-start pass).
void launch_strong_update(const Ptrs &P, int phase, cudaStream_t s);

}  // namespace sph
