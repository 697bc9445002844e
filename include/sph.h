/*
 * sph.h -- C ABI of the GB300 (sm_103a) DFSPH particle pipeline.
 *
 * The calls follow the paper's statement of the problem (arXiv 2403.11156): a scene is
 * configured (Sec. 4.1: fluid and rigid particles, particle radius, rest density,
 * viscosity, domain), simulated step by step (Sec. 4.2: gravity, viscosity, pressure,
 * rigid and fluid update; DFSPH per Sec. 3.4.2 and Sec. 5), and its particles exported
 * (Sec. 4.3).  Every step of the pipeline runs in this library's CUDA kernels on one GPU.
 *
 * Conventions
 *  - Host arrays passed to sph_create are copied; the caller keeps ownership.
 *  - Output buffers are caller-owned; per-particle outputs are in the caller's original
 *    particle order (index = position in the arrays given to sph_create).
 *  - Coordinates are float32, [n][3] row-major (x, y, z), SI units (m, m/s, kg/m^3).
 *  - All device work is enqueued on the stream given at creation (NULL = legacy default
 *    stream).  sph_step returns once the step is enqueued; calls that return data
 *    synchronise that stream.
 *  - A context is not thread-safe.  SPH_ECUDA and SPH_ETIMEOUT poison a context: only
 *    sph_last_error and sph_destroy remain valid.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPH_ABI_VERSION 2

typedef enum sph_status {
    SPH_OK = 0,
    SPH_EINVAL = 1,       /* bad argument or scene descriptor; nothing was changed        */
    SPH_ENOMEM = 2,       /* a device or host allocation failed                           */
    SPH_ECUDA = 3,        /* a CUDA call failed; the context is poisoned                  */
    SPH_ENOCONVERGE = 4,  /* a solver stopped at max_iter above its tolerance; the state  */
                          /* was advanced with the last iterate (see sph_stats)           */
    SPH_ETIMEOUT = 5,     /* a bounded device-side wait gave up; the context is poisoned  */
    SPH_ENUMERIC = 6,     /* a non-finite position or velocity was produced               */
    SPH_EOVERFLOW = 7     /* a particle had more neighbours than the list capacity; that  */
                          /* step dropped the excess (raise max_*_neighbors)              */
} sph_status;

/* viscosity_mode */
#define SPH_VISC_NONE 0      /* gravity only                                               */
#define SPH_VISC_EXPLICIT 1  /* (mu/rho) times the Laplacian of Sec. 3.6.1 Eq. lap        */
#define SPH_VISC_XSPH 2      /* XSPH velocity smoothing with coefficient xsph_c            */
#define SPH_VISC_IMPLICIT 3  /* (I - dt A) v* = v~ of Sec. 3.6.2, matrix-free CG          */

/* pressure_solver */
#define SPH_SOLVER_DFSPH 0   /* divergence-free + constant-density Jacobi solves (Sec. 3.4.2) */
#define SPH_SOLVER_WCSPH 1   /* equation of state p = k ((rho/rho0)^gamma - 1), clamped at 0, */
                             /* applied once per step (Sec. 3.4.1, Alg. general_algorithm);  */
                             /* warm_start, divergence_solve and the iteration limits are    */
                             /* ignored                                                      */
#define SPH_SOLVER_PCISPH 2  /* predictive-corrective PPE solve (Alg. ppe_solver): the total */
                             /* pressure is refined by p <- max(p + delta (rho* - rho0), 0)   */
                             /* with a prototype particle's delta until the density error     */
                             /* meets eta_density (min/max_iter_density); no divergence       */
                             /* solve, no warm start                                          */

/* rigid_coupling */
#define SPH_COUPLING_WEAK 0    /* body velocities fixed during the fluid solves (Sec. 3.5);  */
                               /* the step's total reaction moves the bodies afterwards      */
#define SPH_COUPLING_STRONG 1  /* every pressure application of the solves also pushes the  */
                               /* bodies (dt F/M, dt I^-1 tau) and their boundary particles  */
                               /* follow before the next source term (the paper's stated    */
                               /* future work)                                               */

/* warm_start of the two DFSPH solves */
#define SPH_WARM_ZERO 0      /* kappa starts at zero                                       */
#define SPH_WARM_PREVIOUS 1  /* a fraction (warm_start_fraction, default half) of the       */
                             /* previous step's kappa where the fluid compresses          */
#define SPH_WARM_LEARNED 2   /* density solve: a fraction (learned_fraction) of a          */
                             /* per-particle network prediction (see sph_set_mlp) where   */
                             /* the fluid compresses; divergence solve as                 */
                             /* SPH_WARM_PREVIOUS                                          */

/* A rigid body (Sec. 3.5, two-way weak coupling; Sec. 4.1 initial pose and velocity). */
typedef struct sph_rigid_desc {
    double mass;       /* kg                                                        */
    double inertia[3]; /* principal moments in the body frame, kg m^2 (all > 0)     */
    double com[3];     /* initial centre of mass, m                                 */
    double quat[4];    /* initial orientation (w, x, y, z), unit                    */
    double vel[3];     /* initial linear velocity, m/s                              */
    double omega[3];   /* initial angular velocity (world frame), rad/s             */
} sph_rigid_desc;

/* One scene (Sec. 4.1).  Zero-initialise and fill; zero means "default" where noted. */
typedef struct sph_scene_desc {
    int64_t n_fluid;              /* fluid particles (>= 1)                           */
    const float *fluid_x;         /* host [n_fluid][3] positions                      */
    const float *fluid_v;         /* host [n_fluid][3] velocities, or NULL for zero   */
    int64_t n_boundary;           /* Akinci boundary particles (>= 0)                 */
    const float *boundary_x;      /* host [n_boundary][3]                             */
    const int32_t *boundary_body; /* host [n_boundary]: body index, -1 = static wall; */
                                  /* NULL = all static                                */
    int32_t n_bodies;             /* rigid bodies (0..SPH_MAX_BODIES)                 */
    const sph_rigid_desc *bodies; /* host [n_bodies]                                  */
    float radius;                 /* particle radius r; support h = 4r, mass          */
                                  /* rho0 (2r)^3 (Sec. 5)                             */
    float rest_density;           /* rho0, kg/m^3                                     */
    float viscosity;              /* kinematic nu at rest density (mu = nu rho0)      */
    float xsph_c;                 /* XSPH coefficient (SPH_VISC_XSPH only)            */
    float gravity[3];             /* m/s^2                                            */
    float domain_min[3];          /* grid extent; particles outside are clamped into  */
    float domain_max[3];          /* the edge cells (still correct, only slower)      */
    float cell_size;              /* 0 = h (1 + 2^-8) (27-cell stencil); >= h/2 (1 +  */
                                  /* 2^-8) for a 125-cell stencil; < 0 = autotune     */
    float eta_density;            /* mean relative density error tolerance (1e-3)     */
    float eta_divergence;         /* mean dt Drho/Dt / rho0 tolerance (1e-3)          */
    float dt_max;                 /* largest step, s                                  */
    float cfl;                    /* > 0: dt = min(dt_max, cfl 2r / max|v|)           */
    int32_t min_iter_density, max_iter_density;   /* max_iter is the hard cap (>= 0)  */
    int32_t min_iter_divergence, max_iter_divergence;
    int32_t viscosity_mode;       /* SPH_VISC_*                                       */
    int32_t warm_start;           /* SPH_WARM_*                                       */
    int32_t divergence_solve;     /* 1 = run the divergence-free solve                */
    int32_t max_fluid_neighbors;  /* list capacity per particle, 0 = 96               */
    int32_t max_boundary_neighbors; /* 0 = 64                                         */
    float cg_tol;                 /* relative residual of the implicit viscosity CG   */
    int32_t cg_max_iter;
    int32_t lanes_per_particle;   /* threads per fluid particle in the neighbour      */
                                  /* sweeps: 1, 2, 4 or 8 (they share the particle's  */
                                  /* list); 0 = by size (8 up to 38,912 fluid         */
                                  /* particles in the context, 4 up to twice that, 2  */
                                  /* up to four times, else 1).  A batch uses the     */
                                  /* largest value given by its scenes.                                   */
    int32_t pressure_solver;      /* SPH_SOLVER_*                                     */
    float eos_stiffness;          /* WCSPH k, Pa (> 0)                                */
    float eos_exponent;           /* WCSPH gamma (>= 1; 0 = 7)                        */
    float warm_start_fraction;    /* SPH_WARM_PREVIOUS: fraction of the previous      */
                                  /* step's stiffness (0..1; 0 = 0.5)                 */
    int32_t rigid_coupling;       /* SPH_COUPLING_*                                   */
    float learned_fraction;       /* SPH_WARM_LEARNED: fraction of the network's      */
                                  /* predicted stiffness applied (0..1; 0 = 0.6)      */
    int32_t learned_gate;         /* SPH_WARM_LEARNED: the network runs in a step     */
                                  /* only if the scene's previous density solve took  */
                                  /* more than this many iterations, else the step    */
                                  /* takes the previous-step warm start (0 = always   */
                                  /* the network; min_iter_density: skip it while the */
                                  /* solve sits at its floor)                         */
} sph_scene_desc;

#define SPH_MAX_BODIES 64

/* Statistics of one scene (the last completed step unless noted). */
typedef struct sph_stats {
    int64_t steps;               /* steps completed since creation                   */
    int32_t div_iters;           /* divergence-solve iterations                      */
    int32_t dens_iters;          /* constant-density iterations                      */
    double div_err;              /* last divergence error (mean dt Drho/Dt / rho0)   */
    double dens_err;             /* last density error (mean max(rho*-rho0,0)/rho0)  */
    double div_err0, dens_err0;  /* errors at the first iteration                    */
    float dt;                    /* step size used                                   */
    float dt_next;               /* CFL step size for the next step                  */
    float max_speed;             /* max |v| after the step                           */
    int32_t max_fluid_nbrs;      /* largest fluid neighbour count of the step        */
    int32_t max_boundary_nbrs;
    int32_t cg_iters;            /* implicit viscosity CG iterations                 */
    float cg_residual;           /* its final relative residual                      */
    int32_t clamps;              /* rigid-body domain clamps since creation          */
    int32_t flags;               /* SPH_FLAG_* seen since creation (sticky)          */
    int64_t total_div_iters;     /* since creation                                   */
    int64_t total_dens_iters;
} sph_stats;

#define SPH_FLAG_OVERFLOW 1
#define SPH_FLAG_NOCONVERGE 2
#define SPH_FLAG_NONFINITE 4
#define SPH_FLAG_TIMEOUT 8

/* Device memory callbacks (for example a framework's caching allocator).  alloc returns
 * NULL on failure; both are called only inside sph_create / sph_destroy. */
typedef struct sph_allocator {
    void *(*alloc)(void *user, size_t bytes, void *stream);
    void (*free)(void *user, void *ptr, size_t bytes, void *stream);
    void *user;
} sph_allocator;

typedef struct sph_ctx sph_ctx;

/* Library ABI version (SPH_ABI_VERSION). */
int32_t sph_abi_version(void);

/* Create a context for one scene (Sec. 4.1).  Copies the host arrays to the device,
 * builds the static boundary grid and its pseudo-masses Psi (Sec. 3.5) and captures the
 * step as a CUDA graph.  alloc may be NULL (cudaMalloc); stream is a cudaStream_t or
 * NULL.  On error *out is NULL and nothing leaks. */
sph_status sph_create(const sph_scene_desc *scene, const sph_allocator *alloc, void *stream,
                      sph_ctx **out);

/* Create a context holding n independent scenes of any sizes that step together: every
 * kernel of the step covers all scenes in one launch, and each scene's solver stops at
 * its own tolerance.  Scene s keeps index s in the calls below. */
sph_status sph_create_batch(const sph_scene_desc *scenes, int32_t n, const sph_allocator *alloc,
                            void *stream, sph_ctx **out);

/* Enqueue one DFSPH step of every scene (Sec. 4.2 order; Sec. 3.3 Alg. general_algorithm,
 * Sec. 3.4.2 Alg. ppe_solver for both solves).  dt > 0: that step size for all scenes;
 * dt <= 0: each scene's CFL step (dt_max when cfl <= 0).  Returns without waiting;
 * errors of the step surface at the next synchronising call. */
sph_status sph_step(sph_ctx *ctx, float dt);

/* Enqueue n steps (same dt rule). */
sph_status sph_steps(sph_ctx *ctx, int32_t n, float dt);

/* Wait for all enqueued work; returns SPH_ENOCONVERGE / SPH_EOVERFLOW / SPH_ENUMERIC if a
 * step since the previous call raised that condition in any scene, else SPH_OK. */
sph_status sph_synchronize(sph_ctx *ctx);

/* Copy the state of one scene out, in original particle order.  Any pointer may be NULL.
 * x, v: [n_fluid][3]; rho, pressure: [n_fluid] (pressure p = kappa rho of the last
 * constant-density solve, Sec. 3.3 Eq. pressure_acceleration; zero before the first
 * step).  on_device == 0: host memory, synchronises; 1: device memory, synchronises;
 * 2: device memory, only enqueued on the context's stream (order later work after it with
 * an event on that stream), so a caller can copy a step's result out while the next step
 * runs; 3: host memory, only enqueued: the fields are unpermuted on the context's stream
 * into one of two library staging slots, and a copy stream of the library moves them to
 * the host while later steps run.  With page-locked host buffers the call returns at
 * once; the data is there once sph_read_wait (or sph_synchronize) says so.  With pageable
 * buffers the copy waits for the step.  Other values: SPH_EINVAL. */
sph_status sph_read_state(sph_ctx *ctx, int32_t scene, float *x, float *v, float *rho,
                          float *pressure, int32_t on_device);

/* Wait until at most `keep` of the host reads enqueued with on_device = 3 (sph_read_state
 * or sph_read_field) are still in flight; reads complete in the order they were enqueued.
 * keep = 0 waits for all of them.  keep: 0..7, else SPH_EINVAL.  A caller stepping and
 * reading every step can keep one read in flight (keep = 1) so that each step's copy
 * overlaps the next step. */
sph_status sph_read_wait(sph_ctx *ctx, int32_t keep);

/* Overwrite the dynamic state of one scene (checkpoint restore); NULL keeps a field.
 * kappa_prev = previous step's total density stiffness times dt^2, kappa_v_prev =
 * divergence stiffness times dt (what SPH_FIELD_KAPPA_PREV / _V_PREV return).  Positions
 * and velocities are taken in original particle order.  Synchronises. */
sph_status sph_write_state(sph_ctx *ctx, int32_t scene, const float *x, const float *v,
                           const float *kappa_prev, const float *kappa_v_prev, int32_t on_device);

/* Per-particle fields for inspection and checkpointing, original order unless noted. */
#define SPH_FIELD_RHO 0          /* float [n_fluid]: density of the last step          */
#define SPH_FIELD_ALPHA 1        /* float: DFSPH factor alpha                          */
#define SPH_FIELD_KAPPA 2        /* float: total density stiffness of the last step    */
#define SPH_FIELD_KAPPA_V 3      /* float: total divergence stiffness of the last step */
#define SPH_FIELD_NN_FLUID 4     /* int32: fluid neighbours of the last step           */
#define SPH_FIELD_NN_BOUNDARY 5  /* int32: boundary neighbours of the last step        */
#define SPH_FIELD_V_DIV 6        /* float [n][3]: velocity after the divergence solve  */
#define SPH_FIELD_KAPPA_PREV 7   /* float: warm-start memory, kappa dt^2               */
#define SPH_FIELD_KAPPA_V_PREV 8 /* float: warm-start memory, kappa_v dt               */
#define SPH_FIELD_CELL_KEY 9     /* uint32: grid cell key at the start of the last step */
#define SPH_FIELD_SORTED_ID 10   /* int32, NOT reordered: original ids in grid order   */
#define SPH_FIELD_PSI 11         /* float [n_boundary]: boundary pseudo-mass Psi        */
#define SPH_FIELD_BOUNDARY_SORTED_ID 12 /* int32 [n_boundary], grid order              */
#define SPH_FIELD_BOUNDARY_CELL_KEY 13  /* uint32 [n_boundary], original order         */
#define SPH_FIELD_FEATURES 14    /* float [n][4]: warm-start network inputs            */
#define SPH_FIELD_KAPPA0 15      /* float: density warm-start stiffness of the last step */
sph_status sph_read_field(sph_ctx *ctx, int32_t scene, int32_t field, void *out,
                          int32_t on_device);   /* on_device as for sph_read_state */

/* Statistics of one scene (synchronises). */
sph_status sph_get_stats(sph_ctx *ctx, int32_t scene, sph_stats *out);

/* Rigid bodies of one scene: per body 19 doubles: com[3], quat[4], vel[3], omega[3],
 * force[3], torque[3] (fluid pressure force and torque of the last step). */
sph_status sph_read_bodies(sph_ctx *ctx, int32_t scene, double *out);

/* Rigid state into one scene (checkpoint resume, with sph_write_state for the fluid): per
 * body the first 13 doubles of the sph_read_bodies layout, com[3], quat[4], vel[3],
 * omega[3]. The force and torque columns are ignored, so a sph_read_bodies buffer can be
 * passed back as it is. Values are stored as given (the integrator renormalises the
 * quaternion every step); the body's boundary particles take the new pose at the next
 * step start, where they are placed from it anyway. Host buffer, caller-owned, read during
 * the call; synchronises. SPH_EINVAL for a bad scene index, a NULL buffer with bodies in
 * the scene, a non-finite value or a quaternion of zero norm (nothing is written then). */
sph_status sph_write_bodies(sph_ctx *ctx, int32_t scene, const double *in);

/* Execution mode: graph != 0 replays the step as one CUDA graph with device-side loop
 * control (default); 0 launches kernels one by one with host-side loop control.
 * timing != 0 (eager mode only) brackets every kernel with CUDA events on the context
 * stream. */
sph_status sph_set_mode(sph_ctx *ctx, int32_t graph, int32_t timing);

/* Autotuning.  A scene created with cell_size < 0 lets sph_create choose its grid cell
 * size (h (1 + 2^-8), 27-cell stencil, or h/2 (1 + 2^-8), 125-cell stencil), the threads
 * per particle of the neighbour sweeps (1, 2 or 4, or 8 instead of 2 for contexts small
 * enough for 8; kept fixed when lanes_per_particle is set) and, with one thread per
 * particle, the number of neighbours each thread keeps in flight in the Jacobi passes (4
 * or 8) by timing a few CUDA-graph steps of every candidate on temporary contexts,
 * twice, keeping each candidate's faster time (the default configuration is kept unless
 * a candidate is more than 3 % faster); the choice is cached per process for the same
 * device and workload size (log2 of the fluid count, scene count, bodies, viscosity
 * mode, lanes_per_particle).  Neighbour sets do not depend on the choice; the summation
 * order, and so the last bits of FP32 results, may. */
typedef struct sph_tuning {
    int32_t tuned;            /* 1 if this context was autotuned                     */
    int32_t from_cache;       /* the choice came from the per-process cache          */
    int32_t gather_batch;     /* chosen neighbours in flight per thread              */
    float cell_factor;        /* chosen cell size / h                                */
    int32_t n_trials;
    float trial_cell_factor[8];
    int32_t trial_batch[8];
    float trial_ms[8];        /* mean milliseconds per step of each candidate        */
    int32_t lanes;            /* chosen threads per particle                         */
    int32_t trial_lanes[8];
} sph_tuning;
sph_status sph_get_tuning(sph_ctx *ctx, sph_tuning *out);

/* Per-kernel timing collected in eager timing mode: up to cap entries of name (63
 * chars + NUL), launches and total milliseconds; returns the entry count in *n. */
typedef struct sph_kernel_time {
    char name[64];
    int64_t launches;
    double total_ms;
} sph_kernel_time;
sph_status sph_kernel_times(sph_ctx *ctx, sph_kernel_time *out, int32_t cap, int32_t *n,
                            int32_t reset);

/* Learned warm start (this library's addition; the paper has no learned component).
 * A per-particle network y = W3 gelu(W2 gelu(W1 f + b1) + b2) + b3 (hidden width 64,
 * exact-erf GELU, BF16 tensor-core layers with FP32 accumulation) maps the standardised
 * features f = (rho/rho0 - 1, dt Drho/Dt(v*)/rho0, (n_f + n_b)/33, kappa_prev/(9.81 h))
 * to the standardised converged density stiffness; the warm start of the constant-
 * density solve is kappa0 = max((y std_y + mean_y) 9.81 h, 0) where the fluid compresses.
 * Parameter block, float [SPH_MLP_PARAMS]: W1[64][4], b1[64], W2[64][64], b2[64],
 * W3[64], b3, feature mean[4], feature std[4], label mean, label std. */
#define SPH_MLP_PARAMS 4555
#define SPH_MLP_WEIGHTS 4545

/* Load the network used by scenes with warm_start = SPH_WARM_LEARNED (host array,
 * copied).  Until it is called those scenes start the density solve from zero. */
sph_status sph_set_mlp(sph_ctx *ctx, const float *params, int64_t n);

/* Network forward on device arrays: params [SPH_MLP_PARAMS], standardised features
 * [n][4] -> y [n] (standardised output).  *error (device int32) is set to 1 if a
 * tensor-core wait gave up.  Enqueued on stream; returns after enqueueing. */
sph_status sph_mlp_forward(const float *params, const float *features, int64_t n, float *y,
                           int32_t *error, void *stream);

/* Gradient of the mean squared error (1/n) sum (y - label)^2 of the network over n
 * standardised samples (device arrays: features [n][4], labels [n]) with respect to the
 * first SPH_MLP_WEIGHTS parameters -> grad (device float [SPH_MLP_WEIGHTS]); *loss (device
 * double) receives the sum of squared errors.  BF16 tensor-core forward and backward with
 * FP32 accumulation.  *error (device int32) is set to 1 if a tensor-core wait gave up. */
sph_status sph_mlp_grad(const float *params, const float *features, const float *labels, int64_t n,
                        float *grad, double *loss, int32_t *error, void *stream);

/* Train the network on raw (unstandardised) samples, device arrays features [n][4] and
 * labels [n]: the call computes the standardisation statistics into params, then runs
 * `epochs` passes of Adam (lr, beta = 0.9/0.999, eps = 1e-8) over mini-batches of
 * `batch` samples in a seeded per-epoch order, updating params (device, FP32 master
 * weights) and adam_state (device float [2 * SPH_MLP_WEIGHTS], zero for a fresh start).
 * loss_history (device float [epochs], may be NULL) receives each epoch's mean squared
 * error in standardised units.  Allocates its scratch with cudaMallocAsync on stream. */
sph_status sph_mlp_train(const float *features, const float *labels, int64_t n, float *params,
                         float *adam_state, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                         float *loss_history, int32_t *error, void *stream);

/* Kernel ids of the device trace (sph_set_trace / sph_read_trace). */
#define SPH_KID_STEP_BEGIN 1      /* step begin */
#define SPH_KID_KEY_HIST_F 2      /* fluid cell-key histogram */
#define SPH_KID_KEY_HIST_B 3      /* boundary cell-key histogram */
#define SPH_KID_SCAN 4            /* look-back scan */
#define SPH_KID_SCATTER_F 5       /* fluid scatter */
#define SPH_KID_SCATTER_B 6       /* boundary scatter */
#define SPH_KID_RANK_F 7          /* fluid rank and gather */
#define SPH_KID_RANK_B 8          /* boundary rank and gather */
#define SPH_KID_DENSITY 9         /* density, alpha, lists */
#define SPH_KID_PASS_A0 10        /* divergence pass A */
#define SPH_KID_PASS_A1 11        /* density pass A */
#define SPH_KID_PASS_B0 12        /* divergence pass B */
#define SPH_KID_PASS_B1 13        /* density pass B */
#define SPH_KID_PASS_B0W 14       /* divergence warm start */
#define SPH_KID_PASS_B1W 15       /* density warm start / EOS */
#define SPH_KID_NONP 16           /* non-pressure forces */
#define SPH_KID_WARM 17           /* warm-start gate and features */
#define SPH_KID_ADVECT 18         /* advection */
#define SPH_KID_STEP_END 19       /* step end, rigid integration */
#define SPH_KID_SET_DT 20         /* fixed step */
#define SPH_KID_BUPDATE 21        /* boundary pose update */
#define SPH_KID_PSI 22            /* boundary Psi */
#define SPH_KID_BFORCE 23         /* body force (weak) */
#define SPH_KID_BREDUCE 24        /* body force reduction */
#define SPH_KID_CG_INIT 25        /* CG initial residual */
#define SPH_KID_CG_AP 26          /* CG matrix sweep */
#define SPH_KID_CG_XR 27          /* CG update */
#define SPH_KID_CG_P 28           /* CG direction */
#define SPH_KID_MLP_WARM 29       /* warm-start network */
#define SPH_KID_BFORCE_INC 30     /* body force (strong) */
#define SPH_KID_BAPPLY 31         /* body impulse (strong) */
#define SPH_KID_BVEL 32           /* boundary velocities (strong) */
#define SPH_KID_CHECK0 33         /* divergence convergence test */
#define SPH_KID_CHECK1 34         /* density convergence test */
#define SPH_KID_CG_ALPHA 35       /* CG alpha */
#define SPH_KID_CG_BETA 36        /* CG beta and stopping test */
#define SPH_KID_BTOUCH 37         /* bodies touched per block (strong) */
#define SPH_KID_RANK_LARGE_F 38   /* crowded cells of the fluid sort, block-sorted */
#define SPH_KID_RANK_LARGE_B 39   /* crowded cells of the boundary sort, block-sorted */

/* Device trace for profiling graph replays: with capacity > 0 every kernel's first thread
 * records (globaltimer_ns << 8 | kernel id) in a device ring of that many entries (the
 * library allocates it; 0 turns tracing off and frees it).  sph_read_trace copies up to
 * cap entries to host memory, returns the count recorded in *n and, with reset != 0,
 * restarts recording.  Kernel ids are the SPH_KID_* values of the library's kernels. */
sph_status sph_set_trace(sph_ctx *ctx, int32_t capacity);
sph_status sph_read_trace(sph_ctx *ctx, uint64_t *out, int32_t cap, int32_t *n, int32_t reset);

/* Failure-path probe: enqueues one thread that waits, spin_limit times about 1 us each, on a
 * device flag that nothing sets.  The wait runs out and records a device error, so the next
 * sph_synchronize returns SPH_ETIMEOUT and the context is poisoned (only sph_destroy stays
 * valid), as after any bounded device wait of the library that gave up.  For tests of the
 * error path; it neither faults nor hangs the GPU.  spin_limit: 1..10^6, else SPH_EINVAL. */
sph_status sph_probe_wait_timeout(sph_ctx *ctx, int32_t spin_limit);

/* Kernel launches enqueued since creation (counted on the device for graph replays). */
sph_status sph_launch_count(sph_ctx *ctx, int64_t *out);

/* Grid order of a point set with no memory allocation (this library's addition; the paper
 * has no counterpart).  For callers that cannot let a library allocate: code enqueueing
 * work while another component captures a CUDA graph, applications that own the GPU's
 * memory budget, real-time loops.  Runs the per-step counting sort of the neighbour search
 * (same float cell-key contract and (cell key, index) order as sph_step) on
 *   x     device float [n][3] positions,
 *   domain_min, domain_max  host float[3], cell_size > 0 (grid as in sph_scene_desc),
 * writing
 *   order device int32 [n]: point indices in (cell key, index) order,
 *   keys  device uint32 [n] or NULL: each point's cell key (input order),
 * on stream (a cudaStream_t, NULL = legacy default).  Returns after enqueueing.
 * Its scratch is one static device array of about 12 MB that every GPU loading this
 * library holds until the process exits, shared by all calls: n above
 * SPH_NOALLOC_MAX_POINTS or a grid above SPH_NOALLOC_MAX_CELLS cells returns SPH_EINVAL,
 * and calls whose work overlaps on the GPU (different streams, or host threads) race on
 * that array.  The first call on a device looks up the array's device address (with that
 * device current) and should come before any stream capture.  Calls no allocator.
 * Points outside [domain_min, domain_max] (and NaN coordinates) are clamped into the edge
 * cells of the padded grid, as in sph_step.  Inside a cell of up to 64 points the order
 * comes from counting each point's smaller indices; a more crowded cell is sorted by one
 * thread block (a stable radix sort on the index), so the work stays linear in n however
 * the points crowd into cells.
 * SPH_OK means the work was enqueued; whether its prefix scan completed is reported by
 * sph_grid_order_noalloc_status. */
#define SPH_NOALLOC_MAX_POINTS 262144
#define SPH_NOALLOC_MAX_CELLS 1048576
sph_status sph_grid_order_noalloc(const float *x, int64_t n, const float *domain_min,
                                  const float *domain_max, float cell_size, int32_t *order,
                                  uint32_t *keys, void *stream);

/* Outcome of the last sph_grid_order_noalloc call on the current device: synchronises
 * stream (the one that call used), then reads the scratch array's error word into host
 * memory with a copy from the symbol (no allocation).  SPH_ETIMEOUT: a bounded wait of the
 * call's look-back prefix scan ran out, so its order is not valid (the GPU stays usable);
 * SPH_OK: it completed; SPH_ECUDA: the synchronisation or the copy failed.  The word is
 * cleared by every call, so a later or overlapping call replaces it.  Not for use inside a
 * stream capture (it synchronises). */
sph_status sph_grid_order_noalloc_status(void *stream);

/* Post-processing (Sec. 4.3: surface reconstruction of the fluid particles, then rendering;
 * the paper uses SplashSurf and Blender, these are CUDA kernels writing device buffers).
 *
 * sph_surface_field: the fluid's volume fraction phi(g) = sum_j (m / rho_j) W(|g - x_j|)
 * (the SPH interpolant of Sec. 3.2 applied to 1: about 1 inside, 0 outside) at the grid
 * nodes origin + spacing (i, j, k), 0 <= i < dims[0] ..., for scene `scene` at its
 * current positions, rho_j the density of the last step (rho0 before the first step).
 * field: device float [dims[2]][dims[1]][dims[0]], caller-owned.  Enqueued on the
 * context's stream; returns after enqueueing.  The reconstruction of a surface is the
 * iso-level 0.5 of this field (sph_surface_mesh).  SPH_EINVAL for a scene out of range,
 * NULL pointers, a spacing that is not positive and finite, dims < 1, a non-finite origin
 * or more than 2^31 nodes; SPH_ECUDA if scratch cannot be allocated. */
sph_status sph_surface_field(sph_ctx *ctx, int32_t scene, const float origin[3], float spacing,
                             const int32_t dims[3], float *field);

/* Iso-surface phi = iso of a device grid field laid out as above, by marching tetrahedra:
 * each grid cube is split into the six tetrahedra around its diagonal from node (i, j, k)
 * to (i+1, j+1, k+1); per tetrahedron the corners with phi > iso are cut off by one or
 * two triangles whose vertices interpolate linearly along the cut edges, oriented with
 * the normal pointing from phi > iso towards phi <= iso (outward for a fluid).  tris:
 * device float [cap][3][3], triangles in cube order (x fastest); *n_tris (host) receives
 * the total, which may exceed cap (then only cap triangles are written and SPH_EOVERFLOW
 * is returned).  Enqueued on stream, which the call synchronises.  SPH_EINVAL for NULL
 * pointers (tris may be NULL with cap = 0, to count), cap < 0, dims < 2, a spacing that is
 * not positive and finite, or a non-finite iso or origin. */
sph_status sph_surface_mesh(const float *field, const int32_t dims[3], const float origin[3],
                            float spacing, float iso, float *tris, int64_t cap, int64_t *n_tris,
                            void *stream);

/* Headless orthographic height map of scene `scene` viewed down the -z axis: pixel (i, j)
 * (centre lo + ((i + 0.5)(hi - lo)_x / width, (j + 0.5)(hi - lo)_y / height)) receives the
 * largest z + sqrt(radius^2 - d^2) over particles whose disk of the given radius covers
 * it (d < radius), NaN where none does.  out: device float [height][width], caller-owned.
 * Enqueued on the context's stream; returns after enqueueing.  SPH_EINVAL for a scene out
 * of range, NULL pointers, width or height < 1 or more than 2^31 pixels, or a bad view
 * rectangle or radius. */
sph_status sph_render_heightmap(sph_ctx *ctx, int32_t scene, const float lo[2], const float hi[2],
                                int32_t width, int32_t height, float radius, float *out);

const char *sph_status_string(sph_status s);

/* Message of the last failing call on ctx (never NULL). */
const char *sph_last_error(const sph_ctx *ctx);

/* Free everything (waits for the stream first).  NULL is a no-op. */
void sph_destroy(sph_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
