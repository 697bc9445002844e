// sph_api.cu -- host runtime behind include/sph.h: scene validation, device layout,
// the step as a CUDA graph (conditional while-nodes run the Jacobi loops on the device),
// an eager mode with optional per-kernel CUDA-event timing, and the read/write paths.
#include "sph.h"
#include "sph_internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace sph;

namespace {

constexpr int kDefaultCapF = 96;
constexpr int kDefaultCapB = 64;
constexpr int64_t kAutoLaneThreads = 152 * 2048;  // resident threads of a full GB300

// Threads per particle chosen by context size: the most (8, 4, 2, 1) whose threads still
// fit the GPU's resident threads.
int auto_lanes(int64_t nf)
{
    for (int l = 8; l > 1; l /= 2)
        if (nf * l <= kAutoLaneThreads) return l;
    return 1;
}

// PCISPH stiffness of a prototype particle with a full neighbourhood on the lattice of
// spacing 2r (the predictive-corrective solver's constant): delta dt^2 = 1 / (2 (m/rho0)^2
// (|sum grad W|^2 + sum |grad W|^2)), the cubic spline's gradient dW/dr = 48/(pi h^4) g(q),
// g = q (3q - 2) for q <= 1/2 and -(1 - q)^2 up to q = 1.
double pcisph_prototype(double r)
{
    const double h = 4.0 * r, s = 2.0 * r, pi = 3.14159265358979323846;
    const int n = (int)std::ceil(h / s) + 1;
    double sum[3] = {0.0, 0.0, 0.0}, sq = 0.0;
    for (int a = -n; a <= n; ++a)
        for (int b = -n; b <= n; ++b)
            for (int e = -n; e <= n; ++e) {
                const double x[3] = {a * s, b * s, e * s};
                const double d = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                const double q = d / h;
                if (!(d > 0.0) || q > 1.0) continue;
                const double g = q <= 0.5 ? q * (3.0 * q - 2.0) : -(1.0 - q) * (1.0 - q);
                const double f = 48.0 / (pi * h * h * h * h) * g / d;
                for (int k = 0; k < 3; ++k) sum[k] += f * x[k];
                sq += f * f * d * d;
            }
    const double mr = s * s * s;   // m / rho0
    return 1.0 / (2.0 * mr * mr * (sum[0] * sum[0] + sum[1] * sum[1] + sum[2] * sum[2] + sq));
}
constexpr double kPi = 3.14159265358979323846;

struct Alloc {
    void *p;
    size_t bytes;
};

struct PendingTime {
    const char *name;
    cudaEvent_t a, b;
};

}  // namespace

struct sph_ctx {
    cudaStream_t stream = nullptr;       // caller's stream (may be the legacy default)
    cudaStream_t cap0 = nullptr, cap1 = nullptr;  // capture streams
    cudaStream_t side = nullptr;         // branch of the step that runs beside the fluid sort
    cudaEvent_t fork = nullptr, join = nullptr;
    sph_allocator alloc{};
    bool use_alloc = false;
    std::vector<Alloc> allocs;
    std::string err;
    bool poisoned = false;
    int device = 0;

    int nscenes = 0;
    std::vector<SceneDev> scenes;        // host copies
    std::vector<int32_t> fblk_scene, bblk_scene, tblk_scene;
    std::vector<int32_t> nbody_scene;
    int max_bodies = 0;
    bool any_moving = false, any_div = false, any_warm_div = false, any_warm = false,
         any_learned = false, any_bodies = false, any_implicit = false, any_wcsph = false, any_strong = false;
    Ptrs P{};
    SceneDev *d_scenes = nullptr;

    // graph
    bool graph_mode = true;
    bool timing = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float last_dt = -1.0f;

    // timing
    std::vector<PendingTime> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<int64_t, double>> times;
    int64_t host_launches = 0;

    std::vector<int32_t> reported_flags;
    unsigned long long *trace = nullptr; // device trace ring (cudaMalloc, owned)
    int32_t trace_cap = 0;
    int batch = 4;                       // neighbours in flight per thread in the Jacobi passes
    sph_tuning tuning{};
    uint32_t *h_flag = nullptr;          // pinned word for eager loop control

    // enqueued host reads (on_device = 3): the unpermuted fields go to one of two device
    // staging slots on the context stream, and a copy stream moves them to the host while
    // later work runs; every read records a completion event in a ring
    static constexpr int kReadRing = 8;
    cudaStream_t copy = nullptr;
    void *stage[2] = {nullptr, nullptr};
    size_t stage_bytes[2] = {0, 0};
    cudaEvent_t staged[2] = {nullptr, nullptr};
    cudaEvent_t read_done[kReadRing] = {};
    int64_t reads = 0;                   // host reads enqueued so far
};

namespace {

sph_status fail(sph_ctx *c, sph_status st, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
        if (st == SPH_ECUDA || st == SPH_ETIMEOUT) c->poisoned = true;
    }
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, SPH_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

void *dev_alloc(sph_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (c->use_alloc) {
        p = c->alloc.alloc(c->alloc.user, bytes, (void *)c->stream);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) c->allocs.push_back({p, bytes});
    return p;
}

template <typename T>
bool dalloc(sph_ctx *c, T *&ptr, size_t count)
{
    ptr = static_cast<T *>(dev_alloc(c, sizeof(T) * count));
    return ptr != nullptr;
}

float default_cell(float radius)
{
    float h = 4.0f * radius;
    return h * 1.00390625f;
}

// smallest cell the 5 x 5 x 5 stencil supports: h/2 (1 + 2^-8)
float half_cell(float radius)
{
    float h = 4.0f * radius;
    return h * 0.501953125f;
}

sph_status validate(sph_ctx *c, const sph_scene_desc &d, int idx)
{
    auto bad = [&](const char *what) { return fail(c, SPH_EINVAL, "scene %d: %s", idx, what); };
    if (d.n_fluid < 1 || d.n_fluid > (int64_t)1 << 30) return bad("n_fluid out of range");
    if (!d.fluid_x) return bad("fluid_x is NULL");
    if (d.n_boundary < 0 || d.n_boundary > (int64_t)1 << 30) return bad("n_boundary out of range");
    if (d.n_boundary > 0 && !d.boundary_x) return bad("boundary_x is NULL");
    if (!(d.radius > 0.0f) || !std::isfinite(d.radius)) return bad("radius must be > 0");
    if (!(d.rest_density > 0.0f)) return bad("rest_density must be > 0");
    if (!(d.viscosity >= 0.0f)) return bad("viscosity must be >= 0");
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(d.domain_min[a]) || !std::isfinite(d.domain_max[a]) ||
            !(d.domain_max[a] > d.domain_min[a]))
            return bad("domain_max must exceed domain_min");
        if (!std::isfinite(d.gravity[a])) return bad("gravity not finite");
    }
    if (!(d.dt_max > 0.0f)) return bad("dt_max must be > 0");
    if (d.cfl < 0.0f || !std::isfinite(d.cfl)) return bad("cfl must be >= 0");
    if (d.eta_density < 0.0f || d.eta_divergence < 0.0f) return bad("tolerances must be >= 0");
    // max_iter is the hard cap; min_iter above it simply never binds
    if (d.min_iter_density < 0 || d.max_iter_density < 0 || d.max_iter_density > 100000)
        return bad("density iteration bounds");
    if (d.min_iter_divergence < 0 || d.max_iter_divergence < 0 || d.max_iter_divergence > 100000)
        return bad("divergence iteration bounds");
    if (d.viscosity_mode < 0 || d.viscosity_mode > 3) return bad("viscosity_mode");
    if (d.warm_start < 0 || d.warm_start > 2) return bad("warm_start");
    if (d.max_fluid_neighbors < 0 || d.max_fluid_neighbors > 1024) return bad("max_fluid_neighbors");
    if (d.max_boundary_neighbors < 0 || d.max_boundary_neighbors > 1024) return bad("max_boundary_neighbors");
    if (d.lanes_per_particle != 0 && d.lanes_per_particle != 1 && d.lanes_per_particle != 2 &&
        d.lanes_per_particle != 4 && d.lanes_per_particle != 8)
        return bad("lanes_per_particle (0, 1, 2, 4 or 8)");
    if (!(d.warm_start_fraction >= 0.0f && d.warm_start_fraction <= 1.0f)) return bad("warm_start_fraction (0..1)");
    if (!(d.learned_fraction >= 0.0f && d.learned_fraction <= 1.0f)) return bad("learned_fraction (0..1)");
    if (d.learned_gate < 0) return bad("learned_gate (>= 0)");
    if (d.rigid_coupling != SPH_COUPLING_WEAK && d.rigid_coupling != SPH_COUPLING_STRONG) return bad("rigid_coupling");
    if (d.pressure_solver != SPH_SOLVER_DFSPH && d.pressure_solver != SPH_SOLVER_WCSPH &&
        d.pressure_solver != SPH_SOLVER_PCISPH)
        return bad("pressure_solver");
    if (d.pressure_solver == SPH_SOLVER_WCSPH &&
        (!(d.eos_stiffness > 0.0f) || !std::isfinite(d.eos_stiffness) || !(d.eos_exponent == 0.0f || d.eos_exponent >= 1.0f) ||
         !std::isfinite(d.eos_exponent)))
        return bad("eos_stiffness / eos_exponent");
    if (d.cell_size > 0.0f && !(d.cell_size >= half_cell(d.radius))) return bad("cell_size below h/2 (1 + 2^-8)");
    if (!std::isfinite(d.cell_size)) return bad("cell_size not finite");
    if (d.n_bodies < 0 || d.n_bodies > SPH_MAX_BODIES) return bad("n_bodies out of range");
    if (d.n_bodies > 0 && !d.bodies) return bad("bodies is NULL");
    for (int k = 0; k < d.n_bodies; ++k) {
        const sph_rigid_desc &b = d.bodies[k];
        if (!(b.mass > 0.0) || !(b.inertia[0] > 0.0) || !(b.inertia[1] > 0.0) || !(b.inertia[2] > 0.0))
            return bad("body mass and inertia must be > 0");
        double qn = b.quat[0] * b.quat[0] + b.quat[1] * b.quat[1] + b.quat[2] * b.quat[2] + b.quat[3] * b.quat[3];
        if (!(std::fabs(qn - 1.0) < 1e-6)) return bad("body quaternion must be unit");
    }
    if (d.boundary_body) {
        for (int64_t b = 0; b < d.n_boundary; ++b)
            if (d.boundary_body[b] < -1 || d.boundary_body[b] >= d.n_bodies) return bad("boundary_body index");
    }
    for (int64_t i = 0; i < 3 * d.n_fluid; ++i)
        if (!std::isfinite(d.fluid_x[i]) || (d.fluid_v && !std::isfinite(d.fluid_v[i])))
            return bad("non-finite fluid input");
    for (int64_t i = 0; i < 3 * d.n_boundary; ++i)
        if (!std::isfinite(d.boundary_x[i])) return bad("non-finite boundary input");
    float c0 = d.cell_size > 0.0f ? d.cell_size : half_cell(d.radius);
    double cells = 1.0;
    for (int a = 0; a < 3; ++a) {
        float ext = (d.domain_max[a] - d.domain_min[a]) / c0;
        cells *= (double)((int64_t)std::ceil(ext) + 2);
    }
    if (cells > 1.5e9) return bad("grid too large (domain / cell size)");
    return SPH_OK;
}

// ------------------------------------------------------------------ read / write kernels
// One thread waits on a flag that nothing sets, a bounded number of times; when the wait
// runs out it records the same error as the library's other bounded waits.
__global__ void k_probe_wait(Control *ctl, uint32_t limit)
{
    const volatile uint32_t *flag = &ctl->probe_flag;
    for (uint32_t k = 0; k < limit; ++k) {
        if (*flag != 0u) return;
        __nanosleep(1000);
    }
    atomicExch(&ctl->error, 6);
}

__global__ void k_read_fluid(Ptrs P, int scene, int field, void *out)
{
    const SceneDev &sc = P.scenes[scene];
    int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= sc.nf) return;
    int64_t i = sc.f_off + local;
    // canonical arrays (state) use id_c; per-step arrays use id_s (equal after a step)
    switch (field) {
    case 100: {  // x
        float4 p = P.pos_c[i];
        float *o = (float *)out + 3 * P.id_c[i];
        o[0] = p.x; o[1] = p.y; o[2] = p.z;
        break;
    }
    case 101: {  // v
        float4 v = P.vel_c[i];
        float *o = (float *)out + 3 * P.id_c[i];
        o[0] = v.x; o[1] = v.y; o[2] = v.z;
        break;
    }
    case 102: ((float *)out)[P.id_c[i]] = P.vel_c[i].w; break;            // rho
    case 103: ((float *)out)[P.id_c[i]] = P.ksum[i] * P.vel_c[i].w; break; // pressure
    case SPH_FIELD_RHO: ((float *)out)[P.id_s[i]] = P.vel_s[i].w; break;
    case SPH_FIELD_ALPHA: ((float *)out)[P.id_s[i]] = P.alpha[i]; break;
    case SPH_FIELD_KAPPA: ((float *)out)[P.id_s[i]] = P.ksum[i]; break;
    case SPH_FIELD_KAPPA_V: ((float *)out)[P.id_s[i]] = P.kvsum[i]; break;
    case SPH_FIELD_NN_FLUID: ((int32_t *)out)[P.id_s[i]] = P.nnf[i]; break;
    case SPH_FIELD_NN_BOUNDARY: ((int32_t *)out)[P.id_s[i]] = P.nnb[i]; break;
    case SPH_FIELD_V_DIV: {
        float4 v = P.vel_s[i];
        float *o = (float *)out + 3 * P.id_s[i];
        o[0] = v.x; o[1] = v.y; o[2] = v.z;
        break;
    }
    case SPH_FIELD_KAPPA_PREV: ((float *)out)[P.id_c[i]] = P.kprev_c[i]; break;
    case SPH_FIELD_KAPPA_V_PREV: ((float *)out)[P.id_c[i]] = P.kvprev_c[i]; break;
    case SPH_FIELD_CELL_KEY: {
        float4 p = P.pos_s[i];
        int32_t ix = cell_coord(p.x, sc.origin[0], sc.cell, sc.dims[0]);
        int32_t iy = cell_coord(p.y, sc.origin[1], sc.cell, sc.dims[1]);
        int32_t iz = cell_coord(p.z, sc.origin[2], sc.cell, sc.dims[2]);
        ((uint32_t *)out)[P.id_s[i]] =
            (uint32_t)ix + (uint32_t)sc.dims[0] * ((uint32_t)iy + (uint32_t)sc.dims[1] * (uint32_t)iz);
        break;
    }
    case SPH_FIELD_SORTED_ID: ((int32_t *)out)[local] = P.id_s[i]; break;
    case SPH_FIELD_FEATURES: {
        float4 f = reinterpret_cast<const float4 *>(P.feat)[i];
        float *o = (float *)out + 4 * P.id_s[i];
        o[0] = f.x; o[1] = f.y; o[2] = f.z; o[3] = f.w;
        break;
    }
    case SPH_FIELD_KAPPA0: ((float *)out)[P.id_s[i]] = P.k0[i]; break;
    default: break;
    }
}

__global__ void k_read_boundary(Ptrs P, int scene, int field, void *out)
{
    const SceneDev &sc = P.scenes[scene];
    int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= sc.nb) return;
    int64_t b = sc.b_off + local;
    switch (field) {
    case SPH_FIELD_PSI: ((float *)out)[P.bid_s[b]] = P.bpos_s[b].w; break;
    case SPH_FIELD_BOUNDARY_SORTED_ID: ((int32_t *)out)[local] = P.bid_s[b]; break;
    case SPH_FIELD_BOUNDARY_CELL_KEY: {
        float4 p = P.bx_o[b];
        int32_t ix = cell_coord(p.x, sc.origin[0], sc.cell, sc.dims[0]);
        int32_t iy = cell_coord(p.y, sc.origin[1], sc.cell, sc.dims[1]);
        int32_t iz = cell_coord(p.z, sc.origin[2], sc.cell, sc.dims[2]);
        ((uint32_t *)out)[local] =
            (uint32_t)ix + (uint32_t)sc.dims[0] * ((uint32_t)iy + (uint32_t)sc.dims[1] * (uint32_t)iz);
        break;
    }
    default: break;
    }
}

// Bring one scene's canonical arrays back to original particle order (through the
// sorted arrays as scratch), so that a checkpoint can be written in that order.
__global__ void k_unpermute_to_sorted(Ptrs P, int scene)
{
    const SceneDev &sc = P.scenes[scene];
    int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= sc.nf) return;
    int64_t i = sc.f_off + local;
    int64_t d = sc.f_off + P.id_c[i];
    P.pos_s[d] = P.pos_c[i];
    P.vel_s[d] = P.vel_c[i];
    P.kprev_s[d] = P.kprev_c[i];
    P.kvprev_s[d] = P.kvprev_c[i];
}
__global__ void k_sorted_to_canonical(Ptrs P, int scene)
{
    const SceneDev &sc = P.scenes[scene];
    int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= sc.nf) return;
    int64_t i = sc.f_off + local;
    P.pos_c[i] = P.pos_s[i];
    float4 v = P.vel_s[i];
    v.w = 0.0f;
    P.vel_c[i] = v;
    P.kprev_c[i] = P.kprev_s[i];
    P.kvprev_c[i] = P.kvprev_s[i];
    P.id_c[i] = (int32_t)local;
    P.id_s[i] = (int32_t)local;
    P.ksum[i] = 0.0f;
    P.kvsum[i] = 0.0f;
}
// Write [n][3] (packed) into a float4 array, original order == canonical order here.
__global__ void k_pack3(float4 *dst, const float *src, int64_t n, float w)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    dst[k] = make_float4(src[3 * k], src[3 * k + 1], src[3 * k + 2], w);
}
__global__ void k_scene_cfl(Ptrs P, int scene)
{
    __shared__ float sh[256];
    const SceneDev &sc = P.scenes[scene];
    float m = 0.0f;
    for (int64_t k = threadIdx.x; k < sc.nf; k += blockDim.x) {
        float4 v = P.vel_c[sc.f_off + k];
        m = fmaxf(m, v.x * v.x + v.y * v.y + v.z * v.z);
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float vm = sqrtf(sh[0]);
        float dt = sc.dt_max;
        if (sc.cfl > 0.0f && vm > 0.0f) dt = fminf(dt, sc.cfl * sc.two_r / vm);
        P.st[scene].dt_next = dt;
    }
}

// ------------------------------------------------------------------ launch plumbing
cudaEvent_t get_event(sph_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

sph_status harvest(sph_ctx *c)
{
    if (c->pending.empty()) return SPH_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (auto &p : c->pending) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto &t = c->times[p.name];
        t.first += 1;
        t.second += ms;
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
    return SPH_OK;
}

template <typename F>
void run(sph_ctx *c, cudaStream_t s, const char *name, F &&f)
{
    if (c->timing && !c->graph_mode) {
        cudaEvent_t a = get_event(c), b = get_event(c);
        cudaEventRecord(a, s);
        f();
        cudaEventRecord(b, s);
        c->pending.push_back({name, a, b});
    } else {
        f();
    }
    c->host_launches += 1;
}

// Enqueue one step.  In capture mode the two Jacobi loops become conditional while
// nodes whose bodies are captured on a second stream; in eager mode the host reads the
// loop flag after every iteration.
sph_status enqueue_step(sph_ctx *c, cudaStream_t s, bool capture)
{
    const Ptrs &P = c->P;
    run(c, s, "step_begin", [&] { launch_step_begin(P, s); });
    // Moving bodies: their boundary particles' update, grid order and Psi touch nothing
    // the fluid sort does (each sort has its own scan state), so they run as a branch on
    // the side stream beside it (a parallel branch of the captured graph) and join before
    // the density sweep.
    if (c->any_moving) {
        cudaStream_t b = c->side;
        CK(cudaEventRecord(c->fork, s));
        CK(cudaStreamWaitEvent(b, c->fork, 0));
        run(c, b, "boundary_update", [&] { launch_boundary_update(P, b); });
        run(c, b, "bsort_key_hist", [&] { launch_key_hist(P, SORT_BOUNDARY, b); });
        run(c, b, "bsort_scan", [&] { launch_scan_cells(P, SORT_BOUNDARY, b); });
        run(c, b, "bsort_scatter", [&] { launch_scatter(P, SORT_BOUNDARY, b); });
        run(c, b, "bsort_rank_gather", [&] { launch_rank_gather(P, SORT_BOUNDARY, b); });
        run(c, b, "boundary_psi", [&] { launch_boundary_psi(P, b); });
        CK(cudaEventRecord(c->join, b));
    }
    run(c, s, "sort_key_hist", [&] { launch_key_hist(P, SORT_FLUID, s); });
    run(c, s, "sort_scan", [&] { launch_scan_cells(P, SORT_FLUID, s); });
    run(c, s, "sort_scatter", [&] { launch_scatter(P, SORT_FLUID, s); });
    run(c, s, "sort_rank_gather", [&] { launch_rank_gather(P, SORT_FLUID, s); });
    if (c->any_moving) CK(cudaStreamWaitEvent(s, c->join, 0));
    run(c, s, "density_alpha", [&] { launch_density_alpha(P, s); });
    if (c->any_strong) run(c, s, "body_touch", [&] { launch_body_touch(P, s); });

    // A device-controlled loop: in capture mode a conditional while node whose body is
    // captured on the second stream; in eager mode the host reads the loop flag.
    auto device_loop = [&](auto &&body) -> sph_status {
        if (capture) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t g;
            const cudaGraphNode_t *deps = nullptr;
            size_t ndeps = 0;
            CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps));
            cudaGraphConditionalHandle h;
            CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
            cudaGraph_t bodyg = np.conditional.phGraph_out[0];
            CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
            CK(cudaStreamBeginCaptureToGraph(c->cap1, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            body(c->cap1, h, 1);
            cudaGraph_t out = nullptr;
            CK(cudaStreamEndCapture(c->cap1, &out));
        } else {
            for (int guard = 0; guard < 200000; ++guard) {
                body(s, (cudaGraphConditionalHandle)0, 0);
                CK(cudaMemcpyAsync(c->h_flag, &P.ctl->loop_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (*c->h_flag == 0) break;
            }
        }
        return SPH_OK;
    };
    auto loop = [&](int solver) -> sph_status {
        const char *na = solver == 0 ? "div_pass_a" : "dens_pass_a";
        const char *nb = solver == 0 ? "div_pass_b" : "dens_pass_b";
        const char *nc = solver == 0 ? "div_check" : "dens_check";
        return device_loop([&](cudaStream_t q, cudaGraphConditionalHandle h, int use) {
            run(c, q, na, [&] { launch_pass_a(P, solver, c->batch, q); });
            run(c, q, nb, [&] { launch_pass_b(P, solver, 0, c->batch, q); });
            if (c->any_strong) run(c, q, "strong_coupling", [&] { launch_strong_update(P, solver, q); });
            run(c, q, nc, [&] { launch_solver_check(P, solver, h, use, q); });
        });
    };

    sph_status st;
    if (c->any_div) {
        if (c->any_warm_div) {
            run(c, s, "div_warm_pass_b", [&] { launch_pass_b(P, 0, 1, c->batch, s); });
            if (c->any_strong) run(c, s, "strong_coupling", [&] { launch_strong_update(P, 2, s); });
        }
        if ((st = loop(0)) != SPH_OK) return st;
    }
    run(c, s, "nonpressure", [&] { launch_nonpressure(P, s); });
    if (c->any_implicit) {
        run(c, s, "cg_init", [&] { launch_cg_init(P, s); });
        st = device_loop([&](cudaStream_t q, cudaGraphConditionalHandle h, int use) {
            run(c, q, "cg_ap", [&] { launch_cg_ap(P, q); });
            run(c, q, "cg_alpha", [&] { launch_cg_alpha(P, q); });
            run(c, q, "cg_xr", [&] { launch_cg_xr(P, q); });
            run(c, q, "cg_beta", [&] { launch_cg_beta(P, h, use, q); });
            run(c, q, "cg_p", [&] { launch_cg_p(P, q); });
        });
        if (st != SPH_OK) return st;
    }
    if (c->any_warm) {
        run(c, s, "warm_density", [&] { launch_warm_density(P, s); });
        if (c->any_learned) run(c, s, "mlp_warm", [&] { launch_mlp_warm(P, s); });
    }
    // the warm-start pressure of the density solve, or the WCSPH equation-of-state pressure
    // (written by the non-pressure kernel), applied once
    if (c->any_warm || c->any_wcsph) {
        run(c, s, "dens_warm_pass_b", [&] { launch_pass_b(P, 1, 1, c->batch, s); });
        if (c->any_strong) run(c, s, "strong_coupling", [&] { launch_strong_update(P, 3, s); });
    }
    if ((st = loop(1)) != SPH_OK) return st;
    if (c->any_bodies) {
        run(c, s, "body_force", [&] { launch_body_force(P, s); });
        run(c, s, "body_reduce", [&] { launch_body_reduce(P, s); });
    }
    run(c, s, "advect", [&] { launch_advect(P, s); });
    run(c, s, "step_end", [&] { launch_step_end(P, s); });
    return SPH_OK;
}

sph_status build_graph(sph_ctx *c)
{
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    CK(cudaStreamBeginCapture(c->cap0, cudaStreamCaptureModeRelaxed));
    sph_status st = enqueue_step(c, c->cap0, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap0, &g);
    if (st != SPH_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    c->graph = g;
    CK(cudaGraphInstantiate(&c->exec, g, 0));
    return SPH_OK;
}

sph_status check_async(sph_ctx *c)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return SPH_OK;
}

sph_status create_impl(const sph_scene_desc *descs, int32_t n, const sph_allocator *alloc, void *stream,
                       sph_ctx **out, int batch = 4)
{
    if (!out) return SPH_EINVAL;
    *out = nullptr;
    sph_ctx *c = new sph_ctx();
    auto bail = [&](sph_status st) {
        sph_destroy(c);
        return st;
    };
    if (!descs || n < 1) {
        delete c;
        return SPH_EINVAL;
    }
    c->stream = (cudaStream_t)stream;
    c->batch = batch == 8 ? 8 : 4;
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->use_alloc = true;
    }
    for (int s = 0; s < n; ++s) {
        sph_status st = validate(c, descs[s], s);
        if (st != SPH_OK) {
            delete c;
            return st;
        }
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return SPH_ECUDA;
    }
    c->nscenes = n;
    c->scenes.resize(n);
    int64_t NF = 0, NB = 0, NC = 0;
    int32_t nfblk = 0, nbblk = 0, ntblk = 0, nbodies = 0;
    int cap_f = 0, cap_b = 0;
    // threads per particle in the neighbour sweeps: one value for the whole context, the
    // largest one given, else by size: enough threads to fill every SM (8 lanes up to
    // 152 x 2048 / 8 particles, 4 up to twice that, 2 up to four times)
    int lanes = 0;
    for (int s = 0; s < n; ++s) lanes = std::max(lanes, (int)descs[s].lanes_per_particle);
    if (lanes == 0) {
        int64_t nf = 0;
        for (int s = 0; s < n; ++s) nf += descs[s].n_fluid;
        lanes = auto_lanes(nf);
    }
    for (int s = 0; s < n; ++s) {
        const sph_scene_desc &d = descs[s];
        SceneDev &q = c->scenes[s];
        memset(&q, 0, sizeof q);
        q.f_off = NF;
        q.nf = d.n_fluid;
        q.b_off = NB;
        q.nb = d.n_boundary;
        q.c_off = NC;
        q.cell = d.cell_size > 0.0f ? d.cell_size : default_cell(d.radius);
        q.R = q.cell >= default_cell(d.radius) ? 1 : 2;
        int64_t nc = 1;
        for (int a = 0; a < 3; ++a) {
            q.origin[a] = d.domain_min[a] - q.cell;
            float ext = (d.domain_max[a] - d.domain_min[a]) / q.cell;
            q.dims[a] = (int32_t)std::ceil(ext) + 2;
            nc *= q.dims[a];
        }
        q.ncell = (int32_t)nc;
        const double r = d.radius, h = 4.0 * r;
        q.h = (float)h;
        q.h2 = q.h * q.h;
        q.inv_h = (float)(1.0 / h);
        q.m = (float)((double)d.rest_density * 8.0 * r * r * r);
        q.rho0 = d.rest_density;
        q.err_scale = d.n_fluid > 0 ? 1.0 / ((double)d.n_fluid * (double)d.rest_density) : 0.0;
        q.sigma = (float)(8.0 / (kPi * h * h * h));
        q.kgrad = (float)(48.0 / (kPi * h * h * h * h));
        double gs = (double)q.m * 48.0 / (kPi * h * h * h * h);
        q.eps_alpha = (float)(1e-6 * gs * gs);
        q.mu = d.viscosity * d.rest_density;
        q.xsph = d.xsph_c;
        for (int a = 0; a < 3; ++a) q.g[a] = d.gravity[a];
        q.eta[0] = d.eta_divergence;
        q.eta[1] = d.eta_density;
        q.dt_max = d.dt_max;
        q.cfl = d.cfl;
        q.two_r = 2.0f * d.radius;
        const bool eos = d.pressure_solver == SPH_SOLVER_WCSPH;   // no iterative solves
        const bool no_div = eos || d.pressure_solver == SPH_SOLVER_PCISPH;
        q.min_it[0] = no_div ? 0 : d.min_iter_divergence;
        q.max_it[0] = no_div ? 0 : d.max_iter_divergence;
        q.min_it[1] = eos ? 0 : d.min_iter_density;
        q.max_it[1] = eos ? 0 : d.max_iter_density;
        q.visc_mode = d.viscosity_mode;
        q.solver = d.pressure_solver;
        const bool wc = d.pressure_solver == SPH_SOLVER_WCSPH;
        q.eos_k = wc ? d.eos_stiffness : 0.0f;
        q.eos_gamma = wc ? (d.eos_exponent > 0.0f ? d.eos_exponent : 7.0f) : 0.0f;
        const bool pci = d.pressure_solver == SPH_SOLVER_PCISPH;
        q.warm = (wc || pci) ? 0 : d.warm_start;
        q.div_on = (d.divergence_solve && !wc && !pci) ? 1 : 0;
        q.pci_c = pci ? (float)pcisph_prototype(d.radius) : 0.0f;
        q.warm_frac = d.warm_start_fraction > 0.0f ? d.warm_start_fraction : 0.5f;
        q.learned_frac = d.learned_fraction > 0.0f ? d.learned_fraction : 0.6f;
        q.learned_gate = d.learned_gate;
        q.strong = (d.rigid_coupling == SPH_COUPLING_STRONG && d.n_bodies > 0) ? 1 : 0;
        q.has_moving = d.n_bodies > 0 ? 1 : 0;
        q.body_off = nbodies;
        q.nbody = d.n_bodies;
        q.fblk_first = nfblk;
        q.fblk_count = (int32_t)((d.n_fluid + kBlock - 1) / kBlock);
        q.bblk_first = nbblk;
        q.bblk_count = (int32_t)((d.n_boundary + kBlock - 1) / kBlock);
        q.tblk_first = ntblk;
        q.tblk_count = (int32_t)((d.n_fluid * lanes + kBlock - 1) / kBlock);
        q.cap_f = d.max_fluid_neighbors > 0 ? d.max_fluid_neighbors : kDefaultCapF;
        q.cap_b = d.max_boundary_neighbors > 0 ? d.max_boundary_neighbors : kDefaultCapB;
        {
            // stencil culling margin: 1e-3 h, plus a bound on the rounding of cell bounds and
            // coordinates of the domain's magnitude (a few float ulps)
            double mag = 0.0;
            for (int a = 0; a < 3; ++a)
                mag = std::max(mag, std::max(std::fabs((double)d.domain_min[a]), std::fabs((double)d.domain_max[a])));
            mag += 2.0 * q.cell;
            const double margin = 1e-3 * h + 1e-6 * mag;
            q.cull2 = (float)((h + margin) * (h + margin));
        }
        q.cg_tol = d.cg_tol > 0.0f ? d.cg_tol : 1e-4f;
        q.cg_max = d.cg_max_iter > 0 ? d.cg_max_iter : 500;
        cap_f = std::max(cap_f, q.cap_f);
        cap_b = std::max(cap_b, q.cap_b);
        for (int k = 0; k < q.fblk_count; ++k) c->fblk_scene.push_back(s);
        for (int k = 0; k < q.bblk_count; ++k) c->bblk_scene.push_back(s);
        for (int k = 0; k < q.tblk_count; ++k) c->tblk_scene.push_back(s);
        NF += d.n_fluid;
        NB += d.n_boundary;
        NC += nc;
        nfblk += q.fblk_count;
        nbblk += q.bblk_count;
        ntblk += q.tblk_count;
        nbodies += d.n_bodies;
        c->max_bodies = std::max(c->max_bodies, (int)d.n_bodies);
        c->any_moving |= d.n_bodies > 0;
        c->any_bodies |= d.n_bodies > 0;
        c->any_div |= q.div_on != 0;
        c->any_warm_div |= q.div_on != 0 && q.warm != 0;
        c->any_warm |= q.warm != 0;
        c->any_learned |= q.warm == 2;
        c->any_wcsph |= q.solver == SPH_SOLVER_WCSPH;
        c->any_strong |= q.strong != 0;
        c->any_implicit |= d.viscosity_mode == 3;
    }
    if (NC >= ((int64_t)1 << 32) - 1 || NF >= ((int64_t)1 << 31) || (double)NF * cap_f > 4.0e10)
        return bail(fail(c, SPH_EINVAL, "context too large"));
    Ptrs &P = c->P;
    P.nfblk = nfblk;
    P.nbblk = nbblk;
    P.ntblk = ntblk;
    P.lanes = lanes;
    P.nscenes = n;
    P.nbodies_total = nbodies;
    P.NF = NF;
    P.NB = NB;
    P.NC = NC;
    c->reported_flags.assign(n, 0);

    bool ok = true;
    SceneState *st = nullptr;
    ok &= dalloc(c, c->d_scenes, n);
    ok &= dalloc(c, st, n);
    ok &= dalloc(c, P.ctl, 1);
    ok &= dalloc(c, P.bodies, std::max(nbodies, 1));
    int32_t *fbs = nullptr, *bbs = nullptr, *tbs = nullptr;
    ok &= dalloc(c, fbs, std::max(nfblk, 1));
    ok &= dalloc(c, bbs, std::max(nbblk, 1));
    ok &= dalloc(c, tbs, std::max(ntblk, 1));
    ok &= dalloc(c, P.pos_s, NF) && dalloc(c, P.vel_s, NF) && dalloc(c, P.pos_c, NF) && dalloc(c, P.vel_c, NF);
    ok &= dalloc(c, P.kprev_c, NF) && dalloc(c, P.kvprev_c, NF) && dalloc(c, P.kprev_s, NF) &&
          dalloc(c, P.kvprev_s, NF);
    ok &= dalloc(c, P.ksum, NF) && dalloc(c, P.kvsum, NF) && dalloc(c, P.alpha, NF) && dalloc(c, P.k0, NF);
    ok &= dalloc(c, P.id_c, NF) && dalloc(c, P.id_s, NF) && dalloc(c, P.nnf, NF) && dalloc(c, P.nnb, NF);
    ok &= dalloc(c, P.nbr, (size_t)NF * cap_f) && dalloc(c, P.bnbr, (size_t)NF * cap_b);
    ok &= dalloc(c, P.feat, (size_t)NF * 4);
    ok &= dalloc(c, P.cell_count, NC) && dalloc(c, P.cell_start, NC + 1);
    ok &= dalloc(c, P.key_tmp, NF) && dalloc(c, P.slot_tmp, NF) && dalloc(c, P.sid_tmp, NF) &&
          dalloc(c, P.src_tmp, NF) && dalloc(c, P.cell_tmp, NF);
    int64_t NBa = std::max<int64_t>(NB, 1);
    ok &= dalloc(c, P.bx_o, NBa) && dalloc(c, P.bv_o, NBa) && dalloc(c, P.br0, NBa) && dalloc(c, P.bbody, NBa);
    ok &= dalloc(c, P.bpos_s, NBa) && dalloc(c, P.bvel_s, NBa) && dalloc(c, P.bid_s, NBa) &&
          dalloc(c, P.bbody_s, NBa);
    ok &= dalloc(c, P.bcell_count, NC) && dalloc(c, P.bcell_start, NC + 1);
    ok &= dalloc(c, P.large_f, large_capacity(NF)) && dalloc(c, P.large_b, large_capacity(NBa));
    ok &= dalloc(c, P.bkey_tmp, NBa) && dalloc(c, P.bslot_tmp, NBa) && dalloc(c, P.bsid_tmp, NBa) &&
          dalloc(c, P.bsrc_tmp, NBa) && dalloc(c, P.bcell_tmp, NBa);
    ok &= dalloc(c, P.partial, std::max(ntblk, 1));
    ok &= dalloc(c, P.partial2, std::max(ntblk, 1));
    ok &= dalloc(c, P.body_partial, (size_t)std::max(ntblk, 1) * std::max(nbodies, 1) * 6);
    ok &= dalloc(c, P.blk_touch, std::max(ntblk, 1));
    if (c->any_implicit) {
        ok &= dalloc(c, P.cg_r, NF) && dalloc(c, P.cg_p, NF) && dalloc(c, P.cg_ap, NF);
        ok &= dalloc(c, P.cg_dots, 2 * (size_t)std::max(std::max(nfblk, ntblk), 1));
    }
    ok &= dalloc(c, P.mlp_w, SPH_MLP_PARAMS);
    if (c->any_learned) {
        int64_t nl = 0;
        for (int32_t k = 0; k < n; ++k)
            if (c->scenes[k].warm == 2) nl += c->scenes[k].nf;
        P.nlearned = nl;
        ok &= dalloc(c, P.mlp_rows, std::max<int64_t>(nl, 1));
    }
    P.scan_tiles = scan_tiles_for(NC);
    ok &= dalloc(c, P.scan_status, std::max(P.scan_tiles, 1));
    ok &= dalloc(c, P.bscan_status, std::max(P.scan_tiles, 1));
    if (!ok) return bail(fail(c, SPH_ENOMEM, "device allocation failed"));
    P.scenes = c->d_scenes;
    P.st = st;
    P.fblk_scene = fbs;
    P.bblk_scene = bbs;
    P.tblk_scene = tbs;
    if (cudaMallocHost(&c->h_flag, sizeof(uint32_t)) != cudaSuccess)
        return bail(fail(c, SPH_ENOMEM, "pinned allocation failed"));

    // streams used only for capture
    if (cudaStreamCreateWithFlags(&c->cap0, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap1, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(c, SPH_ECUDA, "stream creation failed"));

    // ---- upload
    cudaStream_t s = c->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    std::vector<SceneState> hst(n);
    memset(hst.data(), 0, sizeof(SceneState) * n);
    std::vector<float4> f4;
    std::vector<float> zf;
    std::vector<int32_t> ids;
    std::vector<BodyDev> hb(std::max(nbodies, 1));
    memset(hb.data(), 0, sizeof(BodyDev) * hb.size());
    std::vector<float4> bx, bv, br;
    std::vector<int32_t> bbody;
    for (int sc = 0; sc < n; ++sc) {
        const sph_scene_desc &d = descs[sc];
        SceneDev &q = c->scenes[sc];
        // initial CFL step from the initial velocities
        double vmax = 0.0;
        f4.resize(d.n_fluid);
        for (int64_t i = 0; i < d.n_fluid; ++i)
            f4[i] = make_float4(d.fluid_x[3 * i], d.fluid_x[3 * i + 1], d.fluid_x[3 * i + 2], 0.0f);
        ok &= up(P.pos_c + q.f_off, f4.data(), sizeof(float4) * d.n_fluid);
        ok &= up(P.pos_s + q.f_off, f4.data(), sizeof(float4) * d.n_fluid);
        for (int64_t i = 0; i < d.n_fluid; ++i) {
            float vx = d.fluid_v ? d.fluid_v[3 * i] : 0.f, vy = d.fluid_v ? d.fluid_v[3 * i + 1] : 0.f,
                  vz = d.fluid_v ? d.fluid_v[3 * i + 2] : 0.f;
            f4[i] = make_float4(vx, vy, vz, 0.0f);
            vmax = std::max(vmax, std::sqrt((double)vx * vx + (double)vy * vy + (double)vz * vz));
        }
        ok &= up(P.vel_c + q.f_off, f4.data(), sizeof(float4) * d.n_fluid);
        ok &= up(P.vel_s + q.f_off, f4.data(), sizeof(float4) * d.n_fluid);
        ids.resize(d.n_fluid);
        for (int64_t i = 0; i < d.n_fluid; ++i) ids[i] = (int32_t)i;
        ok &= up(P.id_c + q.f_off, ids.data(), sizeof(int32_t) * d.n_fluid);
        ok &= up(P.id_s + q.f_off, ids.data(), sizeof(int32_t) * d.n_fluid);
        float dt0 = d.dt_max;
        if (d.cfl > 0.0f && vmax > 0.0) dt0 = std::min(dt0, (float)(d.cfl * 2.0 * d.radius / vmax));
        hst[sc].dt_next = dt0;
        hst[sc].dt = dt0;
        // boundary
        bx.resize(d.n_boundary);
        bv.resize(d.n_boundary);
        br.resize(d.n_boundary);
        bbody.resize(d.n_boundary);
        for (int64_t b = 0; b < d.n_boundary; ++b) {
            bx[b] = make_float4(d.boundary_x[3 * b], d.boundary_x[3 * b + 1], d.boundary_x[3 * b + 2], 0.0f);
            bv[b] = make_float4(0.f, 0.f, 0.f, 0.f);
            br[b] = make_float4(0.f, 0.f, 0.f, 0.f);
            bbody[b] = d.boundary_body ? d.boundary_body[b] : -1;
        }
        for (int k = 0; k < d.n_bodies; ++k) {
            const sph_rigid_desc &rd = d.bodies[k];
            BodyDev &B = hb[q.body_off + k];
            B.mass = rd.mass;
            B.inv_mass = 1.0 / rd.mass;
            for (int a = 0; a < 3; ++a) {
                B.inertia[a] = rd.inertia[a];
                B.inv_inertia[a] = 1.0 / rd.inertia[a];
                B.com[a] = rd.com[a];
                B.vel[a] = rd.vel[a];
                B.omega[a] = rd.omega[a];
            }
            for (int a = 0; a < 4; ++a) B.quat[a] = rd.quat[a];
            B.scene = sc;
            double w = rd.quat[0], x = rd.quat[1], y = rd.quat[2], z = rd.quat[3];
            double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                              {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                              {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
            double rad = 0.0;
            for (int64_t b = 0; b < d.n_boundary; ++b) {
                if (bbody[b] != k) continue;
                double dd[3] = {d.boundary_x[3 * b] - rd.com[0], d.boundary_x[3 * b + 1] - rd.com[1],
                                d.boundary_x[3 * b + 2] - rd.com[2]};
                double r0[3];
                for (int a = 0; a < 3; ++a) r0[a] = R[0][a] * dd[0] + R[1][a] * dd[1] + R[2][a] * dd[2];
                br[b] = make_float4((float)r0[0], (float)r0[1], (float)r0[2], 0.0f);
                rad = std::max(rad, std::sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]));
                double rw[3] = {dd[0], dd[1], dd[2]};
                bv[b] = make_float4((float)(rd.vel[0] + rd.omega[1] * rw[2] - rd.omega[2] * rw[1]),
                                    (float)(rd.vel[1] + rd.omega[2] * rw[0] - rd.omega[0] * rw[2]),
                                    (float)(rd.vel[2] + rd.omega[0] * rw[1] - rd.omega[1] * rw[0]), 0.0f);
            }
            B.radius = rad;
            for (int a = 0; a < 3; ++a) {
                B.lo[a] = (double)d.domain_min[a] + rad;
                B.hi[a] = (double)d.domain_max[a] - rad;
            }
        }
        if (d.n_boundary > 0) {
            ok &= up(P.bx_o + q.b_off, bx.data(), sizeof(float4) * d.n_boundary);
            ok &= up(P.bv_o + q.b_off, bv.data(), sizeof(float4) * d.n_boundary);
            ok &= up(P.br0 + q.b_off, br.data(), sizeof(float4) * d.n_boundary);
            ok &= up(P.bbody + q.b_off, bbody.data(), sizeof(int32_t) * d.n_boundary);
        }
        if (!ok) break;
    }
    if (!ok) return bail(fail(c, SPH_ECUDA, "upload failed"));
    Control hctl;
    memset(&hctl, 0, sizeof hctl);
    hctl.nscenes = n;
    ok &= up(c->d_scenes, c->scenes.data(), sizeof(SceneDev) * n);
    ok &= up(st, hst.data(), sizeof(SceneState) * n);
    ok &= up(P.ctl, &hctl, sizeof hctl);
    ok &= up(P.bodies, hb.data(), sizeof(BodyDev) * hb.size());
    ok &= up(fbs, c->fblk_scene.data(), sizeof(int32_t) * std::max(nfblk, 0));
    ok &= up(tbs, c->tblk_scene.data(), sizeof(int32_t) * std::max(ntblk, 0));
    if (nbblk) ok &= up(bbs, c->bblk_scene.data(), sizeof(int32_t) * nbblk);
    ok &= cudaMemsetAsync(P.cell_count, 0, sizeof(uint32_t) * NC, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.bcell_count, 0, sizeof(uint32_t) * NC, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.scan_status, 0, sizeof(uint64_t) * std::max(P.scan_tiles, 1), s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.bscan_status, 0, sizeof(uint64_t) * std::max(P.scan_tiles, 1), s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.kprev_c, 0, sizeof(float) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.kvprev_c, 0, sizeof(float) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.ksum, 0, sizeof(float) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.kvsum, 0, sizeof(float) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.alpha, 0, sizeof(float) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.k0, 0, sizeof(float) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.nnf, 0, sizeof(int32_t) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.nnb, 0, sizeof(int32_t) * NF, s) == cudaSuccess;
    ok &= cudaMemsetAsync(P.feat, 0, sizeof(float) * 4 * NF, s) == cudaSuccess;
    if (!ok) return bail(fail(c, SPH_ECUDA, "upload failed"));

    // ---- static boundary: grid order and pseudo-masses (moving bodies redo it per step)
    if (nbblk) {
        launch_key_hist(P, SORT_BOUNDARY, s);
        launch_scan_cells(P, SORT_BOUNDARY, s);
        launch_scatter(P, SORT_BOUNDARY, s);
        launch_rank_gather(P, SORT_BOUNDARY, s);
        launch_boundary_psi(P, s);
        sph_status cs = check_async(c);
        if (cs != SPH_OK) return bail(cs);
    }
    if (c->any_learned && mlp_prepare_kernels() != cudaSuccess)
        return bail(fail(c, SPH_ECUDA, "network kernel attributes could not be set"));
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(c, SPH_ECUDA, "create: %s", cudaGetErrorString(cudaGetLastError())));
    sph_status gs = build_graph(c);
    if (gs != SPH_OK) return bail(gs);
    *out = c;
    return SPH_OK;
}

// ------------------------------------------------------------------ autotuning
std::mutex g_tune_mu;
std::map<std::string, sph_tuning> g_tune_cache;

std::string tune_key(const sph_scene_desc *d, int32_t n)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    char name[256] = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) snprintf(name, sizeof name, "%s", prop.name);
    int64_t nf = 0;
    for (int s = 0; s < n; ++s) nf += d[s].n_fluid;
    int bucket = 0;
    while ((int64_t)1 << (bucket + 1) <= nf) ++bucket;
    char buf[512];
    snprintf(buf, sizeof buf, "%s|fluid2^%d|scenes%d|bodies%d|visc%d|lanes%d", name, bucket, n, d[0].n_bodies,
             d[0].viscosity_mode, d[0].lanes_per_particle);
    return buf;
}

// Time `steps` CUDA-graph steps of one configuration on a temporary context.
sph_status time_config(const std::vector<sph_scene_desc> &descs, const sph_allocator *alloc, void *stream,
                       int batch, int steps, float *ms)
{
    sph_ctx *t = nullptr;
    sph_status st = create_impl(descs.data(), (int32_t)descs.size(), alloc, stream, &t, batch);
    if (st != SPH_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    st = sph_steps(t, 2, 0.0f);
    if (st == SPH_OK) {
        cudaEventRecord(a, s);
        st = sph_steps(t, steps, 0.0f);
        cudaEventRecord(b, s);
    }
    if (st == SPH_OK && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(ms, a, b);
    else if (st == SPH_OK) st = SPH_ECUDA;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    sph_destroy(t);
    *ms /= (float)steps;
    return st;
}

// Scenes with cell_size < 0: pick the cell size (27- or 125-cell stencil), the threads
// per particle of the sweeps and the gather batch by timing each candidate (two rounds,
// the faster time of each), cache the choice, and build the context with it.
sph_status create_tuned(const sph_scene_desc *descs, int32_t n, const sph_allocator *alloc, void *stream,
                        sph_ctx **out)
{
    std::vector<sph_scene_desc> trial(descs, descs + n);
    const std::string key = tune_key(descs, n);
    sph_tuning best{};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    // lanes given by the caller stay fixed
    int fixed_lanes = 0;
    for (int s = 0; s < n; ++s) fixed_lanes = std::max(fixed_lanes, (int)descs[s].lanes_per_particle);
    auto set_trial = [&](float factor, int lanes) {
        for (int s = 0; s < n; ++s) {
            trial[s].cell_size = descs[s].cell_size < 0.0f ? 4.0f * descs[s].radius * factor : descs[s].cell_size;
            trial[s].lanes_per_particle = lanes;
        }
    };
    if (!cached) {
        const float factors[2] = {1.00390625f, 0.501953125f};
        int64_t nf_tot = 0;
        for (int s = 0; s < n; ++s) nf_tot += descs[s].n_fluid;
        // (lanes, batch) candidates; contexts small enough for 8 lanes try them instead of 2
        // (unless the caller fixed the lanes: then only that count's candidates count)
        int lanes_c[4] = {1, 1, 2, 4};
        const int batch_c[4] = {4, 8, 4, 4};
        if (fixed_lanes ? fixed_lanes == 8 : auto_lanes(nf_tot) == 8) lanes_c[2] = 8;
        best.n_trials = 0;
        for (int f = 0; f < 2; ++f)
            for (int b = 0; b < 4; ++b) {
                if (fixed_lanes && lanes_c[b] != fixed_lanes) continue;
                const int k = best.n_trials++;
                best.trial_cell_factor[k] = factors[f];
                best.trial_batch[k] = batch_c[b];
                best.trial_lanes[k] = lanes_c[b];
                best.trial_ms[k] = 1e30f;
            }
        // every candidate is timed in two rounds and keeps its faster time: the first
        // candidate of the first round also meets the process's cold start
        for (int round = 0; round < 2; ++round)
            for (int k = 0; k < best.n_trials; ++k) {
                set_trial(best.trial_cell_factor[k], best.trial_lanes[k]);
                float ms = 0.0f;
                sph_status st = time_config(trial, alloc, stream, best.trial_batch[k], 5, &ms);
                if (st != SPH_OK) return st;
                best.trial_ms[k] = std::min(best.trial_ms[k], ms);
            }
        float best_ms = 1e30f;
        for (int k = 0; k < best.n_trials; ++k)
            if (best.trial_ms[k] < best_ms) {
                best_ms = best.trial_ms[k];
                best.cell_factor = best.trial_cell_factor[k];
                best.gather_batch = best.trial_batch[k];
                best.lanes = best.trial_lanes[k];
            }
        // keep the default configuration (27-cell stencil, gather batch 4, lanes by size)
        // unless a candidate is more than 3 % faster: short trials are noisy, and the
        // default is the one whose kernels are profiled
        int64_t nf_all = 0;
        for (int s = 0; s < n; ++s) nf_all += descs[s].n_fluid;
        const int def_lanes = fixed_lanes ? fixed_lanes : auto_lanes(nf_all);
        for (int k = 0; k < best.n_trials; ++k)
            if (best.trial_cell_factor[k] == factors[0] && best.trial_batch[k] == 4 &&
                best.trial_lanes[k] == def_lanes && best.trial_ms[k] <= 1.03f * best_ms) {
                best.cell_factor = factors[0];
                best.gather_batch = 4;
                best.lanes = def_lanes;
            }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    best.tuned = 1;
    best.from_cache = cached ? 1 : 0;
    set_trial(best.cell_factor, best.lanes);
    sph_status st = create_impl(trial.data(), n, alloc, stream, out, best.gather_batch);
    if (st == SPH_OK) (*out)->tuning = best;
    return st;
}

sph_status check_ctx(sph_ctx *c)
{
    if (!c) return SPH_EINVAL;
    if (c->poisoned) return SPH_ECUDA;
    return SPH_OK;
}

}  // namespace

// ===================================================================================== ABI
extern "C" {

int32_t sph_abi_version(void) { return SPH_ABI_VERSION; }

static bool wants_tuning(const sph_scene_desc *d, int32_t n)
{
    for (int s = 0; d && s < n; ++s)
        if (d[s].cell_size < 0.0f) return true;
    return false;
}

sph_status sph_create(const sph_scene_desc *scene, const sph_allocator *alloc, void *stream, sph_ctx **out)
{
    return sph_create_batch(scene, 1, alloc, stream, out);
}

sph_status sph_create_batch(const sph_scene_desc *scenes, int32_t n, const sph_allocator *alloc, void *stream,
                            sph_ctx **out)
{
    if (wants_tuning(scenes, n)) {
        // validate once (a negative cell size is the tuning request)
        std::vector<sph_scene_desc> v(scenes, scenes + n);
        for (auto &d : v)
            if (d.cell_size < 0.0f) d.cell_size = 0.0f;
        sph_ctx probe;
        for (int s = 0; s < n; ++s) {
            sph_status st = validate(&probe, v[s], s);
            if (st != SPH_OK) return st;
        }
        return create_tuned(scenes, n, alloc, stream, out);
    }
    return create_impl(scenes, n, alloc, stream, out);
}

sph_status sph_surface_field(sph_ctx *c, int32_t scene, const float origin[3], float spacing, const int32_t dims[3],
                             float *field)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (scene < 0 || scene >= c->nscenes) return fail(c, SPH_EINVAL, "scene %d out of range", scene);
    if (!origin || !dims || !field || !(spacing > 0.0f) || !std::isfinite(spacing))
        return fail(c, SPH_EINVAL, "surface field: bad grid");
    int64_t nodes = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || !std::isfinite(origin[a])) return fail(c, SPH_EINVAL, "surface field: bad grid");
        nodes *= dims[a];
    }
    if (nodes > ((int64_t)1 << 31)) return fail(c, SPH_EINVAL, "surface field: grid too large");
    const SceneDev &q = c->scenes[scene];
    cudaError_t e = post_surface_field(q, c->P.pos_c + q.f_off, c->P.vel_c + q.f_off, origin, spacing, dims, field,
                                       c->stream);
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "surface field: %s", cudaGetErrorString(e));
    return SPH_OK;
}

sph_status sph_render_heightmap(sph_ctx *c, int32_t scene, const float lo[2], const float hi[2], int32_t width,
                                int32_t height, float radius, float *out)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (scene < 0 || scene >= c->nscenes) return fail(c, SPH_EINVAL, "scene %d out of range", scene);
    if (!lo || !hi || !out || width < 1 || height < 1 || (int64_t)width * height > ((int64_t)1 << 31) ||
        !(radius > 0.0f) || !std::isfinite(radius) || !(hi[0] > lo[0]) || !(hi[1] > lo[1]) ||
        !std::isfinite(lo[0]) || !std::isfinite(lo[1]) || !std::isfinite(hi[0]) || !std::isfinite(hi[1]))
        return fail(c, SPH_EINVAL, "height map: bad view");
    const SceneDev &q = c->scenes[scene];
    cudaError_t e = post_height_map(c->P.pos_c + q.f_off, q.nf, lo, hi, width, height, radius, out, c->stream);
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "height map: %s", cudaGetErrorString(e));
    return SPH_OK;
}

sph_status sph_get_tuning(sph_ctx *c, sph_tuning *out)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (!out) return fail(c, SPH_EINVAL, "out is NULL");
    *out = c->tuning;
    if (!c->tuning.tuned) {
        out->gather_batch = c->batch;
        out->lanes = c->P.lanes;
        out->cell_factor = c->scenes[0].cell / (4.0f * (float)(c->scenes[0].two_r * 0.5f));
    }
    return SPH_OK;
}

sph_status sph_step(sph_ctx *c, float dt)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (!std::isfinite(dt)) return fail(c, SPH_EINVAL, "dt not finite");
    float want = dt > 0.0f ? dt : 0.0f;
    if (want != c->last_dt) {
        launch_set_dt(c->P, want, c->stream);
        c->last_dt = want;
        c->host_launches += 1;
    }
    if (c->graph_mode) {
        CK(cudaGraphLaunch(c->exec, c->stream));
    } else {
        st = enqueue_step(c, c->stream, false);
        if (st != SPH_OK) return st;
    }
    return check_async(c);
}

sph_status sph_steps(sph_ctx *c, int32_t n, float dt)
{
    if (n < 0) return fail(c, SPH_EINVAL, "negative step count");
    for (int32_t k = 0; k < n; ++k) {
        sph_status st = sph_step(c, dt);
        if (st != SPH_OK) return st;
    }
    return SPH_OK;
}

sph_status sph_probe_wait_timeout(sph_ctx *c, int32_t spin_limit)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (spin_limit < 1 || spin_limit > 1000000) return fail(c, SPH_EINVAL, "spin_limit (1..10^6)");
    k_probe_wait<<<1, 1, 0, c->stream>>>(c->P.ctl, (uint32_t)spin_limit);
    return check_async(c);
}

sph_status sph_synchronize(sph_ctx *c)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    if (c->copy) CK(cudaStreamSynchronize(c->copy));
    Control hctl;
    CK(cudaMemcpy(&hctl, c->P.ctl, sizeof hctl, cudaMemcpyDeviceToHost));
    if (hctl.error)
        return fail(c, SPH_ETIMEOUT, "a bounded device wait gave up (code %d)", hctl.error);
    std::vector<SceneState> hs(c->nscenes);
    CK(cudaMemcpy(hs.data(), c->P.st, sizeof(SceneState) * c->nscenes, cudaMemcpyDeviceToHost));
    sph_status result = SPH_OK;
    for (int s = 0; s < c->nscenes; ++s) {
        int fresh = hs[s].flags & ~c->reported_flags[s];
        c->reported_flags[s] |= hs[s].flags;
        if (fresh & SPH_FLAG_NONFINITE) result = fail(c, SPH_ENUMERIC, "scene %d: non-finite state", s);
        else if ((fresh & SPH_FLAG_OVERFLOW) && result == SPH_OK)
            result = fail(c, SPH_EOVERFLOW, "scene %d: neighbour list capacity exceeded", s);
        else if ((fresh & SPH_FLAG_NOCONVERGE) && result == SPH_OK)
            result = fail(c, SPH_ENOCONVERGE, "scene %d: solver stopped at max_iter", s);
    }
    return result;
}

sph_status sph_read_wait(sph_ctx *c, int32_t keep)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (keep < 0 || keep >= sph_ctx::kReadRing) return fail(c, SPH_EINVAL, "keep %d not in 0..%d", keep,
                                                             sph_ctx::kReadRing - 1);
    const int64_t last = c->reads - 1 - keep;   // the newest read that must be complete
    if (last >= 0) CK(cudaEventSynchronize(c->read_done[last % sph_ctx::kReadRing]));
    return SPH_OK;
}

static sph_status scene_ok(sph_ctx *c, int32_t scene)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (scene < 0 || scene >= c->nscenes) return fail(c, SPH_EINVAL, "scene index %d out of range", scene);
    return SPH_OK;
}

// One enqueued host read (on_device = 3) of several fields of one scene: each field's
// unpermute kernel writes its slice of a staging slot on the context stream, then the copy
// stream copies the slot to the caller's host buffers and records the read's completion
// event.  A slot is refilled only after the read that last used it (two reads back) has
// been copied out.
struct HostField {
    int field;
    void *out;
    size_t bytes;
    bool boundary;
};
static sph_status read_host_async(sph_ctx *c, int32_t scene, const HostField *f, int nf)
{
    size_t total = 0;
    for (int k = 0; k < nf; ++k)
        if (f[k].out) total += (f[k].bytes + 255) & ~size_t(255);
    if (total == 0) return SPH_OK;
    if (!c->copy) {
        CK(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) CK(cudaEventCreateWithFlags(&c->staged[k], cudaEventDisableTiming));
        for (int k = 0; k < sph_ctx::kReadRing; ++k) CK(cudaEventCreateWithFlags(&c->read_done[k], cudaEventDisableTiming));
    }
    const int slot = (int)(c->reads & 1);
    if (c->reads >= 2) CK(cudaStreamWaitEvent(c->stream, c->read_done[(c->reads - 2) % sph_ctx::kReadRing], 0));
    if (c->stage_bytes[slot] < total) {
        void *p = dev_alloc(c, total);
        if (!p) return fail(c, SPH_ENOMEM, "host read staging (%zu bytes)", total);
        c->stage[slot] = p;
        c->stage_bytes[slot] = total;
    }
    const SceneDev &q = c->scenes[scene];
    unsigned char *base = static_cast<unsigned char *>(c->stage[slot]);
    size_t off = 0;
    for (int k = 0; k < nf; ++k) {
        if (!f[k].out) continue;
        const int64_t n = f[k].boundary ? q.nb : q.nf;
        if (n > 0) {
            const int blocks = (int)((n + 255) / 256);
            if (f[k].boundary) k_read_boundary<<<blocks, 256, 0, c->stream>>>(c->P, scene, f[k].field, base + off);
            else k_read_fluid<<<blocks, 256, 0, c->stream>>>(c->P, scene, f[k].field, base + off);
        }
        off += (f[k].bytes + 255) & ~size_t(255);
    }
    sph_status st = check_async(c);
    if (st != SPH_OK) return st;
    CK(cudaEventRecord(c->staged[slot], c->stream));
    CK(cudaStreamWaitEvent(c->copy, c->staged[slot], 0));
    off = 0;
    for (int k = 0; k < nf; ++k) {
        if (!f[k].out) continue;
        if (f[k].bytes) CK(cudaMemcpyAsync(f[k].out, base + off, f[k].bytes, cudaMemcpyDeviceToHost, c->copy));
        off += (f[k].bytes + 255) & ~size_t(255);
    }
    CK(cudaEventRecord(c->read_done[c->reads % sph_ctx::kReadRing], c->copy));
    c->reads += 1;
    return SPH_OK;
}

static sph_status read_into(sph_ctx *c, int32_t scene, int field, void *out, size_t bytes, bool boundary,
                            int32_t on_device)
{
    if (!out) return SPH_OK;
    const SceneDev &q = c->scenes[scene];
    int64_t n = boundary ? q.nb : q.nf;
    if (n == 0) return SPH_OK;
    void *dst = out;
    void *tmp = nullptr;
    const bool host = on_device == 0 || on_device == 3;
    if (host) {
        CK(cudaMallocAsync(&tmp, bytes, c->stream));
        dst = tmp;
    }
    int blocks = (int)((n + 255) / 256);
    if (boundary) k_read_boundary<<<blocks, 256, 0, c->stream>>>(c->P, scene, field, dst);
    else k_read_fluid<<<blocks, 256, 0, c->stream>>>(c->P, scene, field, dst);
    sph_status st = check_async(c);
    if (st != SPH_OK) return st;
    if (host) {
        CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaFreeAsync(tmp, c->stream));
    }
    return SPH_OK;
}

sph_status sph_read_state(sph_ctx *c, int32_t scene, float *x, float *v, float *rho, float *pressure,
                          int32_t on_device)
{
    sph_status st = scene_ok(c, scene);
    if (st != SPH_OK) return st;
    if (on_device < 0 || on_device > 3) return fail(c, SPH_EINVAL, "on_device %d not in 0..3", on_device);
    size_t nf = (size_t)c->scenes[scene].nf;
    if (on_device == 3) {
        const HostField f[4] = {{100, x, 12 * nf, false}, {101, v, 12 * nf, false}, {102, rho, 4 * nf, false},
                                {103, pressure, 4 * nf, false}};
        return read_host_async(c, scene, f, 4);
    }
    if ((st = read_into(c, scene, 100, x, 12 * nf, false, on_device)) != SPH_OK) return st;
    if ((st = read_into(c, scene, 101, v, 12 * nf, false, on_device)) != SPH_OK) return st;
    if ((st = read_into(c, scene, 102, rho, 4 * nf, false, on_device)) != SPH_OK) return st;
    if ((st = read_into(c, scene, 103, pressure, 4 * nf, false, on_device)) != SPH_OK) return st;
    if (on_device <= 1) CK(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_read_field(sph_ctx *c, int32_t scene, int32_t field, void *out, int32_t on_device)
{
    sph_status st = scene_ok(c, scene);
    if (st != SPH_OK) return st;
    size_t nf = (size_t)c->scenes[scene].nf, nb = (size_t)c->scenes[scene].nb;
    size_t bytes;
    bool boundary = false;
    switch (field) {
    case SPH_FIELD_V_DIV: bytes = 12 * nf; break;
    case SPH_FIELD_FEATURES: bytes = 16 * nf; break;
    case SPH_FIELD_PSI:
    case SPH_FIELD_BOUNDARY_SORTED_ID:
    case SPH_FIELD_BOUNDARY_CELL_KEY:
        bytes = 4 * nb;
        boundary = true;
        break;
    case SPH_FIELD_RHO: case SPH_FIELD_ALPHA: case SPH_FIELD_KAPPA: case SPH_FIELD_KAPPA_V:
    case SPH_FIELD_NN_FLUID: case SPH_FIELD_NN_BOUNDARY: case SPH_FIELD_KAPPA_PREV:
    case SPH_FIELD_KAPPA_V_PREV: case SPH_FIELD_CELL_KEY: case SPH_FIELD_SORTED_ID: case SPH_FIELD_KAPPA0:
        bytes = 4 * nf;
        break;
    default: return fail(c, SPH_EINVAL, "unknown field %d", field);
    }
    if (on_device < 0 || on_device > 3) return fail(c, SPH_EINVAL, "on_device %d not in 0..3", on_device);
    if (on_device == 3) {
        const HostField f[1] = {{field, out, bytes, boundary}};
        return read_host_async(c, scene, f, 1);
    }
    if ((st = read_into(c, scene, field, out, bytes, boundary, on_device)) != SPH_OK) return st;
    if (on_device <= 1) CK(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_write_state(sph_ctx *c, int32_t scene, const float *x, const float *v, const float *kappa_prev,
                           const float *kappa_v_prev, int32_t on_device)
{
    sph_status st = scene_ok(c, scene);
    if (st != SPH_OK) return st;
    const SceneDev &q = c->scenes[scene];
    const int64_t nf = q.nf;
    cudaStream_t s = c->stream;
    int blocks = (int)((nf + 255) / 256);
    // host inputs are staged into one device buffer before anything of the scene changes,
    // so that a failed staging leaves it as it was; the buffer is freed on every exit
    struct Stage {
        float *p = nullptr;
        cudaStream_t s;
        ~Stage() { if (p) cudaFreeAsync(p, s); }
    } stage{nullptr, s};
    const float *dx = x, *dv = v;
    if (!on_device && (x || v)) {
        if (cudaMallocAsync(&stage.p, 24 * (size_t)nf, s) != cudaSuccess) {
            stage.p = nullptr;
            return fail(c, SPH_ECUDA, "write_state staging failed");
        }
        if (x) {
            if (cudaMemcpyAsync(stage.p, x, 12 * nf, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return fail(c, SPH_ECUDA, "write_state staging failed");
            dx = stage.p;
        }
        if (v) {
            if (cudaMemcpyAsync(stage.p + 3 * nf, v, 12 * nf, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return fail(c, SPH_ECUDA, "write_state staging failed");
            dv = stage.p + 3 * nf;
        }
    }
    k_unpermute_to_sorted<<<blocks, 256, 0, s>>>(c->P, scene);
    k_sorted_to_canonical<<<blocks, 256, 0, s>>>(c->P, scene);
    if ((st = check_async(c)) != SPH_OK) return st;
    if (x) k_pack3<<<blocks, 256, 0, s>>>(c->P.pos_c + q.f_off, dx, nf, 0.0f);
    if (v) k_pack3<<<blocks, 256, 0, s>>>(c->P.vel_c + q.f_off, dv, nf, 0.0f);
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (kappa_prev) CK(cudaMemcpyAsync(c->P.kprev_c + q.f_off, kappa_prev, 4 * nf, kind, s));
    if (kappa_v_prev) CK(cudaMemcpyAsync(c->P.kvprev_c + q.f_off, kappa_v_prev, 4 * nf, kind, s));
    k_scene_cfl<<<1, 256, 0, s>>>(c->P, scene);
    if ((st = check_async(c)) != SPH_OK) return st;
    CK(cudaStreamSynchronize(s));
    return SPH_OK;
}

sph_status sph_get_stats(sph_ctx *c, int32_t scene, sph_stats *out)
{
    sph_status st = scene_ok(c, scene);
    if (st != SPH_OK) return st;
    if (!out) return fail(c, SPH_EINVAL, "out is NULL");
    CK(cudaStreamSynchronize(c->stream));
    SceneState h;
    CK(cudaMemcpy(&h, c->P.st + scene, sizeof h, cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof *out);
    out->steps = h.steps;
    out->div_iters = h.it[0];
    out->dens_iters = h.it[1];
    out->div_err = std::isinf(h.err[0]) ? 0.0 : h.err[0];
    out->dens_err = std::isinf(h.err[1]) ? 0.0 : h.err[1];
    out->div_err0 = h.err0[0];
    out->dens_err0 = h.err0[1];
    out->dt = h.dt;
    out->dt_next = h.dt_next;
    out->max_speed = std::sqrt(h.maxv2);
    out->max_fluid_nbrs = h.max_nn_f;
    out->max_boundary_nbrs = h.max_nn_b;
    out->cg_iters = h.cg_it;
    out->cg_residual = h.cg_res;
    out->clamps = h.clamps;
    out->flags = h.flags;
    out->total_div_iters = h.total_it[0];
    out->total_dens_iters = h.total_it[1];
    return SPH_OK;
}

sph_status sph_read_bodies(sph_ctx *c, int32_t scene, double *out)
{
    sph_status st = scene_ok(c, scene);
    if (st != SPH_OK) return st;
    const SceneDev &q = c->scenes[scene];
    if (q.nbody == 0 || !out) return SPH_OK;
    CK(cudaStreamSynchronize(c->stream));
    std::vector<BodyDev> hb(q.nbody);
    CK(cudaMemcpy(hb.data(), c->P.bodies + q.body_off, sizeof(BodyDev) * q.nbody, cudaMemcpyDeviceToHost));
    for (int k = 0; k < q.nbody; ++k) {
        double *o = out + 19 * k;
        for (int a = 0; a < 3; ++a) {
            o[a] = hb[k].com[a];
            o[7 + a] = hb[k].vel[a];
            o[10 + a] = hb[k].omega[a];
            o[13 + a] = hb[k].force[a];
            o[16 + a] = hb[k].torque[a];
        }
        for (int a = 0; a < 4; ++a) o[3 + a] = hb[k].quat[a];
    }
    return SPH_OK;
}

sph_status sph_write_bodies(sph_ctx *c, int32_t scene, const double *in)
{
    sph_status st = scene_ok(c, scene);
    if (st != SPH_OK) return st;
    const SceneDev &q = c->scenes[scene];
    if (q.nbody == 0) return SPH_OK;
    if (!in) return fail(c, SPH_EINVAL, "sph_write_bodies: NULL buffer");
    for (int k = 0; k < q.nbody; ++k) {
        const double *o = in + 19 * k;
        double n2 = 0.0;
        for (int a = 0; a < 13; ++a)
            if (!std::isfinite(o[a])) return fail(c, SPH_EINVAL, "sph_write_bodies: body %d not finite", k);
        for (int a = 0; a < 4; ++a) n2 += o[3 + a] * o[3 + a];
        if (!(n2 > 0.0)) return fail(c, SPH_EINVAL, "sph_write_bodies: body %d has a zero quaternion", k);
    }
    CK(cudaStreamSynchronize(c->stream));
    std::vector<BodyDev> hb(q.nbody);
    CK(cudaMemcpy(hb.data(), c->P.bodies + q.body_off, sizeof(BodyDev) * q.nbody, cudaMemcpyDeviceToHost));
    for (int k = 0; k < q.nbody; ++k) {
        const double *o = in + 19 * k;
        for (int a = 0; a < 3; ++a) {
            hb[k].com[a] = o[a];
            hb[k].vel[a] = o[7 + a];
            hb[k].omega[a] = o[10 + a];
        }
        for (int a = 0; a < 4; ++a) hb[k].quat[a] = o[3 + a];
    }
    CK(cudaMemcpy(c->P.bodies + q.body_off, hb.data(), sizeof(BodyDev) * q.nbody, cudaMemcpyHostToDevice));
    return SPH_OK;
}

sph_status sph_set_mode(sph_ctx *c, int32_t graph, int32_t timing)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    c->graph_mode = graph != 0;
    c->timing = timing != 0;
    return SPH_OK;
}

sph_status sph_kernel_times(sph_ctx *c, sph_kernel_time *out, int32_t cap, int32_t *n, int32_t reset)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if ((st = harvest(c)) != SPH_OK) return st;
    int32_t k = 0;
    for (auto &kv : c->times) {
        if (out && k < cap) {
            memset(out[k].name, 0, sizeof out[k].name);
            strncpy(out[k].name, kv.first.c_str(), sizeof out[k].name - 1);
            out[k].launches = kv.second.first;
            out[k].total_ms = kv.second.second;
        }
        ++k;
    }
    if (n) *n = k;
    if (reset) c->times.clear();
    return SPH_OK;
}

sph_status sph_set_mlp(sph_ctx *c, const float *params, int64_t n)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (!params || n != SPH_MLP_PARAMS) return fail(c, SPH_EINVAL, "network parameter block must hold %d floats", SPH_MLP_PARAMS);
    for (int k = SPH_MLP_WEIGHTS + 4; k < SPH_MLP_WEIGHTS + 8; ++k)
        if (!(params[k] > 0.0f)) return fail(c, SPH_EINVAL, "feature std must be > 0");
    if (!(params[SPH_MLP_PARAMS - 1] > 0.0f)) return fail(c, SPH_EINVAL, "label std must be > 0");
    for (int64_t k = 0; k < n; ++k)
        if (!std::isfinite(params[k])) return fail(c, SPH_EINVAL, "non-finite network parameter");
    CK(cudaMemcpyAsync(c->P.mlp_w, params, sizeof(float) * SPH_MLP_PARAMS, cudaMemcpyHostToDevice, c->stream));
    const int32_t one = 1;
    CK(cudaMemcpyAsync(&c->P.ctl->have_mlp, &one, sizeof one, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_set_trace(sph_ctx *c, int32_t capacity)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (capacity < 0 || capacity > (1 << 26)) return fail(c, SPH_EINVAL, "trace capacity out of range");
    CK(cudaStreamSynchronize(c->stream));
    unsigned long long *nt = nullptr;
    if (capacity > 0) CK(cudaMalloc(&nt, sizeof(unsigned long long) * capacity));
    const uint32_t counts[2] = {0u, (uint32_t)capacity};
    CK(cudaMemcpy(&c->P.ctl->trace, &nt, sizeof nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(&c->P.ctl->trace_n, counts, sizeof counts, cudaMemcpyHostToDevice));
    if (c->trace) cudaFree(c->trace);
    c->trace = nt;
    c->trace_cap = capacity;
    return SPH_OK;
}

sph_status sph_read_trace(sph_ctx *c, uint64_t *out, int32_t cap, int32_t *n, int32_t reset)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    uint32_t cnt = 0;
    CK(cudaMemcpy(&cnt, &c->P.ctl->trace_n, sizeof cnt, cudaMemcpyDeviceToHost));
    const uint32_t avail = std::min<uint32_t>(cnt, (uint32_t)c->trace_cap);
    if (out && c->trace && cap > 0)
        CK(cudaMemcpy(out, c->trace, sizeof(uint64_t) * std::min<uint32_t>(avail, (uint32_t)cap), cudaMemcpyDeviceToHost));
    if (n) *n = (int32_t)cnt;
    if (reset) {
        const uint32_t zero = 0;
        CK(cudaMemcpy(&c->P.ctl->trace_n, &zero, sizeof zero, cudaMemcpyHostToDevice));
    }
    return SPH_OK;
}

sph_status sph_launch_count(sph_ctx *c, int64_t *out)
{
    sph_status st = check_ctx(c);
    if (st != SPH_OK) return st;
    if (!out) return fail(c, SPH_EINVAL, "out is NULL");
    CK(cudaStreamSynchronize(c->stream));
    Control h;
    CK(cudaMemcpy(&h, c->P.ctl, sizeof h, cudaMemcpyDeviceToHost));
    *out = h.launches;
    return SPH_OK;
}

const char *sph_status_string(sph_status s)
{
    switch (s) {
    case SPH_OK: return "ok";
    case SPH_EINVAL: return "invalid argument";
    case SPH_ENOMEM: return "out of memory";
    case SPH_ECUDA: return "CUDA error";
    case SPH_ENOCONVERGE: return "solver did not converge";
    case SPH_ETIMEOUT: return "device wait timed out";
    case SPH_ENUMERIC: return "non-finite state";
    case SPH_EOVERFLOW: return "neighbour list overflow";
    }
    return "unknown status";
}

const char *sph_last_error(const sph_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

void sph_destroy(sph_ctx *c)
{
    if (!c) return;
    if (c->stream || true) cudaStreamSynchronize(c->stream);
    if (c->copy) {
        cudaStreamSynchronize(c->copy);
        cudaStreamDestroy(c->copy);
        for (auto e : c->staged)
            if (e) cudaEventDestroy(e);
        for (auto e : c->read_done)
            if (e) cudaEventDestroy(e);
    }
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (auto &a : c->allocs) {
        if (c->use_alloc) c->alloc.free(c->alloc.user, a.p, a.bytes, (void *)c->stream);
        else cudaFree(a.p);
    }
    if (c->h_flag) cudaFreeHost(c->h_flag);
    if (c->trace) cudaFree(c->trace);
    if (c->cap0) cudaStreamDestroy(c->cap0);
    if (c->cap1) cudaStreamDestroy(c->cap1);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    delete c;
}

}  // extern "C"
