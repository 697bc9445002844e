/*
 * dfsph_oracle.c -- plain FP64 CPU oracle of the per-step DFSPH particle pipeline.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header, table or
 * constant with the CUDA library: every formula below is restated from the paper
 * (arXiv 2403.11156, "Journey into SPH Simulation") and, where the paper is silent, from
 * the published DFSPH / Akinci / Monaghan definitions it cites, with each reading named.
 *
 * Everything is FP64 except two bit-exact contracts that are defined in FP32 on purpose:
 * the uniform-grid cell key and the neighbour predicate (both evaluated in `float` with
 * IEEE round-to-nearest and no FMA contraction; build with -ffp-contract=off).
 *
 * Fields are kept in the caller's original particle order; nothing is sorted, blocked or
 * fused.  Per-particle loops may run under OpenMP because each iteration writes only its
 * own outputs; every reduction is a plain serial loop, so results do not depend on the
 * thread count.
 *
 * Besides DFSPH the step implements the paper's EOS solver (WCSPH, Sec. 3.4.1) and
 * PCISPH (an iterative PPE solver of Alg. ppe_solver) on the same density, non-pressure
 * and pressure-acceleration building blocks.
 *
 * Pins (see tests/test_oracle_*.py): kernel normalisation and gradient antisymmetry,
 * lattice rest density, the boundary pseudo-mass of a flat wall lattice, the DFSPH factor alpha (closed-form lattice value, and the exact
 * cancellation of a lone compression next to a wall by one Jacobi update), brute-force
 * neighbour sets, momentum antisymmetry of pressure, viscosity and boundary forces,
 * hydrostatic pressure in a resting tank (weight on the walls, interior gradient within
 * 5 %), depth-independent buoyancy of a submerged body, operator symmetry of implicit
 * viscosity, MLP gradients against finite differences, and a run resumed through the
 * state setters (fluid and rigid) continuing bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------ */
/* Smoothing kernel (Sec. 3.2, Eq. density).  The paper names W and its support h = 4r    */
/* (Sec. 5) but prints no formula; the cubic spline is the reading:                       */
/*   q = |x|/h, sigma = 8/(pi h^3)                                                        */
/*   W = sigma (6q^3 - 6q^2 + 1)        for q <= 1/2                                      */
/*   W = sigma 2 (1-q)^3                for 1/2 < q <= 1, and 0 beyond.                   */
/* ------------------------------------------------------------------------------------ */
double or_W(double r, double h)
{
    double q = r / h;
    double sigma = 8.0 / (M_PI * h * h * h);
    if (q <= 0.5) return sigma * (6.0 * q * q * q - 6.0 * q * q + 1.0);
    if (q <= 1.0) {
        double t = 1.0 - q;
        return sigma * 2.0 * t * t * t;
    }
    return 0.0;
}

/* dW/dr of the spline above, times x/|x|:  grad W = (48/(pi h^3)) g(q) x / (|x| h)       */
/* with g = q(3q-2) for q <= 1/2 and g = -(1-q)^2 for 1/2 < q <= 1; zero at x = 0, q > 1. */
void or_gradW(const double *x, double h, double *out)
{
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double q = r / h;
    out[0] = out[1] = out[2] = 0.0;
    if (r <= 0.0 || q > 1.0) return;
    double g = (q <= 0.5) ? q * (3.0 * q - 2.0) : -(1.0 - q) * (1.0 - q);
    double f = 48.0 / (M_PI * h * h * h) * g / (r * h);
    out[0] = f * x[0];
    out[1] = f * x[1];
    out[2] = f * x[2];
}

/* ------------------------------------------------------------------------------------ */
/* Uniform grid contract (Sec. 5.6 names a prefix-sum grid; the layout is a reading).     */
/* All in float: origin o = dmin - c, n = ceil((dmax-dmin)/c) + 2 per axis,               */
/* i = clamp(floor((x - o)/c), 0, n-1), key = ix + nx (iy + ny iz).                       */
/* Default cell size c = h * (1 + 2^-8): a hair above h so that every pair passing the    */
/* float predicate lies in adjacent cells despite rounding.                               */
/* ------------------------------------------------------------------------------------ */
float or_default_cell_size(float radius)
{
    float h = 4.0f * radius;
    return h * 1.00390625f;
}

void or_grid_dims(const float *dmin, const float *dmax, float c, int32_t *dims, float *origin)
{
    for (int a = 0; a < 3; ++a) {
        origin[a] = dmin[a] - c;
        float ext = (dmax[a] - dmin[a]) / c;
        dims[a] = (int32_t)ceilf(ext) + 2;
    }
}

static int32_t cell_coord_f(float x, float o, float c, int32_t n)
{
    float t = (x - o) / c;
    if (!(t > 0.0f)) return 0; /* also catches NaN */
    if (t >= (float)(n - 1)) return n - 1;
    return (int32_t)floorf(t);
}

void or_cell_keys(int64_t n, const float *x, const float *dmin, const float *dmax, float c,
                  uint32_t *keys)
{
    int32_t dims[3];
    float o[3];
    or_grid_dims(dmin, dmax, c, dims, o);
    for (int64_t i = 0; i < n; ++i) {
        int32_t ix = cell_coord_f(x[3 * i + 0], o[0], c, dims[0]);
        int32_t iy = cell_coord_f(x[3 * i + 1], o[1], c, dims[1]);
        int32_t iz = cell_coord_f(x[3 * i + 2], o[2], c, dims[2]);
        keys[i] = (uint32_t)ix + (uint32_t)dims[0] * ((uint32_t)iy + (uint32_t)dims[1] * (uint32_t)iz);
    }
}

/* Sort order contract: lexicographic (cell key, original particle id). */
typedef struct { uint32_t key; int64_t id; } key_id;
static int cmp_key_id(const void *a, const void *b)
{
    const key_id *p = (const key_id *)a, *q = (const key_id *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->id != q->id) return p->id < q->id ? -1 : 1;
    return 0;
}

void or_sort_order(int64_t n, const uint32_t *keys, int64_t *ids_out)
{
    key_id *t = (key_id *)malloc(sizeof(key_id) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { t[i].key = keys[i]; t[i].id = i; }
    qsort(t, (size_t)n, sizeof(key_id), cmp_key_id);
    for (int64_t i = 0; i < n; ++i) ids_out[i] = t[i].id;
    free(t);
}

/* Neighbour predicate contract: j != i and d2 < h2 with dx = xi - xj in float and       */
/* d2 = ((dx*dx) + (dy*dy)) + (dz*dz) in float, h2 = h*h in float (strict '<').          */
static int nbr_pred(const float *a, const float *b, float h2)
{
    float dx = a[0] - b[0];
    float dy = a[1] - b[1];
    float dz = a[2] - b[2];
    float sx = dx * dx;
    float sy = dy * dy;
    float sz = dz * dz;
    float d2 = (sx + sy) + sz;
    return d2 < h2;
}

/* Brute-force O(n m) neighbour counts: for each point of x, how many points of y pass    */
/* the predicate (exclude_self: skip j == i, for x == y).                                  */
void or_neighbor_counts_brute(int64_t n, const float *x, int64_t m, const float *y, float h,
                              int exclude_self, int32_t *counts)
{
    float h2 = h * h;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = 0;
        for (int64_t j = 0; j < m; ++j) {
            if (exclude_self && i == j) continue;
            if (nbr_pred(x + 3 * i, y + 3 * j, h2)) ++c;
        }
        counts[i] = c;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Neighbour lists (CSR).  A plain cell-bucket search used only to avoid O(n^2); the      */
/* predicate above decides membership, so the sets equal brute force (pinned in tests).   */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t *start; /* [n+1] */
    int64_t *idx;   /* [start[n]] */
} csr;

static void csr_free(csr *c)
{
    free(c->start);
    free(c->idx);
    c->start = NULL;
    c->idx = NULL;
}

typedef struct {
    double o[3], c;
    int64_t n[3];
    int64_t *cell_start; /* [ncell+1] */
    int64_t *items;      /* point indices grouped by cell, ascending within a cell */
} bucket_grid;

static int64_t bucket_coord(double x, double o, double c, int64_t n)
{
    double t = (x - o) / c;
    if (!(t > 0.0)) return 0;
    if (t >= (double)(n - 1)) return n - 1;
    return (int64_t)floor(t);
}

static void bucket_build(bucket_grid *g, const double *lo, const double *hi, double c,
                         int64_t np, const float *pts)
{
    g->c = c;
    for (int a = 0; a < 3; ++a) {
        g->o[a] = lo[a] - c;
        g->n[a] = (int64_t)ceil((hi[a] - lo[a]) / c) + 2;
    }
    int64_t nc = g->n[0] * g->n[1] * g->n[2];
    g->cell_start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    g->items = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    for (int64_t i = 0; i < np; ++i) {
        int64_t ix = bucket_coord(pts[3 * i + 0], g->o[0], c, g->n[0]);
        int64_t iy = bucket_coord(pts[3 * i + 1], g->o[1], c, g->n[1]);
        int64_t iz = bucket_coord(pts[3 * i + 2], g->o[2], c, g->n[2]);
        cell_of[i] = ix + g->n[0] * (iy + g->n[1] * iz);
        g->cell_start[cell_of[i] + 1] += 1;
    }
    for (int64_t k = 0; k < nc; ++k) g->cell_start[k + 1] += g->cell_start[k];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    memcpy(fill, g->cell_start, sizeof(int64_t) * (size_t)nc);
    for (int64_t i = 0; i < np; ++i) g->items[fill[cell_of[i]]++] = i;
    free(fill);
    free(cell_of);
}

static void bucket_free(bucket_grid *g)
{
    free(g->cell_start);
    free(g->items);
}

/* Lists of y-points within h of each x-point (predicate in float). */
static void build_lists(csr *out, int64_t nx, const float *xs, const bucket_grid *g,
                        const float *ys, float h, int exclude_self)
{
    float h2 = h * h;
    out->start = (int64_t *)calloc((size_t)nx + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < nx; ++i) {
            const float *p = xs + 3 * i;
            int64_t cx = bucket_coord(p[0], g->o[0], g->c, g->n[0]);
            int64_t cy = bucket_coord(p[1], g->o[1], g->c, g->n[1]);
            int64_t cz = bucket_coord(p[2], g->o[2], g->c, g->n[2]);
            int64_t cnt = 0;
            int64_t w = pass ? out->start[i] : 0;
            for (int64_t dz = -1; dz <= 1; ++dz)
                for (int64_t dy = -1; dy <= 1; ++dy)
                    for (int64_t dx = -1; dx <= 1; ++dx) {
                        int64_t ax = cx + dx, ay = cy + dy, az = cz + dz;
                        if (ax < 0 || ay < 0 || az < 0 || ax >= g->n[0] || ay >= g->n[1] || az >= g->n[2])
                            continue;
                        int64_t k = ax + g->n[0] * (ay + g->n[1] * az);
                        for (int64_t t = g->cell_start[k]; t < g->cell_start[k + 1]; ++t) {
                            int64_t j = g->items[t];
                            if (exclude_self && j == i) continue;
                            if (!nbr_pred(p, ys + 3 * j, h2)) continue;
                            if (pass) out->idx[w++] = j;
                            else ++cnt;
                        }
                    }
            if (!pass) out->start[i + 1] = cnt;
        }
        if (!pass) {
            for (int64_t i = 0; i < nx; ++i) out->start[i + 1] += out->start[i];
            out->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(out->start[nx] > 0 ? out->start[nx] : 1));
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Learned warm start network (not in the paper): y = W3 gelu(W2 gelu(W1 f + b1) + b2)+b3 */
/* with exact-erf GELU.  Layout: W1 [64][4], b1[64], W2[64][64], b2[64], W3[64], b3[1],   */
/* then feature mean[4], feature std[4], label mean, label std (total OR_MLP_NPARAM).     */
/* ------------------------------------------------------------------------------------ */
#define OR_H 64
#define OR_F 4
#define OR_MLP_NW (OR_H * OR_F + OR_H + OR_H * OR_H + OR_H + OR_H + 1)
#define OR_MLP_NPARAM (OR_MLP_NW + 2 * OR_F + 2)

int64_t or_mlp_nparam(void) { return OR_MLP_NPARAM; }
int64_t or_mlp_nweights(void) { return OR_MLP_NW; }

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_d(double x)
{
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

/* Forward on already-standardised features f[n][4] -> standardised output y[n]. */
void or_mlp_forward(const double *w, int64_t n, const double *f, double *y)
{
    const double *W1 = w, *b1 = W1 + OR_H * OR_F, *W2 = b1 + OR_H, *b2 = W2 + OR_H * OR_H;
    const double *W3 = b2 + OR_H, *b3 = W3 + OR_H;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        double a1[OR_H], a2[OR_H];
        for (int o = 0; o < OR_H; ++o) {
            double z = b1[o];
            for (int k = 0; k < OR_F; ++k) z += W1[o * OR_F + k] * f[s * OR_F + k];
            a1[o] = gelu(z);
        }
        for (int o = 0; o < OR_H; ++o) {
            double z = b2[o];
            for (int k = 0; k < OR_H; ++k) z += W2[o * OR_H + k] * a1[k];
            a2[o] = gelu(z);
        }
        double z = b3[0];
        for (int k = 0; k < OR_H; ++k) z += W3[k] * a2[k];
        y[s] = z;
    }
}

/* Mean-squared-error loss L = (1/n) sum (y - t)^2 and its gradient w.r.t. the weights   */
/* (the first OR_MLP_NW entries of the parameter block).  Returns L.                     */
double or_mlp_loss_grad(const double *w, int64_t n, const double *f, const double *t, double *grad)
{
    const double *W1 = w, *b1 = W1 + OR_H * OR_F, *W2 = b1 + OR_H, *b2 = W2 + OR_H * OR_H;
    const double *W3 = b2 + OR_H, *b3 = W3 + OR_H;
    memset(grad, 0, sizeof(double) * OR_MLP_NW);
    double *gW1 = grad, *gb1 = gW1 + OR_H * OR_F, *gW2 = gb1 + OR_H, *gb2 = gW2 + OR_H * OR_H;
    double *gW3 = gb2 + OR_H, *gb3 = gW3 + OR_H;
    double loss = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        double z1[OR_H], a1[OR_H], z2[OR_H], a2[OR_H], d2[OR_H], d1[OR_H];
        const double *fs = f + s * OR_F;
        for (int o = 0; o < OR_H; ++o) {
            double z = b1[o];
            for (int k = 0; k < OR_F; ++k) z += W1[o * OR_F + k] * fs[k];
            z1[o] = z;
            a1[o] = gelu(z);
        }
        for (int o = 0; o < OR_H; ++o) {
            double z = b2[o];
            for (int k = 0; k < OR_H; ++k) z += W2[o * OR_H + k] * a1[k];
            z2[o] = z;
            a2[o] = gelu(z);
        }
        double y = b3[0];
        for (int k = 0; k < OR_H; ++k) y += W3[k] * a2[k];
        double e = y - t[s];
        loss += e * e;
        double dy = 2.0 * e / (double)n;
        gb3[0] += dy;
        for (int k = 0; k < OR_H; ++k) {
            gW3[k] += dy * a2[k];
            d2[k] = dy * W3[k] * gelu_d(z2[k]);
        }
        for (int o = 0; o < OR_H; ++o) {
            gb2[o] += d2[o];
            for (int k = 0; k < OR_H; ++k) gW2[o * OR_H + k] += d2[o] * a1[k];
        }
        for (int k = 0; k < OR_H; ++k) {
            double acc = 0.0;
            for (int o = 0; o < OR_H; ++o) acc += W2[o * OR_H + k] * d2[o];
            d1[k] = acc * gelu_d(z1[k]);
        }
        for (int o = 0; o < OR_H; ++o) {
            gb1[o] += d1[o];
            for (int k = 0; k < OR_F; ++k) gW1[o * OR_F + k] += d1[o] * fs[k];
        }
    }
    return loss / (double)(n > 0 ? n : 1);
}

/* One Adam step (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,             */
/* w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps), t counted from 1.              */
void or_adam_step(double *w, double *m, double *v, const double *g, int64_t n, int64_t t,
                  double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t k = 0; k < n; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        w[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Scene state and the DFSPH step.                                                        */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double radius, rest_density, viscosity;
    double gravity[3];
    double eta_density, eta_divergence, dt_max, cfl;
    int32_t min_iter_density, max_iter_density, min_iter_divergence, max_iter_divergence;
    int32_t viscosity_mode; /* 0 none, 1 explicit Laplacian (Eq. lap), 2 XSPH, 3 implicit CG */
    int32_t warm_start;     /* 0 zero, 1 previous-step kappa, 2 learned network */
    int32_t divergence_solve;
    float domain_min[3], domain_max[3];
    double xsph_c, cg_tol;
    int32_t cg_max_iter, pad_;
    int32_t pressure_solver; /* 0 DFSPH, 1 WCSPH (equation of state, Sec. 3.4.1), 2 PCISPH  */
    int32_t pad2_;
    double eos_stiffness, eos_exponent;
    double warm_start_fraction; /* fraction of the previous stiffness (0 = one half)       */
    int32_t rigid_coupling;     /* 0 weak (body velocities fixed during the solves), 1 strong */
    int32_t pad3_;
    double learned_fraction;    /* fraction of the network's stiffness applied (0 = 0.6)   */
} or_params;

typedef struct {
    double mass, inertia[3], com[3], quat[4], vel[3], omega[3];
} or_body;

enum {
    OR_X = 0, OR_V, OR_RHO, OR_ALPHA, OR_KAPPA, OR_KAPPA_V, OR_PRESSURE, OR_NN_F, OR_NN_B,
    OR_V_DIV, OR_V_NONP, OR_PSI, OR_XB, OR_VB, OR_KAPPA0, OR_FEAT, OR_DIV_ERR_I, OR_DENS_ERR_I,
    OR_FLUID_BOUNDARY_IMPULSE, OR_NFIELDS
};

typedef struct {
    or_params p;
    double h, m, cell;
    int64_t nf, nb;
    int32_t nbody;
    double *x, *v, *rho, *alpha, *kappa, *kappa_v, *kappa_prev, *kappa_v_prev, *pressure;
    double *v_div, *v_nonp, *kappa0, *feat, *e_div, *e_dens, *fb_impulse;
    int32_t *nn_f, *nn_b;
    double *xb, *vb, *psi, *r0;
    int32_t *body;
    or_body *bodies;
    double *body_force; /* [nbody][6]: force, torque from fluid in the last step */
    double *mlp;
    int have_mlp;
    csr ff, fb;
    double dt_next;
    double stats[16];
} or_ctx;

/* stats layout */
enum {
    ST_DIV_ITERS = 0, ST_DENS_ITERS, ST_DIV_ERR, ST_DENS_ERR, ST_DT, ST_DT_NEXT, ST_MAXV,
    ST_CLAMPS, ST_CG_ITERS, ST_CG_RES, ST_DIV_ERR0, ST_DENS_ERR0, ST_STEPS
};

static void quat_to_R(const double *q, double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static double *dalloc(int64_t n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static double max_speed(const or_ctx *c)
{
    double mx = 0.0;
    for (int64_t i = 0; i < c->nf; ++i) {
        double s = sqrt(c->v[3 * i] * c->v[3 * i] + c->v[3 * i + 1] * c->v[3 * i + 1] + c->v[3 * i + 2] * c->v[3 * i + 2]);
        if (s > mx) mx = s;
    }
    return mx;
}

/* CFL reading (not in the paper): dt = min(dt_max, cfl * 2r / max|v|). */
static double cfl_dt(const or_ctx *c)
{
    double vm = max_speed(c);
    double dt = c->p.dt_max;
    if (c->p.cfl > 0.0 && vm > 0.0) {
        double d = c->p.cfl * 2.0 * c->p.radius / vm;
        if (d < dt) dt = d;
    }
    return dt;
}

static void set_boundary_from_bodies(or_ctx *c)
{
    for (int32_t k = 0; k < c->nbody; ++k) {
        or_body *B = &c->bodies[k];
        double R[3][3];
        quat_to_R(B->quat, R);
        for (int64_t b = 0; b < c->nb; ++b) {
            if (c->body[b] != k) continue;
            const double *r0 = c->r0 + 3 * b;
            double rw[3];
            for (int a = 0; a < 3; ++a) rw[a] = R[a][0] * r0[0] + R[a][1] * r0[1] + R[a][2] * r0[2];
            for (int a = 0; a < 3; ++a) c->xb[3 * b + a] = B->com[a] + rw[a];
            c->vb[3 * b + 0] = B->vel[0] + (B->omega[1] * rw[2] - B->omega[2] * rw[1]);
            c->vb[3 * b + 1] = B->vel[1] + (B->omega[2] * rw[0] - B->omega[0] * rw[2]);
            c->vb[3 * b + 2] = B->vel[2] + (B->omega[0] * rw[1] - B->omega[1] * rw[0]);
        }
    }
}

or_ctx *or_create(const or_params *p, int64_t nf, const float *xf, const float *vf, int64_t nb,
                  const float *xb, const int32_t *body, int32_t nbody, const double *bodies)
{
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->p = *p;
    /* h = 4r (Sec. 5); particle mass m = rho0 (2r)^3 (a reading: the lattice volume). */
    c->h = 4.0 * p->radius;
    c->m = p->rest_density * 8.0 * p->radius * p->radius * p->radius;
    c->cell = (double)or_default_cell_size((float)p->radius);
    c->nf = nf;
    c->nb = nb;
    c->nbody = nbody;
    c->x = dalloc(3 * nf); c->v = dalloc(3 * nf);
    c->rho = dalloc(nf); c->alpha = dalloc(nf); c->kappa = dalloc(nf); c->kappa_v = dalloc(nf);
    c->kappa_prev = dalloc(nf); c->kappa_v_prev = dalloc(nf); c->pressure = dalloc(nf);
    c->v_div = dalloc(3 * nf); c->v_nonp = dalloc(3 * nf); c->kappa0 = dalloc(nf);
    c->feat = dalloc(4 * nf); c->e_div = dalloc(nf); c->e_dens = dalloc(nf);
    c->fb_impulse = dalloc(3 * nf);
    c->nn_f = (int32_t *)calloc((size_t)(nf > 0 ? nf : 1), sizeof(int32_t));
    c->nn_b = (int32_t *)calloc((size_t)(nf > 0 ? nf : 1), sizeof(int32_t));
    c->xb = dalloc(3 * nb); c->vb = dalloc(3 * nb); c->psi = dalloc(nb); c->r0 = dalloc(3 * nb);
    c->body = (int32_t *)calloc((size_t)(nb > 0 ? nb : 1), sizeof(int32_t));
    c->bodies = (or_body *)calloc((size_t)(nbody > 0 ? nbody : 1), sizeof(or_body));
    c->body_force = dalloc(6 * (nbody > 0 ? nbody : 1));
    c->mlp = dalloc(OR_MLP_NPARAM);
    for (int64_t i = 0; i < 3 * nf; ++i) { c->x[i] = xf[i]; c->v[i] = vf ? vf[i] : 0.0; }
    for (int64_t i = 0; i < 3 * nb; ++i) c->xb[i] = xb[i];
    for (int64_t b = 0; b < nb; ++b) c->body[b] = body ? body[b] : -1;
    for (int32_t k = 0; k < nbody; ++k) {
        const double *d = bodies + 19 * k; /* mass, inertia[3], com[3], quat[4], vel[3], omega[3], pad[2] */
        or_body *B = &c->bodies[k];
        B->mass = d[0];
        for (int a = 0; a < 3; ++a) { B->inertia[a] = d[1 + a]; B->com[a] = d[4 + a]; B->vel[a] = d[11 + a]; B->omega[a] = d[14 + a]; }
        for (int a = 0; a < 4; ++a) B->quat[a] = d[7 + a];
        double R[3][3];
        quat_to_R(B->quat, R);
        /* body-frame offsets r0 = R^T (x - com) */
        for (int64_t b = 0; b < nb; ++b) {
            if (c->body[b] != k) continue;
            double d3[3] = {c->xb[3 * b] - B->com[0], c->xb[3 * b + 1] - B->com[1], c->xb[3 * b + 2] - B->com[2]};
            for (int a = 0; a < 3; ++a) c->r0[3 * b + a] = R[0][a] * d3[0] + R[1][a] * d3[1] + R[2][a] * d3[2];
        }
    }
    if (nbody > 0) set_boundary_from_bodies(c);
    c->dt_next = cfl_dt(c);
    return c;
}

void or_destroy(or_ctx *c)
{
    if (!c) return;
    double **ptrs[] = {&c->x, &c->v, &c->rho, &c->alpha, &c->kappa, &c->kappa_v, &c->kappa_prev,
                       &c->kappa_v_prev, &c->pressure, &c->v_div, &c->v_nonp, &c->kappa0, &c->feat,
                       &c->e_div, &c->e_dens, &c->fb_impulse, &c->xb, &c->vb, &c->psi, &c->r0,
                       &c->body_force, &c->mlp};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(*ptrs[k]);
    free(c->nn_f); free(c->nn_b); free(c->body); free(c->bodies);
    csr_free(&c->ff); csr_free(&c->fb);
    free(c);
}

void or_set_mlp(or_ctx *c, const double *params)
{
    memcpy(c->mlp, params, sizeof(double) * OR_MLP_NPARAM);
    c->have_mlp = 1;
}

/* Overwrite the dynamic state (checkpoint restore); NULL leaves a field as is. */
void or_set_state(or_ctx *c, const double *x, const double *v, const double *kappa_prev,
                  const double *kappa_v_prev)
{
    if (x) memcpy(c->x, x, sizeof(double) * 3 * c->nf);
    if (v) memcpy(c->v, v, sizeof(double) * 3 * c->nf);
    if (kappa_prev) memcpy(c->kappa_prev, kappa_prev, sizeof(double) * c->nf);
    if (kappa_v_prev) memcpy(c->kappa_v_prev, kappa_v_prev, sizeof(double) * c->nf);
    c->dt_next = cfl_dt(c);
}

/* Boundary pseudo-mass (Sec. 3.5): Psi_b = rho0 / sum_k W_bk over boundary particles k    */
/* within h, the particle itself included (reading: walls and all bodies count).          */
static void compute_psi(or_ctx *c, const float *xbf, const bucket_grid *gb)
{
    float h = (float)c->h;
    float h2 = h * h;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t b = 0; b < c->nb; ++b) {
        const float *p = xbf + 3 * b;
        int64_t cx = bucket_coord(p[0], gb->o[0], gb->c, gb->n[0]);
        int64_t cy = bucket_coord(p[1], gb->o[1], gb->c, gb->n[1]);
        int64_t cz = bucket_coord(p[2], gb->o[2], gb->c, gb->n[2]);
        double s = or_W(0.0, c->h);
        for (int64_t dz = -1; dz <= 1; ++dz)
            for (int64_t dy = -1; dy <= 1; ++dy)
                for (int64_t dx = -1; dx <= 1; ++dx) {
                    int64_t ax = cx + dx, ay = cy + dy, az = cz + dz;
                    if (ax < 0 || ay < 0 || az < 0 || ax >= gb->n[0] || ay >= gb->n[1] || az >= gb->n[2]) continue;
                    int64_t k = ax + gb->n[0] * (ay + gb->n[1] * az);
                    for (int64_t t = gb->cell_start[k]; t < gb->cell_start[k + 1]; ++t) {
                        int64_t j = gb->items[t];
                        if (j == b || !nbr_pred(p, xbf + 3 * j, h2)) continue;
                        double d[3] = {c->xb[3 * b] - c->xb[3 * j], c->xb[3 * b + 1] - c->xb[3 * j + 1], c->xb[3 * b + 2] - c->xb[3 * j + 2]};
                        s += or_W(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), c->h);
                    }
                }
        c->psi[b] = c->p.rest_density / s;
    }
}

static void diffx(const or_ctx *c, int64_t i, int64_t j, double *d)
{
    for (int a = 0; a < 3; ++a) d[a] = c->x[3 * i + a] - c->x[3 * j + a];
}
static void diffxb(const or_ctx *c, int64_t i, int64_t b, double *d)
{
    for (int a = 0; a < 3; ++a) d[a] = c->x[3 * i + a] - c->xb[3 * b + a];
}

/* Density (Sec. 3.2 Eq. density with the boundary term of Sec. 3.5) and the DFSPH factor */
/* alpha_i = rho_i / (|sum_j m grad W_ij + sum_b Psi_b grad W_ib|^2 + sum_j |m grad W_ij|^2) */
/* (DFSPH, cited by the paper; boundary in the first sum only, a reading).  alpha = 0 when */
/* the denominator is below 1e-6 (m * 48/(pi h^4))^2.                                     */
static void density_alpha(or_ctx *c)
{
    double h = c->h, m = c->m;
    double gs = m * 48.0 / (M_PI * h * h * h * h);
    double eps = 1e-6 * gs * gs;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->nf; ++i) {
        double rho = m * or_W(0.0, h);
        double s1[3] = {0, 0, 0}, s2 = 0.0;
        for (int64_t t = c->ff.start[i]; t < c->ff.start[i + 1]; ++t) {
            int64_t j = c->ff.idx[t];
            double d[3], g[3];
            diffx(c, i, j, d);
            rho += m * or_W(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), h);
            or_gradW(d, h, g);
            for (int a = 0; a < 3; ++a) s1[a] += m * g[a];
            s2 += m * m * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        }
        for (int64_t t = c->fb.start[i]; t < c->fb.start[i + 1]; ++t) {
            int64_t b = c->fb.idx[t];
            double d[3], g[3];
            diffxb(c, i, b, d);
            rho += c->psi[b] * or_W(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), h);
            or_gradW(d, h, g);
            for (int a = 0; a < 3; ++a) s1[a] += c->psi[b] * g[a];
        }
        double den = s1[0] * s1[0] + s1[1] * s1[1] + s1[2] * s1[2] + s2;
        c->rho[i] = rho;
        c->alpha[i] = (den > eps) ? rho / den : 0.0;
        c->nn_f[i] = (int32_t)(c->ff.start[i + 1] - c->ff.start[i]);
        c->nn_b[i] = (int32_t)(c->fb.start[i + 1] - c->fb.start[i]);
    }
}

/* SPH rate of density change (Sec. 3.2 divergence, continuity Eq. 1 in mass form):       */
/* D rho_i/Dt = sum_j m (v_i - v_j).grad W_ij + sum_b Psi_b (v_i - v_b).grad W_ib.        */
static double drho_dt(const or_ctx *c, int64_t i)
{
    double s = 0.0;
    for (int64_t t = c->ff.start[i]; t < c->ff.start[i + 1]; ++t) {
        int64_t j = c->ff.idx[t];
        double d[3], g[3];
        diffx(c, i, j, d);
        or_gradW(d, c->h, g);
        for (int a = 0; a < 3; ++a) s += c->m * (c->v[3 * i + a] - c->v[3 * j + a]) * g[a];
    }
    for (int64_t t = c->fb.start[i]; t < c->fb.start[i + 1]; ++t) {
        int64_t b = c->fb.idx[t];
        double d[3], g[3];
        diffxb(c, i, b, d);
        or_gradW(d, c->h, g);
        for (int a = 0; a < 3; ++a) s += c->psi[b] * (c->v[3 * i + a] - c->vb[3 * b + a]) * g[a];
    }
    return s;
}

/* Pressure acceleration (Sec. 3.3 Eq. pressure_acceleration with p/rho^2 = kappa/rho) and */
/* the boundary term of Sec. 3.5 Eq. rigid_pressure divided by m_f:                       */
/* v_i -= dt [ sum_j m (k_i/rho_i + k_j/rho_j) grad W_ij + sum_b Psi_b (k_i/rho_i) grad W_ib ] */
/* Jacobi: every particle reads the kappas of this sweep, velocities are written after.   */
static void apply_kappa(or_ctx *c, const double *k, double dt)
{
    double *dv = dalloc(3 * c->nf);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->nf; ++i) {
        double ki = k[i] / c->rho[i];
        double acc[3] = {0, 0, 0};
        for (int64_t t = c->ff.start[i]; t < c->ff.start[i + 1]; ++t) {
            int64_t j = c->ff.idx[t];
            double d[3], g[3];
            diffx(c, i, j, d);
            or_gradW(d, c->h, g);
            double f = c->m * (ki + k[j] / c->rho[j]);
            for (int a = 0; a < 3; ++a) acc[a] += f * g[a];
        }
        for (int64_t t = c->fb.start[i]; t < c->fb.start[i + 1]; ++t) {
            int64_t b = c->fb.idx[t];
            double d[3], g[3];
            diffxb(c, i, b, d);
            or_gradW(d, c->h, g);
            for (int a = 0; a < 3; ++a) acc[a] += c->psi[b] * ki * g[a];
        }
        for (int a = 0; a < 3; ++a) dv[3 * i + a] = -dt * acc[a];
    }
    for (int64_t i = 0; i < 3 * c->nf; ++i) c->v[i] += dv[i];
    free(dv);
}

/* Implicit viscosity operator (Sec. 3.6.2): (A v)_i = sum_j A_ij (v_j - v_i) with        */
/* A_ij = -2(d+2) mu mbar_ij/(rho_i rho_j) grad W_ij x_ij^T / (|x_ij|^2 + 0.01 h^2),       */
/* d = 3, mbar = m (uniform mass).  The denominator takes |x_ij|^2 as in Eq. lap (the     */
/* printed |x_ij| is read as a typo).  out = (I - dt A) v.                                */
static void visc_apply(const or_ctx *c, double mu, double dt, const double *v, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->nf; ++i) {
        double acc[3] = {0, 0, 0};
        for (int64_t t = c->ff.start[i]; t < c->ff.start[i + 1]; ++t) {
            int64_t j = c->ff.idx[t];
            double d[3], g[3];
            diffx(c, i, j, d);
            or_gradW(d, c->h, g);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double s = -10.0 * mu * c->m / (c->rho[i] * c->rho[j]) / (r2 + 0.01 * c->h * c->h);
            double xv = 0.0;
            for (int a = 0; a < 3; ++a) xv += d[a] * (v[3 * j + a] - v[3 * i + a]);
            for (int a = 0; a < 3; ++a) acc[a] += s * g[a] * xv; /* (grad W x^T)(v_j - v_i) */
        }
        for (int a = 0; a < 3; ++a) out[3 * i + a] = v[3 * i + a] - dt * acc[a];
    }
}

/* Exposed for the symmetry pin: out = (I - dt A) v on the current neighbour lists. */
void or_visc_operator(or_ctx *c, double dt, const double *v, double *out)
{
    visc_apply(c, c->p.viscosity * c->p.rest_density, dt, v, out);
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* Matrix-free conjugate gradient (Sec. 3.6.2, Sec. 4.2) on (I - dt A) v* = vtilde,       */
/* started from vtilde, stopped at |r| <= tol |b| or cg_max_iter.                          */
static void visc_cg(or_ctx *c, double dt)
{
    int64_t n = 3 * c->nf;
    double mu = c->p.viscosity * c->p.rest_density;
    double *b = dalloc(n), *r = dalloc(n), *p = dalloc(n), *Ap = dalloc(n);
    memcpy(b, c->v, sizeof(double) * n);
    visc_apply(c, mu, dt, c->v, Ap);
    for (int64_t k = 0; k < n; ++k) { r[k] = b[k] - Ap[k]; p[k] = r[k]; }
    double rr = dot(n, r, r), bb = dot(n, b, b);
    int it = 0;
    double tol2 = c->p.cg_tol * c->p.cg_tol * bb;
    while (rr > tol2 && it < c->p.cg_max_iter) {
        visc_apply(c, mu, dt, p, Ap);
        double pAp = dot(n, p, Ap);
        if (!(pAp > 0.0)) break;
        double a = rr / pAp;
        for (int64_t k = 0; k < n; ++k) { c->v[k] += a * p[k]; r[k] -= a * Ap[k]; }
        double rr2 = dot(n, r, r);
        double beta = rr2 / rr;
        for (int64_t k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        rr = rr2;
        ++it;
    }
    c->stats[ST_CG_ITERS] = it;
    c->stats[ST_CG_RES] = bb > 0 ? sqrt(rr / bb) : 0.0;
    free(b); free(r); free(p); free(Ap);
}

/* Non-pressure forces (Sec. 3.3 Alg. general_algorithm, Sec. 4.2 order: gravity then     */
/* viscosity): v* = v + dt (g + (mu/rho_i) lap v_i) with the explicit Laplacian of Eq. lap */
/* lap v_i = 2(d+2) sum_j (m/rho_j) (v_ij.x_ij)/(|x_ij|^2 + 0.01 h^2) grad W_ij, d = 3,   */
/* and mu = nu rho0 (the scene's viscosity is kinematic at rest density; mu/rho as in the  */
/* Navier-Stokes equation of Sec. 3.1 and in Sec. 3.6.2); XSPH instead adds               */
/* c sum_j (m/rho_j)(v_j - v_i) W_ij; the implicit mode solves Sec. 3.6.2.                */
static void non_pressure(or_ctx *c, double dt)
{
    double *vn = dalloc(3 * c->nf);
    int mode = c->p.viscosity_mode;
    double mu = c->p.viscosity * c->p.rest_density, h = c->h;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->nf; ++i) {
        double acc[3] = {c->p.gravity[0], c->p.gravity[1], c->p.gravity[2]};
        double xs[3] = {0, 0, 0};
        if (mode == 1 || mode == 2) {
            for (int64_t t = c->ff.start[i]; t < c->ff.start[i + 1]; ++t) {
                int64_t j = c->ff.idx[t];
                double d[3], vij[3];
                diffx(c, i, j, d);
                for (int a = 0; a < 3; ++a) vij[a] = c->v[3 * i + a] - c->v[3 * j + a];
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (mode == 1) {
                    double g[3];
                    or_gradW(d, h, g);
                    double s = 10.0 * mu / c->rho[i] * (c->m / c->rho[j]) * (vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2]) / (r2 + 0.01 * h * h);
                    for (int a = 0; a < 3; ++a) acc[a] += s * g[a];
                } else {
                    double w = (c->m / c->rho[j]) * or_W(sqrt(r2), h);
                    for (int a = 0; a < 3; ++a) xs[a] -= w * vij[a];
                }
            }
        }
        for (int a = 0; a < 3; ++a) vn[3 * i + a] = c->v[3 * i + a] + dt * acc[a] + c->p.xsph_c * xs[a];
    }
    memcpy(c->v, vn, sizeof(double) * 3 * c->nf);
    free(vn);
    if (mode == 3) visc_cg(c, dt);
}

/* Learned warm start features (a reading; the paper has no learned component):           */
/* f = (rho/rho0 - 1, dt Drho/Dt(v*)/rho0, (n_f + n_b)/33, kappa_prev/(9.81 h)) with the  */
/* previous total stiffness rescaled to this step (stored as kappa dt^2).                 */
static void warm_features(or_ctx *c, double dt)
{
    double kref = 9.81 * c->h;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->nf; ++i) {
        c->feat[4 * i + 0] = c->rho[i] / c->p.rest_density - 1.0;
        c->feat[4 * i + 1] = dt * drho_dt(c, i) / c->p.rest_density;
        c->feat[4 * i + 2] = (double)(c->nn_f[i] + c->nn_b[i]) / 33.0;
        c->feat[4 * i + 3] = c->kappa_prev[i] / (dt * dt) / kref;
    }
}

/* Steps 1-3 of a time step: neighbour lists, boundary pseudo-masses, density and alpha. */
static void prepare(or_ctx *c)
{
    int64_t nf = c->nf, nb = c->nb;
    float h = (float)c->h;
    /* 1. neighbourhoods (predicate in float on the float-rounded positions) */
    float *xf = (float *)malloc(sizeof(float) * (size_t)(3 * nf > 0 ? 3 * nf : 1));
    float *xbf = (float *)malloc(sizeof(float) * (size_t)(3 * nb > 0 ? 3 * nb : 1));
    for (int64_t k = 0; k < 3 * nf; ++k) xf[k] = (float)c->x[k];
    for (int64_t k = 0; k < 3 * nb; ++k) xbf[k] = (float)c->xb[k];
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = c->p.domain_min[a]; hi[a] = c->p.domain_max[a]; }
    double bc = c->h * 1.001;
    bucket_grid gf, gb;
    bucket_build(&gf, lo, hi, bc, nf, xf);
    bucket_build(&gb, lo, hi, bc, nb, xbf);
    csr_free(&c->ff);
    csr_free(&c->fb);
    build_lists(&c->ff, nf, xf, &gf, xf, h, 1);
    build_lists(&c->fb, nf, xf, &gb, xbf, h, 0);

    /* 2. boundary pseudo-masses */
    compute_psi(c, xbf, &gb);
    bucket_free(&gf);
    bucket_free(&gb);
    free(xf);
    free(xbf);

    /* 3. density and alpha */
    density_alpha(c);
}

void or_prepare(or_ctx *c) { prepare(c); }

/* Solve (I - dt A) x = b by the matrix-free CG above on the current lists; x starts at b. */
int32_t or_visc_solve(or_ctx *c, double dt, const double *b, double *x)
{
    double *save = c->v;
    c->v = x;
    memcpy(x, b, sizeof(double) * 3 * c->nf);
    visc_cg(c, dt);
    c->v = save;
    return (int32_t)c->stats[ST_CG_ITERS];
}

/* Strong rigid-fluid coupling (the paper's stated future work, Sec. 6, after its cited  */
/* interlinked solver; a reading): every pressure application of the solves also pushes  */
/* the bodies.  With the applied stiffness k (p/rho^2 = k/rho), the reaction of Eq.       */
/* rigid_pressure_symmetric on boundary particle b is m Psi_b (k_i/rho_i) grad W_ib; its */
/* sum over a body's particles changes the body's velocity by dt F / M and its angular    */
/* velocity by dt I^-1 tau (world inertia of the step's orientation), and the boundary   */
/* particle velocities follow before the next source term.  The sums are accumulated in  */
/* body_force for output; the step's rigid integration then adds only gravity and the     */
/* gyroscopic term.                                                                        */
static void strong_impulse(or_ctx *c, const double *k, double dt)
{
    if (c->p.rigid_coupling != 1 || c->nbody == 0) return;
    double *F = dalloc(6 * (size_t)c->nbody);
    for (int64_t i = 0; i < c->nf; ++i) {
        double kt = k[i] / c->rho[i];
        for (int64_t t = c->fb.start[i]; t < c->fb.start[i + 1]; ++t) {
            int64_t b = c->fb.idx[t];
            int32_t kb = c->body[b];
            if (kb < 0) continue;
            double d[3], g[3], f[3];
            diffxb(c, i, b, d);
            or_gradW(d, c->h, g);
            for (int a = 0; a < 3; ++a) f[a] = c->m * c->psi[b] * kt * g[a];
            const or_body *B = &c->bodies[kb];
            double r[3] = {c->xb[3 * b] - B->com[0], c->xb[3 * b + 1] - B->com[1], c->xb[3 * b + 2] - B->com[2]};
            double *fb = F + 6 * kb;
            for (int a = 0; a < 3; ++a) fb[a] += f[a];
            fb[3] += r[1] * f[2] - r[2] * f[1];
            fb[4] += r[2] * f[0] - r[0] * f[2];
            fb[5] += r[0] * f[1] - r[1] * f[0];
        }
    }
    for (int32_t kb = 0; kb < c->nbody; ++kb) {
        or_body *B = &c->bodies[kb];
        double *fb = F + 6 * kb, R[3][3], Iinv[3][3];
        quat_to_R(B->quat, R);
        for (int a = 0; a < 3; ++a)
            for (int e = 0; e < 3; ++e) {
                Iinv[a][e] = 0.0;
                for (int q = 0; q < 3; ++q) Iinv[a][e] += R[a][q] / B->inertia[q] * R[e][q];
            }
        for (int a = 0; a < 3; ++a) B->vel[a] += dt * fb[a] / B->mass;
        for (int a = 0; a < 3; ++a) B->omega[a] += dt * (Iinv[a][0] * fb[3] + Iinv[a][1] * fb[4] + Iinv[a][2] * fb[5]);
        for (int a = 0; a < 6; ++a) c->body_force[6 * kb + a] += fb[a];
    }
    free(F);
    set_boundary_from_bodies(c);
}

/* PCISPH stiffness of a prototype particle (the PCISPH reading of Alg. ppe_solver; the   */
/* paper cites the method without restating it): with a full neighbourhood on the lattice */
/* of spacing 2r, delta = 1 / (beta (|sum_j grad W_ij|^2 + sum_j |grad W_ij|^2)), beta =   */
/* 2 (dt m / rho0)^2.  Returned without the 1/dt^2 factor.                                */
double or_pcisph_factor(const or_ctx *c)
{
    double s = 2.0 * c->p.radius, gs[3] = {0, 0, 0}, g2 = 0.0;
    int n = (int)ceil(c->h / s) + 1;
    for (int a = -n; a <= n; ++a)
        for (int b = -n; b <= n; ++b)
            for (int e = -n; e <= n; ++e) {
                double d[3] = {a * s, b * s, e * s}, g[3];
                or_gradW(d, c->h, g);
                for (int k = 0; k < 3; ++k) gs[k] += g[k];
                g2 += g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            }
    double mr = c->m / c->p.rest_density;
    return 1.0 / (2.0 * mr * mr * (gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2] + g2));
}

void or_step(or_ctx *c, double dt_in)
{
    double dt = dt_in > 0.0 ? dt_in : c->dt_next;
    double rho0 = c->p.rest_density;
    /* warm starts take this fraction of the previous step's stiffness (a reading; 1/2 by
     * default) */
    double wf = c->p.warm_start_fraction > 0.0 ? c->p.warm_start_fraction : 0.5;
    int64_t nf = c->nf, nb = c->nb;
    c->stats[ST_DT] = dt;

    prepare(c);

    int strong = c->p.rigid_coupling == 1;
    for (int64_t k6 = 0; k6 < 6 * c->nbody; ++k6) c->body_force[k6] = 0.0;

    /* 4. divergence-free solve (Eq. velocity_source, Alg. ppe_solver, Jacobi updates) */
    for (int64_t i = 0; i < nf; ++i) c->kappa_v[i] = 0.0;
    int div_it = 0;
    double div_err = 0.0;
    if (c->p.divergence_solve && c->p.pressure_solver == 0) {   /* DFSPH only */
        double *kv = dalloc(nf);
        if (c->p.warm_start != 0) {
            /* warm start (DFSPH practice, a reading): half the previous step's total      */
            /* divergence stiffness, stored as kappa_v dt, only where the fluid currently  */
            /* compresses (D rho/Dt > 0); elsewhere zero.                                   */
            for (int64_t i = 0; i < nf; ++i) {
                double d = drho_dt(c, i);
                kv[i] = d > 0.0 ? wf * c->kappa_v_prev[i] / dt : 0.0;
                c->kappa_v[i] = kv[i];
            }
            apply_kappa(c, kv, dt);
            strong_impulse(c, kv, dt);
        }
        for (;;) {
            if (div_it >= c->p.max_iter_divergence) break;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < nf; ++i) {
                double d = drho_dt(c, i);
                c->e_div[i] = d > 0.0 ? d : 0.0;
            }
            double s = 0.0;
            for (int64_t i = 0; i < nf; ++i) s += c->e_div[i];
            div_err = nf > 0 ? s / (double)nf * dt / rho0 : 0.0;
            if (div_it == 0) c->stats[ST_DIV_ERR0] = div_err;
            for (int64_t i = 0; i < nf; ++i) {
                kv[i] = c->alpha[i] * c->e_div[i] / dt;
                c->kappa_v[i] += kv[i];
            }
            apply_kappa(c, kv, dt);
            strong_impulse(c, kv, dt);
            ++div_it;
            if (!((div_err > c->p.eta_divergence) || div_it < c->p.min_iter_divergence)) break;
        }
        free(kv);
    }
    memcpy(c->v_div, c->v, sizeof(double) * 3 * nf);
    c->stats[ST_DIV_ITERS] = div_it;
    c->stats[ST_DIV_ERR] = div_err;

    /* 5. non-pressure forces -> v* */
    non_pressure(c, dt);
    memcpy(c->v_nonp, c->v, sizeof(double) * 3 * nf);

    /* 6. warm start of the constant-density solve */
    double *k = dalloc(nf);
    for (int64_t i = 0; i < nf; ++i) { c->kappa[i] = 0.0; c->kappa0[i] = 0.0; }
    int wcsph = c->p.pressure_solver == 1, pcisph = c->p.pressure_solver == 2;
    if (wcsph) {
        /* WCSPH (Sec. 3.4.1 EOS solver inside Alg. general_algorithm): the pressure comes   */
        /* from the current density by p = k ((rho/rho0)^gamma - 1), clamped at zero (a     */
        /* reading: no tension at the free surface), and the pressure acceleration of Eq.    */
        /* pressure_acceleration (plus the Akinci boundary term) is applied to v* once.  In  */
        /* the stiffness form used by apply_kappa, kappa_i = p_i / rho_i (p/rho^2 =          */
        /* kappa/rho).                                                                       */
        for (int64_t i = 0; i < nf; ++i) {
            double p = c->p.eos_stiffness * (pow(c->rho[i] / rho0, c->p.eos_exponent) - 1.0);
            if (p < 0.0) p = 0.0;
            k[i] = p / c->rho[i];
            c->kappa[i] = k[i];
        }
        apply_kappa(c, k, dt);
        strong_impulse(c, k, dt);
    }
    if (c->p.warm_start != 0 && !wcsph && !pcisph) {
        /* gate: predicted density deviation with v* before any pressure of this step */
        double *dev = dalloc(nf);
        for (int64_t i = 0; i < nf; ++i) dev[i] = (c->rho[i] - rho0) + dt * drho_dt(c, i);
        if (c->p.warm_start == 1) {
            /* half the previous step's total stiffness, stored as kappa dt^2 (a reading) */
            for (int64_t i = 0; i < nf; ++i)
                c->kappa0[i] = dev[i] > 0.0 ? wf * c->kappa_prev[i] / (dt * dt) : 0.0;
        } else if (c->p.warm_start == 2 && c->have_mlp) {
            warm_features(c, dt);
            const double *mu_f = c->mlp + OR_MLP_NW, *sd_f = mu_f + OR_F;
            double mu_y = c->mlp[OR_MLP_NW + 2 * OR_F], sd_y = c->mlp[OR_MLP_NW + 2 * OR_F + 1];
            double *fn = dalloc(4 * nf), *y = dalloc(nf);
            for (int64_t i = 0; i < nf; ++i)
                for (int a = 0; a < 4; ++a) fn[4 * i + a] = (c->feat[4 * i + a] - mu_f[a]) / sd_f[a];
            or_mlp_forward(c->mlp, nf, fn, y);
            /* like the previous-step start, only a fraction of the predicted stiffness is
               applied (a reading: the full prediction overshoots where it errs high) */
            double kref = 9.81 * c->h;
            double lf = c->p.learned_fraction > 0.0 ? c->p.learned_fraction : 0.6;
            for (int64_t i = 0; i < nf; ++i) {
                double kk = (y[i] * sd_y + mu_y) * kref;
                c->kappa0[i] = (dev[i] > 0.0 && kk > 0.0) ? lf * kk : 0.0;
            }
            free(fn);
            free(y);
        }
        free(dev);
        for (int64_t i = 0; i < nf; ++i) { k[i] = c->kappa0[i]; c->kappa[i] = k[i]; }
        apply_kappa(c, k, dt);
        strong_impulse(c, k, dt);
    }

    /* 7. constant-density solve (Eq. density_source with rho* = rho - dt rho div v*).       */
    /* PCISPH refines the total pressure instead: p <- max(p + delta (rho* - rho0), 0) with  */
    /* the prototype's delta, and the velocity moves by the pressure acceleration of the      */
    /* change (Eq. pressure_acceleration is linear in p, so this equals v* plus the          */
    /* acceleration of the total pressure).  Same error measure and iteration limits.        */
    int dens_it = 0;
    double dens_err = 0.0;
    double *ptot = pcisph ? dalloc(nf) : NULL;
    double delta = pcisph ? or_pcisph_factor(c) / (dt * dt) : 0.0;
    for (; !wcsph;) {
        if (dens_it >= c->p.max_iter_density) break;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < nf; ++i) {
            double dev = (c->rho[i] - rho0) + dt * drho_dt(c, i);
            c->e_dens[i] = dev > 0.0 ? dev : 0.0;
        }
        double s = 0.0;
        for (int64_t i = 0; i < nf; ++i) s += c->e_dens[i];
        dens_err = nf > 0 ? s / (double)nf / rho0 : 0.0;
        if (dens_it == 0) c->stats[ST_DENS_ERR0] = dens_err;
        if (pcisph) {
            for (int64_t i = 0; i < nf; ++i) {
                double dev = (c->rho[i] - rho0) + dt * drho_dt(c, i);
                double pn = ptot[i] + delta * dev;
                if (pn < 0.0) pn = 0.0;
                k[i] = (pn - ptot[i]) / c->rho[i];     /* pressure change as stiffness p/rho */
                ptot[i] = pn;
                c->kappa[i] += k[i];
            }
        } else {
            for (int64_t i = 0; i < nf; ++i) {
                k[i] = c->alpha[i] * c->e_dens[i] / (dt * dt);
                c->kappa[i] += k[i];
            }
        }
        apply_kappa(c, k, dt);
        strong_impulse(c, k, dt);
        ++dens_it;
        if (!((dens_err > c->p.eta_density) || dens_it < c->p.min_iter_density)) break;
    }
    if (pcisph) /* the total pressure itself (the increments' sum, without their rounding) */
        for (int64_t i = 0; i < nf; ++i) c->kappa[i] = ptot[i] / c->rho[i];
    free(k);
    free(ptot);
    c->stats[ST_DENS_ITERS] = dens_it;
    c->stats[ST_DENS_ERR] = dens_err;

    /* 8a. boundary reaction (Sec. 3.5 Eq. rigid_pressure_symmetric) with the total applied  */
    /* kappa of this step; the fluid-side impulse is recorded for the antisymmetry pin.     */
    if (!strong)
        for (int64_t k6 = 0; k6 < 6 * c->nbody; ++k6) c->body_force[k6] = 0.0;
    for (int64_t i = 0; i < nf; ++i) {
        double kt = (c->kappa[i] + c->kappa_v[i]) / c->rho[i];
        double imp[3] = {0, 0, 0};
        for (int64_t t = c->fb.start[i]; t < c->fb.start[i + 1]; ++t) {
            int64_t b = c->fb.idx[t];
            double d[3], g[3];
            diffxb(c, i, b, d);
            or_gradW(d, c->h, g);
            double F[3];
            for (int a = 0; a < 3; ++a) {
                F[a] = c->m * c->psi[b] * kt * g[a]; /* force on b from i */
                imp[a] -= dt * F[a];
            }
            int32_t kb = c->body[b];
            if (kb >= 0 && !strong) {
                or_body *B = &c->bodies[kb];
                double r[3] = {c->xb[3 * b] - B->com[0], c->xb[3 * b + 1] - B->com[1], c->xb[3 * b + 2] - B->com[2]};
                double *bf = c->body_force + 6 * kb;
                for (int a = 0; a < 3; ++a) bf[a] += F[a];
                bf[3] += r[1] * F[2] - r[2] * F[1];
                bf[4] += r[2] * F[0] - r[0] * F[2];
                bf[5] += r[0] * F[1] - r[1] * F[0];
            }
        }
        for (int a = 0; a < 3; ++a) c->fb_impulse[3 * i + a] = imp[a];
    }

    /* 8b. advect fluid (symplectic Euler, Sec. 3.3): x += dt v */
    for (int64_t k3 = 0; k3 < 3 * nf; ++k3) c->x[k3] += dt * c->v[k3];

    /* 8c. rigid bodies: symplectic Euler with a renormalised quaternion, weak coupling; no */
    /* contact (the paper delegates it to PyBullet): bodies are clamped inside the domain.  */
    int clamps = 0;
    for (int32_t kb = 0; kb < c->nbody; ++kb) {
        or_body *B = &c->bodies[kb];
        double *bf = c->body_force + 6 * kb;
        /* strong coupling applied the fluid's impulses during the solves already */
        const double fscale = strong ? 0.0 : 1.0;
        for (int a = 0; a < 3; ++a) B->vel[a] += dt * (fscale * bf[a] / B->mass + c->p.gravity[a]);
        for (int a = 0; a < 3; ++a) B->com[a] += dt * B->vel[a];
        double R[3][3];
        quat_to_R(B->quat, R);
        /* world inertia I = R diag(I0) R^T; omega += dt I^-1 (tau - omega x I omega) */
        double Iw[3][3], Iinv[3][3];
        for (int a = 0; a < 3; ++a)
            for (int e = 0; e < 3; ++e) {
                Iw[a][e] = 0.0;
                Iinv[a][e] = 0.0;
                for (int s = 0; s < 3; ++s) {
                    Iw[a][e] += R[a][s] * B->inertia[s] * R[e][s];
                    Iinv[a][e] += R[a][s] / B->inertia[s] * R[e][s];
                }
            }
        double Iwo[3], rhs[3];
        for (int a = 0; a < 3; ++a) Iwo[a] = Iw[a][0] * B->omega[0] + Iw[a][1] * B->omega[1] + Iw[a][2] * B->omega[2];
        rhs[0] = fscale * bf[3] - (B->omega[1] * Iwo[2] - B->omega[2] * Iwo[1]);
        rhs[1] = fscale * bf[4] - (B->omega[2] * Iwo[0] - B->omega[0] * Iwo[2]);
        rhs[2] = fscale * bf[5] - (B->omega[0] * Iwo[1] - B->omega[1] * Iwo[0]);
        for (int a = 0; a < 3; ++a) B->omega[a] += dt * (Iinv[a][0] * rhs[0] + Iinv[a][1] * rhs[1] + Iinv[a][2] * rhs[2]);
        double w = B->quat[0], qx = B->quat[1], qy = B->quat[2], qz = B->quat[3];
        double ox = B->omega[0], oy = B->omega[1], oz = B->omega[2];
        /* dq/dt = 1/2 (0, omega) (x) q */
        double dw = 0.5 * (-ox * qx - oy * qy - oz * qz);
        double dx = 0.5 * (ox * w + oy * qz - oz * qy);
        double dy = 0.5 * (oy * w + oz * qx - ox * qz);
        double dz = 0.5 * (oz * w + ox * qy - oy * qx);
        w += dt * dw; qx += dt * dx; qy += dt * dy; qz += dt * dz;
        double nq = sqrt(w * w + qx * qx + qy * qy + qz * qz);
        B->quat[0] = w / nq; B->quat[1] = qx / nq; B->quat[2] = qy / nq; B->quat[3] = qz / nq;
        /* clamp the bounding sphere inside the domain */
        double rad = 0.0;
        for (int64_t b = 0; b < nb; ++b)
            if (c->body[b] == kb) {
                double r2 = c->r0[3 * b] * c->r0[3 * b] + c->r0[3 * b + 1] * c->r0[3 * b + 1] + c->r0[3 * b + 2] * c->r0[3 * b + 2];
                if (r2 > rad * rad) rad = sqrt(r2);
            }
        for (int a = 0; a < 3; ++a) {
            double lo_a = (double)c->p.domain_min[a] + rad, hi_a = (double)c->p.domain_max[a] - rad;
            if (B->com[a] < lo_a) { B->com[a] = lo_a; if (B->vel[a] < 0) B->vel[a] = 0; ++clamps; }
            if (B->com[a] > hi_a) { B->com[a] = hi_a; if (B->vel[a] > 0) B->vel[a] = 0; ++clamps; }
        }
    }
    if (c->nbody > 0) set_boundary_from_bodies(c);
    c->stats[ST_CLAMPS] += clamps;

    /* 9. bookkeeping: pressure p = kappa rho (Eq. pressure_acceleration with p/rho^2 =   */
    /* kappa/rho), warm-start memory, next CFL step.                                      */
    for (int64_t i = 0; i < nf; ++i) {
        c->pressure[i] = c->kappa[i] * c->rho[i];
        c->kappa_prev[i] = c->kappa[i] * dt * dt;
        c->kappa_v_prev[i] = c->kappa_v[i] * dt;
    }
    c->stats[ST_MAXV] = max_speed(c);
    c->dt_next = cfl_dt(c);
    c->stats[ST_DT_NEXT] = c->dt_next;
    c->stats[ST_STEPS] += 1;
}

int64_t or_field_width(int32_t f)
{
    switch (f) {
    case OR_X: case OR_V: case OR_V_DIV: case OR_V_NONP: case OR_XB: case OR_VB:
    case OR_FLUID_BOUNDARY_IMPULSE: return 3;
    case OR_FEAT: return 4;
    default: return 1;
    }
}

/* Copy a field out (FP64, original particle order).  Returns the element count or -1. */
int64_t or_get(const or_ctx *c, int32_t f, double *out)
{
    int64_t n = (f == OR_PSI || f == OR_XB || f == OR_VB) ? c->nb : c->nf;
    int64_t w = or_field_width(f);
    const double *src = NULL;
    switch (f) {
    case OR_X: src = c->x; break;
    case OR_V: src = c->v; break;
    case OR_RHO: src = c->rho; break;
    case OR_ALPHA: src = c->alpha; break;
    case OR_KAPPA: src = c->kappa; break;
    case OR_KAPPA_V: src = c->kappa_v; break;
    case OR_PRESSURE: src = c->pressure; break;
    case OR_V_DIV: src = c->v_div; break;
    case OR_V_NONP: src = c->v_nonp; break;
    case OR_PSI: src = c->psi; break;
    case OR_XB: src = c->xb; break;
    case OR_VB: src = c->vb; break;
    case OR_KAPPA0: src = c->kappa0; break;
    case OR_FEAT: src = c->feat; break;
    case OR_DIV_ERR_I: src = c->e_div; break;
    case OR_DENS_ERR_I: src = c->e_dens; break;
    case OR_FLUID_BOUNDARY_IMPULSE: src = c->fb_impulse; break;
    case OR_NN_F:
        for (int64_t i = 0; i < n; ++i) out[i] = c->nn_f[i];
        return n;
    case OR_NN_B:
        for (int64_t i = 0; i < n; ++i) out[i] = c->nn_b[i];
        return n;
    default: return -1;
    }
    memcpy(out, src, sizeof(double) * (size_t)(n * w));
    return n * w;
}

void or_get_stats(const or_ctx *c, double *out) { memcpy(out, c->stats, sizeof(c->stats)); }

/* Rigid state out: per body com[3], quat[4], vel[3], omega[3], force[3], torque[3]. */
void or_get_bodies(const or_ctx *c, double *out)
{
    for (int32_t k = 0; k < c->nbody; ++k) {
        const or_body *B = &c->bodies[k];
        double *o = out + 19 * k;
        for (int a = 0; a < 3; ++a) { o[a] = B->com[a]; o[7 + a] = B->vel[a]; o[10 + a] = B->omega[a]; }
        for (int a = 0; a < 4; ++a) o[3 + a] = B->quat[a];
        for (int a = 0; a < 6; ++a) o[13 + a] = c->body_force[6 * k + a];
    }
}

/* Rigid state in (test set-up: resuming from another implementation's state): per body    */
/* com[3], quat[4], vel[3], omega[3] in the layout of or_get_bodies (its force and torque   */
/* columns are ignored); the bodies' boundary particles are placed at the new pose.         */
void or_set_bodies(or_ctx *c, const double *in)
{
    for (int32_t k = 0; k < c->nbody; ++k) {
        or_body *B = &c->bodies[k];
        const double *o = in + 19 * k;
        for (int a = 0; a < 3; ++a) { B->com[a] = o[a]; B->vel[a] = o[7 + a]; B->omega[a] = o[10 + a]; }
        for (int a = 0; a < 4; ++a) B->quat[a] = o[3 + a];
    }
    if (c->nbody > 0) set_boundary_from_bodies(c);
    c->dt_next = cfl_dt(c);
}

double or_mass(const or_ctx *c) { return c->m; }
double or_dt_next(const or_ctx *c) { return c->dt_next; }

int32_t or_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel regions (timing only; results do not depend on it). */
void or_set_num_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
