// sph_post.cu -- the post-processing phase (Sec. 4.3) as CUDA kernels: the fluid's
// volume-fraction field on a regular grid (surface reconstruction input), its iso-surface
// by marching tetrahedra, and a headless orthographic height map of the particles.
//
//  * field: phi(g) = sum_j (m / rho_j) W(|g - x_j|), the SPH interpolant (Sec. 3.2) of the
//    constant 1: about 1 inside the fluid, 0 outside.  The scene's particles are first
//    sorted into its cell grid (counting sort, then a rank by index inside each cell, so
//    the summation order and the result are reproducible); one thread per grid node then
//    walks the node's stencil of cells.
//  * mesh: each grid cube is split into the six tetrahedra around its diagonal from corner
//    0 to corner 7 (corner index = dx + 2 dy + 4 dz); per tetrahedron the corners above the
//    iso-level are cut off by one triangle (one or three corners above) or two (two
//    above), vertices interpolated linearly along the cut edges from the corner above to
//    the corner below (the same arithmetic in every cube sharing an edge), each triangle oriented
//    so its normal points from the corners above to those below.  A counting pass, a
//    prefix sum and an emitting pass write the triangles in cube order.
//  * height map: per particle, the pixels of its disk receive z + sqrt(R^2 - d^2) through
//    an atomic maximum on an order-preserving integer image of the float.
#include "sph.h"
#include "sph_sweep.cuh"

#include <algorithm>
#include <cmath>

namespace sph {

namespace {

constexpr int kPostBlock = 256;

// ------------------------------------------------------------------ field
__global__ void k_pf_hist(const float4 *__restrict__ pos, int64_t n, SceneDev sc, uint32_t *count,
                          uint32_t *key, uint32_t *slot)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos[i];
    const int32_t ix = cell_coord(p.x, sc.origin[0], sc.cell, sc.dims[0]);
    const int32_t iy = cell_coord(p.y, sc.origin[1], sc.cell, sc.dims[1]);
    const int32_t iz = cell_coord(p.z, sc.origin[2], sc.cell, sc.dims[2]);
    const uint32_t k = (uint32_t)ix + (uint32_t)sc.dims[0] * ((uint32_t)iy + (uint32_t)sc.dims[1] * (uint32_t)iz);
    key[i] = k;
    slot[i] = atomicAdd(&count[k], 1u);
}

// Place each particle in its cell's range (order inside a cell not yet fixed).
__global__ void k_pf_place(int64_t n, const uint32_t *__restrict__ key, const uint32_t *__restrict__ slot,
                           const uint32_t *__restrict__ start, uint32_t *cellidx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cellidx[start[key[i]] + slot[i]] = (uint32_t)i;
}

// Rank inside the cell by particle index (reproducible order) and write (x, m / rho), rho
// the particle's density of the last step (the rest density before the first step).
__global__ void k_pf_rank(const float4 *__restrict__ pos, const float4 *__restrict__ vel, int64_t n, float mass,
                          float rho0, const uint32_t *__restrict__ key, const uint32_t *__restrict__ start,
                          const uint32_t *__restrict__ cellidx, float4 *sorted)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = cellidx[s];
    const uint32_t k = key[i];
    const uint32_t b = start[k], e = start[k + 1];
    uint32_t rank = 0;
    for (uint32_t t = b; t < e; ++t) rank += cellidx[t] < i ? 1u : 0u;
    const float4 p = pos[i];
    const float rho = vel[i].w;
    sorted[b + rank] = make_float4(p.x, p.y, p.z, mass / (rho > 0.0f ? rho : rho0));
}

__global__ void k_pf_field(const float4 *__restrict__ sorted, const uint32_t *__restrict__ start, SceneDev sc,
                           float ox, float oy, float oz, float spacing, int32_t nx, int32_t ny, int32_t nz,
                           float *__restrict__ out)
{
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nx * ny * nz;
    if (node >= total) return;
    const int32_t i = (int32_t)(node % nx), j = (int32_t)((node / nx) % ny), k = (int32_t)(node / ((int64_t)nx * ny));
    const float gx = fmaf((float)i, spacing, ox), gy = fmaf((float)j, spacing, oy), gz = fmaf((float)k, spacing, oz);
    const int32_t cx = cell_coord(gx, sc.origin[0], sc.cell, sc.dims[0]);
    const int32_t cy = cell_coord(gy, sc.origin[1], sc.cell, sc.dims[1]);
    const int32_t cz = cell_coord(gz, sc.origin[2], sc.cell, sc.dims[2]);
    const int32_t R = sc.R;
    const int32_t x0 = max(cx - R, 0), x1 = min(cx + R, sc.dims[0] - 1);
    float phi = 0.0f;
    for (int32_t dz = -R; dz <= R; ++dz) {
        const int32_t z = cz + dz;
        if (z < 0 || z >= sc.dims[2]) continue;
        for (int32_t dy = -R; dy <= R; ++dy) {
            const int32_t y = cy + dy;
            if (y < 0 || y >= sc.dims[1]) continue;
            const int64_t row = (int64_t)sc.dims[0] * (y + (int64_t)sc.dims[1] * z);
            for (uint32_t t = start[row + x0]; t < start[row + x1 + 1]; ++t) {
                const float4 p = __ldg(sorted + t);
                const float dx = gx - p.x, dy2 = gy - p.y, dz2 = gz - p.z;
                const float d2 = fmaf(dx, dx, fmaf(dy2, dy2, dz2 * dz2));
                if (d2 < sc.h2) phi = fmaf(p.w, sc.sigma * spline_w(sqrtf(d2) * sc.inv_h), phi);
            }
        }
    }
    out[node] = phi;
}

// ------------------------------------------------------------------ marching tetrahedra
__constant__ int8_t c_tets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                    {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

struct Cube {
    float v[8];
    float p[8][3];
    int above;   // bit c: corner c is above the iso-level
};

__device__ __forceinline__ bool load_cube(const float *__restrict__ f, int32_t nx, int32_t ny, int64_t cube,
                                          int32_t cx_, int32_t cy_, float ox, float oy, float oz, float sp,
                                          float iso, Cube &c)
{
    const int32_t i = (int32_t)(cube % cx_), j = (int32_t)((cube / cx_) % cy_), k = (int32_t)(cube / ((int64_t)cx_ * cy_));
    c.above = 0;
    for (int q = 0; q < 8; ++q) {
        const int32_t di = q & 1, dj = (q >> 1) & 1, dk = (q >> 2) & 1;
        const int64_t a = (int64_t)(i + di) + (int64_t)nx * ((j + dj) + (int64_t)ny * (k + dk));
        c.v[q] = f[a];
        c.p[q][0] = fmaf((float)(i + di), sp, ox);
        c.p[q][1] = fmaf((float)(j + dj), sp, oy);
        c.p[q][2] = fmaf((float)(k + dk), sp, oz);
        if (c.v[q] > iso) c.above |= 1 << q;
    }
    return c.above != 0 && c.above != 0xff;
}

__device__ __forceinline__ int tet_count(int above, int t)
{
    int n = 0;
    for (int q = 0; q < 4; ++q) n += (above >> c_tets[t][q]) & 1;
    return (n == 0 || n == 4) ? 0 : (n == 2 ? 2 : 1);
}

__device__ __forceinline__ void cut(const Cube &c, int a, int b, float iso, float *out)
{
    const float t = (iso - c.v[a]) / (c.v[b] - c.v[a]);
    for (int d = 0; d < 3; ++d) out[d] = fmaf(t, c.p[b][d] - c.p[a][d], c.p[a][d]);
}

// Write triangle (q0, q1, q2), flipped if its normal points from the outside corners'
// centroid towards the inside corners' centroid.
__device__ __forceinline__ void emit(const float *q0, const float *q1, const float *q2, const float *cin,
                                     const float *cout, float *dst)
{
    const float e1[3] = {q1[0] - q0[0], q1[1] - q0[1], q1[2] - q0[2]};
    const float e2[3] = {q2[0] - q0[0], q2[1] - q0[1], q2[2] - q0[2]};
    const float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const float dot = n[0] * (cout[0] - cin[0]) + n[1] * (cout[1] - cin[1]) + n[2] * (cout[2] - cin[2]);
    const float *b = dot < 0.0f ? q2 : q1, *c = dot < 0.0f ? q1 : q2;
    for (int d = 0; d < 3; ++d) {
        dst[d] = q0[d];
        dst[3 + d] = b[d];
        dst[6 + d] = c[d];
    }
}

__global__ void k_mt_count(const float *__restrict__ f, int32_t nx, int32_t ny, int32_t nz, float iso,
                           uint32_t *count)
{
    const int32_t cx_ = nx - 1, cy_ = ny - 1, cz_ = nz - 1;
    const int64_t cube = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cube >= (int64_t)cx_ * cy_ * cz_) return;
    Cube c;
    uint32_t n = 0;
    if (load_cube(f, nx, ny, cube, cx_, cy_, 0.0f, 0.0f, 0.0f, 1.0f, iso, c))
        for (int t = 0; t < 6; ++t) n += (uint32_t)tet_count(c.above, t);
    count[cube] = n;
}

__global__ void k_mt_emit(const float *__restrict__ f, int32_t nx, int32_t ny, int32_t nz, float ox, float oy,
                          float oz, float sp, float iso, const uint32_t *__restrict__ start, float *tris, int64_t cap)
{
    const int32_t cx_ = nx - 1, cy_ = ny - 1, cz_ = nz - 1;
    const int64_t cube = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cube >= (int64_t)cx_ * cy_ * cz_) return;
    Cube c;
    if (!load_cube(f, nx, ny, cube, cx_, cy_, ox, oy, oz, sp, iso, c)) return;
    int64_t o = start[cube];
    for (int t = 0; t < 6; ++t) {
        int ins[4], outs[4], ni = 0, no = 0;
        for (int q = 0; q < 4; ++q) {
            const int v = c_tets[t][q];
            if ((c.above >> v) & 1) ins[ni++] = v;
            else outs[no++] = v;
        }
        if (ni == 0 || ni == 4) continue;
        float cin[3] = {0, 0, 0}, cout[3] = {0, 0, 0};
        for (int q = 0; q < ni; ++q)
            for (int d = 0; d < 3; ++d) cin[d] += c.p[ins[q]][d] / (float)ni;
        for (int q = 0; q < no; ++q)
            for (int d = 0; d < 3; ++d) cout[d] += c.p[outs[q]][d] / (float)no;
        if (ni == 1 || ni == 3) {
            // every cut runs from the corner above to the corner below, so the tetrahedra
            // sharing a grid edge compute the same vertex (a watertight mesh)
            float q[3][3];
            for (int e = 0; e < 3; ++e) {
                if (ni == 1) cut(c, ins[0], outs[e], iso, q[e]);
                else cut(c, ins[e], outs[0], iso, q[e]);
            }
            if (o < cap) emit(q[0], q[1], q[2], cin, cout, tris + 9 * o);
            ++o;
        } else {
            float q[4][3];
            cut(c, ins[0], outs[0], iso, q[0]);
            cut(c, ins[0], outs[1], iso, q[1]);
            cut(c, ins[1], outs[1], iso, q[2]);
            cut(c, ins[1], outs[0], iso, q[3]);
            if (o < cap) emit(q[0], q[1], q[2], cin, cout, tris + 9 * o);
            ++o;
            if (o < cap) emit(q[0], q[2], q[3], cin, cout, tris + 9 * o);
            ++o;
        }
    }
}

// ------------------------------------------------------------------ height map
__device__ __forceinline__ uint32_t order_key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float order_value(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_hm_clear(uint32_t *img, int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) img[k] = 0u;
}

__global__ void k_hm_splat(const float4 *__restrict__ pos, int64_t n, float lox, float loy, float du, float dv,
                           int32_t w, int32_t h, float R, uint32_t *img)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos[i];
    // pixel range of the disk's bounding box, clamped in float before the conversion
    auto px = [](float v, int32_t n) { return (int32_t)fminf(fmaxf(v, -1.0f), (float)n); };
    const int32_t i0 = max(px(floorf((p.x - R - lox) / du - 0.5f), w), 0);
    const int32_t i1 = min(px(ceilf((p.x + R - lox) / du - 0.5f), w), w - 1);
    const int32_t j0 = max(px(floorf((p.y - R - loy) / dv - 0.5f), h), 0);
    const int32_t j1 = min(px(ceilf((p.y + R - loy) / dv - 0.5f), h), h - 1);
    const float R2 = R * R;
    for (int32_t j = j0; j <= j1; ++j) {
        const float v = fmaf((float)j + 0.5f, dv, loy) - p.y;
        for (int32_t ii = i0; ii <= i1; ++ii) {
            const float u = fmaf((float)ii + 0.5f, du, lox) - p.x;
            const float d2 = fmaf(u, u, v * v);
            if (d2 < R2) atomicMax(img + (int64_t)j * w + ii, order_key(p.z + sqrtf(R2 - d2)));
        }
    }
}

__global__ void k_hm_decode(const uint32_t *img, int64_t n, float *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t v = img[k];
    out[k] = v == 0u ? __int_as_float(0x7fc00000) : order_value(v);
}

int blocks_for(int64_t n) { return (int)((n + kPostBlock - 1) / kPostBlock); }

// Scratch for a prefix sum: status words and control block, zeroed.
cudaError_t scan_scratch(int64_t n, uint64_t **status, Control **ctl, cudaStream_t s)
{
    const int32_t tiles = scan_tiles_for(n);
    cudaError_t e = cudaMallocAsync((void **)status, sizeof(uint64_t) * (size_t)std::max(tiles, 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)ctl, sizeof(Control), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(*status, 0, sizeof(uint64_t) * (size_t)std::max(tiles, 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(*ctl, 0, sizeof(Control), s);
    return e;
}

}  // namespace

cudaError_t post_surface_field(const SceneDev &sc, const float4 *pos, const float4 *vel, const float origin[3],
                               float spacing, const int32_t dims[3], float *out, cudaStream_t s)
{
    const int64_t n = sc.nf, ncell = sc.ncell;
    uint32_t *count = nullptr, *start = nullptr, *key = nullptr, *slot = nullptr, *cellidx = nullptr;
    float4 *sorted = nullptr;
    uint64_t *status = nullptr;
    Control *ctl = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&count, sizeof(uint32_t) * ncell, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&start, sizeof(uint32_t) * (ncell + 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&key, sizeof(uint32_t) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&slot, sizeof(uint32_t) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cellidx, sizeof(uint32_t) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&sorted, sizeof(float4) * n, s);
    if (e == cudaSuccess) e = scan_scratch(ncell, &status, &ctl, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * ncell, s);
    if (e == cudaSuccess) {
        k_pf_hist<<<blocks_for(n), kPostBlock, 0, s>>>(pos, n, sc, count, key, slot);
        launch_scan(count, start, ncell, status, scan_tiles_for(ncell), &ctl->scan[0], ctl, s);
        k_pf_place<<<blocks_for(n), kPostBlock, 0, s>>>(n, key, slot, start, cellidx);
        k_pf_rank<<<blocks_for(n), kPostBlock, 0, s>>>(pos, vel, n, sc.m, sc.rho0, key, start, cellidx, sorted);
        const int64_t nodes = (int64_t)dims[0] * dims[1] * dims[2];
        k_pf_field<<<blocks_for(nodes), kPostBlock, 0, s>>>(sorted, start, sc, origin[0], origin[1], origin[2],
                                                             spacing, dims[0], dims[1], dims[2], out);
        e = cudaGetLastError();
    }
    for (void *p : {(void *)count, (void *)start, (void *)key, (void *)slot, (void *)cellidx, (void *)sorted,
                    (void *)status, (void *)ctl})
        if (p) cudaFreeAsync(p, s);
    return e;
}

cudaError_t post_height_map(const float4 *pos, int64_t n, const float lo[2], const float hi[2], int32_t w,
                            int32_t h, float radius, float *out, cudaStream_t s)
{
    const int64_t px = (int64_t)w * h;
    uint32_t *img = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&img, sizeof(uint32_t) * px, s);
    if (e != cudaSuccess) return e;
    const float du = (hi[0] - lo[0]) / (float)w, dv = (hi[1] - lo[1]) / (float)h;
    k_hm_clear<<<blocks_for(px), kPostBlock, 0, s>>>(img, px);
    if (n > 0) k_hm_splat<<<blocks_for(n), kPostBlock, 0, s>>>(pos, n, lo[0], lo[1], du, dv, w, h, radius, img);
    k_hm_decode<<<blocks_for(px), kPostBlock, 0, s>>>(img, px, out);
    e = cudaGetLastError();
    cudaFreeAsync(img, s);
    return e;
}

}  // namespace sph

using namespace sph;

extern "C" sph_status sph_surface_mesh(const float *field, const int32_t dims[3], const float origin[3],
                                       float spacing, float iso, float *tris, int64_t cap, int64_t *n_tris,
                                       void *stream)
{
    if (!field || !dims || !origin || !n_tris || cap < 0 || (cap > 0 && !tris)) return SPH_EINVAL;
    if (!(spacing > 0.0f) || !std::isfinite(spacing) || !std::isfinite(iso)) return SPH_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || !std::isfinite(origin[a])) return SPH_EINVAL;
    const int64_t cubes = (int64_t)(dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1);
    if ((int64_t)dims[0] * dims[1] * dims[2] > ((int64_t)1 << 31)) return SPH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *count = nullptr, *start = nullptr;
    uint64_t *status = nullptr;
    Control *ctl = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&count, sizeof(uint32_t) * cubes, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&start, sizeof(uint32_t) * (cubes + 1), s);
    if (e == cudaSuccess) e = scan_scratch(cubes, &status, &ctl, s);
    uint32_t total = 0;
    if (e == cudaSuccess) {
        k_mt_count<<<blocks_for(cubes), kPostBlock, 0, s>>>(field, dims[0], dims[1], dims[2], iso, count);
        launch_scan(count, start, cubes, status, scan_tiles_for(cubes), &ctl->scan[0], ctl, s);
        if (cap > 0)
            k_mt_emit<<<blocks_for(cubes), kPostBlock, 0, s>>>(field, dims[0], dims[1], dims[2], origin[0],
                                                               origin[1], origin[2], spacing, iso, start, tris, cap);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, start + cubes, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    }
    int32_t scan_err = 0;
    if (e == cudaSuccess && ctl) e = cudaMemcpyAsync(&scan_err, &ctl->error, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    for (void *p : {(void *)count, (void *)start, (void *)status, (void *)ctl})
        if (p) cudaFreeAsync(p, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return SPH_ECUDA;
    if (scan_err) return SPH_ETIMEOUT;
    *n_tris = (int64_t)total;
    return (int64_t)total > cap ? SPH_EOVERFLOW : SPH_OK;
}
