"""FP64 CPU oracle of the post-processing phase (test infrastructure; the paper's Phase
Three, Sec. 4.3: surface reconstruction of the fluid particles, then rendering).

Only the test suite may import this module.  It restates three plain definitions and
shares nothing with the CUDA library:

* surface_field: the SPH interpolation of the fluid's volume fraction on a regular grid,
  phi(g) = sum_j (m / rho_j) W(|g - x_j|) (Sec. 3.2 Eq. density's interpolant applied to
  the constant 1; about 1 inside the fluid, 0 outside), the cubic spline with h = 4r.
* marching_tetrahedra: the iso-surface phi = iso of a grid field, each grid cube split
  into the six tetrahedra around its main diagonal; per tetrahedron the corners above the
  iso-level (in float32, as the field is float32) are cut off by one triangle (one or
  three corners above) or a quad split into two triangles (two above), vertices linearly
  interpolated along the cut edges from the corner above to the corner below, triangles
  oriented with the normal pointing from the corners above to the corners below (outward
  for a fluid).
* height_map: a headless orthographic view down the -z axis of the particles as spheres
  of radius R: per pixel centre (u, v), the largest z + sqrt(R^2 - d^2) over particles
  whose disk covers it (d < R), else no hit.

Parity unpinned: none; tests/test_oracle_post.py pins each against closed forms.
"""
from __future__ import annotations

import math

import numpy as np

# cube corners, corner index = dx + 2 dy + 4 dz
CORNERS = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0],
                    [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]], dtype=np.int64)
# the six tetrahedra around the diagonal 0 - 7 (one per order of the x, y, z unit steps)
TETS = [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)]


def spline_w(r: np.ndarray, h: float) -> np.ndarray:
    """Cubic spline W(r) with support h (sigma = 8 / (pi h^3))."""
    q = np.asarray(r, np.float64) / h
    w = np.where(q <= 0.5, 6 * q ** 3 - 6 * q ** 2 + 1, np.where(q <= 1.0, 2 * (1 - q) ** 3, 0.0))
    return 8.0 / (math.pi * h ** 3) * w


def surface_field(x, rho, mass, h, origin, spacing, dims) -> np.ndarray:
    """phi on the grid nodes origin + spacing (i, j, k), array [dims[2]][dims[1]][dims[0]]."""
    from scipy.spatial import cKDTree
    x = np.asarray(x, np.float64)
    vol = mass / np.asarray(rho, np.float64)
    nx, ny, nz = (int(d) for d in dims)
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    g = np.asarray(origin, np.float64) + spacing * g.reshape(-1, 3).astype(np.float64)
    tree = cKDTree(x)
    phi = np.zeros(len(g))
    for n, js in enumerate(tree.query_ball_point(g, h)):
        if js:
            js = np.asarray(js)
            phi[n] = np.sum(vol[js] * spline_w(np.linalg.norm(x[js] - g[n], axis=1), h))
    # meshgrid "ij" order is x-major; return [z][y][x]
    return phi.reshape(nx, ny, nz).transpose(2, 1, 0).copy()


def _cut(pa, pb, fa, fb, iso):
    t = (iso - fa) / (fb - fa)
    return pa + t * (pb - pa)


def marching_tetrahedra(field, origin, spacing, iso) -> np.ndarray:
    """Triangles [n][3][3] of the iso-surface of a float32 grid field [nz][ny][nx], cubes
    in x-fastest order, tetrahedra in TETS order, within a tetrahedron the corners and the
    cut edges in ascending corner order."""
    f = np.asarray(field)
    iso32 = np.float32(iso)
    above_all = f.astype(np.float32) > iso32            # the classification, in float32
    f64 = f.astype(np.float64)
    nz, ny, nx = f.shape
    org = np.asarray(origin, np.float64)
    out = []
    for k in range(nz - 1):
        for j in range(ny - 1):
            for i in range(nx - 1):
                idx = [(k + c[2], j + c[1], i + c[0]) for c in CORNERS]
                ab = [bool(above_all[t]) for t in idx]
                if all(ab) or not any(ab):
                    continue
                pos = [org + spacing * np.array([i + c[0], j + c[1], k + c[2]], np.float64) for c in CORNERS]
                val = [float(f64[t]) for t in idx]
                for tet in TETS:
                    ins = [c for c in tet if ab[c]]
                    outs = [c for c in tet if not ab[c]]
                    if len(ins) in (0, 4):
                        continue
                    if len(ins) == 1:
                        a = ins[0]
                        tris = [[_cut(pos[a], pos[b], val[a], val[b], iso) for b in outs]]
                    elif len(ins) == 3:
                        b = outs[0]
                        tris = [[_cut(pos[a], pos[b], val[a], val[b], iso) for a in ins]]
                    else:
                        a0, a1 = ins
                        b0, b1 = outs
                        q = [_cut(pos[a0], pos[b0], val[a0], val[b0], iso),
                             _cut(pos[a0], pos[b1], val[a0], val[b1], iso),
                             _cut(pos[a1], pos[b1], val[a1], val[b1], iso),
                             _cut(pos[a1], pos[b0], val[a1], val[b0], iso)]
                        tris = [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
                    cin = np.mean([pos[c] for c in ins], axis=0)
                    cout = np.mean([pos[c] for c in outs], axis=0)
                    for t in tris:
                        nrm = np.cross(t[1] - t[0], t[2] - t[0])
                        if np.dot(nrm, cout - cin) < 0.0:
                            t = [t[0], t[2], t[1]]
                        out.append(np.array(t))
    return np.array(out, np.float64).reshape(-1, 3, 3)


def height_map(x, radius, lo, hi, width, height):
    """Heights [height][width] (NaN where no particle covers the pixel centre) of the view
    down -z over the rectangle [lo, hi] of the x-y plane."""
    x = np.asarray(x, np.float64)
    du = (hi[0] - lo[0]) / width
    dv = (hi[1] - lo[1]) / height
    hm = np.full((height, width), -np.inf)
    for p in x:
        i0 = max(int(math.floor((p[0] - radius - lo[0]) / du - 0.5)), 0)
        i1 = min(int(math.ceil((p[0] + radius - lo[0]) / du - 0.5)), width - 1)
        j0 = max(int(math.floor((p[1] - radius - lo[1]) / dv - 0.5)), 0)
        j1 = min(int(math.ceil((p[1] + radius - lo[1]) / dv - 0.5)), height - 1)
        if i1 < i0 or j1 < j0:
            continue
        u = lo[0] + (np.arange(i0, i1 + 1) + 0.5) * du
        v = lo[1] + (np.arange(j0, j1 + 1) + 0.5) * dv
        d2 = (u[None, :] - p[0]) ** 2 + (v[:, None] - p[1]) ** 2
        z = np.where(d2 < radius * radius, p[2] + np.sqrt(np.maximum(radius * radius - d2, 0.0)), -np.inf)
        hm[j0:j1 + 1, i0:i1 + 1] = np.maximum(hm[j0:j1 + 1, i0:i1 + 1], z)
    hm[~np.isfinite(hm)] = np.nan
    return hm
