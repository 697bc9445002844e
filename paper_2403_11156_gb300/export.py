"""Export of the post-processing results to files (the paper's Phase Three, Sec. 4.3, hands
particles to SplashSurf and Blender; here the surface and the view are computed by the
library's kernels and only written out on the host):

* write_obj: a triangle mesh from sph_surface_mesh as a Wavefront OBJ file, vertices
  shared between triangles (the kernels compute a shared edge's vertex bit-identically);
* write_pgm: a height map from sph_render_heightmap as an 8-bit greyscale PGM image,
  shaded by the slope of the height field (Lambert with a light from the upper left),
  empty pixels black.
"""
from __future__ import annotations

import numpy as np


def write_obj(tris, path: str) -> int:
    """Write triangles [n][3][3] (array or tensor); returns the vertex count."""
    t = tris.detach().cpu().numpy() if hasattr(tris, "detach") else np.asarray(tris)
    t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1, 3)
    verts, inv = np.unique(t.view(np.dtype((np.void, 12))), return_inverse=True)
    v = verts.view(np.float32).reshape(-1, 3)
    faces = inv.reshape(-1, 3) + 1
    with open(path, "w") as f:
        f.write("# %d vertices, %d triangles\n" % (len(v), len(faces)))
        np.savetxt(f, v, fmt="v %.7g %.7g %.7g")
        np.savetxt(f, faces, fmt="f %d %d %d")
    return len(v)


def shade(height, pixel: float):
    """Greyscale shading [h][w] uint8 of a height map (NaN = empty) with square pixels of
    the given size: n = (-dz/dx, -dz/dy, 1) normalised, light (-1, 1, 2) normalised."""
    hm = height.detach().cpu().numpy() if hasattr(height, "detach") else np.asarray(height)
    hm = np.asarray(hm, np.float64)
    full = np.where(np.isfinite(hm), hm, np.nanmin(hm) if np.isfinite(hm).any() else 0.0)
    gy, gx = np.gradient(full, pixel)
    n = np.stack([-gx, -gy, np.ones_like(full)], -1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    light = np.array([-1.0, 1.0, 2.0]) / np.sqrt(6.0)
    lum = np.clip(n @ light, 0.0, 1.0)
    img = (40 + 215 * lum).astype(np.uint8)
    img[~np.isfinite(hm)] = 0
    return img[::-1]                      # image rows top-down: +y up


def write_pgm(height, pixel: float, path: str) -> None:
    img = shade(height, pixel)
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        f.write(img.tobytes())
