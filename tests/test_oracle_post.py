"""Pins of the post-processing oracle (oracle/postprocess.py): the volume-fraction field of
one particle in closed form and of a uniform lattice (exactly 1 at the particles, where
every rho_j equals the lattice density), marching tetrahedra on a plane (every vertex on
it, the exact area, normals up), on a sphere (a closed 2-manifold, vertices on the sphere
within the grid interpolation error, area within 2 %, outward normals), and the height map
of one and two spheres."""
import math

import numpy as np
import pytest

import oracle
from oracle import postprocess as post


def test_field_of_one_particle():
    h, m, rho = 0.04, 0.008, 1000.0
    x = np.array([[0.1, 0.1, 0.1]])
    phi = post.surface_field(x, [rho], m, h, (0.05, 0.06, 0.07), 0.01, (11, 9, 8))
    g = np.stack(np.meshgrid(0.05 + 0.01 * np.arange(11), 0.06 + 0.01 * np.arange(9),
                             0.07 + 0.01 * np.arange(8), indexing="ij"), -1)
    r = np.linalg.norm(g - x[0], axis=-1)
    q = r / h
    w = np.where(q <= 0.5, 6 * q ** 3 - 6 * q ** 2 + 1, np.where(q <= 1, 2 * (1 - q) ** 3, 0))
    want = (m / rho) * 8 / (math.pi * h ** 3) * w
    np.testing.assert_allclose(phi, want.transpose(2, 1, 0), rtol=1e-12, atol=1e-15)


def test_field_is_one_inside_a_lattice():
    r = 2.0 ** -7
    s, h = 2 * r, 4 * r
    m = 1000.0 * s ** 3
    g = np.arange(9) * s
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.25
    # the interior particles' SPH density: the lattice sum (rest density S/pi of the pins)
    rho_lat = m * post.spline_w(np.linalg.norm(x - x[4 + 9 * (4 + 9 * 4)], axis=1), h).sum()
    rho = np.full(len(x), rho_lat)
    phi = post.surface_field(x, rho, m, h, (0.25 + 4 * s,) * 3, s, (1, 1, 1))
    assert phi[0, 0, 0] == pytest.approx(1.0, rel=1e-12)


def _edges(tris):
    key = lambda p: tuple(np.round(p, 9))
    e = {}
    for t in tris:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            k = tuple(sorted((key(t[a]), key(t[b]))))
            e[k] = e.get(k, 0) + 1
    return e


def test_marching_tetrahedra_plane():
    n = 6
    z = np.arange(n)[:, None, None] * np.ones((n, n, n))
    field = (2.3 - z).astype(np.float32)                 # above 0 below z = 2.3
    tris = post.marching_tetrahedra(field, (0, 0, 0), 1.0, 0.0)
    assert len(tris) > 0
    np.testing.assert_allclose(tris[..., 2], 2.3, rtol=0, atol=1e-6)
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert np.all(nrm[:, 2] > 0)                          # from the high side to the low side
    assert 0.5 * np.linalg.norm(nrm, axis=1).sum() == pytest.approx((n - 1) ** 2, rel=1e-6)


def test_marching_tetrahedra_sphere_is_closed():
    n, R = 24, 7.3
    c = np.array([11.6, 11.4, 11.5])
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    field = (R - np.linalg.norm(g - c, axis=-1)).transpose(2, 1, 0).astype(np.float32)
    tris = post.marching_tetrahedra(field, (0, 0, 0), 1.0, 0.0)
    # every edge shared by exactly two triangles, Euler characteristic 2
    e = _edges(tris)
    assert set(e.values()) == {2}
    verts = {tuple(np.round(p, 9)) for t in tris for p in t}
    assert len(verts) - len(e) + len(tris) == 2
    r = np.linalg.norm(tris.reshape(-1, 3) - c, axis=1)
    assert np.abs(r - R).max() < 0.1 * R
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    area = 0.5 * np.linalg.norm(nrm, axis=1).sum()
    assert area == pytest.approx(4 * math.pi * R * R, rel=0.02)
    assert np.all(np.einsum("ij,ij->i", nrm, tris.mean(axis=1) - c) > 0)   # outward


def test_height_map_spheres():
    R = 0.05
    x = np.array([[0.3, 0.3, 0.1], [0.34, 0.3, 0.12]])
    hm = post.height_map(x[:1], R, (0.2, 0.2), (0.4, 0.4), 40, 40)   # 5 mm pixels
    # pixel (i, j) centre: 0.2 + (i + 0.5) 0.005; the centre pixel nearest (0.3, 0.3)
    u = 0.2 + (np.arange(40) + 0.5) * 0.005
    d2 = (u[None, :] - 0.3) ** 2 + (u[:, None] - 0.3) ** 2
    want = np.where(d2 < R * R, 0.1 + np.sqrt(np.maximum(R * R - d2, 0)), np.nan)
    np.testing.assert_allclose(hm, want, rtol=0, atol=1e-15)
    two = post.height_map(x, R, (0.2, 0.2), (0.4, 0.4), 40, 40)
    one_b = post.height_map(x[1:], R, (0.2, 0.2), (0.4, 0.4), 40, 40)
    np.testing.assert_allclose(two, np.fmax(hm, one_b), rtol=0, atol=0)
