"""Seeded synthetic scene generators.

This module is the only code the CUDA path and the CPU oracle share: it places particles
(lattices, jitter, box surfaces) and fills in parameter dictionaries.  It holds none of
the method's arithmetic -- no kernel, density, mass or solver formula -- so both sides
compute everything physical on their own.

The paper's scenes need meshes and render assets that are not available (dragons,
biscuit, nine rigid objects, Sec. 5); the dam-break, rigid-box and column scenes below
stand in for them with the paper's particle radius, support radius and rest density
(r = 0.01 m, h = 4r, rho0 = 1000 kg/m^3, Sec. 5) where the workload does not fix them.

A scene is a dict with keys ``fluid_x`` [n,3] f32, ``fluid_v`` [n,3] f32, ``boundary_x``
[nb,3] f32, ``boundary_body`` [nb] i32 (-1 = static wall), ``bodies`` (list of dicts with
mass, inertia, com, quat, vel, omega) and the solver parameters.
"""
from __future__ import annotations

import math

import numpy as np

VISC_NONE, VISC_EXPLICIT, VISC_XSPH, VISC_IMPLICIT = 0, 1, 2, 3
WARM_ZERO, WARM_PREVIOUS, WARM_LEARNED = 0, 1, 2
SOLVER_DFSPH, SOLVER_WCSPH, SOLVER_PCISPH = 0, 1, 2
COUPLING_WEAK, COUPLING_STRONG = 0, 1


def params(radius=0.01, rest_density=1000.0, viscosity=0.01, gravity=(0.0, 0.0, -9.81),
           domain_min=(0.0, 0.0, 0.0), domain_max=(1.0, 1.0, 1.0), eta_density=1e-3,
           eta_divergence=1e-3, dt_max=4e-4, cfl=0.0, min_iter_density=2,
           max_iter_density=100, min_iter_divergence=1, max_iter_divergence=100,
           viscosity_mode=VISC_EXPLICIT, warm_start=WARM_PREVIOUS, divergence_solve=1,
           xsph_c=0.0, cg_tol=1e-4, cg_max_iter=500, max_fluid_neighbors=0,
           max_boundary_neighbors=0, cell_size=0.0, lanes_per_particle=0, pressure_solver=0,
           eos_stiffness=0.0, eos_exponent=7.0, warm_start_fraction=0.0, rigid_coupling=0,
           learned_fraction=0.0, learned_gate=0):
    return dict(radius=float(radius), rest_density=float(rest_density),
                viscosity=float(viscosity), gravity=tuple(float(g) for g in gravity),
                domain_min=tuple(float(a) for a in domain_min),
                domain_max=tuple(float(a) for a in domain_max),
                eta_density=float(eta_density), eta_divergence=float(eta_divergence),
                dt_max=float(dt_max), cfl=float(cfl), min_iter_density=int(min_iter_density),
                max_iter_density=int(max_iter_density),
                min_iter_divergence=int(min_iter_divergence),
                max_iter_divergence=int(max_iter_divergence),
                viscosity_mode=int(viscosity_mode), warm_start=int(warm_start),
                divergence_solve=int(divergence_solve), xsph_c=float(xsph_c),
                cg_tol=float(cg_tol), cg_max_iter=int(cg_max_iter),
                max_fluid_neighbors=int(max_fluid_neighbors),
                max_boundary_neighbors=int(max_boundary_neighbors),
                cell_size=float(cell_size), lanes_per_particle=int(lanes_per_particle),
                pressure_solver=int(pressure_solver), eos_stiffness=float(eos_stiffness),
                eos_exponent=float(eos_exponent), warm_start_fraction=float(warm_start_fraction),
                rigid_coupling=int(rigid_coupling), learned_fraction=float(learned_fraction),
                learned_gate=int(learned_gate))


def lattice_block(n, spacing, origin, jitter=0.0, rng=None):
    """Points origin + spacing * (i, j, k), 0 <= i < n[0] ..., x fastest, plus uniform
    jitter in [-jitter, jitter] per coordinate."""
    nx, ny, nz = (int(a) for a in n)
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    k = np.arange(nz, dtype=np.float64)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    p = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1) * spacing + np.asarray(origin)
    if jitter > 0.0:
        rng = rng if rng is not None else np.random.default_rng(0)
        p = p + rng.uniform(-jitter, jitter, size=p.shape)
    return p.astype(np.float32)


def box_surface(n, spacing, origin):
    """Surface points of the lattice origin + spacing * (i, j, k), 0 <= i <= n[0] ...:
    every lattice point with at least one index on its minimum or maximum.  `spacing`
    may be a scalar or one value per axis."""
    nx, ny, nz = (int(a) for a in n)
    sp = np.broadcast_to(np.asarray(spacing, dtype=np.float64), (3,))
    i = np.arange(nx + 1)
    j = np.arange(ny + 1)
    k = np.arange(nz + 1)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    idx = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    on = ((idx[:, 0] == 0) | (idx[:, 0] == nx) | (idx[:, 1] == 0) | (idx[:, 1] == ny)
          | (idx[:, 2] == 0) | (idx[:, 2] == nz))
    pts = idx[on] * sp + np.asarray(origin, dtype=np.float64)
    return pts.astype(np.float32)


def tank_walls(extent, spacing):
    """One wall layer lining [0, extent[a]] per axis, sampled with round(extent/spacing)
    intervals per axis (so the spacing is within a hair of `spacing`)."""
    n = [max(1, int(round(e / spacing))) for e in extent]
    sp = [e / m for e, m in zip(extent, n)]
    return box_surface(n, sp, (0.0, 0.0, 0.0))


# Gap between the first fluid layer and a one-layer wall, in units of the spacing 2r.
# At 1.1 spacings the wall's Akinci contribution reproduces the rest density of the
# first fluid layer (about +0.1 %); at 1.0 spacing it over-counts by 6-15 % (corners),
# and the solver turns that into a 16 m/s kick in the first step.
WALL_GAP = 1.1


def plane(n, spacing, origin):
    """One layer z = origin[2] of (n[0]+1) x (n[1]+1) points."""
    pts = lattice_block((n[0] + 1, n[1] + 1, 1), spacing, origin)
    return pts


def cube_body(center, edge, spacing, density):
    """A solid-cube rigid body sampled on its surface; returns (points, body dict).
    The inertia is the solid cube's, mass density * edge^3 (inputs, not solver math)."""
    n = int(round(edge / spacing))
    origin = np.asarray(center, dtype=np.float64) - 0.5 * edge
    pts = box_surface((n, n, n), spacing, origin)
    mass = density * edge ** 3
    inertia = mass * edge * edge / 6.0
    body = dict(mass=mass, inertia=(inertia, inertia, inertia), com=tuple(center),
                quat=(1.0, 0.0, 0.0, 0.0), vel=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0))
    return pts, body


def _scene(fluid_x, boundary_x, p, fluid_v=None, boundary_body=None, bodies=None):
    fluid_x = np.ascontiguousarray(fluid_x, dtype=np.float32).reshape(-1, 3)
    boundary_x = np.ascontiguousarray(boundary_x, dtype=np.float32).reshape(-1, 3)
    d = dict(p)
    d["fluid_x"] = fluid_x
    d["fluid_v"] = (np.zeros_like(fluid_x) if fluid_v is None
                    else np.ascontiguousarray(fluid_v, dtype=np.float32).reshape(-1, 3))
    d["boundary_x"] = boundary_x
    d["boundary_body"] = (np.full(len(boundary_x), -1, dtype=np.int32) if boundary_body is None
                          else np.ascontiguousarray(boundary_body, dtype=np.int32))
    d["bodies"] = list(bodies or [])
    return d


# ------------------------------------------------------------------------------ workloads
def dam_break_small(seed=1, n=(20, 20, 20), radius=0.01, box=0.8, jitter=1e-4, **kw):
    """Dam break: an n[0] x n[1] x n[2] lattice at spacing 2r (min corner 2.2r from the
    walls, uniform jitter) inside one layer of wall particles lining [0, box]^3 at 2r.
    With the defaults: 8,000 fluid and 41^3 - 39^3 = 9,602 wall particles, nu = 0.01,
    dt = 4e-4 s, eta = 0.1 %."""
    rng = np.random.default_rng(seed)
    s = 2.0 * radius
    g = WALL_GAP * s
    fx = lattice_block(n, s, (g, g, g), jitter, rng)
    bx = tank_walls((box, box, box), s)
    defaults = dict(radius=radius, domain_min=(0.0, 0.0, 0.0), domain_max=(box, box, box),
                    viscosity=0.01, dt_max=4e-4)
    defaults.update(kw)
    return _scene(fx, bx, params(**defaults))


def wcsph_parameters(height, radius, rest_density=1000.0, gamma=7.0, mach=0.1, cfl=0.4):
    """Equation-of-state parameters for a column of the given height (WCSPH practice; the
    paper fixes none): a numerical sound speed c with the largest free-fall speed
    sqrt(2 g height) at Mach `mach`, stiffness k = rho0 c^2 / gamma, and the acoustic step
    dt = cfl h / c with h = 4r."""
    c = np.sqrt(2.0 * 9.81 * height) / mach
    return dict(pressure_solver=SOLVER_WCSPH, eos_stiffness=float(rest_density * c * c / gamma),
                eos_exponent=float(gamma), dt_max=float(cfl * 4.0 * radius / c),
                warm_start=WARM_ZERO, divergence_solve=0)


def dam_break_wcsph(seed=1, n=(20, 20, 20), radius=0.01, box=0.8, **kw):
    """The small dam break under the WCSPH pressure solver (Sec. 3.4.1), with the
    equation-of-state parameters of wcsph_parameters for the column's height."""
    p = wcsph_parameters(n[2] * 2.0 * radius, radius)
    p.update(kw)
    return dam_break_small(seed=seed, n=n, radius=radius, box=box, **p)


def dam_break_pcisph(seed=1, n=(20, 20, 20), radius=0.01, box=0.8, **kw):
    """The small dam break under PCISPH (pressure refined iteratively to the same 0.1 %
    density tolerance; no divergence solve, no warm start)."""
    p = dict(pressure_solver=SOLVER_PCISPH, warm_start=WARM_ZERO, divergence_solve=0,
             min_iter_density=3)
    p.update(kw)
    return dam_break_small(seed=seed, n=n, radius=radius, box=box, **p)


def body_in_fluid(seed=3, n=(14, 14, 14), radius=0.01, edge=0.06, density=300.0, compress=0.95,
                  jitter=2e-4, **kw):
    """A cube body (surface-sampled at 2r, given density) in the middle of a fluid lattice
    block at spacing compress * 2r (slightly compressed, so the first step has pressure),
    fluid particles closer than 1.1 spacings to the cube removed; no walls, no gravity
    unless given."""
    rng = np.random.default_rng(seed)
    s = 2.0 * radius
    fx = lattice_block(n, compress * s, (0.1, 0.1, 0.1), jitter, rng)
    c = fx.astype(np.float64).mean(axis=0)
    pts, body = cube_body(tuple(c), edge, s, density)
    keep = np.any(np.abs(fx - c) > 0.5 * edge + WALL_GAP * s, axis=1)
    ext = 0.2 + n[0] * s
    defaults = dict(radius=radius, domain_min=(0.0, 0.0, 0.0), domain_max=(ext, ext, ext),
                    gravity=(0.0, 0.0, 0.0), viscosity=0.0, viscosity_mode=VISC_NONE)
    defaults.update(kw)
    return _scene(fx[keep], pts, params(**defaults), boundary_body=np.zeros(len(pts), np.int32),
                  bodies=[body])


def dam_break_rigid(seed=2, n=(125, 98, 98), radius=0.005, tank=(2.0, 1.0, 1.0),
                    n_boxes=3, box_edge=0.1, box_density=500.0, jitter=None, **kw):
    """Large dam break with two-way rigid coupling: a 125 x 98 x 98 = 1,200,500-particle
    lattice at spacing 2r = 0.01 m, 1.1 spacings from the x = 0, y = 0, z = 0 walls, in a
    closed 2 x 1 x 1 m tank of one wall layer at spacing 2r (100,002 particles); n_boxes
    surface-sampled cubes (edge 0.1 m, density 500 kg/m^3, 602 particles each) at rest at
    x = 1.45, 1.65, 1.85, y = 0.5, z = 0.8.  CFL dt <= 1e-3 s, eta = 0.1 %.
    (A 120 x 100 x 100 block at that spacing fills the 1 m cross-section with no room for
    a wall gap; 125 x 98 x 98 keeps the particle count and the tank.)"""
    rng = np.random.default_rng(seed)
    s = 2.0 * radius
    jit = 0.01 * s if jitter is None else jitter
    g = WALL_GAP * s
    fx = lattice_block(n, s, (g, g, g), jit, rng)
    walls = tank_walls(tank, s)
    parts = [walls]
    body_ids = [np.full(len(walls), -1, dtype=np.int32)]
    bodies = []
    centers = [(1.45, 0.5, 0.8), (1.65, 0.5, 0.8), (1.85, 0.5, 0.8)]
    for k in range(n_boxes):
        c = centers[k % len(centers)]
        c = (c[0] * tank[0] / 2.0, c[1] * tank[1], c[2] * tank[2])
        pts, body = cube_body(c, box_edge, s, box_density)
        parts.append(pts)
        body_ids.append(np.full(len(pts), k, dtype=np.int32))
        bodies.append(body)
    defaults = dict(radius=radius, domain_min=(0.0, 0.0, 0.0), domain_max=tuple(tank),
                    viscosity=0.01, dt_max=1e-3, cfl=0.4)
    defaults.update(kw)
    return _scene(fx, np.concatenate(parts), params(**defaults),
                  boundary_body=np.concatenate(body_ids), bodies=bodies)


def viscous_column(seed=3, n=(50, 50, 100), radius=0.0025, gap=0.1, plane_size=1.0,
                   **kw):
    """High-viscosity column: an n lattice at spacing 2r (0.25 x 0.25 x 0.5 m with the
    defaults) whose bottom sits `gap` above a one-layer plane of (plane_size/2r + 1)^2
    particles; nu = 0.1 m^2/s with the implicit solve, CG tolerance 1e-4."""
    rng = np.random.default_rng(seed)
    s = 2.0 * radius
    ext = np.array(n) * s
    origin = (-0.5 * ext[0], -0.5 * ext[1], gap)
    fx = lattice_block(n, s, origin, 0.01 * s, rng)
    m = int(round(plane_size / s))
    px = plane((m, m), s, (-0.5 * plane_size, -0.5 * plane_size, 0.0))
    top = gap + ext[2] + 0.2
    defaults = dict(radius=radius, viscosity=0.1, viscosity_mode=VISC_IMPLICIT,
                    domain_min=(-0.5 * plane_size, -0.5 * plane_size, 0.0),
                    domain_max=(0.5 * plane_size, 0.5 * plane_size, top), dt_max=1e-3,
                    cfl=0.4, cg_tol=1e-4)
    defaults.update(kw)
    return _scene(fx, px, params(**defaults))


def dam_break_random(seed, n_target, radius=0.005, aspect=None, fill=None, **kw):
    """A dam break with about n_target fluid particles in a closed tank of aspect ratio
    `aspect` (length / width, drawn from U[1, 3] when None) whose fluid block fills the
    fraction `fill` of the tank volume (U[0.2, 0.6] when None).  The block spans the full
    tank width and height 0.8 of the tank; its length sets the fill."""
    rng = np.random.default_rng(seed)
    aspect = float(rng.uniform(1.0, 3.0)) if aspect is None else float(aspect)
    fill = float(rng.uniform(0.2, 0.6)) if fill is None else float(fill)
    s = 2.0 * radius
    vol = n_target * s ** 3 / fill
    width = (vol / aspect) ** (1.0 / 3.0)
    length = aspect * width
    ny = max(2, int(round(width / s)) - 2)
    nz = max(2, int(round(0.8 * width / s)))
    nx = max(2, int(round(n_target / (ny * nz))))
    nx = min(nx, int(round(length / s)) - 1)
    g = WALL_GAP * s
    fx = lattice_block((nx, ny, nz), s, (g, g, g), 0.01 * s, rng)
    tank = (length, (ny - 1) * s + 2.0 * g, width)
    walls = tank_walls(tank, s)
    defaults = dict(radius=radius, domain_min=(0.0, 0.0, 0.0), domain_max=tank,
                    viscosity=0.01, dt_max=1e-3, cfl=0.4)
    defaults.update(kw)
    return _scene(fx, walls, params(**defaults))


def batch_scene_sizes(n_scenes=64, lo=2e4, hi=2e5, seed=5):
    """Fluid particle counts drawn log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(n_scenes)]


def batch_dam_break(n_scenes=64, lo=2e4, hi=2e5, seed=5, radius=0.01, fill=0.4, **kw):
    """n_scenes independent dam breaks with log-uniform particle counts in [lo, hi]; each
    cubic tank is scaled so that the fluid fills `fill` of it.  Fixed dt = 4e-4 s."""
    sizes = batch_scene_sizes(n_scenes, lo, hi, seed)
    out = []
    for k, n in enumerate(sizes):
        defaults = dict(dt_max=4e-4, cfl=0.0)
        defaults.update(kw)
        out.append(dam_break_random(seed * 1000 + k, n, radius=radius, aspect=1.0, fill=fill,
                                    **defaults))
    return out


def resting_tank(n=(8, 8, 8), radius=0.01, jitter=0.0, seed=0, **kw):
    """A fluid block filling the bottom of a closed one-layer tank of its own footprint
    (1.1 spacings of wall gap on every side), twice the block's height, for hydrostatic
    checks."""
    rng = np.random.default_rng(seed)
    s = 2.0 * radius
    g = WALL_GAP * s
    fx = lattice_block(n, s, (g, g, g), jitter, rng)
    tank = ((n[0] - 1) * s + 2 * g, (n[1] - 1) * s + 2 * g, 2.0 * n[2] * s)
    walls = tank_walls(tank, s)
    defaults = dict(radius=radius, domain_min=(0.0, 0.0, 0.0), domain_max=tank,
                    viscosity=0.05, dt_max=1e-3)
    defaults.update(kw)
    return _scene(fx, walls, params(**defaults))


def random_cloud(n, seed=0, radius=0.01, extent=0.2, **kw):
    """n fluid particles uniform in a cube of side `extent`, no boundary."""
    rng = np.random.default_rng(seed)
    fx = rng.uniform(0.0, extent, size=(n, 3)).astype(np.float32)
    defaults = dict(radius=radius, domain_min=(0.0, 0.0, 0.0),
                    domain_max=(extent, extent, extent))
    defaults.update(kw)
    return _scene(fx, np.zeros((0, 3), np.float32), params(**defaults))
