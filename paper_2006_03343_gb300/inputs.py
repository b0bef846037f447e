"""Seeded synthetic inputs for the wall-stress stage.

This module holds no arithmetic of the method: it only draws terrain level sets,
velocity fields, roughness and caller-side stresses, in float64 with
``numpy.random.default_rng(seed)``.  The same arrays feed the CUDA library and
the CPU oracle.

Terrain shapes follow the paper's test geometries (Sec. 4): the cosine-squared
ridge (Eq. 31), the cosine-squared hill (Eq. 32) and the wall-mounted cube
array (Sec. 4.2), plus random Gaussian-hill terrain for batched ensembles.
The mean velocity is the log law of Eq. 29 evaluated at each node's own
distance to the surface, with u* = 1 and kappa = 0.4; seeded Gaussian noise is
added to all three components everywhere, and the "fluid" stresses that an SGS
model would supply are seeded N(0, (0.1 u*^2)^2) fields.

Node positions (Eq. 12 and Sec. 2.4): x_i = i dx, y_j = j dy, uv-nodes at
z = (k + 1/2) dz, w-nodes at z = k dz, with dz = lz / (nz - 1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

KAPPA = 0.4
USTAR = 1.0
TAU_NAMES = ("txx", "txy", "tyy", "tzz", "txz", "tyz")
# grid each stress component lives on (Sec. 3.3): uv-nodes or w-nodes
TAU_ON_W = {"txx": False, "txy": False, "tyy": False, "tzz": False, "txz": True, "tyz": True}


@dataclasses.dataclass
class Case:
    name: str
    grid: tuple            # (nx, ny, nz, lx, ly, lz)
    phi_uv: np.ndarray     # [nz, ny, nx] float64 signed distance at uv-nodes
    phi_w: np.ndarray      # [nz, ny, nx] float64 signed distance at w-nodes
    z0: object             # float or [nz, ny, nx] float64 per-cell roughness
    phi_c: float           # sample distance above the surface (the offset Delta)
    phi_b: float           # half band width
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    tau: dict              # fluid-region stresses, 6 x [nz, ny, nx]
    dtype: str = "f32"     # arithmetic the configuration is run in on the GPU
    seed: int = 0

    @property
    def shape(self):
        nx, ny, nz = self.grid[:3]
        return (nz, ny, nx)

    @property
    def npoints(self):
        nx, ny, nz = self.grid[:3]
        return nx * ny * nz

    @property
    def dz(self):
        return self.grid[5] / (self.grid[2] - 1)


def node_coords(grid):
    """Return (x[nx], y[ny], z_uv[nz], z_w[nz]) node coordinates."""
    nx, ny, nz, lx, ly, lz = grid
    dx, dy, dz = lx / nx, ly / ny, lz / (nz - 1)
    x = np.arange(nx, dtype=np.float64) * dx
    y = np.arange(ny, dtype=np.float64) * dy
    z_uv = (np.arange(nz, dtype=np.float64) + 0.5) * dz
    z_w = np.arange(nz, dtype=np.float64) * dz
    return x, y, z_uv, z_w


def _min_image(d, period):
    return d - period * np.round(d / period)


# --------------------------------------------------------------------------- #
# terrain
# --------------------------------------------------------------------------- #
def heightfield_phi(grid, h2d):
    """phi = z - h(x, y) on both grids for a height field h2d[ny, nx]."""
    _, _, z_uv, z_w = node_coords(grid)
    phi_uv = z_uv[:, None, None] - h2d[None, :, :]
    phi_w = z_w[:, None, None] - h2d[None, :, :]
    return np.ascontiguousarray(phi_uv), np.ascontiguousarray(phi_w)


def ridge_height(grid, height=0.1, half_width=0.3, centre_frac=0.25):
    """2D cosine-squared ridge, Eq. 31, centred at x = centre_frac * lx."""
    nx, ny, nz, lx, ly, lz = grid
    x, y, _, _ = node_coords(grid)
    xr = _min_image(x - centre_frac * lx, lx)
    h1 = np.where(np.abs(xr) < half_width, height * np.cos(np.pi * xr / (2 * half_width)) ** 2, 0.0)
    return np.broadcast_to(h1[None, :], (ny, nx)).copy()


def hill_height(grid, height=0.13, radius=0.5, centre=(0.25, 0.5)):
    """3D cosine-squared hill, Eq. 32, centred at (centre[0] lx, centre[1] ly)."""
    nx, ny, nz, lx, ly, lz = grid
    x, y, _, _ = node_coords(grid)
    xr = _min_image(x - centre[0] * lx, lx)
    yr = _min_image(y - centre[1] * ly, ly)
    r = np.sqrt(xr[None, :] ** 2 + yr[:, None] ** 2)
    return np.where(r < radius, height * np.cos(np.pi * r / (2 * radius)) ** 2, 0.0)


def gaussian_hills_height(grid, rng, nhills=None):
    """Sum of 1-8 periodic Gaussian hills A exp(-r^2 / (2 w^2))."""
    nx, ny, nz, lx, ly, lz = grid
    x, y, _, _ = node_coords(grid)
    if nhills is None:
        nhills = int(rng.integers(1, 9))
    h = np.zeros((ny, nx))
    for _ in range(nhills):
        a = rng.uniform(0.02, 0.2)
        wd = rng.uniform(0.05, 0.4)
        cx = rng.uniform(0.0, lx)
        cy = rng.uniform(0.0, ly)
        xr = _min_image(x - cx, lx)
        yr = _min_image(y - cy, ly)
        h += a * np.exp(-(xr[None, :] ** 2 + yr[:, None] ** 2) / (2 * wd * wd))
    return h


def cube_array_phi(grid, side=0.25, centres_x=(0.5, 1.5, 2.5, 3.5), centres_y=(0.25, 0.75, 1.25, 1.75)):
    """Exact signed distance to an array of wall-mounted cubes (top face at z = side).

    The cubes stand on the floor z = 0; the floor is not part of the immersed
    surface, so each cube is treated as a column reaching below z = 0 (no bottom
    face).  Periodic images in x and y are handled by the minimum image."""
    nx, ny, nz, lx, ly, lz = grid
    x, y, z_uv, z_w = node_coords(grid)
    half = side / 2.0
    out = []
    for z in (z_uv, z_w):
        best = np.full((nz, ny, nx), np.inf)
        for cx in centres_x:
            qx = np.abs(_min_image(x - cx, lx)) - half                 # [nx]
            for cy in centres_y:
                qy = np.abs(_min_image(y - cy, ly)) - half             # [ny]
                qz = z - side                                          # [nz]
                QX = qx[None, None, :]
                QY = qy[None, :, None]
                QZ = qz[:, None, None]
                outside = np.sqrt(np.maximum(QX, 0) ** 2 + np.maximum(QY, 0) ** 2 + np.maximum(QZ, 0) ** 2)
                inside = np.minimum(np.maximum(np.maximum(QX, QY), QZ), 0.0)
                best = np.minimum(best, outside + inside)
        out.append(np.ascontiguousarray(best))
    return out[0], out[1]


# --------------------------------------------------------------------------- #
# fields
# --------------------------------------------------------------------------- #
def log_profile(phi, z0):
    """Eq. 29 mean streamwise velocity at distance phi from the surface; 0 below z0."""
    z0a = np.asarray(z0, dtype=np.float64)
    safe = np.maximum(phi, z0a)
    return np.where(phi > z0a, (USTAR / KAPPA) * np.log(safe / z0a), 0.0)


def velocity(phi_uv, phi_w, z0, rng, sigma):
    u = log_profile(phi_uv, z0) + rng.normal(0.0, sigma, phi_uv.shape)
    v = rng.normal(0.0, sigma, phi_uv.shape)
    w = rng.normal(0.0, sigma, phi_w.shape)
    return u, v, w


def fluid_stress(shape, rng, scale=0.1):
    return {name: rng.normal(0.0, scale * USTAR * USTAR, shape) for name in TAU_NAMES}


def _finish(name, grid, phi_uv, phi_w, z0, phi_c, phi_b, rng, sigma, dtype, seed):
    if not np.isscalar(z0):
        z0 = np.ascontiguousarray(z0)
    u, v, w = velocity(phi_uv, phi_w, z0, rng, sigma)
    tau = fluid_stress(phi_uv.shape, rng)
    return Case(name=name, grid=grid, phi_uv=phi_uv, phi_w=phi_w, z0=z0, phi_c=phi_c, phi_b=phi_b,
                u=np.ascontiguousarray(u), v=np.ascontiguousarray(v), w=np.ascontiguousarray(w),
                tau={k: np.ascontiguousarray(t) for k, t in tau.items()}, dtype=dtype, seed=seed)


# --------------------------------------------------------------------------- #
# the named workloads
# --------------------------------------------------------------------------- #
RIDGE_SHAPE = (32, 32, 32)
CUBES_SHAPE = (256, 128, 128)
HILL_SHAPE = (512, 256, 256)
ENSEMBLE_SHAPES = ((64, 64, 64), (128, 64, 64), (192, 96, 96), (256, 128, 64))
ADJOINT_SHAPE = (256, 128, 128)


def ridge(shape=RIDGE_SHAPE, seed=1, dtype="f64"):
    """2D cosine-squared ridge (H = 0.1, half-width 0.3) in a 2pi x pi x 1 box."""
    nx, ny, nz = shape
    grid = (nx, ny, nz, 2 * math.pi, math.pi, 1.0)
    rng = np.random.default_rng(seed)
    phi_uv, phi_w = heightfield_phi(grid, ridge_height(grid))
    dz = 1.0 / (nz - 1)
    return _finish("ridge", grid, phi_uv, phi_w, 1e-4, 1.5 * dz, 0.5 * dz, rng, 0.1, dtype, seed)


def cubes(shape=CUBES_SHAPE, seed=2, dtype="f32"):
    """4 x 4 wall-mounted cubes of side 0.25 in a 4 x 2 x 1 domain."""
    nx, ny, nz = shape
    grid = (nx, ny, nz, 4.0, 2.0, 1.0)
    rng = np.random.default_rng(seed)
    phi_uv, phi_w = cube_array_phi(grid)
    dz = 1.0 / (nz - 1)
    return _finish("cubes", grid, phi_uv, phi_w, 1e-4, 1.5 * dz, 0.5 * dz, rng, 0.15, dtype, seed)


def hill(shape=HILL_SHAPE, seed=3, dtype="f32"):
    """3D cosine-squared hill (H = 0.13, R = 0.5) with a lognormal per-cell z0."""
    nx, ny, nz = shape
    grid = (nx, ny, nz, 2 * math.pi, math.pi, 1.0)
    rng = np.random.default_rng(seed)
    phi_uv, phi_w = heightfield_phi(grid, hill_height(grid))
    z0 = 1e-4 * np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    dz = 1.0 / (nz - 1)
    return _finish("hill", grid, phi_uv, phi_w, z0, 1.5 * dz, 0.5 * dz, rng, 0.1, dtype, seed)


def ensemble_member(m, shape=None, seed_base=4000, dtype="f32"):
    """Member m of the random Gaussian-hill ensemble (own grid, offset and roughness)."""
    seed = seed_base + m
    rng = np.random.default_rng(seed)
    if shape is None:
        shape = ENSEMBLE_SHAPES[int(rng.integers(0, len(ENSEMBLE_SHAPES)))]
    nx, ny, nz = shape
    grid = (nx, ny, nz, 2 * math.pi, math.pi, 1.0)
    phi_uv, phi_w = heightfield_phi(grid, gaussian_hills_height(grid, rng))
    dz = 1.0 / (nz - 1)
    phi_c = float(rng.uniform(1.0, 2.0)) * dz
    z0 = float(10.0 ** rng.uniform(-5.0, -3.0))
    return _finish(f"ensemble{m}", grid, phi_uv, phi_w, z0, phi_c, 0.5 * dz, rng, 0.1, dtype, seed)


def ensemble(count=64, seed_base=4000, shapes=None, dtype="f32"):
    return [ensemble_member(m, None if shapes is None else shapes[m % len(shapes)], seed_base, dtype)
            for m in range(count)]


def adjoint_case(shape=ADJOINT_SHAPE, seed=5, dtype="f32"):
    """Random multi-hill terrain with a per-cell log-roughness field and a seeded
    weight g on the three forcing components (the linear functional L = <g, f>)."""
    nx, ny, nz = shape
    grid = (nx, ny, nz, 2 * math.pi, math.pi, 1.0)
    rng = np.random.default_rng(seed)
    phi_uv, phi_w = heightfield_phi(grid, gaussian_hills_height(grid, rng))
    z0 = 1e-4 * np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    dz = 1.0 / (nz - 1)
    case = _finish("adjoint", grid, phi_uv, phi_w, z0, 1.5 * dz, 0.5 * dz, rng, 0.1, dtype, seed)
    g = [np.ascontiguousarray(rng.standard_normal((nz, ny, nx))) for _ in range(3)]
    return case, g


def flat(shape, wall_height=0.0, z0=1e-4, phi_c_cells=1.5, phi_b_cells=0.5, lengths=(1.0, 1.0, 1.0),
         sigma=0.0, seed=0, dtype="f64"):
    """Flat terrain with the wall at z = wall_height (the raised walls of Sec. 4.1)."""
    nx, ny, nz = shape
    grid = (nx, ny, nz) + tuple(lengths)
    dz = lengths[2] / (nz - 1)
    rng = np.random.default_rng(seed)
    h = np.full((ny, nx), float(wall_height))
    phi_uv, phi_w = heightfield_phi(grid, h)
    return _finish("flat", grid, phi_uv, phi_w, z0, phi_c_cells * dz, phi_b_cells * dz, rng, sigma, dtype, seed)


CONFIGS = {
    "ridge": ridge,
    "cubes": cubes,
    "hill": hill,
}


def make(name: str, shape: Optional[tuple] = None, **kw) -> Case:
    fn = CONFIGS[name]
    return fn(shape=shape, **kw) if shape is not None else fn(**kw)
